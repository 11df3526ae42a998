// vbgs_estep_cc.cu -- E-step and fused statistics contraction on the CUDA
// cores, in FP64 (the plain form) or FP32.
//
// `compute_elbo_delta` (Alg. 1) needs, for every point n and component k,
//   log rho_nk = c_k - 1/2 |M_k (x_n - m_k)|^2 - psi(sum alpha),
// with M_k = sqrt(nu_k) L_k^-1 lower triangular (W_k^-1 = L_k L_k^T): the
// factored quadratic form, no expansion, so no cancellation between large
// terms.  The two passes never store an N x K array:
//   pass 1  point-parallel: each thread owns PPT points and streams the
//           component records of one K-split through shared memory,
//           keeping an online (max, sum of exp) pair; a merge kernel
//           combines the splits into lse_n and fixed-order block sums.
//   pass 2  component-parallel: each thread owns one component and streams
//           the points of one N-split (x, lse, upper(x x^T)) through shared
//           memory, accumulating r_nk [1, x, upper(x x^T)] -- the fused
//           contraction Delta S = R^T S_u of Eq. 3 with R recomputed on the
//           fly instead of materialised (Alg. 3 instead of Alg. 2).
//   reduce  sums the N-split partials of Delta S in a fixed order (FP64).
// FP64 form: everything in double, exp() from the CUDA math library.
// FP32 form: records in float and log2 units, ex2.approx on the MUFU, FP32
// accumulation inside a split, FP64 partials and reduction.
#include "vbgs_internal.cuh"
#include <algorithm>
#include <mutex>
#include <string>

namespace vbgs {

namespace {

constexpr int kThreads = 128;
constexpr int kChunkK = 64;   // component records per shared-memory chunk (pass 1)
constexpr int kChunkN = 64;   // points per shared-memory chunk (pass 2)

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <typename T> struct Arith;
template <> struct Arith<double> {
    // r = exp(l - ref) in natural units
    static __device__ __forceinline__ double expd(double v) { return exp(v); }
    static __device__ __forceinline__ double lse_scale() { return 1.0; }
};
template <> struct Arith<float> {
    // records are in log2 units: r = 2^(l2 - ref2)
    static __device__ __forceinline__ float expd(float v) { return ex2_approx(v); }
    static __device__ __forceinline__ float lse_scale() { return 1.4426950408889634f; }
};

// logit (without the -psi(sum alpha) term) of point x under record r:
// c - 1/2 |M (x - m)|^2, M packed lower triangle at r[6..26].
template <typename T>
__device__ __forceinline__ T logit(const T *__restrict__ r, const T x[6])
{
    T d[6];
#pragma unroll
    for (int i = 0; i < 6; i++) d[i] = x[i] - r[i];
    T q = T(0);
#pragma unroll
    for (int i = 0; i < 6; i++) {
        T y = T(0);
#pragma unroll
        for (int j = 0; j <= i; j++) y = fma(r[6 + tri(i, j)], d[j], y);
        q = fma(y, y, q);
    }
    return fma(T(-0.5), q, r[27]);
}

// Pass 1.  grid = (point blocks, K splits).  part[split * N + n] = (max, sum)
// with max in natural units and sum = sum_k exp(l_k - max).  When tmax is
// given, also the largest logit of every (256-point block, 64-component
// chunk) in natural units, tmax[block * nkc + chunk]; this needs kps to be a
// multiple of kChunkK so chunks align across splits.
template <typename T, int PPT>
__global__ void __launch_bounds__(kThreads) k_pass1(const double *__restrict__ X, int64_t N,
                                                    const T *__restrict__ rec, int K, int kps,
                                                    double2 *__restrict__ part, float *__restrict__ tmax)
{
    __shared__ T srec[kChunkK * 28];
    __shared__ float sred[kThreads / 32];
    const int split = blockIdx.y;
    const int k0 = split * kps;
    const int k1 = min(K, k0 + kps);
    const int nkc = (K + kChunkK - 1) / kChunkK;
    T x[PPT][6], mx[PPT], s[PPT];
    int64_t nb = (int64_t)blockIdx.x * kThreads * PPT + threadIdx.x;
#pragma unroll
    for (int p = 0; p < PPT; p++) {
        int64_t n = nb + (int64_t)p * kThreads;
        int64_t nn = n < N ? n : N - 1;
#pragma unroll
        for (int i = 0; i < 6; i++) x[p][i] = (T)X[nn * VBGS_XS + i];
        mx[p] = -INFINITY;
        s[p] = T(0);
    }
    for (int kc = k0; kc < k1; kc += kChunkK) {
        const int cnt = min(kChunkK, k1 - kc);
        __syncthreads();
        for (int i = threadIdx.x; i < cnt * 28; i += kThreads)
            srec[i] = rec[(size_t)(kc + i / 28) * VBGS_REC + (i % 28)];
        __syncthreads();
        T cmax = -INFINITY;
        for (int j = 0; j < cnt; j++) {
            const T *r = srec + j * 28;
#pragma unroll
            for (int p = 0; p < PPT; p++) {
                T l = logit<T>(r, x[p]);
                cmax = l > cmax ? l : cmax;
                if (l > mx[p]) {
                    s[p] = fma(s[p], Arith<T>::expd(mx[p] - l), T(1));
                    mx[p] = l;
                } else {
                    s[p] += Arith<T>::expd(l - mx[p]);
                }
            }
        }
        if (tmax) {
            float v = (float)((double)cmax / (double)Arith<T>::lse_scale());
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
            if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = v;
            __syncthreads();
            if (threadIdx.x == 0) {
                float w = sred[0];
#pragma unroll
                for (int i = 1; i < kThreads / 32; i++) w = fmaxf(w, sred[i]);
                tmax[(size_t)blockIdx.x * nkc + kc / kChunkK] = w;
            }
        }
    }
#pragma unroll
    for (int p = 0; p < PPT; p++) {
        int64_t n = nb + (int64_t)p * kThreads;
        if (n < N) {
            double m = (double)mx[p] / (double)Arith<T>::lse_scale();
            part[(size_t)split * N + n] = make_double2(m, (double)s[p]);
        }
    }
}

// Merge the K-split partials into lse_n and per-block sums of lse (fixed order).
// Without item_start the partials are split-major, part[j * N + n]; with it
// they are per work item of 128 points, part[q * 128 + n % 128] for the items
// q = item_start[n / 128] .. item_start[n / 128 + 1] - 1 of the point's tile.
__global__ void __launch_bounds__(256) k_merge(const double2 *__restrict__ part, int nsplit, int64_t N,
                                               const int *__restrict__ item_start, double *__restrict__ lse,
                                               double *__restrict__ lse_part, float *__restrict__ minlse)
{
    __shared__ double sh[8];
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (n < N) {
        size_t base = (size_t)n, stride = (size_t)N;
        int cnt = nsplit;
        if (item_start) {
            const int64_t P = n >> 7;
            base = (size_t)item_start[P] * 128 + (size_t)(n & 127);
            stride = 128;
            cnt = item_start[P + 1] - item_start[P];
        }
        double M = -INFINITY;
        for (int j = 0; j < cnt; j++) M = fmax(M, part[base + (size_t)j * stride].x);
        double s = 0.0;
        for (int j = 0; j < cnt; j++) {
            double2 p = part[base + (size_t)j * stride];
            if (p.y > 0.0) s += p.y * exp(p.x - M);
        }
        v = M + log(s);
        lse[n] = v;
    }
    float vm = n < N ? (float)v : INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v += __shfl_down_sync(0xffffffffu, v, o);
        vm = fminf(vm, __shfl_down_sync(0xffffffffu, vm, o));
    }
    // minlse per 32 points (one warp), the skip bound's lower bound on lse
    if ((threadIdx.x & 31) == 0) {
        sh[threadIdx.x >> 5] = v;
        const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
        if (minlse && w * 32 < N) minlse[w] = vm;
    }
    __syncthreads();
    if (threadIdx.x == 0 && lse_part) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += sh[i];
        lse_part[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024) k_sum(const double *__restrict__ v, int n, double *__restrict__ out)
{
    pdl_wait();
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += sh[i];
        *out = t;
    }
}

// Pass 2.  grid = (component tiles of 128, N splits).  part[(split * K + k) * 28 + f].
// FP64: raw moments [1, x, upper(x x^T)] (the plain form).  FP32: moments of
// d = x - a_k about the component's anchor a_k = m_k (the record's mean), so
// that FP32 accumulation never forms the large, cancelling raw second
// moments; k_reduce_splits shifts them back to raw moments in FP64.
// With tile maxima (tmax: largest logit of every (tpb-point block, tkc-
// component block), nkc column blocks) and per-32-point minima of lse, a
// 64-point chunk is skipped when the largest of the maxima it touches minus
// the smallest lse of its points is below -skip_nats (uniform across the CTA).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_pass2(const double *__restrict__ X,
                                                    const double *__restrict__ lse, int64_t N,
                                                    int64_t nps, const T *__restrict__ rec, int K,
                                                    double *__restrict__ part,
                                                    const float *__restrict__ tmax,
                                                    const float *__restrict__ minlse,
                                                    int tpb, int tkc, unsigned long long *__restrict__ pairs,
                                                    float skip_nats)
{
    constexpr bool kAnchored = sizeof(T) == 4;
    __shared__ T spt[kChunkN * 28];   // per point: x[6], lse, upper(x x^T)[21] (FP64 only)
    const int k = blockIdx.x * kThreads + threadIdx.x;
    const int split = blockIdx.y;
    const int64_t n0 = (int64_t)split * nps;
    const int64_t n1 = min(N, n0 + nps);
    T r[28];
    const int kk = k < K ? k : K - 1;
#pragma unroll
    for (int i = 0; i < 28; i++) r[i] = rec[(size_t)kk * VBGS_REC + i];
    T acc[28];
#pragma unroll
    for (int f = 0; f < 28; f++) acc[f] = T(0);

    const int nkc = (K + tkc - 1) / (tkc > 0 ? tkc : 1);
    const int kt0 = blockIdx.x * kThreads;
    const int c_lo = kt0 / (tkc > 0 ? tkc : 1), c_hi = min(K - 1, kt0 + kThreads - 1) / (tkc > 0 ? tkc : 1);
    for (int64_t nc = n0; nc < n1; nc += kChunkN) {
        const int cnt = (int)min((int64_t)kChunkN, n1 - nc);
        if (tmax) {
            float b = -INFINITY, lmin = INFINITY;
            for (int64_t r = nc / tpb; r <= (nc + cnt - 1) / tpb; r++)
                for (int c = c_lo; c <= c_hi; c++) b = fmaxf(b, tmax[r * nkc + c]);
            for (int64_t w = nc / 32; w <= (nc + cnt - 1) / 32; w++) lmin = fminf(lmin, minlse[w]);
            if (b - lmin < -skip_nats) continue;
        }
        if (pairs && threadIdx.x == 0) atomicAdd(pairs, (unsigned long long)cnt * (unsigned long long)min(kThreads, K - kt0));
        __syncthreads();
        for (int p = threadIdx.x; p < cnt; p += kThreads) {
            const double *xp = X + (nc + p) * VBGS_XS;
            T *o = spt + p * 28;
            double xd[6];
#pragma unroll
            for (int i = 0; i < 6; i++) { xd[i] = xp[i]; o[i] = (T)xd[i]; }
            o[6] = (T)(lse[nc + p] * (double)Arith<T>::lse_scale());
            if (!kAnchored) {
                int u = 7;
#pragma unroll
                for (int i = 0; i < 6; i++)
#pragma unroll
                    for (int j = i; j < 6; j++) o[u++] = (T)(xd[i] * xd[j]);
            }
        }
        __syncthreads();
        for (int p = 0; p < cnt; p++) {
            const T *o = spt + p * 28;
            T x[6];
#pragma unroll
            for (int i = 0; i < 6; i++) x[i] = o[i];
            const T w = Arith<T>::expd(logit<T>(r, x) - o[6]);
            acc[0] += w;
            if (kAnchored) {
                T d[6], wd[6];
#pragma unroll
                for (int i = 0; i < 6; i++) { d[i] = x[i] - r[i]; wd[i] = w * d[i]; acc[1 + i] += wd[i]; }
                int u = 7;
#pragma unroll
                for (int i = 0; i < 6; i++)
#pragma unroll
                    for (int j = i; j < 6; j++, u++) acc[u] = fma(wd[i], d[j], acc[u]);
            } else {
#pragma unroll
                for (int i = 0; i < 6; i++) acc[1 + i] = fma(w, x[i], acc[1 + i]);
#pragma unroll
                for (int f = 7; f < 28; f++) acc[f] = fma(w, o[f], acc[f]);
            }
        }
    }
    if (k < K) {
        double *dst = part + ((size_t)split * K + k) * 28;
#pragma unroll
        for (int f = 0; f < 28; f++) dst[f] = (double)acc[f];
    }
}

// dS[k * 28 + f] = sum over splits in order.  With an anchor (FP32 records),
// the split sums are moments about a_k and are shifted to raw moments:
//   S1 = S1' + N a,  S2 = S2' + a S1'^T + S1' a^T + N a a^T   (FP64).
__global__ void k_reduce_splits(const double *__restrict__ part, int nsplit, int K,
                                const float *__restrict__ anchor, const int *__restrict__ kperm,
                                double *__restrict__ dS)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const size_t n = (size_t)K * 28;
    double s[28];
#pragma unroll
    for (int f = 0; f < 28; f++) s[f] = 0.0;
    for (int j = 0; j < nsplit; j++) {
        const double *p = part + (size_t)j * n + (size_t)k * 28;
#pragma unroll
        for (int f = 0; f < 28; f++) s[f] += p[f];
    }
    if (anchor) {
        double a[6], s1[6];
#pragma unroll
        for (int i = 0; i < 6; i++) { a[i] = (double)anchor[(size_t)k * VBGS_REC + i]; s1[i] = s[1 + i]; }
        int u = 7;
#pragma unroll
        for (int i = 0; i < 6; i++)
#pragma unroll
            for (int j = i; j < 6; j++, u++) s[u] += a[i] * s1[j] + s1[i] * a[j] + s[0] * a[i] * a[j];
#pragma unroll
        for (int i = 0; i < 6; i++) s[1 + i] += s[0] * a[i];
    }
    const size_t out = kperm ? (size_t)kperm[k] : (size_t)k;
#pragma unroll
    for (int f = 0; f < 28; f++) dS[out * 28 + f] = s[f];
}

struct Plan {
    int p1_blocks, p1_splits, kps;
    int p2_tiles, p2_splits;
    int64_t nps;
    size_t scratch;   // doubles
};

template <int PPT>
Plan make_plan(int64_t N, int K, int num_sms)
{
    Plan pl{};
    const int target = num_sms * 8;
    pl.p1_blocks = (int)((N + kThreads * PPT - 1) / (kThreads * PPT));
    int s1 = std::max(1, (target + pl.p1_blocks - 1) / std::max(1, pl.p1_blocks));
    s1 = std::min(s1, std::max(1, K / 16));
    pl.kps = (K + s1 - 1) / s1;
    pl.kps = (pl.kps + kChunkK - 1) / kChunkK * kChunkK;   // chunk-aligned splits (tile maxima)
    pl.p1_splits = (K + pl.kps - 1) / pl.kps;
    pl.p2_tiles = (K + kThreads - 1) / kThreads;
    int64_t s2 = std::max<int64_t>(1, (target + pl.p2_tiles - 1) / pl.p2_tiles);
    s2 = std::min<int64_t>(s2, std::max<int64_t>(1, N / 64));
    s2 = std::min<int64_t>(s2, 1024);
    pl.nps = (N + s2 - 1) / s2;
    pl.nps = (pl.nps + 255) / 256 * 256;                   // block-aligned splits (skip bound)
    pl.p2_splits = (int)((N + pl.nps - 1) / pl.nps);
    pl.scratch = std::max((size_t)pl.p1_splits * (size_t)N * 2, (size_t)pl.p2_splits * (size_t)K * 28);
    return pl;
}

constexpr int kPPT64 = 2;
constexpr int kPPT32 = 2;

} // namespace

double skip_nats_for(int precision, int K)
{
    const double t = std::log((double)std::max(K, 1)) + (precision == VBGS_FP64 ? 37.0 : 20.0);
    return std::max(t, 20.0);
}

int launch_block_sum(const double *part, int n, double *sum_out, cudaStream_t st, Prof *pf)
{
    pf->begin(VBGS_PROF_MERGE, st);
    launch_pdl(k_sum, 1, 1024, 0, st, part, n, sum_out);
    pf->end(st);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_lse_merge(const double2 *part, int nsplit, int64_t N, const int *item_start, double *lse,
                     double *lse_part, float *minlse, double *sum_out, cudaStream_t st, Prof *pf)
{
    // 64-point blocks: the FP64 exp/log of the merge is latency bound, so
    // spread it over every SM
    const int mb = (int)((N + 63) / 64);
    pf->begin(VBGS_PROF_MERGE, st);
    k_merge<<<mb, 64, 0, st>>>(part, nsplit, N, item_start, lse, lse_part, minlse);
    pf->end(st);
    pf->begin(VBGS_PROF_MERGE, st);
    launch_pdl(k_sum, 1, 1024, 0, st, lse_part, mb, sum_out);
    pf->end(st);
    return cudaGetLastError() == cudaSuccess ? 2 : -1;
}

int launch_pass2_fp32(const EstepBuffers &B, int tpb, int tkc, cudaStream_t st, Prof *pf)
{
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    Plan pl = make_plan<kPPT32>(B.N, B.K, sms);
    if ((size_t)pl.p2_splits * (size_t)B.K * 28 > B.part_cap) return -2;
    dim3 g2(pl.p2_tiles, pl.p2_splits);
    pf->begin(VBGS_PROF_PASS2, st);
    k_pass2<float><<<g2, kThreads, 0, st>>>(B.X, B.lse, B.N, pl.nps, B.rec32, B.K, B.part, B.tmax, B.minlse, tpb, tkc,
                                            pf->on ? pf->d_pairs : nullptr, B.skip_nats);
    pf->end(st);
    pf->begin(VBGS_PROF_REDUCE, st);
    k_reduce_splits<<<(B.K + 127) / 128, 128, 0, st>>>(B.part, pl.p2_splits, B.K, B.rec32, B.kperm, B.dS);
    pf->end(st);
    return cudaGetLastError() == cudaSuccess ? 2 : -1;
}

size_t estep_cuda_core_scratch(int64_t N, int K, int precision)
{
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    Plan pl = precision == VBGS_FP64 ? make_plan<kPPT64>(N, K, sms) : make_plan<kPPT32>(N, K, sms);
    return pl.scratch;
}

int launch_estep_cuda_core(const EstepBuffers &B, int precision, bool want_stats, cudaStream_t st,
                           Prof *pf)
{
    if (B.N <= 0) return 0;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool f64 = precision == VBGS_FP64;
    Plan pl = f64 ? make_plan<kPPT64>(B.N, B.K, sms) : make_plan<kPPT32>(B.N, B.K, sms);
    if (pl.scratch > B.part_cap) return -2;
    int launches = 0;
    double2 *p1 = reinterpret_cast<double2 *>(B.part);
    dim3 g1(pl.p1_blocks, pl.p1_splits);
    pf->begin(VBGS_PROF_PASS1, st);
    float *tmax = want_stats ? B.tmax : nullptr;
    if (f64) k_pass1<double, kPPT64><<<g1, kThreads, 0, st>>>(B.X, B.N, B.rec, B.K, pl.kps, p1, tmax);
    else     k_pass1<float, kPPT32><<<g1, kThreads, 0, st>>>(B.X, B.N, B.rec32, B.K, pl.kps, p1, tmax);
    pf->end(st);
    const int mb = (int)((B.N + 63) / 64);
    pf->begin(VBGS_PROF_MERGE, st);
    k_merge<<<mb, 64, 0, st>>>(p1, pl.p1_splits, B.N, nullptr, B.lse, B.lse_part, tmax ? B.minlse : nullptr);
    pf->end(st);
    pf->begin(VBGS_PROF_MERGE, st);
    launch_pdl(k_sum, 1, 1024, 0, st, B.lse_part, mb, B.scal + SC_SUM_LSE);
    pf->end(st);
    launches += 3;
    if (want_stats) {
        dim3 g2(pl.p2_tiles, pl.p2_splits);
        pf->begin(VBGS_PROF_PASS2, st);
        if (f64) k_pass2<double><<<g2, kThreads, 0, st>>>(B.X, B.lse, B.N, pl.nps, B.rec, B.K, B.part,
                                                          tmax, B.minlse, 256, kChunkK, pf->on ? pf->d_pairs : nullptr,
                                                          B.skip_nats);
        else     k_pass2<float><<<g2, kThreads, 0, st>>>(B.X, B.lse, B.N, pl.nps, B.rec32, B.K, B.part,
                                                         tmax, B.minlse, 256, kChunkK, pf->on ? pf->d_pairs : nullptr,
                                                         B.skip_nats);
        pf->end(st);
        pf->begin(VBGS_PROF_REDUCE, st);
        k_reduce_splits<<<(B.K + 127) / 128, 128, 0, st>>>(B.part, pl.p2_splits, B.K,
                                                          f64 ? nullptr : B.rec32, B.kperm, B.dS);
        pf->end(st);
        launches += 2;
    }
    return cudaGetLastError() == cudaSuccess ? launches : -1;
}


// ---------------------------------------------------------------------------
// E-step with no allocation (vbgs_estep_noalloc).
//
// Some callers cannot call cudaMalloc: a host runtime that owns all device
// memory through its own pool and forbids side allocations, a process held
// to a fixed device-memory budget, or a latency-critical loop that cannot
// afford an allocation (which may synchronise the device) in the middle of
// a frame.  For them this entry point takes its scratch memory (staged
// points, split partials, fixed-order sums, flags) from one file-scope
// device array of VBGS_NOALLOC_SCRATCH_BYTES instead of the context's
// buffers, and writes its results into buffers the caller passes.
//
// The array lives in the library's device image: every GPU that loads the
// library holds it until the process exits.  Its device address is looked up
// once per device (per CUDA context on it), by the first call made with that
// device current, and passed to the kernels as a pointer.  All
// calls share the one array and it keeps the last call's contents; calls
// that overlap on the GPU (different streams, or contexts on other host
// threads) race on it.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocDoubles = VBGS_NOALLOC_SCRATCH_BYTES / sizeof(double);
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

// The scratch array's device address per CUDA context.  A module is loaded
// into each context that uses it, so the address belongs to the context, not
// to the device ordinal: after cudaDeviceReset (or a primary context released
// and created again) the array may sit elsewhere, and the lookup is repeated
// for the new context.
constexpr int kMaxContexts = 64;
std::mutex g_noalloc_mu;
struct NoallocSlot { void *cuctx; double *addr; };
NoallocSlot g_noalloc_slots[kMaxContexts] = {};
int g_noalloc_used = 0;

typedef int (*CtxGetCurrentFn)(void **);

// Handle of the calling thread's current CUDA context (nullptr if none).
void *current_cuctx()
{
    static CtxGetCurrentFn fn = nullptr;
    static bool looked = false;
    if (!looked) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(f);
        cudaGetLastError();
        looked = true;
    }
    void *c = nullptr;
    if (!fn || fn(&c) != 0) return nullptr;
    return c;
}

// Device address of the scratch array in the current context (set-up on the
// first call per context, with its device current).  Returns nullptr on
// failure with *why set.
double *noalloc_scratch(const char **why)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
        cudaGetLastError();
        *why = "no current CUDA device";
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    void *cc = current_cuctx();
    for (int i = 0; cc && i < g_noalloc_used; i++)
        if (g_noalloc_slots[i].cuctx == cc) return g_noalloc_slots[i].addr;
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        *why = "cudaGetSymbolAddress of the scratch array failed";
        return nullptr;
    }
    // The lookup makes the device's primary context current if no context was.
    if (!cc) cc = current_cuctx();
    if (!cc) return static_cast<double *>(p);
    // A full table starts over: the oldest contexts are the likeliest gone.
    if (g_noalloc_used == kMaxContexts) g_noalloc_used = 0;
    g_noalloc_slots[g_noalloc_used++] = {cc, static_cast<double *>(p)};
    return static_cast<double *>(p);
}

bool on_device(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

__global__ void k_lse_subtract_psi(double *__restrict__ lse, int64_t N, const double *__restrict__ scal)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n < N) lse[n] -= scal[SC_PSI_AHAT];
}

int noalloc_fail(vbgs_ctx *ctx, int code, const std::string &msg)
{
    ctx->err = msg;
    return code;
}

} // namespace

} // namespace vbgs

extern "C" int vbgs_estep_noalloc(vbgs_ctx *ctx, const double *points, int64_t N, double *lse_out,
                                  double *dS_out)
{
    using namespace vbgs;
    if (!ctx) return VBGS_EINVAL;
    if (N < 0 || !dS_out || (N > 0 && (!points || !lse_out)))
        return noalloc_fail(ctx, VBGS_EINVAL, "vbgs_estep_noalloc: need N >= 0 and device points, lse, dS");
    // Host memory handed to a kernel would fault it: every array must be device memory.
    if ((N > 0 && (!on_device(points) || !on_device(lse_out))) || !on_device(dS_out))
        return noalloc_fail(ctx, VBGS_EINVAL, "vbgs_estep_noalloc: points, lse_out and dS_out must be device memory");
    const cudaStream_t st = ctx->stream;
    const int K = ctx->K;
    const char *why = "";
    double *base = noalloc_scratch(&why);
    if (!base) return noalloc_fail(ctx, VBGS_ECUDA, std::string("vbgs_estep_noalloc: ") + why);
    if (N == 0) {
        if (cudaMemsetAsync(dS_out, 0, sizeof(double) * (size_t)K * 28, st) != cudaSuccess)
            return noalloc_fail(ctx, VBGS_ECUDA, "vbgs_estep_noalloc: clearing dS failed");
        return VBGS_OK;
    }
    // Scratch layout (doubles): flags | (unused) | points N x 8 | split partials.
    auto round_up = [](size_t v) { return (v + 31) & ~size_t(31); };
    const size_t o_flags = 0;
    const int mb = (int)((N + 255) / 256);
    const size_t o_X = 32;
    const size_t o_part = o_X + round_up((size_t)N * VBGS_XS);
    const size_t avail = o_part < kNoAllocDoubles ? kNoAllocDoubles - o_part : 0;
    if (avail < (size_t)N * 2 || avail < (size_t)K * 28)
        return noalloc_fail(ctx, VBGS_EINVAL,
                            "vbgs_estep_noalloc: N = " + std::to_string(N) + ", K = " + std::to_string(K) +
                            " need more than the " + std::to_string(VBGS_NOALLOC_SCRATCH_BYTES) +
                            "-byte scratch array (32 + 8 N + max(2 N, 28 K) doubles)");
    int *flags = reinterpret_cast<int *>(base + o_flags);
    double *X = base + o_X;
    double *part = base + o_part;

    // Stage and validate the points; the flags must start at zero.
    Prof off;
    if (cudaMemsetAsync(flags, 0, sizeof(int) * FL_COUNT, st) != cudaSuccess ||
        launch_stage_points(points, N, X, flags, st, &off) < 0)
        return noalloc_fail(ctx, VBGS_ECUDA, "vbgs_estep_noalloc: staging failed");
    int bad = 0;
    if (cudaMemcpyAsync(&bad, flags + FL_BAD_POINT, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return noalloc_fail(ctx, VBGS_ECUDA, "vbgs_estep_noalloc: reading the staging flag failed");
    if (bad) return noalloc_fail(ctx, VBGS_EINVAL, "vbgs_estep_noalloc: non-finite point coordinate");

    // The launch plan of the context path, with split counts capped so the
    // partials fit the array.
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool f64 = ctx->precision == VBGS_FP64;
    Plan pl = f64 ? make_plan<kPPT64>(N, K, sms) : make_plan<kPPT32>(N, K, sms);
    const int s1max = (int)std::min<size_t>(avail / ((size_t)N * 2), (size_t)pl.p1_splits);
    pl.kps = (K + s1max - 1) / s1max;
    pl.p1_splits = (K + pl.kps - 1) / pl.kps;
    const int64_t s2max = (int64_t)std::min<size_t>(avail / ((size_t)K * 28), (size_t)pl.p2_splits);
    pl.nps = (N + s2max - 1) / s2max;
    pl.p2_splits = (int)((N + pl.nps - 1) / pl.nps);

    double2 *p1 = reinterpret_cast<double2 *>(part);
    dim3 g1(pl.p1_blocks, pl.p1_splits);
    if (f64) k_pass1<double, kPPT64><<<g1, kThreads, 0, st>>>(X, N, ctx->d_rec, K, pl.kps, p1, nullptr);
    else     k_pass1<float, kPPT32><<<g1, kThreads, 0, st>>>(X, N, ctx->d_rec32, K, pl.kps, p1, nullptr);
    k_merge<<<mb, 256, 0, st>>>(p1, pl.p1_splits, N, nullptr, lse_out, nullptr, nullptr);
    dim3 g2(pl.p2_tiles, pl.p2_splits);
    if (f64) k_pass2<double><<<g2, kThreads, 0, st>>>(X, lse_out, N, pl.nps, ctx->d_rec, K, part, nullptr, nullptr, 1, 1, nullptr,
                                                        0.f);
    else     k_pass2<float><<<g2, kThreads, 0, st>>>(X, lse_out, N, pl.nps, ctx->d_rec32, K, part, nullptr, nullptr, 1, 1, nullptr,
                                                       0.f);
    k_reduce_splits<<<(K + 127) / 128, 128, 0, st>>>(part, pl.p2_splits, K, f64 ? nullptr : ctx->d_rec32,
                                                    ctx->d_kperm, dS_out);
    k_lse_subtract_psi<<<mb, 256, 0, st>>>(lse_out, N, ctx->d_scal);
    if (cudaGetLastError() != cudaSuccess) return noalloc_fail(ctx, VBGS_ECUDA, "vbgs_estep_noalloc: launch failed");
    // memset + 2 staging kernels, pass 1, merge, pass 2, reduce, lse shift
    ctx->launches = 8;
    return VBGS_OK;
}
