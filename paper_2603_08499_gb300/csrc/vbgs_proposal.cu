// vbgs_proposal.cu -- learned candidate proposal for the E-step.
//
// With many components, nearly every (point, component) responsibility is
// negligible.  A small MLP over the point (x, y, z, r, g, b) proposes the 4
// most likely of G = 1024 component clusters (k-means of the posterior means,
// refreshed after every posterior update); the E-step then scores only the
// components of those clusters.  A certificate bounds, per point, the mass the
// other clusters can hold:
//   for a cluster g with constant cmax_g = max_k c_k, precision lower bound
//   lmin_g = min_k nu_k / tr(W_k^-1) <= lambda_min(nu_k W_k) and bounding box
//   of the means bbox_g, every logit of g is <= cmax_g - lmin_g/2 d^2(x, bbox_g),
//   so the missed mass is <= sum_{g not proposed} |g| 2^(ub_g - lse2_cand).
// Points whose bound exceeds 1e-3 (and a seeded 1% audit sample) run the exact
// E-step over all components; the audit also measures the true missed mass.
// The MLP is trained on the GPU by the kernels below (forward, backward, Adam)
// on the cluster masses q_ng = sum_{k in g} r_nk of the exact E-steps.
//
// All logits here are in log2 units (FP32 records: c and M scaled by log2 e).
#include "vbgs_internal.cuh"
#include <cub/device/device_radix_sort.cuh>
#include <algorithm>

namespace vbgs {

namespace {

constexpr int kG = VBGS_PROP_CLUSTERS;
constexpr int kTop = VBGS_PROP_TOP;
constexpr int kMaxCand = VBGS_PROP_MAXCAND;

__device__ __forceinline__ float ex2a(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// log2-unit logit of point x (FP32) under FP32 record r (c - 1/2 |M (x - m)|^2).
__device__ __forceinline__ float logit32(const float *__restrict__ r, const float x[6])
{
    float d[6];
#pragma unroll
    for (int i = 0; i < 6; i++) d[i] = x[i] - r[i];
    float q = 0.f;
#pragma unroll
    for (int i = 0; i < 6; i++) {
        float y = 0.f;
#pragma unroll
        for (int j = 0; j <= i; j++) y = fmaf(r[6 + tri(i, j)], d[j], y);
        q = fmaf(y, y, q);
    }
    return fmaf(-0.5f, q, r[27]);
}

// Certificate terms of a cluster (kCS floats): [0] cmax, [1] lp, [2..7] box
// low, [8..13] box high, [14] size, [15] lc, [16] la; log2 units.
constexpr int kCS = 20;

// Upper bound of every logit of a cluster at point x.
__device__ __forceinline__ float cluster_ub(const float *__restrict__ c, const float x[6])
{
    float dp = 0.f, dc = 0.f;
#pragma unroll
    for (int q = 0; q < 3; q++) {
        const float o = fmaxf(fmaxf(c[2 + q] - x[q], x[q] - c[8 + q]), 0.f);
        dp = fmaf(o, o, dp);
        const float oc = fmaxf(fmaxf(c[5 + q] - x[3 + q], x[3 + q] - c[11 + q]), 0.f);
        dc = fmaf(oc, oc, dc);
    }
    return c[0] - 0.5f * fmaxf(fmaxf(c[1] * dp, c[15] * dc), c[16] * (dp + dc));
}

// ---------------------------------------------------------------- k-means ----
// Clustering features of the components (at record positions): the mean
// with the colour scaled by csc.
__global__ void k_means_of_records(const float *__restrict__ rec32, int K, float csc, float *__restrict__ pts)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= K) return;
#pragma unroll
    for (int i = 0; i < 6; i++) pts[(size_t)p * 6 + i] = rec32[(size_t)p * VBGS_REC + i] * (i < 3 ? 1.f : csc);
}

// Nearest centroid (squared distance in FP32, ties to the lower index).
__global__ void __launch_bounds__(256) k_assign(const float *__restrict__ pts, int K, const float *__restrict__ cent,
                                                unsigned int *__restrict__ key, int *__restrict__ idx)
{
    __shared__ float sc[kG * 6];
    for (int i = threadIdx.x; i < kG * 6; i += blockDim.x) sc[i] = cent[i];
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= K) return;
    float x[6];
#pragma unroll
    for (int i = 0; i < 6; i++) x[i] = pts[(size_t)p * 6 + i];
    float best = INFINITY;
    int bg = 0;
    for (int g = 0; g < kG; g++) {
        float d2 = 0.f;
#pragma unroll
        for (int i = 0; i < 6; i++) {
            const float t = x[i] - sc[g * 6 + i];
            d2 = fmaf(t, t, d2);
        }
        if (d2 < best) { best = d2; bg = g; }
    }
    key[p] = (unsigned int)bg;
    idx[p] = p;
}

// Cluster boundaries of the sorted assignment (cstart[g] .. cstart[g+1]).
__global__ void k_cluster_bounds(const unsigned int *__restrict__ skey, int K, int *__restrict__ cstart)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > K) return;
    const int cur = i < K ? (int)skey[i] : kG;
    const int prev = i > 0 ? (int)skey[i - 1] : -1;
    for (int g = prev + 1; g <= cur; g++) cstart[g] = i;
}

// Centroid update: mean of the members in sorted order (deterministic); an
// empty cluster keeps its centroid.
__global__ void __launch_bounds__(128) k_centroids(const float *__restrict__ pts, const int *__restrict__ order,
                                                   const int *__restrict__ cstart, float *__restrict__ cent)
{
    __shared__ float sh[6][4];
    const int g = blockIdx.x, t = threadIdx.x;
    const int b = cstart[g], e = cstart[g + 1];
    float s[6] = {0, 0, 0, 0, 0, 0};
    for (int i = b + t; i < e; i += blockDim.x)
#pragma unroll
        for (int q = 0; q < 6; q++) s[q] += pts[(size_t)order[i] * 6 + q];
#pragma unroll
    for (int q = 0; q < 6; q++) {
        float v = s[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((t & 31) == 0) sh[q][t >> 5] = v;
    }
    __syncthreads();
    if (t < 6 && e > b) cent[g * 6 + t] = ((sh[t][0] + sh[t][1]) + (sh[t][2] + sh[t][3])) / (float)(e - b);
}

// Certificate terms of every cluster (layout of cluster_ub).  The FP32
// record holds the per-component bounds lp at [28], lc at [29], la at [30].
__global__ void __launch_bounds__(128) k_cluster_stats(const float *__restrict__ rec32,
                                                       const int *__restrict__ order, const int *__restrict__ cstart,
                                                       float *__restrict__ cstat)
{
    __shared__ float sh[16][4];
    const int g = blockIdx.x, t = threadIdx.x;
    const int b = cstart[g], e = cstart[g + 1];
    float cm = -INFINITY, lm = INFINITY, lc = INFINITY, la = INFINITY, lo[6], hi[6];
#pragma unroll
    for (int q = 0; q < 6; q++) { lo[q] = INFINITY; hi[q] = -INFINITY; }
    for (int i = b + t; i < e; i += blockDim.x) {
        const float *r = rec32 + (size_t)order[i] * VBGS_REC;
        cm = fmaxf(cm, r[27]);
        lm = fminf(lm, r[28]);
        lc = fminf(lc, r[29]);
        la = fminf(la, r[30]);
#pragma unroll
        for (int q = 0; q < 6; q++) { lo[q] = fminf(lo[q], r[q]); hi[q] = fmaxf(hi[q], r[q]); }
    }
    float v[16] = {cm, lm, lo[0], lo[1], lo[2], lo[3], lo[4], lo[5], hi[0], hi[1], hi[2], hi[3], hi[4], hi[5], lc, la};
#pragma unroll
    for (int q = 0; q < 16; q++) {
        float x = v[q];
        const bool mx = (q == 0) || (q >= 8 && q < 14);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float y = __shfl_xor_sync(0xffffffffu, x, o);
            x = mx ? fmaxf(x, y) : fminf(x, y);
        }
        if ((t & 31) == 0) sh[q][t >> 5] = x;
    }
    __syncthreads();
    if (t < 16) {
        const bool mx = (t == 0) || (t >= 8 && t < 14);
        float x = sh[t][0];
        for (int w = 1; w < 4; w++) x = mx ? fmaxf(x, sh[t][w]) : fminf(x, sh[t][w]);
        cstat[g * kCS + (t < 14 ? t : t + 1)] = x;   // lc -> [15], la -> [16]
    }
    if (t == 16) cstat[g * kCS + 14] = (float)(e - b);
}

// ------------------------------------------------------------------ MLP -----
// Generic tiled FP32 GEMM with strides: C[m][n] = act(sum_k A[m][k] B[k][n] + bias[n]) (+ C if accumulate).
// A(m,k) = A[m * sam + k * sak], B(k,n) = B[k * sbk + n * sbn], C row-major ldc.
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float *__restrict__ A, int sam, int sak,
                                              const float *__restrict__ B, int sbk, int sbn, float *__restrict__ C,
                                              int ldc, const float *__restrict__ bias, int relu, int accumulate)
{
    __shared__ float As[16][65];
    __shared__ float Bs[16][65];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float acc[4][4] = {};
    // tile loads walk the operand's unit-stride dimension across threads
    const bool a_kfast = (sak == 1), b_nfast = (sbn == 1);
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int i = threadIdx.x; i < 16 * 64; i += 256) {
            const int kk = a_kfast ? (i & 15) : (i >> 6), mm = a_kfast ? (i >> 4) : (i & 63);
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < M && k < K) ? A[(size_t)m * sam + (size_t)k * sak] : 0.f;
            const int kb = b_nfast ? (i >> 6) : (i & 15), nn = b_nfast ? (i & 63) : (i >> 4);
            const int n = n0 + nn, k2 = k0 + kb;
            Bs[kb][nn] = (n < N && k2 < K) ? B[(size_t)k2 * sbk + (size_t)n * sbn] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; kk++) {
            float a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; i++) { a[i] = As[kk][ty * 4 + i]; bb[i] = Bs[kk][tx * 4 + i]; }
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
            if (m < M && n < N) {
                float v = acc[i][j] + (bias ? bias[n] : 0.f);
                if (relu) v = fmaxf(v, 0.f);
                float *c = C + (size_t)m * ldc + n;
                *c = accumulate ? *c + v : v;
            }
        }
}

// Column sums (bias gradients): out[n] = sum_m X[m][n]; a block per 32
// columns, 8 row phases reduced in a fixed order.
__global__ void __launch_bounds__(256) k_colsum(const float *__restrict__ X, int M, int Nc, float *__restrict__ out)
{
    __shared__ float sh[8][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int n = blockIdx.x * 32 + tx;
    float s = 0.f;
    if (n < Nc)
        for (int m = ty; m < M; m += 8) s += X[(size_t)m * Nc + n];
    sh[ty][tx] = s;
    __syncthreads();
    if (ty == 0 && n < Nc) {
        float t = 0.f;
        for (int i = 0; i < 8; i++) t += sh[i][tx];
        out[n] = t;
    }
}

// dH *= (H > 0)
__global__ void k_relu_bwd(float *__restrict__ dH, const float *__restrict__ H, size_t n)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !(H[i] > 0.f)) dH[i] = 0.f;
}

// One warp per row of G logits: top-kTop indices (ties to the lower index)
// and, with labels q, the soft cross-entropy and its gradient (p - q) / B.
__global__ void __launch_bounds__(256) k_softmax_top(const float *__restrict__ Z, int B, const float *__restrict__ Q,
                                                     float *__restrict__ dZ, int *__restrict__ top,
                                                     float *__restrict__ loss_sum)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= B) return;
    const float *z = Z + (size_t)warp * kG;
    float v[kG / 32];
#pragma unroll
    for (int i = 0; i < kG / 32; i++) v[i] = z[i * 32 + lane];
    if (top) {
        float w[kG / 32];
#pragma unroll
        for (int i = 0; i < kG / 32; i++) w[i] = v[i];
        for (int t = 0; t < kTop; t++) {
            float bv = -INFINITY;
            int bi = 0x7fffffff;
#pragma unroll
            for (int i = 0; i < kG / 32; i++)
                if (w[i] > bv) { bv = w[i]; bi = i * 32 + lane; }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
            }
            if (lane == 0) top[(size_t)warp * kTop + t] = bi;
            if ((bi & 31) == lane) w[bi >> 5] = -INFINITY;
        }
    }
    if (Q) {
        float mx = -INFINITY;
#pragma unroll
        for (int i = 0; i < kG / 32; i++) mx = fmaxf(mx, v[i]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < kG / 32; i++) s += expf(v[i] - mx);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const float lse = mx + logf(s);
        const float *q = Q + (size_t)warp * kG;
        float l = 0.f;
#pragma unroll
        for (int i = 0; i < kG / 32; i++) {
            const float qq = q[i * 32 + lane];
            const float lp = v[i] - lse;
            l -= qq * lp;
            dZ[(size_t)warp * kG + i * 32 + lane] = (expf(lp) - qq) / (float)B;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
        if (lane == 0) atomicAdd(loss_sum, l);
    }
}

// Adam on FP32 master weights; wq = the BF16-rounded weights the GEMMs use.
__global__ void k_adam(float *__restrict__ w, float *__restrict__ wq, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, size_t n, float lr, float b1, float b2, float c1, float c2)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
    w[i] = wi;
    wq[i] = __bfloat162float(__float2bfloat16_rn(wi));
}

// Network inputs: positions mapped to [-1, 1] by the Morton box, colours to [-1, 1].
__global__ void k_mlp_inputs(const double *__restrict__ X, const int *__restrict__ rows, int64_t rstride, int64_t n,
                             BoxParams box, float *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t r = rows ? rows[i] : i * rstride;
    const double *x = X + r * VBGS_XS;
#pragma unroll
    for (int q = 0; q < 3; q++) out[i * 6 + q] = (float)((x[q] - box.lo[q]) * box.inv_ext[q] * 2.0 - 1.0);
#pragma unroll
    for (int q = 3; q < 6; q++) out[i * 6 + q] = (float)(x[q] * 2.0 - 1.0);
}

// ------------------------------------------------------- candidate E-step ----
// Per point: log2-sum-exp over the components of its candidate clusters and
// the certified bound of the mass outside them.  The candidates start as the
// network's top-kTop clusters; while the bound exceeds the threshold, the
// cluster with the largest bound term joins the candidates (its components
// are scored exactly, which also tightens every other term through the new
// lse), in rounds that add every cluster within 4x of the largest term, up to
// kMaxCand clusters.  exact[n] = 1 (bound still above the
// threshold: the point takes the exact E-step), 2 (seeded audit sample), 0.
// cand[n * kMaxCand + i]: candidate clusters, -1 padded.
// One warp per point.  Lanes split the members of a cluster when scoring it
// and split the clusters when evaluating the bound; (max, sum) pairs and the
// bound are combined across the warp.
__device__ __forceinline__ void warp_score_cluster(const float *__restrict__ rec32, const int *__restrict__ order,
                                                   int b, int e, const float x[6], int lane, float &mx, float &s)
{
    for (int i = b + lane; i < e; i += 32) {
        const float l = logit32(rec32 + (size_t)order[i] * VBGS_REC, x);
        if (l > mx) { s = s * ex2a(mx - l) + 1.f; mx = l; }
        else s += ex2a(l - mx);
    }
}

__device__ __forceinline__ float warp_l2(float mx, float s)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float om = __shfl_xor_sync(0xffffffffu, mx, o), os = __shfl_xor_sync(0xffffffffu, s, o);
        const float m = fmaxf(mx, om);
        s = (m == -INFINITY) ? 0.f : s * ex2a(mx - m) + os * ex2a(om - m);
        mx = m;
    }
    return mx + __log2f(s);
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__global__ void __launch_bounds__(256) k_cand_pass1(const double *__restrict__ X, int64_t N,
                                                    const float *__restrict__ rec32, const int *__restrict__ order,
                                                    const int *__restrict__ cstart, const float *__restrict__ cstat,
                                                    const int *__restrict__ top, float thresh, uint32_t audit_seed,
                                                    uint32_t audit_per_mille, double *__restrict__ lse_c,
                                                    float *__restrict__ bound, int *__restrict__ exact,
                                                    int *__restrict__ cand, unsigned long long *__restrict__ counters)
{
    extern __shared__ float scs[];   // kG x kCS cluster certificate terms (80 KB)
    for (int i = threadIdx.x; i < kG * kCS; i += blockDim.x) scs[i] = cstat[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t n = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (n >= N) return;
    float x[6];
#pragma unroll
    for (int i = 0; i < 6; i++) x[i] = (float)X[n * VBGS_XS + i];
    // lane l owns the membership bits of clusters 32 l .. 32 l + 31
    uint32_t mine = 0u;
    int nc = 0;
    float mx = -INFINITY, s = 0.f;
    unsigned long long pairs = 0;
    for (int t = 0; t < kTop; t++) {
        const int g = top[n * kTop + t];
        if ((g >> 5) == lane) mine |= 1u << (g & 31);
        if (lane == 0) cand[n * kMaxCand + nc] = g;
        nc++;
        pairs += (unsigned long long)(cstart[g + 1] - cstart[g]);
        warp_score_cluster(rec32, order, cstart[g], cstart[g + 1], x, lane, mx, s);
    }
    // bound term of the non-candidate clusters of this lane
    auto lane_terms = [&](float l2, float &sum, float &best) {
        sum = 0.f;
        best = 0.f;
        for (int j = 0; j < 32; j++) {
            const int g = lane * 32 + j;
            if (mine & (1u << j)) continue;
            const float *c = scs + g * kCS;
            if (c[14] == 0.f) continue;
            const float b = c[14] * ex2a(fminf(cluster_ub(c, x) - l2, 64.f));
            sum += b;
            best = fmaxf(best, b);
        }
    };
    float mm = 0.f;
    for (int round = 0; round < 8; round++) {
        const float l2 = warp_l2(mx, s);
        float ls, lb;
        lane_terms(l2, ls, lb);
        mm = warp_sum(ls);
        const float best = warp_max(lb);
        if (mm <= thresh || nc == kMaxCand) break;
        // add every cluster whose term is within 4x of the largest, in index
        // order, up to the free slots
        const float tau = fmaxf(0.25f * best, thresh * (1.f / 64.f));
        uint32_t add = 0u;
        for (int j = 0; j < 32; j++) {
            const int g = lane * 32 + j;
            if (mine & (1u << j)) continue;
            const float *c = scs + g * kCS;
            if (c[14] == 0.f) continue;
            if (c[14] * ex2a(fminf(cluster_ub(c, x) - l2, 64.f)) >= tau) add |= 1u << j;
        }
        for (int l = 0; l < 32 && nc < kMaxCand; l++) {
            uint32_t a = __shfl_sync(0xffffffffu, add, l);
            while (a && nc < kMaxCand) {
                const int j = __ffs(a) - 1;
                a &= a - 1;
                const int g = l * 32 + j;
                if (lane == l) mine |= 1u << j;
                if (lane == 0) cand[n * kMaxCand + nc] = g;
                nc++;
                pairs += (unsigned long long)(cstart[g + 1] - cstart[g]);
                warp_score_cluster(rec32, order, cstart[g], cstart[g + 1], x, lane, mx, s);
            }
        }
    }
    const float l2 = warp_l2(mx, s);
    {
        float ls, lb;
        lane_terms(l2, ls, lb);
        mm = warp_sum(ls);
    }
    if (lane == 0) {
        for (int i = nc; i < kMaxCand; i++) cand[n * kMaxCand + i] = -1;
        bound[n] = mm;
        // seeded audit sample: a hash of (seed, point index)
        uint32_t h = audit_seed ^ (uint32_t)(n * 0x9E3779B9u);
        h ^= h >> 16; h *= 0x7feb352du; h ^= h >> 15; h *= 0x846ca68bu; h ^= h >> 16;
        const bool audit = (h % 1000u) < audit_per_mille;
        const int ex = !(mm <= thresh) ? 1 : (audit ? 2 : 0);
        exact[n] = ex;
        lse_c[n] = (double)l2 * 0.6931471805599453;   // natural units
        atomicAdd(&counters[0], pairs);
        if (ex == 1) atomicAdd(&counters[1], 1ull);
        if (ex == 2) atomicAdd(&counters[2], 1ull);
        atomicAdd(&counters[3], (unsigned long long)(nc - kTop));
    }
}

// Gather the exact-E-step points (fallback and audit) into X_e (N x 8).
__global__ void k_gather_rows(const double *__restrict__ X, const int *__restrict__ rows, int64_t n,
                              double *__restrict__ Xe)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * VBGS_XS) return;
    Xe[i] = X[(int64_t)rows[i / VBGS_XS] * VBGS_XS + (i % VBGS_XS)];
}

// (cluster, point) keys of the proposal points' candidates, for the per-
// cluster point lists of pass 2; exact points and empty slots get the key kG
// (sorted last).
__global__ void k_cand_keys(const int *__restrict__ cand, const int *__restrict__ exact, int64_t N,
                            unsigned int *__restrict__ key, int *__restrict__ val)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * kMaxCand) return;
    const int64_t n = i / kMaxCand;
    key[i] = (exact[n] || cand[i] < 0) ? (unsigned int)kG : (unsigned int)cand[i];
    val[i] = (int)n;
}

// Candidate pass 2: one CTA per cluster, one thread per member component;
// the cluster's proposal points stream through shared memory and each thread
// accumulates r [1, d, upper(d d^T)] about its component's mean (FP32), then
// writes the moments shifted to raw (FP64) at the component's position.
__global__ void __launch_bounds__(128) k_cand_pass2(const double *__restrict__ X, const double *__restrict__ lse_c,
                                                    const float *__restrict__ rec32, const int *__restrict__ order,
                                                    const int *__restrict__ cstart, const int *__restrict__ pstart,
                                                    const int *__restrict__ plist, const int *__restrict__ kperm,
                                                    double *__restrict__ dS)
{
    __shared__ float sp[64][8];
    const int g = blockIdx.x;
    const int b = cstart[g], e = cstart[g + 1];
    const int pb = pstart[g], pe = pstart[g + 1];
    for (int m0 = b; m0 < e; m0 += blockDim.x) {
        const int mi = m0 + threadIdx.x;
        const bool valid = mi < e;
        const int pos = valid ? order[mi] : order[b];
        float r[28];
#pragma unroll
        for (int i = 0; i < 28; i++) r[i] = rec32[(size_t)pos * VBGS_REC + i];
        float acc[28];
#pragma unroll
        for (int f = 0; f < 28; f++) acc[f] = 0.f;
        for (int p0 = pb; p0 < pe; p0 += 64) {
            const int cnt = min(64, pe - p0);
            __syncthreads();
            for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
                const int n = plist[p0 + t];
#pragma unroll
                for (int q = 0; q < 6; q++) sp[t][q] = (float)X[(int64_t)n * VBGS_XS + q];
                sp[t][6] = (float)(lse_c[n] * 1.4426950408889634);
            }
            __syncthreads();
            for (int t = 0; t < cnt; t++) {
                float x[6];
#pragma unroll
                for (int q = 0; q < 6; q++) x[q] = sp[t][q];
                const float w = ex2a(logit32(r, x) - sp[t][6]);
                acc[0] += w;
                float d[6], wd[6];
#pragma unroll
                for (int q = 0; q < 6; q++) { d[q] = x[q] - r[q]; wd[q] = w * d[q]; acc[1 + q] += wd[q]; }
                int u = 7;
#pragma unroll
                for (int i = 0; i < 6; i++)
#pragma unroll
                    for (int j = i; j < 6; j++, u++) acc[u] = fmaf(wd[i], d[j], acc[u]);
            }
        }
        if (valid) {
            double s[28], a[6];
#pragma unroll
            for (int f = 0; f < 28; f++) s[f] = (double)acc[f];
#pragma unroll
            for (int i = 0; i < 6; i++) a[i] = (double)r[i];
            int u = 7;
#pragma unroll
            for (int i = 0; i < 6; i++)
#pragma unroll
                for (int j = i; j < 6; j++, u++) s[u] += a[i] * s[1 + j] + s[1 + i] * a[j] + s[0] * a[i] * a[j];
#pragma unroll
            for (int i = 0; i < 6; i++) s[1 + i] += s[0] * a[i];
            double *dst = dS + (size_t)kperm[pos] * 28;
#pragma unroll
            for (int f = 0; f < 28; f++) dst[f] += s[f];
        }
    }
}

// Per-cluster point-list boundaries from the sorted keys.
__global__ void k_list_bounds(const unsigned int *__restrict__ skey, int64_t n, int *__restrict__ pstart)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    const int cur = i < n ? (int)min(skey[i], (unsigned int)kG) : kG;
    const int prev = i > 0 ? (int)min(skey[i - 1], (unsigned int)kG) : -1;
    for (int g = prev + 1; g <= cur; g++) pstart[g] = (int)i;
}

// Labels of the exact points: q_ng = sum_{k in g} 2^(l_nk - lse2_n), over the
// clusters the certificate does not rule out (bound mass >= 2^-40).  One warp
// per point: lanes test the clusters, then share the scoring of each kept one.
__global__ void __launch_bounds__(256) k_labels(const double *__restrict__ Xe, const double *__restrict__ lse_e,
                                                int64_t rstride, int64_t ne, const float *__restrict__ rec32,
                                                const int *__restrict__ order, const int *__restrict__ cstart,
                                                const float *__restrict__ cstat, float *__restrict__ Q)
{
    const int lane = threadIdx.x & 31;
    const int64_t n = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (n >= ne) return;
    float x[6];
#pragma unroll
    for (int i = 0; i < 6; i++) x[i] = (float)Xe[n * rstride * VBGS_XS + i];
    const float l2 = (float)(lse_e[n * rstride] * 1.4426950408889634);
    float *q = Q + n * kG;
    for (int g0 = 0; g0 < kG; g0 += 32) {
        const int g = g0 + lane;
        const float *c = cstat + g * kCS;
        const bool keep = c[14] > 0.f && cluster_ub(c, x) - l2 > -40.f;
        if (!keep) q[g] = 0.f;
        uint32_t kb = __ballot_sync(0xffffffffu, keep);
        while (kb) {
            const int j = __ffs(kb) - 1;
            kb &= kb - 1;
            const int gg = g0 + j;
            float v = 0.f;
            for (int i = cstart[gg] + lane; i < cstart[gg + 1]; i += 32)
                v += ex2a(logit32(rec32 + (size_t)order[i] * VBGS_REC, x) - l2);
            v = warp_sum(v);
            if (lane == 0) q[gg] = v;
        }
    }
}

// lse of the frame: proposal points keep the candidate lse, exact points the
// exact one; fixed-order block sums.
__global__ void __launch_bounds__(256) k_lse_combine(double *__restrict__ lse_c, const double *__restrict__ lse_e,
                                                     const int *__restrict__ erows, int64_t ne,
                                                     float *__restrict__ audit_missed)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    const int n = erows[i];
    // true missed mass of the proposal on this point: 1 - exp(lse_cand - lse)
    audit_missed[i] = (float)(-expm1(lse_c[n] - lse_e[i]));
    lse_c[n] = lse_e[i];
}

__global__ void __launch_bounds__(256) k_sum_lse(const double *__restrict__ v, int64_t n, double *__restrict__ part)
{
    __shared__ double sh[8];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double x = i < n ? v[i] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; w++) t += sh[w];
        part[blockIdx.x] = t;
    }
}

__global__ void k_add(double *__restrict__ a, const double *__restrict__ b, size_t n)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] += b[i];
}

} // namespace

// ------------------------------------------------------------ launchers -----
bool g_prop_attr = false;
int prop_set_attributes()
{
    if (g_prop_attr) return 0;
    if (cudaFuncSetAttribute(k_cand_pass1, cudaFuncAttributeMaxDynamicSharedMemorySize, kG * kCS * (int)sizeof(float)) !=
        cudaSuccess)
        return -1;
    g_prop_attr = true;
    return 0;
}

int prop_launch_kmeans(const float *rec32, int K, float csc, float *pts, float *cent, SortBuffers &sb, int *order,
                       unsigned int *skey, int *cstart, int lloyd_iters, cudaStream_t st)
{
    k_means_of_records<<<(K + 255) / 256, 256, 0, st>>>(rec32, K, csc, pts);
    for (int it = 0; it <= lloyd_iters; it++) {
        k_assign<<<(K + 255) / 256, 256, 0, st>>>(pts, K, cent, sb.keys_in, sb.idx_in);
        size_t bytes = sb.temp_bytes;
        if (cub::DeviceRadixSort::SortPairs(sb.temp, bytes, sb.keys_in, skey, sb.idx_in, order, K, 0, 11, st) !=
            cudaSuccess)
            return -1;
        k_cluster_bounds<<<(K + 256) / 256, 256, 0, st>>>(skey, K, cstart);
        if (it < lloyd_iters) k_centroids<<<kG, 128, 0, st>>>(pts, order, cstart, cent);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int prop_launch_cluster_stats(const float *rec32, const int *order, const int *cstart, float *cstat, cudaStream_t st)
{
    k_cluster_stats<<<kG, 128, 0, st>>>(rec32, order, cstart, cstat);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

void prop_gemm(int M, int N, int K, const float *A, int sam, int sak, const float *B, int sbk, int sbn, float *C,
               int ldc, const float *bias, bool relu, bool accumulate, cudaStream_t st)
{
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    k_gemm<<<grid, 256, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, relu ? 1 : 0, accumulate ? 1 : 0);
}

void prop_colsum(const float *X, int M, int Nc, float *out, cudaStream_t st)
{
    k_colsum<<<(Nc + 31) / 32, 256, 0, st>>>(X, M, Nc, out);
}

void prop_relu_bwd(float *dH, const float *H, size_t n, cudaStream_t st)
{
    k_relu_bwd<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(dH, H, n);
}

void prop_softmax_top(const float *Z, int B, const float *Q, float *dZ, int *top, float *loss_sum, cudaStream_t st)
{
    k_softmax_top<<<(B * 32 + 255) / 256, 256, 0, st>>>(Z, B, Q, dZ, top, loss_sum);
}

void prop_adam(float *w, float *wq, float *m, float *v, const float *g, size_t n, float lr, int step, cudaStream_t st)
{
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w, wq, m, v, g, n, lr, b1, b2, c1, c2);
}

void prop_inputs(const double *X, const int *rows, int64_t rstride, int64_t n, const BoxParams &box, float *out,
                 cudaStream_t st)
{
    if (n > 0) k_mlp_inputs<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(X, rows, rstride, n, box, out);
}

int prop_cand_pass1(const double *X, int64_t N, const float *rec32, const int *order, const int *cstart,
                    const float *cstat, const int *top, float thresh, uint32_t seed, uint32_t audit_per_mille,
                    double *lse_c, float *bound, int *exact, int *cand, unsigned long long *counters, cudaStream_t st)
{
    const size_t smem = (size_t)kG * kCS * sizeof(float);
    if (prop_set_attributes()) return -1;
    k_cand_pass1<<<(unsigned)((N * 32 + 255) / 256), 256, smem, st>>>(X, N, rec32, order, cstart, cstat, top, thresh,
                                                                      seed, audit_per_mille, lse_c, bound, exact, cand,
                                                                      counters);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

void prop_gather_rows(const double *X, const int *rows, int64_t n, double *Xe, cudaStream_t st)
{
    if (n > 0) k_gather_rows<<<(unsigned)((n * VBGS_XS + 255) / 256), 256, 0, st>>>(X, rows, n, Xe);
}

int prop_cand_lists(const int *cand, const int *exact, int64_t N, SortBuffers &sb, unsigned int *skey, int *plist,
                    int *pstart, cudaStream_t st)
{
    const int64_t n = N * kMaxCand;
    k_cand_keys<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(cand, exact, N, sb.keys_in, sb.idx_in);
    size_t bytes = sb.temp_bytes;
    if (cub::DeviceRadixSort::SortPairs(sb.temp, bytes, sb.keys_in, skey, sb.idx_in, plist, (int)n, 0, 11, st) !=
        cudaSuccess)
        return -1;
    k_list_bounds<<<(unsigned)((n + 256) / 256), 256, 0, st>>>(skey, n, pstart);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

void prop_cand_pass2(const double *X, const double *lse_c, const float *rec32, const int *order, const int *cstart,
                     const int *pstart, const int *plist, const int *kperm, double *dS, cudaStream_t st)
{
    k_cand_pass2<<<kG, 128, 0, st>>>(X, lse_c, rec32, order, cstart, pstart, plist, kperm, dS);
}

void prop_labels(const double *Xe, const double *lse_e, int64_t rstride, int64_t ne, const float *rec32,
                 const int *order, const int *cstart, const float *cstat, float *Q, cudaStream_t st)
{
    if (ne > 0)
        k_labels<<<(unsigned)((ne * 32 + 255) / 256), 256, 0, st>>>(Xe, lse_e, rstride, ne, rec32, order, cstart,
                                                                     cstat, Q);
}

void prop_lse_combine(double *lse_c, const double *lse_e, const int *erows, int64_t ne, float *audit_missed,
                      cudaStream_t st)
{
    if (ne > 0) k_lse_combine<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(lse_c, lse_e, erows, ne, audit_missed);
}

void prop_sum_lse(const double *v, int64_t n, double *part, int *nparts, cudaStream_t st)
{
    const int nb = (int)((n + 255) / 256);
    *nparts = nb;
    if (nb > 0) k_sum_lse<<<nb, 256, 0, st>>>(v, n, part);
}

void prop_add(double *a, const double *b, size_t n, cudaStream_t st)
{
    k_add<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, b, n);
}

} // namespace vbgs

namespace vbgs {
namespace {

__global__ void k_init_centroids(const float *__restrict__ rec32, int K, float csc, float *__restrict__ cent)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= kG) return;
    const int p = (int)(((long long)g * K) / kG);
#pragma unroll
    for (int i = 0; i < 6; i++) cent[g * 6 + i] = rec32[(size_t)p * VBGS_REC + i] * (i < 3 ? 1.f : csc);
}

__global__ void __launch_bounds__(1024) k_sum_final(const double *__restrict__ part, int n, double *__restrict__ out)
{
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
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

// Exact rows first (stable): key 0 for exact points, 1 otherwise.
__global__ void k_exact_keys(const int *__restrict__ exact, int64_t N, unsigned int *__restrict__ key,
                             int *__restrict__ val)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    key[n] = exact[n] ? 0u : 1u;
    val[n] = (int)n;
}

} // namespace

void prop_init_centroids(const float *rec32, int K, float csc, float *cent, cudaStream_t st)
{
    k_init_centroids<<<(kG + 255) / 256, 256, 0, st>>>(rec32, K, csc, cent);
}

void prop_sum_final(const double *part, int n, double *out, cudaStream_t st)
{
    k_sum_final<<<1, 1024, 0, st>>>(part, n, out);
}

int prop_exact_rows(const int *exact, int64_t N, SortBuffers &sb, unsigned int *skey, int *erows, cudaStream_t st)
{
    k_exact_keys<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(exact, N, sb.keys_in, sb.idx_in);
    size_t bytes = sb.temp_bytes;
    if (cub::DeviceRadixSort::SortPairs(sb.temp, bytes, sb.keys_in, skey, sb.idx_in, erows, (int)N, 0, 1, st) !=
        cudaSuccess)
        return -1;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

} // namespace vbgs
