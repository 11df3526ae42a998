// vbgs_render.cu -- splat rendering of the fitted mixture and the PSNR of
// the paper's quality metric (Sec. 5.1, Setup: PSNR =
// 10 log10(255^2 / MSE) over all pixels and RGB channels on a 0..255 scale).
//
// The paper does not describe its renderer.  Every component that data has
// reached (accumulated count N_k >= 1: at least one point's worth of
// responsibility; the others hold only the prior and are left out) is a
// splat at its spatial posterior mean with the expected spatial covariance
// W_s^-1 / (nu - d - 1) of its Wishart posterior (d = 6 joint, 3 split), the
// colour posterior mean clamped to [0, 1] and opacity 0.99; elliptical
// weighted average projection (perspective Jacobian at the camera-space
// mean, +0.3 px^2 on the screen covariance's diagonal); front-to-back
// compositing at pixel centres in increasing camera depth, ties by component
// index: alpha = min(0.99, 0.99 exp(-q / 2)), q = d^T C^-1 d, contributions
// with alpha < 1/255 skipped, black background.
//
// GB300 layout of the work:
//   k_splat_prep   a thread per component: posterior (FP64, from S_past and
//                  the prior), camera transform, screen covariance and its
//                  inverse, the screen rectangle of 16 x 16
//                  pixel tiles that holds every pixel with alpha >= 1/255
//                  (q <= 2 ln(255 * 0.99): the ellipse's bounding box), a
//                  64-bit depth key.
//   depth rank     one stable CUB radix sort of the depth keys (FP64 depth
//                  bits, components in index order): each splat's rank in
//                  the global front-to-back order, ties by index.
//   k_emit         (tile << 32 | rank) keys, one per covered tile, at
//                  offsets from a CUB exclusive scan of the tile counts.
//   tile sort      CUB radix sort of those keys: every tile's splats
//                  contiguous and front to back.
//   k_raster       a CTA per tile (256 threads, a pixel each): batches of
//                  256 splats staged in shared memory, each pixel composites
//                  them (the quadratic form in FP64, alpha and the colour in
//                  FP32, one expm1 per splat and pixel); a pixel stops
//                  once its transmittance is below 1e-7 (what remains can
//                  change its colour by less than 1e-7), the CTA once all
//                  its pixels have.
//   k_mse_part, k_psnr  FP64 sum of squared differences (0..255 scale) and
//                  the PSNR, on the device.
// The work is splats x covered pixels of a few FP64 and FP32 operations and
// one exp each: no contraction to put on the tensor cores.
#include "vbgs_internal.cuh"
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>
#include <algorithm>

namespace vbgs {
namespace {

constexpr int kTile = 16;                   // tile edge in pixels
constexpr int kRT = kTile * kTile;          // threads per raster CTA
constexpr double kNear = 0.1;               // splats closer to the camera plane are left out
constexpr double kLowPass = 0.3;            // px^2 on the screen covariance's diagonal
constexpr float kOpacity = 0.99f;            // alpha = min(0.99, o e^(-q/2)) with o = 0.99: the cap never binds
constexpr float kOneMinusOpacity = 0.01f;    // 1 - o, rounded once (not 1 - 0.99f)
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTStop = 1e-7f;
constexpr double kMinCount = 1.0;           // components with fewer points' worth of data are not drawn

// A splat as the rasteriser reads it: centre and inverse screen covariance
// in FP64 -- the quadratic form of a thin splat seen edge-on cancels: its
// terms reach 1e3 where q <= 11 matters, so FP32 would move alpha by ~1e-5,
// and a pixel far along a long splat's major axis has a minor-axis offset
// that FP32 cannot resolve -- and the colour in FP32.  64 bytes.
struct __align__(16) Splat {
    double u, v, ca, cb, cc;
    float r, g, b, pad;
};
static_assert(sizeof(Splat) == 64, "splat record size");

struct Camera {
    double o[3], Rwc[9], f;
    int W, H, tiles_x, tiles_y;
};

// Per component: splat record, tile
// rectangle, tile count and depth key (all-ones when left out).
__global__ void k_splat_prep(const double *__restrict__ m0, const double *__restrict__ S, MstepParams P, int d, int K,
                             Camera cam, float4 *__restrict__ sp, int4 *__restrict__ rect, long long *__restrict__ cnt,
                             unsigned long long *__restrict__ zkey, int *__restrict__ zidx)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > K) return;
    if (k == K) {   // the scan's last element: its exclusive sum is the total
        cnt[K] = 0;
        return;
    }
    zidx[k] = k;
    zkey[k] = ~0ull;
    cnt[k] = 0;
    const double *s = S + (size_t)k * VBGS_F;
    const double *a0 = m0 + (size_t)k * 6;
    const double Nk = s[0], beta = P.beta0 + Nk, nu = P.nu0 + Nk;
    if (!(Nk >= kMinCount)) return;
    double m[6];
#pragma unroll
    for (int i = 0; i < 6; i++) m[i] = (P.beta0 * a0[i] + s[1 + i]) / beta;
    const double den = nu - (double)d - 1.0;
    if (!(den > 0.0)) return;
    double Sg[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = i; j < 3; j++) {
            const double w = P.W0inv[i * 6 + j] + s[upper_index(i, j)] + P.beta0 * a0[i] * a0[j] - beta * m[i] * m[j];
            Sg[i][j] = Sg[j][i] = w / den;
        }
    // camera space: xc = Rcw (mu - o), Rcw = Rwc^T
    double xc[3];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        double t = 0.0;
#pragma unroll
        for (int i = 0; i < 3; i++) t += cam.Rwc[i * 3 + j] * (m[i] - cam.o[i]);
        xc[j] = t;
    }
    const double z = xc[2];
    if (!(z > kNear)) return;
    const double u = cam.f * xc[0] / z + 0.5 * cam.W, v = cam.f * xc[1] / z + 0.5 * cam.H;
    // Sc = Rcw Sg Rcw^T; C = J Sc J^T + low-pass
    double Sc[3][3];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) {
            double t = 0.0;
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int j = 0; j < 3; j++) t += cam.Rwc[i * 3 + a] * Sg[i][j] * cam.Rwc[j * 3 + b];
            Sc[a][b] = t;
        }
    const double J[2][3] = {{cam.f / z, 0.0, -cam.f * xc[0] / (z * z)}, {0.0, cam.f / z, -cam.f * xc[1] / (z * z)}};
    double C[2][2];
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
        for (int b = 0; b < 2; b++) {
            double t = 0.0;
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int j = 0; j < 3; j++) t += J[a][i] * Sc[i][j] * J[b][j];
            C[a][b] = t + (a == b ? kLowPass : 0.0);
        }
    const double det = C[0][0] * C[1][1] - C[0][1] * C[1][0];
    if (!(det > 0.0) || !(C[0][0] > 0.0)) return;
    // pixels with alpha >= 1/255 satisfy q <= r2; the bounding box of that
    // ellipse, widened a little for the FP32 evaluation of q
    const double r2 = 2.0 * log(255.0 * (double)kOpacity);
    const double hx = sqrt(r2 * C[0][0]) * 1.0001 + 1e-3, hy = sqrt(r2 * C[1][1]) * 1.0001 + 1e-3;
    // pixel i (centre i + 1/2) with |i + 1/2 - u| <= hx
    const double fx0 = fmax(ceil(u - hx - 0.5), 0.0), fx1 = fmin(floor(u + hx - 0.5), (double)(cam.W - 1));
    const double fy0 = fmax(ceil(v - hy - 0.5), 0.0), fy1 = fmin(floor(v + hy - 0.5), (double)(cam.H - 1));
    if (!(fx0 <= fx1) || !(fy0 <= fy1)) return;
    const int tx0 = (int)fx0 / kTile, tx1 = (int)fx1 / kTile, ty0 = (int)fy0 / kTile, ty1 = (int)fy1 / kTile;
    rect[k] = make_int4(tx0, ty0, tx1, ty1);
    cnt[k] = (long long)(tx1 - tx0 + 1) * (ty1 - ty0 + 1);
    zkey[k] = (unsigned long long)__double_as_longlong(z);   // z > 0: the bits order as the values
    Splat &o = reinterpret_cast<Splat *>(sp)[k];
    o.u = u;
    o.v = v;
    o.ca = C[1][1] / det;
    o.cb = -C[0][1] / det;
    o.cc = C[0][0] / det;
    o.r = (float)fmin(fmax(m[3], 0.0), 1.0);
    o.g = (float)fmin(fmax(m[4], 0.0), 1.0);
    o.b = (float)fmin(fmax(m[5], 0.0), 1.0);
}

__global__ void k_rank(const int *__restrict__ sorted_idx, int K, int *__restrict__ rank)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < K) rank[sorted_idx[i]] = i;
}

__global__ void k_emit(const int4 *__restrict__ rect, const long long *__restrict__ cnt, const long long *__restrict__ off,
                       const int *__restrict__ rank, int K, int tiles_x, unsigned long long *__restrict__ key,
                       int *__restrict__ val)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K || cnt[k] == 0) return;
    const int4 r = rect[k];
    long long o = off[k];
    const unsigned long long rk = (unsigned long long)(unsigned)rank[k];
    for (int ty = r.y; ty <= r.w; ty++)
        for (int tx = r.x; tx <= r.z; tx++, o++) {
            key[o] = ((unsigned long long)(ty * tiles_x + tx) << 32) | rk;
            val[o] = k;
        }
}

__global__ void k_ranges(const unsigned long long *__restrict__ key, long long n, int2 *__restrict__ range)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int t = (int)(key[i] >> 32);
    if (i == 0 || (int)(key[i - 1] >> 32) != t) range[t].x = (int)i;
    if (i == n - 1 || (int)(key[i + 1] >> 32) != t) range[t].y = (int)(i + 1);
}

__global__ void __launch_bounds__(kRT) k_raster(const float4 *__restrict__ sp, const int *__restrict__ val,
                                                const int2 *__restrict__ range, int W, int H, int tiles_x,
                                                float *__restrict__ img)
{
    __shared__ Splat sh[kRT];
    const int tile = blockIdx.x, tid = threadIdx.x;
    const int px = (tile % tiles_x) * kTile + (tid % kTile), py = (tile / tiles_x) * kTile + tid / kTile;
    const bool inside = px < W && py < H;
    const double cx = (double)px + 0.5, cy = (double)py + 0.5;
    const int2 r = range[tile];
    float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f;
    bool done = !inside;
    for (int b = r.x; b < r.y; b += kRT) {
        if (__syncthreads_and(done)) break;
        const int i = b + tid;
        if (i < r.y) {
            const int k = val[i];
            sh[tid] = reinterpret_cast<const Splat *>(sp)[k];
        }
        __syncthreads();
        const int n = min(kRT, r.y - b);
        if (!done) {
            for (int j = 0; j < n; j++) {
                const Splat &a = sh[j];
                const double dx = cx - a.u, dy = cy - a.v;
                const float q = (float)fma(a.ca * dx, dx, fma(2.0 * a.cb * dx, dy, a.cc * dy * dy));
                // alpha = o e^(-q/2) <= 0.99 (the cap never binds at o = 0.99)
                // and 1 - alpha = (1 - o) - o (e^(-q/2) - 1) from expm1:
                // 1 - alpha of a nearly opaque splat is ~0.01, so an exp
                // accurate to a few units of 2^-24 relative to 1 would give it
                // a relative error ~100 times larger, and every splat behind
                // it would inherit that through the transmittance
                const float em = expm1f(-0.5f * q);
                const float al = fmaf(kOpacity, em, kOpacity);
                if (al < kAlphaMin) continue;
                const float w = T * al;
                cr = fmaf(w, a.r, cr);
                cg = fmaf(w, a.g, cg);
                cb = fmaf(w, a.b, cb);
                T *= fmaf(-kOpacity, em, kOneMinusOpacity);
                if (T < kTStop) {
                    done = true;
                    break;
                }
            }
        }
    }
    if (inside) {
        float *o = img + ((size_t)py * W + px) * 3;
        o[0] = cr;
        o[1] = cg;
        o[2] = cb;
    }
}

// Sum of squared differences on the 0..255 scale, per block of 256 values.
__global__ void __launch_bounds__(256) k_mse_part(const float *__restrict__ a, const float *__restrict__ b, size_t n,
                                                  double *__restrict__ part)
{
    __shared__ double sh[8];
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (i < n) {
        const double d = 255.0 * ((double)a[i] - (double)b[i]);
        v = d * d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; w++) t += sh[w];
        part[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024) k_psnr(const double *__restrict__ part, int nb, size_t n, double *__restrict__ out)
{
    __shared__ double sh[32];
    double v = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) v += part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += sh[w];
        const double mse = t / (double)n;
        out[0] = mse;
        out[1] = mse > 0.0 ? 10.0 * log10(255.0 * 255.0 / mse) : INFINITY;
    }
}

template <typename T>
cudaError_t grow(T **p, size_t &cap, size_t n)
{
    if (n <= cap && *p) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc((void **)p, std::max<size_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess) cap = n;
    return e;
}

} // namespace

void render_free(RenderBuffers &B)
{
    void *ptrs[] = {B.sp, B.rect, B.cnt, B.off, B.zkey, B.zkey_s, B.zidx, B.zidx_s, B.rank, B.ekey, B.ekey_s,
                    B.eval, B.eval_s, B.range, B.img, B.ref, B.part, B.out, B.temp};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    B = RenderBuffers{};
}

int render_frame(const double *m0, const double *S, const MstepParams &P, int d, int K, const double *camera,
                 int W, int H, RenderBuffers &B, float *image, const float *ref, double *psnr, double *device_ms,
                 cudaStream_t st, std::string &why)
{
#define RCU(call)                                               \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) {                                \
            why = std::string(#call) + ": " + cudaGetErrorString(e_); \
            return -1;                                          \
        }                                                       \
    } while (0)
    Camera cam;
    for (int i = 0; i < 3; i++) cam.o[i] = camera[i];
    for (int i = 0; i < 9; i++) cam.Rwc[i] = camera[3 + i];
    cam.f = camera[12];
    cam.W = W;
    cam.H = H;
    cam.tiles_x = (W + kTile - 1) / kTile;
    cam.tiles_y = (H + kTile - 1) / kTile;
    const int ntiles = cam.tiles_x * cam.tiles_y;
    const size_t npx = (size_t)W * H * 3;
    int tile_bits = 1;
    while ((1 << tile_bits) < ntiles) tile_bits++;

    RCU(grow(&B.sp, B.cap_sp, (size_t)K * 4));
    RCU(grow(&B.rect, B.cap_rect, (size_t)K));
    RCU(grow(&B.cnt, B.cap_cnt, (size_t)K + 1));
    RCU(grow(&B.off, B.cap_off, (size_t)K + 1));
    RCU(grow(&B.zkey, B.cap_zkey, (size_t)K));
    RCU(grow(&B.zkey_s, B.cap_zkey_s, (size_t)K));
    RCU(grow(&B.zidx, B.cap_zidx, (size_t)K));
    RCU(grow(&B.zidx_s, B.cap_zidx_s, (size_t)K));
    RCU(grow(&B.rank, B.cap_rank, (size_t)K));
    RCU(grow(&B.range, B.cap_range, (size_t)ntiles));
    RCU(grow(&B.img, B.cap_img, npx));
    RCU(grow(&B.ref, B.cap_ref, npx));
    RCU(grow(&B.part, B.cap_part, (npx + 255) / 256));
    RCU(grow(&B.out, B.cap_out, (size_t)2));

    cudaEvent_t ev[4] = {};
    for (auto &e : ev) RCU(cudaEventCreate(&e));
    auto destroy_events = [&]() {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
    };

    // 1. splats, depth ranks, tile counts and their offsets
    size_t t1 = 0, t2 = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, t1, B.zkey, B.zkey_s, B.zidx, B.zidx_s, K, 0, 64, st);
    cub::DeviceScan::ExclusiveSum(nullptr, t2, B.cnt, B.off, K + 1, st);
    size_t need = std::max(t1, t2);
    if (need > B.temp_bytes) {
        if (B.temp) cudaFree(B.temp);
        B.temp = nullptr;
        B.temp_bytes = 0;
        RCU(cudaMalloc(&B.temp, need));
        B.temp_bytes = need;
    }
    RCU(cudaEventRecord(ev[0], st));
    k_splat_prep<<<(K + 1 + 127) / 128, 128, 0, st>>>(m0, S, P, d, K, cam, B.sp, B.rect, B.cnt, B.zkey, B.zidx);
    size_t tb = B.temp_bytes;
    RCU(cub::DeviceRadixSort::SortPairs(B.temp, tb, B.zkey, B.zkey_s, B.zidx, B.zidx_s, K, 0, 64, st));
    k_rank<<<(K + 255) / 256, 256, 0, st>>>(B.zidx_s, K, B.rank);
    tb = B.temp_bytes;
    RCU(cub::DeviceScan::ExclusiveSum(B.temp, tb, B.cnt, B.off, K + 1, st));
    RCU(cudaEventRecord(ev[1], st));
    long long total = 0;
    RCU(cudaMemcpyAsync(&total, B.off + K, sizeof total, cudaMemcpyDeviceToHost, st));
    RCU(cudaStreamSynchronize(st));
    if (total < 0 || total > (long long)0x7fffffff) {
        destroy_events();
        why = "more than 2^31 (splat, tile) pairs";
        return -1;
    }
    // 2. tile keys, sorted; per-tile ranges; compositing; PSNR
    RCU(grow(&B.ekey, B.cap_ekey, (size_t)total));
    RCU(grow(&B.ekey_s, B.cap_ekey_s, (size_t)total));
    RCU(grow(&B.eval, B.cap_eval, (size_t)total));
    RCU(grow(&B.eval_s, B.cap_eval_s, (size_t)total));
    size_t t3 = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, t3, B.ekey, B.ekey_s, B.eval, B.eval_s, (int)std::max<long long>(total, 1),
                                    0, 32 + tile_bits, st);
    if (t3 > B.temp_bytes) {
        cudaFree(B.temp);
        B.temp = nullptr;
        B.temp_bytes = 0;
        RCU(cudaMalloc(&B.temp, t3));
        B.temp_bytes = t3;
    }
    if (ref) RCU(cudaMemcpyAsync(B.ref, ref, sizeof(float) * npx, cudaMemcpyHostToDevice, st));
    RCU(cudaMemsetAsync(B.range, 0, sizeof(int2) * ntiles, st));
    RCU(cudaEventRecord(ev[2], st));
    if (total > 0) {
        k_emit<<<(K + 127) / 128, 128, 0, st>>>(B.rect, B.cnt, B.off, B.rank, K, cam.tiles_x,
                                                B.ekey, B.eval);
        tb = B.temp_bytes;
        RCU(cub::DeviceRadixSort::SortPairs(B.temp, tb, B.ekey, B.ekey_s, B.eval, B.eval_s, (int)total, 0,
                                            32 + tile_bits, st));
        k_ranges<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(B.ekey_s, total, B.range);
    }
    k_raster<<<ntiles, kRT, 0, st>>>(B.sp, B.eval_s, B.range, W, H, cam.tiles_x, B.img);
    const int nb = (int)((npx + 255) / 256);
    if (ref) {
        k_mse_part<<<nb, 256, 0, st>>>(B.img, B.ref, npx, B.part);
        k_psnr<<<1, 1024, 0, st>>>(B.part, nb, npx, B.out);
    }
    RCU(cudaEventRecord(ev[3], st));
    RCU(cudaGetLastError());
    double out[2] = {0.0, 0.0};
    if (image) RCU(cudaMemcpyAsync(image, B.img, sizeof(float) * npx, cudaMemcpyDeviceToHost, st));
    if (ref) RCU(cudaMemcpyAsync(out, B.out, sizeof out, cudaMemcpyDeviceToHost, st));
    RCU(cudaStreamSynchronize(st));
    if (psnr) *psnr = out[1];
    if (device_ms) {
        float a = 0.f, b = 0.f;
        cudaEventElapsedTime(&a, ev[0], ev[1]);
        cudaEventElapsedTime(&b, ev[2], ev[3]);
        *device_ms = (double)a + (double)b;
    }
    destroy_events();
    return 0;
#undef RCU
}

} // namespace vbgs
