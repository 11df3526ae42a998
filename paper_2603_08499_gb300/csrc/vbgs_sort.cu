// vbgs_sort.cu -- spatial (Morton) order of points and components.
//
// The sums of Eq. 3 and the per-point log-sum-exp do not depend on the order
// of points or components, so the library is free to process both in a
// spatially coherent order: 30-bit Morton codes of the position (x, y, z)
// inside a fixed box, sorted with CUB's radix sort.  Neighbouring points and
// components then share tiles, which is what lets pass 2 skip tiles whose
// responsibilities are all negligible.  Only the top 16 bits of the codes
// are sorted (two radix passes instead of four): cells of 1/40 of the box per
// axis, far smaller than the region of a 128-wide tile; the sort is stable,
// so inside a cell the input order stays.
//   points:      pidx[i] = original index of the i-th point in Morton order
//   components:  kperm[p] = original index of the component at position p,
//                kinv[k] = position of component k; positions are ordered
//                by the Morton code of the posterior mean at frame start.
#include "vbgs_internal.cuh"
#include <cub/device/device_radix_sort.cuh>

namespace vbgs {

namespace {

constexpr int kSortLo = 14;   // lowest code bit sorted

__device__ __forceinline__ uint32_t spread10(uint32_t v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ uint32_t morton3(const BoxParams &b, double x, double y, double z)
{
    const double p[3] = {x, y, z};
    uint32_t q[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        double t = (p[i] - b.lo[i]) * b.inv_ext[i] * 1023.0;
        t = fmin(fmax(t, 0.0), 1023.0);
        q[i] = (uint32_t)t;
    }
    return (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
}

__global__ void k_point_codes(const double *__restrict__ X, int64_t N, BoxParams b, uint32_t *__restrict__ keys,
                              int *__restrict__ idx)
{
    pdl_wait();
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const double *x = X + n * VBGS_XS;
    keys[n] = morton3(b, x[0], x[1], x[2]);
    idx[n] = (int)n;
}

// Posterior mean of each component, (beta0 m0 + S1) / (beta0 + N_k), as its key.
__global__ void k_comp_codes(const double *__restrict__ m0, const double *__restrict__ Spast, int K,
                             double beta0, BoxParams b, uint32_t *__restrict__ keys, int *__restrict__ idx)
{
    pdl_wait();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const double *s = Spast + (size_t)k * 28;
    const double inv = 1.0 / (beta0 + s[0]);
    double m[3];
#pragma unroll
    for (int i = 0; i < 3; i++) m[i] = (beta0 * m0[(size_t)k * 6 + i] + s[1 + i]) * inv;
    keys[k] = morton3(b, m[0], m[1], m[2]);
    idx[k] = k;
}

__global__ void k_gather_points(const double *__restrict__ X, const int *__restrict__ pidx, int64_t N,
                                double *__restrict__ Xs)
{
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * 4) return;
    const int64_t n = i >> 2, q = i & 3;   // 4 x 16-byte pieces of a 64-byte row
    const double2 *src = reinterpret_cast<const double2 *>(X + (int64_t)pidx[n] * VBGS_XS);
    reinterpret_cast<double2 *>(Xs + n * VBGS_XS)[q] = src[q];
}

__global__ void k_invert(const int *__restrict__ kperm, int K, int *__restrict__ kinv)
{
    pdl_wait();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < K) kinv[kperm[p]] = p;
}

} // namespace

size_t sort_temp_bytes(int64_t n)
{
    size_t bytes = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, bytes, (uint32_t *)nullptr, (uint32_t *)nullptr, (int *)nullptr,
                                    (int *)nullptr, (int)std::max<int64_t>(n, 1), 0, 30);
    return bytes;
}

int launch_point_order(const double *X, int64_t N, const BoxParams &box, SortBuffers &sb, double *Xs,
                       int *pidx, cudaStream_t st, Prof *pf)
{
    if (N <= 0) return 0;
    pf->begin(VBGS_PROF_MISC, st);
    launch_pdl(k_point_codes, (unsigned)((N + 255) / 256), 256, 0, st, X, N, box, sb.keys_in, sb.idx_in);
    pf->end(st);
    size_t bytes = sb.temp_bytes;
    if (cub::DeviceRadixSort::SortPairs(sb.temp, bytes, sb.keys_in, sb.keys_out, sb.idx_in, pidx, (int)N, kSortLo, 30,
                                        st) != cudaSuccess)
        return -1;
    pf->begin(VBGS_PROF_MISC, st);
    launch_pdl(k_gather_points, (unsigned)((N * 4 + 255) / 256), 256, 0, st, X, pidx, N, Xs);
    pf->end(st);
    return cudaGetLastError() == cudaSuccess ? 4 : -1;
}

int launch_comp_order(const double *m0, const double *Spast, int K, double beta0, const BoxParams &box,
                      SortBuffers &sb, int *kperm, int *kinv, cudaStream_t st, Prof *pf)
{
    pf->begin(VBGS_PROF_MISC, st);
    launch_pdl(k_comp_codes, (K + 255) / 256, 256, 0, st, m0, Spast, K, beta0, box, sb.keys_in, sb.idx_in);
    pf->end(st);
    size_t bytes = sb.temp_bytes;
    if (cub::DeviceRadixSort::SortPairs(sb.temp, bytes, sb.keys_in, sb.keys_out, sb.idx_in, kperm, K, kSortLo, 30, st) !=
        cudaSuccess)
        return -1;
    pf->begin(VBGS_PROF_MISC, st);
    launch_pdl(k_invert, (K + 255) / 256, 256, 0, st, kperm, K, kinv);
    pf->end(st);
    return cudaGetLastError() == cudaSuccess ? 4 : -1;
}

} // namespace vbgs
