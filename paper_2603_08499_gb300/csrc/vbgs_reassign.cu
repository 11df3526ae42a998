// vbgs_reassign.cu -- the reassign step of Alg. 1 (run before fit in every
// frame; Sec. 2.1.2): n points sampled toward low per-point ELBO, the n
// least-used components, and the prior means of those components set to the
// sampled points.
//
//   points      key_n = g_n - lse_n / tau in caller order; the n largest keys
//               are a sample of n distinct points with probability
//               proportional to exp(-lse_n / tau) (Gumbel-top-k; g_n are
//               standard Gumbel variates the caller draws); ties go to the
//               lower index.
//   components  ascending count N_k of S_past, ties by the caller's key v_k
//               (when given), then by the lower index.
//   apply       m0[comp_i] = x[point_i], i < n.
//
// Both orders come from CUB's stable radix sort on 64-bit keys that order as
// the doubles they encode (sign bit set for non-negative values, every bit
// flipped for negative ones; -0 is first mapped to +0, so equal values tie).
// Sorting in caller order makes the sort's stability the tie rule.
#include "vbgs_internal.cuh"
#include <cub/device/device_radix_sort.cuh>

namespace vbgs {
namespace {

__device__ __forceinline__ unsigned long long ord64(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(__dadd_rn(v, 0.0));   // -0 -> +0
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// Point keys, complemented so that an ascending sort puts the largest key
// first.  lse: per-point lse in caller order without the shared
// -psi(sum alpha) term, psi at *psi; the key is g - (lse - psi) / tau with
// each operation rounded once.
__global__ void k_point_keys(const double *__restrict__ lse, int64_t N, const double *__restrict__ psi,
                             const double *__restrict__ g, double inv_tau, unsigned long long *__restrict__ keys,
                             int *__restrict__ idx)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const double l = __dsub_rn(lse[n], *psi);
    keys[n] = ~ord64(__dsub_rn(g[n], __dmul_rn(l, inv_tau)));
    idx[n] = (int)n;
}

// First component pass (only with a caller key): order by v_k.
__global__ void k_comp_tie_keys(const double *__restrict__ v, int K, unsigned long long *__restrict__ keys,
                                int *__restrict__ idx)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    keys[k] = ord64(v[k]);
    idx[k] = k;
}

// Second (or only) component pass: the counts N_k = S[k][0] of the sequence
// `order` (NULL: identity), sorted stably so that ties keep that sequence.
__global__ void k_comp_count_keys(const double *__restrict__ S, const int *__restrict__ order, int K,
                                  unsigned long long *__restrict__ keys, int *__restrict__ idx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K) return;
    const int k = order ? order[i] : i;
    keys[i] = ord64(S[(size_t)k * VBGS_F]);
    idx[i] = k;
}

// m0[comp_i] = x[point_i] (X: staged points, caller order, N x 8); rows and
// picks (points, then components) for the host.
__global__ void k_reassign_apply(const int *__restrict__ pts, const int *__restrict__ comps, int n,
                                 const double *__restrict__ X, double *__restrict__ m0, double *__restrict__ rows,
                                 int *__restrict__ picks)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * 6) return;
    const int i = t / 6, d = t - 6 * i;
    const double x = X[(size_t)pts[i] * VBGS_XS + d];
    m0[(size_t)comps[i] * 6 + d] = x;
    rows[t] = x;
    if (d == 0) {
        picks[i] = pts[i];
        picks[n + i] = comps[i];
    }
}

} // namespace

size_t reassign_temp_bytes(int64_t n)
{
    size_t bytes = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, bytes, (unsigned long long *)nullptr, (unsigned long long *)nullptr,
                                    (int *)nullptr, (int *)nullptr, (int)std::max<int64_t>(n, 1));
    return bytes;
}

int launch_reassign(const ReassignArgs &a, ReassignBuffers &rb, cudaStream_t st)
{
    const int64_t N = a.N;
    const int K = a.K, n = a.n;
    if (n <= 0 || n > N || n > K || N > rb.cap || K > rb.cap) return -1;
    size_t bytes;
    // points: keys in caller order, stable ascending sort of the complemented keys
    k_point_keys<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(a.lse, N, a.psi, rb.g, a.inv_tau, rb.k_in, rb.i_in);
    bytes = rb.temp_bytes;
    if (cub::DeviceRadixSort::SortPairs(rb.temp, bytes, rb.k_in, rb.k_out, rb.i_in, rb.pts, (int)N, 0, 64, st) !=
        cudaSuccess)
        return -1;
    // components: by the caller's key first (when given), then stably by N_k
    const int *order = nullptr;
    int launches = 2;
    if (a.have_v) {
        k_comp_tie_keys<<<(K + 255) / 256, 256, 0, st>>>(rb.v, K, rb.k_in, rb.i_in);
        bytes = rb.temp_bytes;
        if (cub::DeviceRadixSort::SortPairs(rb.temp, bytes, rb.k_in, rb.k_out, rb.i_in, rb.i_out, K, 0, 64, st) !=
            cudaSuccess)
            return -1;
        order = rb.i_out;
        launches += 2;
    }
    k_comp_count_keys<<<(K + 255) / 256, 256, 0, st>>>(a.S, order, K, rb.k_in, rb.i_in);
    bytes = rb.temp_bytes;
    if (cub::DeviceRadixSort::SortPairs(rb.temp, bytes, rb.k_in, rb.k_out, rb.i_in, rb.comps, K, 0, 64, st) !=
        cudaSuccess)
        return -1;
    k_reassign_apply<<<(n * 6 + 255) / 256, 256, 0, st>>>(rb.pts, rb.comps, n, a.X, a.m0, rb.rows, rb.picks);
    launches += 3;
    return cudaGetLastError() == cudaSuccess ? launches : -1;
}

} // namespace vbgs
