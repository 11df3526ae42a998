// vbgs_mlp_tc.cu -- the learned proposal's GEMMs on the tensor cores.
//
// C = act(A B^T + bias) (+ C) for the network 6 -> 128 -> 128 -> 1024 and
// its backward pass, with strided FP32 operands in global memory:
// A(m, k) = A[m * sam + k * sak] (M x K), B(n, k) = B[n * sbn + k * sbk]
// (N x K), C row-major (ldc).  The products run as tcgen05 kind::f16 MMAs
// with BF16 operands and FP32 accumulation in tensor memory.  An operand
// that is not already a BF16 value (activations, gradients) is split into
// hi = bf16(x) and lo = bf16(x - hi), and the product takes the terms
// hi*hi + lo*hi + hi*lo: about 16 significant bits per operand, so the layer
// outputs and gradients keep FP32-level accuracy; the weights are BF16
// values already (one term).
//
// A CTA computes a 128 x 128 tile of C over a range of K: 128 threads stage
// 32-wide K chunks of A and B (FP32 loads along each operand's unit-stride
// dimension, the hi/lo split, 16-byte stores into the K-major core-matrix
// layout) in two shared-memory stages, one thread issues the MMAs of a chunk
// and commits them to the stage's mbarrier, which the threads wait on before
// they overwrite the stage.  Long K (the weight gradients, K = batch) is split
// over gridDim.z CTAs whose partial tiles a second kernel adds in a fixed
// order (no atomics: the same sums on every run).  Ragged M, N and K are
// zero-filled on load and masked on store.  Waits are bounded: one that gives
// up sets the context's timeout flag, and the issuing thread still waits for
// its own MMAs before tensor memory is released.
#include "vbgs_internal.cuh"
#include "vbgs_tc.cuh"
#include <cuda_bf16.h>
#include <algorithm>

namespace vbgs {
namespace {

constexpr int kTM = 128;                  // rows of a C tile (MMA M)
constexpr int kTN = 128;                  // columns of a C tile (MMA N)
constexpr int kKC = 32;                   // K per staged chunk (two MMA K steps)
constexpr int kOpBytes = kTM * kKC * 2;   // one BF16 operand chunk: 8 KB
constexpr int kSBO = (kKC / 8) * 128;     // 8-row group stride of a chunk: 512 B
constexpr long long kGemmSpin = 4000000000LL;

struct __align__(1024) GemmSmem {
    unsigned char a[2][2][kOpBytes];      // [stage][hi, lo]
    unsigned char b[2][2][kOpBytes];
    unsigned long long bar[2];
    unsigned long long bar_final;
    unsigned int tmem_base;
};

__device__ __forceinline__ bool gemm_wait(unsigned long long *b, uint32_t parity, int *flags)
{
    if (mbar_try(b, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(b, parity))
        if (clock64() - t0 > kGemmSpin) {
            if (flags) atomicExch(&flags[FL_TIMEOUT], 1);
            return false;
        }
    return true;
}

// Row r of an operand chunk: kKC values starting at k0 (zero outside K or
// beyond the last row), split and stored in the core-matrix layout.
__device__ __forceinline__ void stage_row(const float *__restrict__ X, int rows, int K, int sr, int sk, int r,
                                          int k0, bool split, unsigned char *hi, unsigned char *lo)
{
    float v[kKC];
    if (r < rows) {
        const float *p = X + (size_t)r * sr;
        if (sk == 1 && k0 + kKC <= K && ((((uintptr_t)(p + k0)) & 15) == 0)) {
#pragma unroll
            for (int q = 0; q < kKC / 4; q++) {
                const float4 t = reinterpret_cast<const float4 *>(p + k0)[q];
                v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < kKC; q++) v[q] = (k0 + q < K) ? p[(size_t)(k0 + q) * sk] : 0.f;
        }
    } else {
#pragma unroll
        for (int q = 0; q < kKC; q++) v[q] = 0.f;
    }
    const int base = (r >> 3) * kSBO + (r & 7) * 16;
#pragma unroll
    for (int g = 0; g < kKC / 8; g++) {
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const float x0 = v[g * 8 + 2 * e], x1 = v[g * 8 + 2 * e + 1];
            const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
            h[e] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            if (split) {
                const __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
                const __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
                l[e] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
            }
        }
        *reinterpret_cast<uint4 *>(hi + base + g * 128) = make_uint4(h[0], h[1], h[2], h[3]);
        if (split) *reinterpret_cast<uint4 *>(lo + base + g * 128) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

__global__ void __launch_bounds__(128) k_gemm_tc(int M, int N, int K, int kchunk, const float *__restrict__ A,
                                                 int sam, int sak, int split_a, const float *__restrict__ B, int sbn,
                                                 int sbk, int split_b, float *__restrict__ C, int ldc,
                                                 const float *__restrict__ bias, int relu, int accumulate,
                                                 float *__restrict__ part, int *__restrict__ flags)
{
    extern __shared__ unsigned char smem_raw[];
    GemmSmem &S = *reinterpret_cast<GemmSmem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    const int nch = (ke - kb + kKC - 1) / kKC;
    if (tid == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        mbar_init(&S.bar_final, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&S.tmem_base)),
                     "r"(kTN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = S.tmem_base;
    constexpr uint32_t idesc = idesc_mn<true>(kTM, kTN);
    bool ok = true;
    int issued = 0;   // chunks whose MMAs thread 0 issued
    for (int c = 0; c < nch; c++) {
        const int s = c & 1;
        // the MMAs of chunk c - 2 read this stage: wait for their commit
        if (c >= 2) ok = __syncthreads_and(ok && gemm_wait(&S.bar[s], (uint32_t)(((c >> 1) - 1) & 1), flags));
        if (!ok) break;
        const int k0 = kb + c * kKC;
        stage_row(A + (size_t)m0 * sam, M - m0, ke, sam, sak, tid, k0, split_a != 0, S.a[s][0], S.a[s][1]);
        stage_row(B + (size_t)n0 * sbn, N - n0, ke, sbn, sbk, tid, k0, split_b != 0, S.b[s][0], S.b[s][1]);
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            fence_after();
            const uint32_t first = (c == 0) ? 0u : 1u;
#pragma unroll
            for (int t = 0; t < kKC / 16; t++) {
                const uint64_t ah = smem_desc_sbo(S.a[s][0] + 256 * t, kSBO), bh = smem_desc_sbo(S.b[s][0] + 256 * t, kSBO);
                mma(tmem, ah, bh, idesc, t == 0 ? first : 1u);
                if (split_a) mma(tmem, smem_desc_sbo(S.a[s][1] + 256 * t, kSBO), bh, idesc, 1u);
                if (split_b) mma(tmem, ah, smem_desc_sbo(S.b[s][1] + 256 * t, kSBO), idesc, 1u);
            }
            mma_commit(&S.bar[s]);
            issued = c + 1;
        }
    }
    // every MMA of this CTA complete (thread 0 committed them all; the final
    // commit tracks them), then the accumulator to registers
    if (tid == 0 && issued > 0) {
        mma_commit(&S.bar_final);
        if (!gemm_wait(&S.bar_final, 0u, flags)) ok = false;
    }
    ok = __syncthreads_and(ok);
    fence_after();
    if (ok) {
        const int m = m0 + warp * 32 + lane;
        float *prow = part ? part + ((size_t)blockIdx.z * M + (size_t)m) * N : nullptr;
#pragma unroll 1
        for (int cb = 0; cb < kTN; cb += 32) {
            uint32_t v[32];
            if (nch > 0) {
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, v);
                tmem_wait_ld();
            } else {
#pragma unroll
                for (int i = 0; i < 32; i++) v[i] = 0u;
            }
            if (m < M) {
#pragma unroll
                for (int i = 0; i < 32; i++) {
                    const int n = n0 + cb + i;
                    if (n >= N) break;
                    float x = __uint_as_float(v[i]);
                    if (prow) {
                        prow[n] = x;
                    } else {
                        if (bias) x += bias[n];
                        if (relu) x = fmaxf(x, 0.f);
                        float *cp = C + (size_t)m * ldc + n;
                        *cp = accumulate ? *cp + x : x;
                    }
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTN) : "memory");
    }
}

// Split-K: C = act(sum_z part[z] + bias) (+ C), the partials added in z order.
__global__ void k_gemm_tc_reduce(int M, int N, int nz, const float *__restrict__ part, float *__restrict__ C,
                                 int ldc, const float *__restrict__ bias, int relu, int accumulate)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)M * N) return;
    const int m = (int)(i / N), n = (int)(i % N);
    float x = 0.f;
    for (int z = 0; z < nz; z++) x += part[(size_t)z * M * N + i];
    if (bias) x += bias[n];
    if (relu) x = fmaxf(x, 0.f);
    float *cp = C + (size_t)m * ldc + n;
    *cp = accumulate ? *cp + x : x;
}

} // namespace

size_t mlp_gemm_part_floats(int M, int N, int K)
{
    const int tiles = ((M + kTM - 1) / kTM) * ((N + kTN - 1) / kTN);
    if (tiles >= 64 || K <= 4 * kKC) return 0;
    const int nz = std::min((K + 8 * kKC - 1) / (8 * kKC), std::max(1, 152 / tiles));
    return nz > 1 ? (size_t)nz * M * N : 0;
}

int mlp_gemm_tc(int M, int N, int K, const float *A, int sam, int sak, bool split_a, const float *B, int sbn,
                int sbk, bool split_b, float *C, int ldc, const float *bias, bool relu, bool accumulate, float *part,
                size_t part_floats, int *flags, cudaStream_t st)
{
    static bool attr = false;
    const size_t smem = sizeof(GemmSmem) + 1024;
    if (!attr) {
        if (cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return -1;
        attr = true;
    }
    if (M <= 0 || N <= 0) return 0;
    const int tm = (M + kTM - 1) / kTM, tn = (N + kTN - 1) / kTN;
    // split K over z when the grid is small and K long (the weight gradients)
    int nz = 1;
    if (tm * tn < 64 && K > 4 * kKC) nz = std::min((K + 8 * kKC - 1) / (8 * kKC), std::max(1, 152 / (tm * tn)));
    if (nz > 1 && (!part || part_floats < (size_t)nz * M * N)) nz = 1;
    int kchunk = (K + nz - 1) / nz;
    kchunk = (kchunk + kKC - 1) / kKC * kKC;
    nz = std::max(1, (K + kchunk - 1) / kchunk);
    dim3 grid(tn, tm, nz);
    k_gemm_tc<<<grid, 128, smem, st>>>(M, N, K, kchunk, A, sam, sak, split_a ? 1 : 0, B, sbn, sbk, split_b ? 1 : 0,
                                       C, ldc, bias, relu ? 1 : 0, accumulate ? 1 : 0, nz > 1 ? part : nullptr, flags);
    if (nz > 1) {
        const size_t n = (size_t)M * N;
        k_gemm_tc_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(M, N, nz, part, C, ldc, bias, relu ? 1 : 0,
                                                                     accumulate ? 1 : 0);
    }
    return cudaGetLastError() == cudaSuccess ? (nz > 1 ? 2 : 1) : -1;
}

} // namespace vbgs
