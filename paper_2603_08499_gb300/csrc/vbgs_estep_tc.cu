// vbgs_estep_tc.cu -- pass 1 of the E-step on the 5th-generation tensor cores.
//
// The expected log-likelihood of compute_elbo_delta (Alg. 1) is a quadratic
// form in the point, so for a block of components it is one GEMM:
//   l2_nk = phi(x_n') . C_k,   phi(x') = [1, x', upper(x' x'^T)] (28 -> 32),
// in log2 units, where x' = (x - o_j) / s_j is the point in the local frame of
// component tile j (o_j the mean of the tile's component means, s_j their
// per-axis spread) and C_k holds the constant, linear and quadratic
// coefficients of component k in that frame.  Local frames keep the terms of
// the expansion small next to the logit, so the cancellation stays within
// FP16 hi/lo operands (about 22 bits) and FP32 accumulation:
//   L = A_hi B_hi + A_hi B_lo + A_lo B_hi     (tcgen05.mma kind::f16, K = 32)
// with A = features of 128 points (one CTA's rows), B = coefficients of 128
// components, the 128 x 128 FP32 accumulator in tensor memory (TMEM).
//
// CTA = 160 threads.  Warps 0-3 (one thread per point row = TMEM lane) build
// the A tile of the next component tile in shared memory, then read the
// finished accumulator with tcgen05.ld and keep the online (max, sum of
// 2^(l - max)) of their row.  Warp 4 issues the coefficient-tile copies
// (cp.async.bulk, completion on an mbarrier) and the MMAs (one elected lane),
// and commits MMA completion to mbarriers.  A and D are double buffered,
// B has kStagesB stages.  Every wait is bounded: on timeout the kernel sets
// the context's timeout flag, stops issuing work, waits (bounded) for the
// copies and MMAs it issued, frees its TMEM and returns.
//
// Shared-memory operand layout (K-major, no swizzle): 8 x 8 fp16 core
// matrices of 128 contiguous bytes; element (row r, feature f) of a 128 x 32
// tile is at byte (r / 8) * 512 + (f / 8) * 128 + (r % 8) * 16 + (f % 8) * 2,
// i.e. leading-dimension (K) core-matrix stride 128 B and stride-dimension
// (8-row group) stride 512 B.  Coefficient tiles are built in global memory
// in exactly this layout so one bulk copy stages them.
#include "vbgs_internal.cuh"
#include "vbgs_tc.cuh"
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <algorithm>
#include <cmath>

namespace vbgs {

// Limit of the waits between warp roles (cycles); vbgs_set_wait_limit.
__device__ long long g_wait_limit = 4000000000LL;

namespace {

constexpr int kRows = 128;          // points per CTA tile (MMA M)
constexpr int kCols = 128;          // components per tile (MMA N)
constexpr int kFeat = 32;           // features (MMA K), 28 used
constexpr int kStagesB = 2;
constexpr int kDB = 1;              // pass-1 accumulator buffers in TMEM (128 columns each)
constexpr int kOperandBytes = kRows * kFeat * 2;          // 8 KB (hi or lo)
constexpr int kTileBytes = 2 * kOperandBytes;             // hi + lo
constexpr int kThreadsTC = 160;
constexpr int kTmemCols = kDB * kCols;
constexpr long long kSpinCycles = 4000000000LL;           // ~2 s at 2 GHz

struct __align__(1024) Smem {
    unsigned char A[2][kTileBytes];
    unsigned char B[kStagesB][kTileBytes];
    unsigned long long bar_bfull[kStagesB];
    unsigned long long bar_bfree[kStagesB];
    unsigned long long bar_afull[2];
    unsigned long long bar_mma[2];
    unsigned long long bar_dfree[2];
    unsigned long long bar_final;
    unsigned int tmem_base;
};

// Bounded wait on a barrier phase; false on timeout.  A normal wait (one
// warp role waiting for another) gives up after g_wait_limit cycles, or as
// soon as another thread of the grid has timed out; a drain wait (for copies
// and MMAs this thread issued, which complete on their own) keeps the full
// kSpinCycles, so that nothing is in flight when the shared memory and TMEM
// are released.
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, uint32_t parity, int *flags, bool drain = false)
{
    if (mbar_try(b, parity)) return true;
    const long long t0 = clock64();
    const long long limit = drain ? kSpinCycles : g_wait_limit;
    // the timeout flag (a global load) and the clock are looked at on every
    // eighth attempt only, so a wait that ends is noticed at the next try_wait
    for (unsigned it = 1;; it++) {
        if (mbar_try(b, parity)) return true;
        if ((it & 7u) != 0u) continue;
        if (!drain && *(volatile int *)&flags[FL_TIMEOUT]) return false;
        if (clock64() - t0 > limit) {
            atomicExch(&flags[FL_TIMEOUT], 1);
            return false;
        }
    }
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(su32(dst)),
                 "l"(src), "r"(bytes), "r"(su32(bar))
                 : "memory");
}

__device__ __forceinline__ uint64_t smem_desc(const void *p)
{
    const uint32_t a = su32(p);
    uint64_t d = (uint64_t)((a & 0x3FFFFu) >> 4);
    d |= (uint64_t)(128u >> 4) << 16;   // leading (K) core-matrix stride
    d |= (uint64_t)(512u >> 4) << 32;   // 8-row group stride
    d |= (uint64_t)1 << 46;             // descriptor version for tcgen05
    return d;                           // base offset 0, no swizzle
}

// kind::f16, FP32 accumulator, A and B K-major, M = 128, N = 128.
template <bool BF16>
__host__ __device__ constexpr uint32_t idesc_f16()
{
    return (1u << 4) | ((BF16 ? 1u : 0u) << 7) | ((BF16 ? 1u : 0u) << 10) | ((uint32_t)(kCols >> 3) << 17) |
           ((uint32_t)(kRows >> 4) << 24);
}


__device__ __forceinline__ float ex2f(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Paired FP32 arithmetic of sm_100 and later (two lanes of a 64-bit register,
// each rounded to nearest like the scalar instruction) and the three-input
// maximum: fewer instructions per logit in the pass-1 reduction, with the
// results of the scalar forms.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 fadd2(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float fmax3(float a, float b, float c)
{
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Double-float arithmetic: a value as an unevaluated FP32 sum h + l (about
// 48 significant bits), on the FP32 pipe.  Error-free transformations of
// Knuth (two-sum), Dekker (fast two-sum) and the FMA product.
struct dfl {
    float h, l;
};
__device__ __forceinline__ dfl df_fast_sum(float a, float b)   // |a| >= |b|
{
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ dfl df_two_sum(float a, float b)
{
    const float s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dfl df_add(dfl x, dfl y)
{
    const dfl s = df_two_sum(x.h, y.h);
    return df_fast_sum(s.h, s.l + (x.l + y.l));
}
__device__ __forceinline__ dfl df_mul(dfl x, dfl y)
{
    const float p = __fmul_rn(x.h, y.h);   // never contracted into a later add
    const float e = fmaf(x.h, y.l, fmaf(x.l, y.h, fmaf(x.h, y.h, -p)));
    return df_fast_sum(p, e);
}
__device__ __forceinline__ dfl df_mulf(dfl x, float f)
{
    const float p = __fmul_rn(x.h, f);
    return df_fast_sum(p, fmaf(x.l, f, fmaf(x.h, f, -p)));
}
// FP64 -> double-float
__device__ __forceinline__ dfl df_from(double v)
{
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}
// The same split from the bit pattern, without FP64 instructions: h = v with
// its significand cut to 24 bits (exact in FP32), l = the remaining 29 bits
// rounded to FP32, for |v| in [2^-74, 2^127]; zeros and FP64 subnormals give
// (+-0, +0): df_from's pair for a zero, and for a subnormal (which rounds to
// zero in FP32) the same up to the sign of a zero; other values take
// df_from.  Zeros are common: a component no data has reached keeps the
// prior's diagonal precision, 15 of its 21 Cholesky entries exactly zero.
__device__ __forceinline__ dfl df_from_bits(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7ff);
    const unsigned sgn = (unsigned)(b >> 63) << 31;
    if (ex == 0) return {__uint_as_float(sgn), 0.f};
    if (ex < 949 || ex > 1150) return df_from(v);
    const float h = __uint_as_float(sgn | ((unsigned)(ex - 1023 + 127) << 23) | (unsigned)((b >> 29) & 0x7fffffu));
    const float scale = __uint_as_float((unsigned)(ex - 1075 + 127) << 23);   // 2^(ex - 1075), a normal float
    const float l = __uint2float_rn((unsigned)(b & 0x1fffffffu)) * scale;
    return {h, sgn ? -l : l};
}
// FP32 -> FP64 without an FP64 instruction: the exponent rebiased and the
// significand widened, exact for zeros and normal numbers; subnormals,
// infinities and NaNs take the conversion instruction.
__device__ __forceinline__ double f2d_exact(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned ex = (b >> 23) & 0xffu;
    const unsigned long long sgn = (unsigned long long)(b & 0x80000000u) << 32;
    if ((b << 1) == 0u) return __longlong_as_double((long long)sgn);
    if (ex == 0u || ex == 0xffu) return (double)f;
    return __longlong_as_double((long long)(sgn | ((unsigned long long)(ex + 896u) << 52) |
                                            ((unsigned long long)(b & 0x7fffffu) << 29)));
}
// sqrt(log2 e) and log2 e as double-float pairs
constexpr float kS2h = 1.2011224031448364f, kS2l = 5.641613398665868e-09f;
constexpr float kL2Eh = 1.4426950216293335f, kL2El = 1.925963033500011e-08f;

// Byte offset of (row, feature) in a 128 x 32 K-major core-matrix operand.
__host__ __device__ constexpr int opnd_off(int r, int f) { return (r >> 3) * 512 + (f >> 3) * 128 + (r & 7) * 16 + (f & 7) * 2; }

template <bool BF16> struct H;
// Scalar conversions (coefficient tiles) and a packed hi/lo split of two
// floats: hi = round(a, b), lo = round((a, b) - hi), two values per cvt.
template <> struct H<false> {
    using T = __half;
    static __device__ __forceinline__ T from_f(float v) { return __float2half_rn(v); }
    static __device__ __forceinline__ float to_f(T v) { return __half2float(v); }
    static __device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo)
    {
        const __half2 h = __floats2half2_rn(a, b);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    }
};
template <> struct H<true> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ T from_f(float v) { return __float2bfloat16_rn(v); }
    static __device__ __forceinline__ float to_f(T v) { return __bfloat162float(v); }
    static __device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo)
    {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    }
};

// ---------------------------------------------------------------------------
// Coefficient tiles.  One CTA per component tile (128 threads = components at
// sorted positions).  In the tile's frame y = (x - o) * inv_s the log2 logit
// is c' - (y - mu)^T P (y - mu) / 2 with P = S Lambda2 S (S = diag(1/inv_s),
// Lambda2 = log2(e) nu W) and mu = (m - o) * inv_s, expanded as
// coef0 + coef1 . y + sum_{a<=b} C_ab y_a y_b and scaled by 2^-e_j (largest
// coefficient of the tile about 2^14) before the hi/lo split.
//
// Double-float arithmetic (FP32 pairs) instead of FP64, whose rate on this
// part is 1/64 of FP32: P from the record's M as FP32 pairs; then coef1 and
// coef0 from the matrix that the stored hi/lo pairs of C represent (Pr), so
// the three parts expand one quadratic form centred exactly at mu and no
// error grows with |mu|.  The record's FP64 values are split into pairs from
// their bit patterns, so the kernel issues no FP64 instruction.
// Header (32 floats): o_hi[6], o_lo[6] (zero), inv_s[6], outscale (2^e_j), pad.
// ---------------------------------------------------------------------------
template <bool BF16>
__device__ __forceinline__ void split_store(dfl v, unsigned char *hi, unsigned char *lo, int off, float &rep)
{
    using HT = typename H<BF16>::T;
    const HT h = H<BF16>::from_f(v.h);
    const HT l = H<BF16>::from_f((v.h - H<BF16>::to_f(h)) + v.l);
    *reinterpret_cast<HT *>(hi + off) = h;
    *reinterpret_cast<HT *>(lo + off) = l;
    rep = H<BF16>::to_f(h) + H<BF16>::to_f(l);
}

template <bool BF16>
__global__ void __launch_bounds__(128) k_coef_tiles(const double *__restrict__ rec, const float *__restrict__ rec32,
                                                    int K, unsigned char *__restrict__ tiles,
                                                    float *__restrict__ hdr, int *__restrict__ dirty, int epoch)
{
    pdl_wait();
    __shared__ float red[7][4];
    __shared__ float frame[12];   // origin o (6), inv_s (6)
    const int t = threadIdx.x, j = blockIdx.x, lane = t & 31, w = t >> 5;
    // a tile whose records were not rewritten since its last build is current;
    // dirty[ntiles + j]: the epoch of the tile's last build
    if (dirty) {
        if (dirty[j] == 0) return;
        __syncthreads();
        if (t == 0) {
            dirty[j] = 0;
            dirty[gridDim.x + j] = epoch;
        }
    }
    const int k = j * kCols + t;
    const bool valid = k < K;
    const size_t rk = (size_t)(valid ? k : K - 1) * VBGS_REC;
    const float *r32 = rec32 + rk;
    const double *r = rec + rk;
    float mf[6];
    dfl M[21];   // sqrt(log2 e) * M from the FP64 record, in double-float
#pragma unroll
    for (int i = 0; i < 6; i++) mf[i] = r32[i];
#pragma unroll
    for (int q = 0; q < 21; q++) M[q] = df_mul(df_from_bits(r[6 + q]), {kS2h, kS2l});
    const int nvalid = min(kCols, K - j * kCols);
    // frame origin: precision-weighted mean of the tile's means (weight
    // tr(nu W), proportional to |M|_F^2), so the tightest components sit
    // near the origin; any origin is exact, it only has to be stored
    float wk = 0.f;
    if (valid)
#pragma unroll
        for (int q = 0; q < 21; q++) wk = fmaf(M[q].h, M[q].h, wk);
#pragma unroll
    for (int i = 0; i < 7; i++) {
        float v = i < 6 ? wk * mf[i] : wk;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[i][w] = v;
    }
    __syncthreads();
    if (t < 6) {
        const float tw = (red[6][0] + red[6][1]) + (red[6][2] + red[6][3]);
        frame[t] = ((red[t][0] + red[t][1]) + (red[t][2] + red[t][3])) / tw;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 6; i++) {
        const float d = valid ? mf[i] - frame[i] : 0.f;
        float v = d * d;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[i][w] = v;
    }
    __syncthreads();
    if (t < 6) {
        const float sd = sqrtf(((red[t][0] + red[t][1]) + (red[t][2] + red[t][3])) / (float)nvalid);
        const float inv = 1.f / fmaxf(sd, 0.05f);
        hdr[(size_t)j * 32 + t] = frame[t];
        hdr[(size_t)j * 32 + 6 + t] = 0.f;
        hdr[(size_t)j * 32 + 12 + t] = inv;
        frame[6 + t] = inv;
    }
    __syncthreads();
    float o[6], inv[6], sa[6];
#pragma unroll
    for (int i = 0; i < 6; i++) {
        o[i] = frame[i];
        inv[i] = frame[6 + i];
        sa[i] = 1.f / inv[i];   // its rounding rescales the frame axis: exact for the form
    }
    // P = S M^T M S (M packed lower triangular: M_la != 0 for l >= a)
    dfl P[21];
#pragma unroll
    for (int a = 0; a < 6; a++)
#pragma unroll
        for (int b = a; b < 6; b++) {
            dfl v = df_mul(M[tri(b, a)], M[tri(b, b)]);
#pragma unroll
            for (int l = b + 1; l < 6; l++) v = df_add(v, df_mul(M[tri(l, a)], M[tri(l, b)]));
            P[tri(b, a)] = df_mulf(df_mulf(v, sa[a]), sa[b]);
        }
    // mu = (m - o) * inv_s
    dfl mu[6];
#pragma unroll
    for (int a = 0; a < 6; a++) mu[a] = df_mulf(df_add(df_from_bits(r[a]), {-o[a], 0.f}), inv[a]);
    // tile-wide largest coefficient (estimate) -> power-of-two scale
    float mx = 0.f;
    if (valid) {
        float c0 = 0.f;
#pragma unroll
        for (int a = 0; a < 6; a++) {
            float bl = 0.f;
#pragma unroll
            for (int b = 0; b < 6; b++) bl = fmaf(P[a >= b ? tri(a, b) : tri(b, a)].h, mu[b].h, bl);
            mx = fmaxf(mx, fabsf(bl));
            c0 = fmaf(mu[a].h, bl, c0);
        }
        mx = fmaxf(mx, fabsf(r32[27] - 0.5f * c0));
#pragma unroll
        for (int q = 0; q < 21; q++) mx = fmaxf(mx, fabsf(P[q].h));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (lane == 0) red[0][w] = mx;
    __syncthreads();
    mx = fmaxf(fmaxf(red[0][0], red[0][1]), fmaxf(red[0][2], red[0][3]));
    int e = 0;
    if (mx > 0.f) e = ilogbf(mx) + 1 - 14;   // 2^(e+13) <= mx < 2^(e+14)
    const float sc = ldexpf(1.f, -e), isc = ldexpf(1.f, e);
    if (t == 0) hdr[(size_t)j * 32 + 18] = isc;
    unsigned char *hi = tiles + (size_t)j * kTileBytes;
    unsigned char *lo = hi + kOperandBytes;
    // quadratic part: C_aa = -P_aa / 2, C_ab = -P_ab (a < b), scaled by a
    // power of two (exact), split; Pr: the matrix the stored pairs represent
    float Pr[21];
    {
        int u = 7;
#pragma unroll
        for (int a = 0; a < 6; a++)
#pragma unroll
            for (int b = a; b < 6; b++, u++) {
                const float f = valid ? (a == b ? -0.5f : -1.f) * sc : 0.f;
                const dfl pv = P[tri(b, a)];
                float rep;
                split_store<BF16>({pv.h * f, pv.l * f}, hi, lo, opnd_off(t, u), rep);
                Pr[tri(b, a)] = (a == b ? -2.f : -1.f) * isc * rep;
            }
    }
#pragma unroll
    for (int f = 28; f < kFeat; f++) {
        float rep;
        split_store<BF16>({0.f, 0.f}, hi, lo, opnd_off(t, f), rep);
    }
    // linear and constant parts: coef1 = Pr mu, coef0 = c' - mu . Pr mu / 2
    dfl quad = {0.f, 0.f};
#pragma unroll
    for (int a = 0; a < 6; a++) {
        dfl bl = df_mulf(mu[0], Pr[tri(a, 0)]);
#pragma unroll
        for (int b = 1; b < 6; b++) bl = df_add(bl, df_mulf(mu[b], Pr[a >= b ? tri(a, b) : tri(b, a)]));
        quad = df_add(quad, df_mul(mu[a], bl));
        const float f = valid ? sc : 0.f;   // padding columns are masked by pass 1
        float rep;
        split_store<BF16>({bl.h * f, bl.l * f}, hi, lo, opnd_off(t, 1 + a), rep);
    }
    const dfl c0 = df_add(df_mul(df_from_bits(r[27]), {kL2Eh, kL2El}), {-0.5f * quad.h, -0.5f * quad.l});
    {
        const float f = valid ? sc : 0.f;
        float rep;
        split_store<BF16>({c0.h * f, c0.l * f}, hi, lo, opnd_off(t, 0), rep);
    }
}

// ---------------------------------------------------------------------------
// Pass 1 on the tensor cores.  grid = work items (point tile, component
// tiles).  part[item * 128 + row] = (max in log2 units, sum of 2^(l - max)).
// tmax[(point tile * 4 + warp) * ntiles + tile]: largest logit (natural units)
// of each 32-point row block and 128-component tile.
// seed (nullable): the seed launch's partials; each row's running maximum
// starts at its seed maximum, and a 64-column batch whose largest logit lies
// more than `drop` (log2 units) below the running maximum in every row of the
// warp is not exponentiated.  With drop = log2 K + 25 the terms left out are
// at most K 2^-drop = 2^-25 of a row's sum over all components (the sum is at
// least its largest term, 1 in units of the final maximum): below FP32
// rounding of the sum.  Its tile maxima are still taken.  pairs (nullable):
// pairs[0] += pairs evaluated, pairs[1] += pairs whose exponential was taken.
// ---------------------------------------------------------------------------
template <bool BF16>
__global__ void __launch_bounds__(kThreadsTC, 3) k_pass1_tc(const float *__restrict__ Xhl, int64_t N, int K,
                                                            const unsigned char *__restrict__ tiles,
                                                            const float *__restrict__ hdr, int ntiles,
                                                            const int *__restrict__ list,
                                                            const int *__restrict__ item_tile,
                                                            const int *__restrict__ item_lo,
                                                            const int *__restrict__ item_hi,
                                                            const int *__restrict__ nitems,
                                                            float2 *__restrict__ part, float *__restrict__ tmax,
                                                            int *__restrict__ flags,
                                                            unsigned long long *__restrict__ pairs, uint32_t knobs,
                                                            const float2 *__restrict__ seed, float drop)
{
    pdl_wait();
    using HT = typename H<BF16>::T;
    extern __shared__ unsigned char smem_raw[];
    Smem &S = *reinterpret_cast<Smem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // this CTA's work item: point tile P, entries [lo, hi) of its component-tile
    // list (all tiles in order without a list); slots beyond the item count
    // leave before any TMEM or barrier
    const int item = blockIdx.x;
    if (item >= *nitems) return;
    const int P = item_tile[item];
    const int lo = item_lo[item];
    const int nt = item_hi[item] - lo;
    auto tile_at = [&](int jj) -> int { return list ? list[(size_t)P * ntiles + lo + jj] : lo + jj; };

    if (tid == 0) {
        for (int i = 0; i < kStagesB; i++) { mbar_init(&S.bar_bfull[i], 1); mbar_init(&S.bar_bfree[i], 1); }
        for (int i = 0; i < 2; i++) { mbar_init(&S.bar_afull[i], 128); mbar_init(&S.bar_mma[i], 1); mbar_init(&S.bar_dfree[i], 128); }
        mbar_init(&S.bar_final, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&S.tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = S.tmem_base;

    if (warp < 4) {
        // ---------------- feature builders + online log-sum-exp ----------------
        const int row = warp * 32 + lane;
        const int64_t n = (int64_t)P * kRows + row;
        const int64_t nn = n < N ? n : N - 1;
        float xh[6], xl[6];
#pragma unroll
        for (int i = 0; i < 6; i++) {
            xh[i] = Xhl[nn * 16 + i];
            xl[i] = Xhl[nn * 16 + 8 + i];
        }
        float mrun = seed && n < N ? seed[n].x : -INFINITY, srun = 0.f;
        unsigned long long ecols = 0;   // columns exponentiated by this warp (with the pair counters)
        bool ok = true;
        // frame header of the next tile to build (o_hi, o_lo, 1/s), prefetched one tile ahead
        float hn[18];
        auto load_hdr = [&](int jj) {
            if (jj < nt) {
                const float4 *h4 = reinterpret_cast<const float4 *>(hdr + (size_t)tile_at(jj) * 32);
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const float4 v = h4[q];
                    hn[4 * q] = v.x; hn[4 * q + 1] = v.y; hn[4 * q + 2] = v.z; hn[4 * q + 3] = v.w;
                }
                const float2 v = reinterpret_cast<const float2 *>(hdr + (size_t)tile_at(jj) * 32)[8];
                hn[16] = v.x; hn[17] = v.y;
            }
        };
        auto build_A = [&](int jj) {
            float h[18];
#pragma unroll
            for (int i = 0; i < 18; i++) h[i] = hn[i];
            load_hdr(jj + 1);
            float d[6];
#pragma unroll
            for (int i = 0; i < 6; i++) d[i] = ((xh[i] - h[i]) + (xl[i] - h[6 + i])) * h[12 + i];
            float f[kFeat];
            f[0] = 1.f;
#pragma unroll
            for (int i = 0; i < 6; i++) f[1 + i] = d[i];
            int u = 7;
#pragma unroll
            for (int a = 0; a < 6; a++)
#pragma unroll
                for (int b = a; b < 6; b++, u++) f[u] = d[a] * d[b];
#pragma unroll
            for (int i = 28; i < kFeat; i++) f[i] = 0.f;
            unsigned char *Ahi = S.A[jj & 1];
            unsigned char *Alo = Ahi + kOperandBytes;
#pragma unroll
            for (int c = 0; c < 4; c++) {
                uint32_t hw[4], lw[4];
#pragma unroll
                for (int e = 0; e < 4; e++) H<BF16>::split2(f[c * 8 + 2 * e], f[c * 8 + 2 * e + 1], hw[e], lw[e]);
                *reinterpret_cast<uint4 *>(Ahi + opnd_off(row, c * 8)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                *reinterpret_cast<uint4 *>(Alo + opnd_off(row, c * 8)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
            fence_async_smem();
            mbar_arrive(&S.bar_afull[jj & 1]);
        };
        load_hdr(0);
        if (nt > 0) build_A(0);
        for (int jj = 0; jj < nt && ok; jj++) {
            if (jj + 1 < nt) build_A(jj + 1);
            const int s = jj % kDB;
            const int tj = tile_at(jj);
            const float scale = hdr[(size_t)tj * 32 + 18];
            ok = __all_sync(0xffffffffu, mbar_wait(&S.bar_mma[s], (uint32_t)((jj / kDB) & 1), flags));
            if (!ok) break;
            fence_after();
            const int nvalid = min(kCols, K - tj * kCols);   // columns past K are padding
            float tmx = -INFINITY;
            const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(s * kCols);
#pragma unroll 1
            for (int c = 0; c < kCols; c += 64) {
                uint32_t v0[32], v1[32];
                tmem_ld32(tbase + c, v0);
                tmem_ld32(tbase + c + 32, v1);
                tmem_wait_ld();
                if (nvalid < kCols) {
#pragma unroll
                    for (int i = 0; i < 32; i++) {
                        if (c + i >= nvalid) v0[i] = 0xff800000u;        // -inf
                        if (c + 32 + i >= nvalid) v1[i] = 0xff800000u;
                    }
                }
                // max and sum over 64 values with 8 independent chains each;
                // three-input maxima, and the scaled exponent arguments and
                // the accumulators taken two at a time (each accumulator adds
                // the same values in the same order as one at a time)
                auto vf = [&](const uint32_t (&v)[32], int i) { return __uint_as_float(v[i]); };
                float mx8[8];
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    float m = fmax3(vf(v0, q), vf(v1, q), vf(v0, q + 8));
                    m = fmax3(m, vf(v1, q + 8), vf(v0, q + 16));
                    m = fmax3(m, vf(v1, q + 16), vf(v0, q + 24));
                    mx8[q] = fmaxf(m, vf(v1, q + 24));
                }
                float cm = fmax3(fmax3(mx8[0], mx8[1], mx8[2]), fmax3(mx8[3], mx8[4], mx8[5]), fmaxf(mx8[6], mx8[7]));
                cm *= scale;
                tmx = fmaxf(tmx, cm);
                if (seed && __all_sync(0xffffffffu, cm < mrun - drop)) continue;   // negligible in every row
                if (pairs) ecols += (unsigned long long)max(0, min(64, nvalid - c));
                if (cm > mrun) {
                    srun *= ex2f(mrun - cm);
                    mrun = cm;
                }
                const float2 sc2 = make_float2(scale, scale), nm2 = make_float2(-mrun, -mrun);
                float2 acc[4];   // acc[q] = (chain 2q, chain 2q + 1)
#pragma unroll
                for (int q = 0; q < 4; q++) acc[q] = make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < 32; i += 2) {
                    const float2 a = ffma2(make_float2(vf(v0, i), vf(v0, i + 1)), sc2, nm2);
                    const float2 b = ffma2(make_float2(vf(v1, i), vf(v1, i + 1)), sc2, nm2);
                    acc[(i & 7) >> 1] = fadd2(acc[(i & 7) >> 1], make_float2(ex2f(a.x), ex2f(a.y)));
                    acc[((i + 4) & 7) >> 1] = fadd2(acc[((i + 4) & 7) >> 1], make_float2(ex2f(b.x), ex2f(b.y)));
                }
                srun += ((acc[0].x + acc[0].y) + (acc[1].x + acc[1].y)) + ((acc[2].x + acc[2].y) + (acc[3].x + acc[3].y));
            }
            fence_before();
            mbar_arrive(&S.bar_dfree[s]);
            // largest logit of this 32-row block and component tile (natural units)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) tmx = fmaxf(tmx, __shfl_xor_sync(0xffffffffu, tmx, o));
            const int64_t rb = (int64_t)P * 4 + warp;
            if (lane == 0 && tmax && rb * 32 < N) tmax[rb * ntiles + tj] = tmx * 0.6931471805599453f;
        }
        if (n < N) part[(size_t)item * kRows + row] = make_float2(mrun, srun);   // log2 units
        if (pairs && tid == 0) {
            unsigned long long cols = 0;
            for (int jj = 0; jj < nt; jj++) cols += (unsigned long long)min(kCols, K - tile_at(jj) * kCols);
            atomicAdd(pairs, cols * (unsigned long long)min((int64_t)kRows, N - (int64_t)P * kRows));
        }
        // pairs[1]: the pairs whose exponential was taken
        const int64_t wrows = min((int64_t)32, N - ((int64_t)P * kRows + warp * 32));
        if (pairs && lane == 0 && wrows > 0) atomicAdd(pairs + 1, ecols * (unsigned long long)wrows);
    } else if (warp == 4 && lane == 0) {
        // ---------------- copy + MMA issuer ----------------
        constexpr uint32_t idesc = idesc_f16<BF16>();
        bool ok = true;
        int n_loads = 0, n_mma = 0;
        const int pre = min(nt, kStagesB - 1);
        for (int jj = 0; jj < pre; jj++) {
            mbar_expect_tx(&S.bar_bfull[jj], kTileBytes);
            bulk_g2s(S.B[jj], tiles + (size_t)tile_at(jj) * kTileBytes, kTileBytes, &S.bar_bfull[jj]);
            n_loads = jj + 1;
        }
        for (int jj = 0; jj < nt && ok; jj++) {
            const int s = jj & 1, ds = jj % kDB, sb = jj % kStagesB;
            ok = mbar_wait(&S.bar_bfull[sb], (uint32_t)((jj / kStagesB) & 1), flags) &&
                 mbar_wait(&S.bar_afull[s], (uint32_t)((jj >> 1) & 1), flags) &&
                 (jj < kDB || mbar_wait(&S.bar_dfree[ds], (uint32_t)(((jj / kDB) - 1) & 1), flags));
            if (!ok) break;
            fence_after();
            const uint32_t d = tmem + (uint32_t)(ds * kCols);
            const unsigned char *Ahi = S.A[s], *Alo = S.A[s] + kOperandBytes;
            const unsigned char *Bhi = S.B[sb], *Blo = S.B[sb] + kOperandBytes;
            // k-steps of 16 features: the descriptor start advances by two core matrices (256 B)
            mma(d, smem_desc(Ahi), smem_desc(Bhi), idesc, 0u);
            mma(d, smem_desc(Ahi + 256), smem_desc(Bhi + 256), idesc, 1u);
            if (!(knobs & VBGS_KNOB_P1_C_LO)) {      // coefficients' lo term
                mma(d, smem_desc(Ahi), smem_desc(Blo), idesc, 1u);
                mma(d, smem_desc(Ahi + 256), smem_desc(Blo + 256), idesc, 1u);
            }
            if (!(knobs & VBGS_KNOB_P1_PHI_LO)) {    // features' lo term
                mma(d, smem_desc(Alo), smem_desc(Bhi), idesc, 1u);
                mma(d, smem_desc(Alo + 256), smem_desc(Bhi + 256), idesc, 1u);
            }
            mma_commit(&S.bar_mma[ds]);
            mma_commit(&S.bar_bfree[sb]);
            n_mma = jj + 1;
            // refill the B stage that the previous tile's MMAs read
            const int nxt = jj + kStagesB - 1;
            if (nxt < nt) {
                const int sn = nxt % kStagesB;
                if (jj >= 1) {
                    ok = mbar_wait(&S.bar_bfree[sn], (uint32_t)(((jj - 1) / kStagesB) & 1), flags);
                    if (!ok) break;
                }
                mbar_expect_tx(&S.bar_bfull[sn], kTileBytes);
                bulk_g2s(S.B[sn], tiles + (size_t)tile_at(nxt) * kTileBytes, kTileBytes, &S.bar_bfull[sn]);
                n_loads = nxt + 1;
            }
        }
        // Drain before the shared memory and TMEM go away: the last phase of
        // every barrier a copy or a commit of this thread arrives on.
        for (int sb = 0; sb < kStagesB; sb++) {
            const int last_load = ((n_loads - 1 - sb) >= 0) ? sb + ((n_loads - 1 - sb) / kStagesB) * kStagesB : -1;
            if (last_load >= 0) mbar_wait(&S.bar_bfull[sb], (uint32_t)((last_load / kStagesB) & 1), flags, true);
            const int last_mma = ((n_mma - 1 - sb) >= 0) ? sb + ((n_mma - 1 - sb) / kStagesB) * kStagesB : -1;
            if (last_mma >= 0) mbar_wait(&S.bar_bfree[sb], (uint32_t)((last_mma / kStagesB) & 1), flags, true);
        }
        for (int s = 0; s < kDB; s++) {
            const int last = ((n_mma - 1 - s) >= 0) ? s + ((n_mma - 1 - s) / kDB) * kDB : -1;
            if (last >= 0) mbar_wait(&S.bar_mma[s], (uint32_t)((last / kDB) & 1), flags, true);
        }
        // a last commit tracks every MMA this thread issued: TMEM is idle after it
        if (n_mma > 0) {
            mma_commit(&S.bar_final);
            mbar_wait(&S.bar_final, 0u, flags, true);
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}


// ---------------------------------------------------------------------------
// Pass-1 tile lists.  For a point tile P (128 Morton-consecutive points, box
// B_P) and a component k, every logit is bounded by the smallest-eigenvalue
// bounds of the record (log2 units, floats 28-30: position Schur complement,
// colour Schur complement, full precision):
//   l_k(x) <= c_k - 1/2 max(lp d_p^2, lc d_c^2, la (d_p^2 + d_c^2)),
// with d_p, d_c the distances of m_k to the position and colour boxes of P.
// A lower bound LB_P of every point's lse is an exact FP32 log-sum over a
// subset of the components, less 1 + 1e-5 |lse| for its rounding.  Tile j
// is evaluated only if one of its components' bounds reaches LB_P less the
// skip threshold; the others hold only pairs with r below e^-threshold.
// ---------------------------------------------------------------------------

// Bounding box (lo[6], hi[6]) of each point tile.
__global__ void __launch_bounds__(128) k_p1_boxes(const double *__restrict__ X, int64_t N, float *__restrict__ boxes)
{
    pdl_wait();
    __shared__ float sbox[2][6][4];
    const int P = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int64_t n = (int64_t)P * kRows + t;
    const int64_t nn = n < N ? n : (int64_t)P * kRows;
#pragma unroll
    for (int i = 0; i < 6; i++) {
        float a = (float)X[nn * VBGS_XS + i], b = a;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a = fminf(a, __shfl_xor_sync(0xffffffffu, a, o));
            b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        if (lane == 0) { sbox[0][i][w] = a; sbox[1][i][w] = b; }
    }
    __syncthreads();
    if (t < 6) {
        boxes[(size_t)P * 12 + t] = fminf(fminf(sbox[0][t][0], sbox[0][t][1]), fminf(sbox[0][t][2], sbox[0][t][3]));
        boxes[(size_t)P * 12 + 6 + t] = fmaxf(fmaxf(sbox[1][t][0], sbox[1][t][1]), fmaxf(sbox[1][t][2], sbox[1][t][3]));
    }
}

// ub[P][j] for every point tile: a CTA per (component tile j, 128 point
// tiles), the tile's bound terms (m, c, lp, lc, la; 16-byte aligned rows for
// vector loads) in shared memory, one thread per point tile.  Branch and
// bound for the maximum: each group of 32 components has a summary (box of
// its means, largest c, smallest lp, lc, la) whose bound dominates every
// member's (each step is monotone, also in FP32); a group whose summary bound
// does not exceed the maximum found so far cannot raise it and is skipped.
// The result equals the maximum over all components.
__device__ __forceinline__ float p1_bound(const float *c, const float lo[6], const float hi[6])
{
    float dp = 0.f, dc = 0.f;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const float o = fmaxf(fmaxf(lo[i] - c[i], c[i] - hi[i]), 0.f);
        dp = fmaf(o, o, dp);
        const float oc = fmaxf(fmaxf(lo[3 + i] - c[3 + i], c[3 + i] - hi[3 + i]), 0.f);
        dc = fmaf(oc, oc, dc);
    }
    return c[6] - 0.5f * fmaxf(fmaxf(c[7] * dp, c[8] * dc), c[9] * (dp + dc));
}
// the same for a group summary g: means box (lo g[0..5], hi g[6..11]), g[12..15] = cmax, lpmin, lcmin, lamin
__device__ __forceinline__ float p1_group_bound(const float *g, const float lo[6], const float hi[6])
{
    float dp = 0.f, dc = 0.f;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const float o = fmaxf(fmaxf(lo[i] - g[6 + i], g[i] - hi[i]), 0.f);
        dp = fmaf(o, o, dp);
        const float oc = fmaxf(fmaxf(lo[3 + i] - g[9 + i], g[3 + i] - hi[3 + i]), 0.f);
        dc = fmaf(oc, oc, dc);
    }
    return g[12] - 0.5f * fmaxf(fmaxf(g[13] * dp, g[14] * dc), g[15] * (dp + dc));
}

// tile_epoch (nullable): bounds of tiles not rebuilt since epoch `since`
// (the last plan for the same points) are current and kept.
__global__ void __launch_bounds__(128) k_p1_ub(const float *__restrict__ boxes, int ptiles, int K, int ntiles,
                                               const float *__restrict__ rec32, float *__restrict__ ub,
                                               const int *__restrict__ tile_epoch, int since)
{
    pdl_wait();
    if (tile_epoch && tile_epoch[blockIdx.x] <= since) return;
    __shared__ __align__(16) float sc[kCols][12];
    __shared__ float sg[kCols / 32][16];
    const int j = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int k = j * kCols + t;
    const int nv = min(kCols, K - j * kCols);
    {
        const float *r = rec32 + (size_t)(k < K ? k : 0) * VBGS_REC;
        float v[16];
#pragma unroll
        for (int i = 0; i < 6; i++) sc[t][i] = r[i];
        sc[t][6] = r[27]; sc[t][7] = r[28]; sc[t][8] = r[29]; sc[t][9] = r[30];
        // group summary over the valid components of this warp's 32
        const bool valid = t < nv;
#pragma unroll
        for (int i = 0; i < 6; i++) {
            v[i] = valid ? r[i] : INFINITY;
            v[6 + i] = valid ? r[i] : -INFINITY;
        }
        v[12] = valid ? r[27] : -INFINITY;
#pragma unroll
        for (int i = 0; i < 3; i++) v[13 + i] = valid ? r[28 + i] : INFINITY;
#pragma unroll
        for (int i = 0; i < 16; i++) {
            const bool mx = i >= 6 && i <= 12;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ov = __shfl_xor_sync(0xffffffffu, v[i], o);
                v[i] = mx ? fmaxf(v[i], ov) : fminf(v[i], ov);
            }
        }
        if (lane < 16) {
            float x = v[0];
#pragma unroll
            for (int i = 1; i < 16; i++) x = lane == i ? v[i] : x;
            sg[w][lane] = x;
        }
    }
    __syncthreads();
    const int P = blockIdx.y * kCols + t;
    if (P < ptiles) {
        float lo[6], hi[6];
#pragma unroll
        for (int i = 0; i < 6; i++) { lo[i] = boxes[(size_t)P * 12 + i]; hi[i] = boxes[(size_t)P * 12 + 6 + i]; }
        static_assert(kCols / 32 == 4, "four component groups per tile");
        float gb[4];
        int g0 = 0;
        float gbest = -INFINITY;
#pragma unroll
        for (int g = 0; g < 4; g++) {
            gb[g] = p1_group_bound(sg[g], lo, hi);
            if (gb[g] > gbest) { gbest = gb[g]; g0 = g; }
        }
        float b = -INFINITY;
        // the group with the largest summary bound first, then the others
#pragma unroll
        for (int gi = 0; gi < kCols / 32; gi++) {
            const int g = gi == 0 ? g0 : (gi <= g0 ? gi - 1 : gi);
            const float bg = g == 0 ? gb[0] : g == 1 ? gb[1] : g == 2 ? gb[2] : gb[3];   // no local-memory index
            if (!(bg > b)) continue;
            const int q1 = min(nv, g * 32 + 32);
            for (int q = g * 32; q < q1; q++) {
                const float4 c0 = *reinterpret_cast<const float4 *>(&sc[q][0]);
                const float4 c1 = *reinterpret_cast<const float4 *>(&sc[q][4]);
                const float4 c2 = *reinterpret_cast<const float4 *>(&sc[q][8]);
                const float c[10] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w, c2.x, c2.y};
                b = fmaxf(b, p1_bound(c, lo, hi));
            }
        }
        ub[(size_t)P * ntiles + j] = b;
    }
}

// Work items: every tile's list cut into items of at most C consecutive
// entries, with C >= cmin chosen so that the items fit the partial buffer
// (tcap items): sum_j ceil(n_j / C) <= total / C + ntiles <= tcap.
// item_start[j] is the first item of tile j (exclusive scan); items are in
// tile order.  One block of blockDim.x threads (a multiple of 32, at most
// 1024) with scan[65] in shared memory; counts == nullptr: nchunks entries
// per tile.
__device__ void build_items(const int *__restrict__ counts, int ntiles, int64_t nchunks, int cmin, int tcap,
                            int *__restrict__ item_start, int *__restrict__ item_tile, int *__restrict__ item_lo,
                            int *__restrict__ item_hi, int *__restrict__ nitems, int *scan)
{
    __shared__ long long red[32];
    __shared__ int C_sh;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5, nt = blockDim.x, nw = nt >> 5;
    auto cnt = [&](int j) -> int { return counts ? __ldcg(counts + j) : (int)nchunks; };
    // each thread takes a contiguous run of tiles
    const int per = (ntiles + nt - 1) / nt, j0 = min(ntiles, t * per), j1 = min(ntiles, j0 + per);
    long long tot = 0;
    for (int j = j0; j < j1; j++) tot += cnt(j);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane == 0) red[w] = tot;
    __syncthreads();
    if (t == 0) {
        long long sum = 0;
        for (int i = 0; i < nw; i++) sum += red[i];
        const long long room = tcap > ntiles ? tcap - ntiles : 1;
        C_sh = (int)max((long long)cmin, (sum + room - 1) / room);
    }
    __syncthreads();
    const int C = C_sh;
    int mine = 0;   // items of this thread's tiles
    for (int j = j0; j < j1; j++) mine += (cnt(j) + C - 1) / C;
    // exclusive block scan: within the warp by shuffles, then the warp totals
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) scan[w] = incl;
    __syncthreads();
    if (w == 0) {
        int v = lane < nw ? scan[lane] : 0, iv = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, iv, o);
            if (lane >= o) iv += u;
        }
        if (lane < nw) scan[32 + lane] = iv - v;   // exclusive prefix of warp lane
        if (lane == nw - 1) scan[64] = iv;         // total
    }
    __syncthreads();
    int start = scan[32 + w] + incl - mine;
    for (int j = j0; j < j1; j++) {
        item_start[j] = start;
        const int c = cnt(j), nj = (c + C - 1) / C;
        for (int i = 0; i < nj; i++) {
            item_tile[start + i] = j;
            item_lo[start + i] = i * C;
            item_hi[start + i] = min(c, (i + 1) * C);
        }
        start += nj;
    }
    if (t == 0) {
        item_start[ntiles] = scan[64];
        *nitems = scan[64];
    }
}

// The work items of a pass, built by the last block of a plan kernel once
// every block has written its count: done counts the finished blocks (zero
// between plans: the last block resets it).
struct ItemsArgs {
    int cmin, tcap;
    int *item_start, *item_tile, *item_lo, *item_hi, *nitems;
    unsigned int *done;
    int *zero2;   // nullable: two ints set to zero for a later kernel of the stream
};
__device__ void items_by_last_block(const int *counts, int ntiles, int64_t nchunks, const ItemsArgs &A, int *scan)
{
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(A.done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    build_items(counts, ntiles, nchunks, A.cmin, A.tcap, A.item_start, A.item_tile, A.item_lo, A.item_hi, A.nitems,
                scan);
    if (threadIdx.x == 0) {
        *A.done = 0u;
        if (A.zero2) { A.zero2[0] = 0; A.zero2[1] = 0; }
    }
}

// Pass-1 plan of point tile P around a first pass-1 launch.  k_p1_ub: the
// largest bound of every component tile over P's box.  k_p1_seed: the seed
// tile (the largest ub, ties to the lower index), evaluated alone by the
// first pass-1 launch.  k_p1_plan: LB_P = the smallest over the tile's
// points of that exact log-sum over a subset of the components, less
// 1 + 1e-5 |lse|; the list holds the other tiles with ub >= LB_P - threshold,
// in increasing order.
constexpr int kPlanThreads = 256;
constexpr int kPlanWarps = kPlanThreads / 32;

// Writes the seed into list[P * ntiles] and the seed launch's work item P
// (point tile P, list entries [0, 1)); sets the point tile's pass-1 tile
// maxima to -inf (pass 1 writes the evaluated tiles).
__global__ void __launch_bounds__(kPlanThreads) k_p1_seed(int64_t N, int ntiles, int ptiles,
                                                          const float *__restrict__ ub, int *__restrict__ list,
                                                          int *__restrict__ sitem_tile, int *__restrict__ sitem_lo,
                                                          int *__restrict__ sitem_hi, int *__restrict__ snitems,
                                                          float *__restrict__ tmax)
{
    pdl_wait();
    const int P = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
    for (int i = t; i < 4 * ntiles; i += kPlanThreads) {
        const int64_t rb = (int64_t)P * 4 + i / ntiles;
        if (rb * 32 < N) tmax[rb * ntiles + i % ntiles] = -INFINITY;
    }
    __shared__ float red[kPlanWarps];
    __shared__ int redi[kPlanWarps];
    const float *u = ub + (size_t)P * ntiles;
    float bv = -INFINITY;
    int bj = 0x7fffffff;
    for (int j = t; j < ntiles; j += kPlanThreads)
        if (u[j] > bv) { bv = u[j]; bj = j; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
        if (ov > bv || (ov == bv && oj < bj)) { bv = ov; bj = oj; }
    }
    if (lane == 0) { red[w] = bv; redi[w] = bj; }
    __syncthreads();
    if (t == 0) {
        float v = -INFINITY;
        int jx = 0x7fffffff;
        for (int q = 0; q < kPlanWarps; q++)
            if (red[q] > v || (red[q] == v && redi[q] < jx)) { v = red[q]; jx = redi[q]; }
        list[(size_t)P * ntiles] = jx == 0x7fffffff ? 0 : jx;
        sitem_tile[P] = P;
        sitem_lo[P] = 0;
        sitem_hi[P] = 1;
        if (P == 0) *snitems = ptiles;
    }
}

// spart: the seed launch's partials (point tile P: rows P * 128 ..).
// The last block to finish also builds the main launch's work items
// (ItemsArgs; the count per point tile is its list's length).
__global__ void __launch_bounds__(kPlanThreads) k_p1_plan(int64_t N, int ntiles, const float2 *__restrict__ spart,
                                                          const float *__restrict__ ub, int *__restrict__ list,
                                                          int *__restrict__ counts, float skip_log2, ItemsArgs items)
{
    pdl_wait();
    const int P = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
    __shared__ float red[kPlanWarps];
    __shared__ int wsum[kPlanWarps];
    __shared__ int base_sh;
    __shared__ int scan[65];
    const float *u = ub + (size_t)P * ntiles;
    int *row = list + (size_t)P * ntiles;
    const int js = row[0];
    // LB: the seed tile's log-sums (log2 units), less 1 + 1e-5 |lse| for the
    // rounding of the partial and of the final merge
    float lb = INFINITY;
    if (t < kRows && (int64_t)P * kRows + t < N) {
        const float2 q = spart[(size_t)P * kRows + t];
        const float l = q.x + __log2f(q.y);
        lb = l - (1.f + 1e-5f * fabsf(l));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lb = fminf(lb, __shfl_xor_sync(0xffffffffu, lb, o));
    if (lane == 0) red[w] = lb;
    if (t == 0) base_sh = 0;
    __syncthreads();
    float LB = red[0];
    for (int q = 1; q < kPlanWarps; q++) LB = fminf(LB, red[q]);
    const float thr = LB - skip_log2;
    // ordered compaction; the reads of a chunk precede its writes, which land
    // at or before the entries read (row[0], the seed, is read above)
    for (int j0 = 0; j0 < ntiles; j0 += kPlanThreads) {
        const int j = j0 + t;
        const bool keep = j < ntiles && j != js && u[j] >= thr;
        const unsigned bb = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) wsum[w] = __popc(bb);
        __syncthreads();
        int off = base_sh;
        for (int i = 0; i < w; i++) off += wsum[i];
        off += __popc(bb & ((1u << lane) - 1u));
        if (keep) row[off] = j;
        __syncthreads();
        if (t == 0) {
            int tot = 0;
            for (int i = 0; i < kPlanWarps; i++) tot += wsum[i];
            base_sh += tot;
        }
        __syncthreads();
    }
    if (t == 0) counts[P] = base_sh;
    items_by_last_block(counts, (int)gridDim.x, 0, items, scan);
}

// ---------------------------------------------------------------------------
// Pass 2 on the tensor cores: the fused statistics contraction of Eq. 3.
// grid = (component tiles, N splits), 160 threads.  A CTA keeps its tile's
// coefficients (the pass-1 tile, A operand) in shared memory and walks the
// 64-point chunks of its split that the pass-1 bound does not rule out:
//   MMA1  D1[128 comps x 64 pts]  = C . phi'^T      (3 hi/lo products, K = 32)
//   epilogue (thread = component row): r = 2^(D1 * scale - lse2_n) -> P hi/lo
//   MMA2  D2[128 comps x 32 feats]  = P_hi phi'_hi + P_hi phi'_lo + P_lo phi'_hi
//         (K = 64 points)
// phi' are the points' features in the tile's frame, so D2 holds the tile-frame
// moments of one chunk; the epilogue adds each chunk's D2 into FP32 registers
// (round to nearest) and k_reduce_splits_tile shifts the sums to raw moments
// in FP64.  One fresh accumulator per chunk keeps the tensor core's FP32
// accumulation (not round-to-nearest) to 64 points: summed over a whole frame
// its bias is of the order of the prior scatter W0^-1 of a thin component.  The
// logits are those of pass 1 (same coefficient tile, same feature arithmetic),
// so the responsibilities of a point sum to one up to the hi/lo rounding of r.
// Operands (K-major, no swizzle, core matrices of 8 rows x 16 bytes):
//   B1 [64 pts  x 32 feats]: LBO 128, SBO 512       (4 KB each for hi, lo)
//   B2 [32 feats x 64 pts ]: LBO 128, SBO 1024      (4 KB each for hi, lo)
//   P  [128 comps x 64 pts]: LBO 128, SBO 1024      (16 KB each for hi, lo)
// TMEM: D1 double buffered at columns 0 / 64, D2 double buffered at 128 / 160.
// ---------------------------------------------------------------------------
constexpr int kChunk2 = 64;
constexpr int kB1Bytes = kChunk2 * kFeat * 2;       // 4 KB
constexpr int kB2Bytes = kFeat * kChunk2 * 2;       // 4 KB
constexpr int kPBytes = kCols * kChunk2 * 2;        // 16 KB

struct __align__(128) Smem2 {
    unsigned char A[kTileBytes];                    // coefficient tile (hi | lo)
    unsigned char B1[2][2 * kB1Bytes];              // hi | lo
    unsigned char B2[2][2 * kB2Bytes];              // hi | lo
    unsigned char P[2][2 * kPBytes];                // hi | lo
    float lse2[3][kChunk2];                         // three stages: a lagging warp may still read the last one
    unsigned long long bar_a, bar_b1full[2], bar_b2full[2], bar_d1full[2], bar_d1free[2], bar_pfull[2], bar_stfree[2],
        bar_d2, bar_final;
    unsigned int tmem_base;
};

__device__ __forceinline__ int b1_off(int pt, int f) { return (pt >> 3) * 512 + (f >> 3) * 128 + (pt & 7) * 16 + (f & 7) * 2; }
__device__ __forceinline__ int b2_off(int f, int pt) { return (f >> 3) * 1024 + (pt >> 3) * 128 + (f & 7) * 16 + (pt & 7) * 2; }
__device__ __forceinline__ int p_off(int m, int pt) { return (m >> 3) * 1024 + (pt >> 3) * 128 + (m & 7) * 16 + (pt & 7) * 2; }

// The pass-2 skip bound of a 64-point chunk against tile j (uniform per CTA).
__device__ __forceinline__ bool chunk_skipped(const float *tmax, const float *minlse, int64_t N, int ntiles, int j,
                                              int64_t c0, float skip_nats)
{
    if (!tmax) return false;
    const int64_t r0 = c0 / 32, r1 = (min(N, c0 + kChunk2) - 1) / 32;
    float b = -INFINITY, l = INFINITY;
    for (int64_t r = r0; r <= r1; r++) {
        b = fmaxf(b, tmax[r * ntiles + j]);
        l = fminf(l, minlse[r]);
    }
    return b - l < -skip_nats;
}


// Work list of pass 2: for every component tile, the 64-point chunks the
// pass-1 bound does not rule out, in increasing order (deterministic).
// One block per tile; counts[j] and list[j * nchunks + i].
// The last block to finish also builds the pass's work items (ItemsArgs).
__global__ void __launch_bounds__(256) k_p2_plan(const float *__restrict__ tmax, const float *__restrict__ minlse,
                                                 int64_t N, int ntiles, int *__restrict__ counts,
                                                 int *__restrict__ list, float skip_nats, ItemsArgs items)
{
    pdl_wait();
    __shared__ int wsum[8];
    __shared__ int base_sh;
    __shared__ int scan[65];
    const int j = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int64_t nchunks = (N + kChunk2 - 1) / kChunk2;
    if (t == 0) base_sh = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < nchunks; c0 += 256) {
        const int64_t c = c0 + t;
        const bool keep = c < nchunks && !chunk_skipped(tmax, minlse, N, ntiles, j, c * kChunk2, skip_nats);
        const unsigned b = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) wsum[w] = __popc(b);
        __syncthreads();
        int off = base_sh;
        for (int i = 0; i < w; i++) off += wsum[i];
        off += __popc(b & ((1u << lane) - 1u));
        if (keep) list[(size_t)j * nchunks + off] = (int)c;
        __syncthreads();
        if (t == 0) {
            int tot = 0;
            for (int i = 0; i < 8; i++) tot += wsum[i];
            base_sh += tot;
        }
        __syncthreads();
    }
    if (t == 0) counts[j] = base_sh;
    items_by_last_block(counts, ntiles, nchunks, items, scan);
}

constexpr int kItemCap = 2048;
// One block of 1024 threads (the passes without skipping).
// zero2 (nullable): two ints set to zero for a later kernel of the stream.
__global__ void __launch_bounds__(1024) k_p2_items(const int *__restrict__ counts, int ntiles, int64_t nchunks,
                                                   int cmin, int tcap, int *__restrict__ item_start,
                                                   int *__restrict__ item_tile, int *__restrict__ item_lo,
                                                   int *__restrict__ item_hi, int *__restrict__ nitems,
                                                   int *__restrict__ zero2)
{
    pdl_wait();
    __shared__ int scan[65];
    if (zero2 && threadIdx.x < 2) zero2[threadIdx.x] = 0;
    build_items(counts, ntiles, nchunks, cmin, tcap, item_start, item_tile, item_lo, item_hi, nitems, scan);
}

template <bool BF16>
__global__ void __launch_bounds__(kThreadsTC, 2) k_pass2_tc(const float *__restrict__ Xhl, const float *__restrict__ lse2f,
                                                            int64_t N, int K, const unsigned char *__restrict__ tiles,
                                                            const float *__restrict__ hdr, int ntiles,
                                                            const int *__restrict__ counts,
                                                            const int *__restrict__ list,
                                                            const int *__restrict__ item_tile,
                                                            const int *__restrict__ item_lo,
                                                            const int *__restrict__ item_hi,
                                                            const int *__restrict__ nitems,
                                                            const double *__restrict__ rec,
                                                            float *__restrict__ part, int *__restrict__ flags,
                                                            unsigned long long *__restrict__ pairs, uint32_t knobs)
{
    pdl_wait();
    using HT = typename H<BF16>::T;
    extern __shared__ unsigned char smem_raw[];
    Smem2 &S = *reinterpret_cast<Smem2 *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // this CTA's work item: list entries [ibeg, iend) of tile j (never empty);
    // CTAs beyond the item count leave before any TMEM or barrier
    const int item = blockIdx.x;
    if (item >= *nitems) return;
    const int j = item_tile[item];
    const int64_t nchunks = (N + kChunk2 - 1) / kChunk2;
    const int ibeg = item_lo[item], iend = item_hi[item];
    // list entry i -> chunk index
    auto chunk_at = [&](int i) -> int64_t { return counts ? (int64_t)list[(size_t)j * nchunks + i] : (int64_t)i; };
    const int64_t cbeg = ibeg, cend = iend;   // iterate over list positions

    if (tid == 0) {
        mbar_init(&S.bar_a, 1);
        mbar_init(&S.bar_d2, 1);
        mbar_init(&S.bar_final, 1);
        for (int i = 0; i < 2; i++) {
            mbar_init(&S.bar_b1full[i], 64); mbar_init(&S.bar_b2full[i], 64);
            mbar_init(&S.bar_d1full[i], 1); mbar_init(&S.bar_d1free[i], 128);
            mbar_init(&S.bar_pfull[i], 128); mbar_init(&S.bar_stfree[i], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&S.tmem_base)), "r"(256)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = S.tmem_base;
    const float *h = hdr + (size_t)j * 32;
    const float scale = h[18];

    // the list holds only chunks to evaluate: positions advance one by one
    auto next_chunk = [&](int64_t c) { return c; };

    if (warp < 4) {
        // ---------------- builders + responsibilities ----------------
        const float *hf = h;   // tile frame (header), read where used (uniform, cached)
        const int m = tid;                          // component row of the epilogue
        bool ok = true;
        // The next chunk's inputs, loaded one chunk ahead of their use: this
        // thread's point (FP32 hi/lo) and, for threads 0..63, its lse2.  The
        // chunk origin (its first point, which thread 0 loads too) is read
        // where it is used.
        float nx[12], nl = INFINITY;
        int64_t nc0 = 0;
        // list entry of the chunk after the one load_next(c) is called for,
        // read one call ahead
        int64_t c0_ahead = cbeg < cend ? chunk_at((int)cbeg) * kChunk2 : 0;
        auto load_next = [&](int64_t c) {
            nc0 = c0_ahead;
            if (c + 1 < cend) c0_ahead = chunk_at((int)(c + 1)) * kChunk2;
            const int64_t n = nc0 + (tid & 63);
            const float4 *xp = reinterpret_cast<const float4 *>(Xhl + (n < N ? n : N - 1) * 16);
            const float4 p0 = xp[0], p1 = xp[1], p2 = xp[2], p3 = xp[3];
            nx[0] = p0.x; nx[1] = p0.y; nx[2] = p0.z; nx[3] = p0.w; nx[4] = p1.x; nx[5] = p1.y;
            nx[6] = p2.x; nx[7] = p2.y; nx[8] = p2.z; nx[9] = p2.w; nx[10] = p3.x; nx[11] = p3.y;
            if (tid < 64) nl = n < N ? lse2f[n] : INFINITY;
        };
        auto build = [&](int st, int sl) {
            // threads 0..63 write B1 (point-major) and lse2, 64..127 write B2
            // (feature-major); each half arrives on its own barrier
            const int pt = tid & 63;
            float d[6];
            if (tid < 64) {
                // logits: the tile's frame, like the coefficients
#pragma unroll
                for (int i = 0; i < 6; i++) d[i] = ((nx[i] - hf[i]) + (nx[6 + i] - hf[6 + i])) * hf[12 + i];
            } else {
                // statistics: the chunk's frame, origin at its first point
                const float *xo = Xhl + nc0 * 16;
#pragma unroll
                for (int i = 0; i < 6; i++) d[i] = ((nx[i] - xo[i]) + (nx[6 + i] - xo[8 + i])) * hf[12 + i];
            }
            float f[kFeat];
            f[0] = 1.f;
#pragma unroll
            for (int i = 0; i < 6; i++) f[1 + i] = d[i];
            int u = 7;
#pragma unroll
            for (int a = 0; a < 6; a++)
#pragma unroll
                for (int b = a; b < 6; b++, u++) f[u] = d[a] * d[b];
#pragma unroll
            for (int i = 28; i < kFeat; i++) f[i] = 0.f;
            uint32_t hw[16], lw[16];
#pragma unroll
            for (int e = 0; e < 16; e++) H<BF16>::split2(f[2 * e], f[2 * e + 1], hw[e], lw[e]);
            if (tid < 64) {
                unsigned char *bh = S.B1[st], *bl = S.B1[st] + kB1Bytes;
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    *reinterpret_cast<uint4 *>(bh + b1_off(pt, 8 * q)) = make_uint4(hw[4 * q], hw[4 * q + 1], hw[4 * q + 2], hw[4 * q + 3]);
                    *reinterpret_cast<uint4 *>(bl + b1_off(pt, 8 * q)) = make_uint4(lw[4 * q], lw[4 * q + 1], lw[4 * q + 2], lw[4 * q + 3]);
                }
                S.lse2[sl][pt] = nl;
            } else {
                unsigned char *bh = S.B2[st], *bl = S.B2[st] + kB2Bytes;
#pragma unroll
                for (int e = 0; e < 16; e++) {
                    *reinterpret_cast<unsigned short *>(bh + b2_off(2 * e, pt)) = (unsigned short)(hw[e] & 0xffffu);
                    *reinterpret_cast<unsigned short *>(bh + b2_off(2 * e + 1, pt)) = (unsigned short)(hw[e] >> 16);
                    *reinterpret_cast<unsigned short *>(bl + b2_off(2 * e, pt)) = (unsigned short)(lw[e] & 0xffffu);
                    *reinterpret_cast<unsigned short *>(bl + b2_off(2 * e + 1, pt)) = (unsigned short)(lw[e] >> 16);
                }
            }
            fence_async_smem();
            mbar_arrive(tid < 64 ? &S.bar_b1full[st] : &S.bar_b2full[st]);
        };
        // Statistics of component row m about its own mean m_k (FP32), from
        // each chunk's moments about the chunk origin o_c (first point),
        // delta = o_c - m_k, per-axis scale s of the features:
        //   S1 += s S1' + N' delta,
        //   S2_ab += s_a s_b S2'_ab + delta_a s_b S1'_b + s_a S1'_a delta_b + N' delta_a delta_b.
        float st[28];
#pragma unroll
        for (int i = 0; i < 28; i++) st[i] = 0.f;
        float sc[6];
#pragma unroll
        for (int i = 0; i < 6; i++) sc[i] = 1.f / hf[12 + i];
        const int kcomp = j * kCols + m;
        float mh[6], ml[6];   // the component's mean as an FP32 hi/lo pair
        {
            const double *mrec = rec + (size_t)(kcomp < K ? kcomp : K - 1) * VBGS_REC;
#pragma unroll
            for (int i = 0; i < 6; i++) {
                const double v = mrec[i];
                mh[i] = (float)v;
                ml[i] = (float)(v - (double)mh[i]);
            }
        }
        int64_t org0 = 0, org1 = 0;   // origin (first point) of the chunk in each stage
        auto add_d2 = [&](int stage) {
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + 128u + (uint32_t)(stage * kFeat), v);
            tmem_wait_ld();
            const float *xo = Xhl + (stage ? org1 : org0) * 16;
            float dl[6], s1[6];
#pragma unroll
            for (int i = 0; i < 6; i++) dl[i] = (xo[i] - mh[i]) + (xo[8 + i] - ml[i]);
            const float nn = __uint_as_float(v[0]);
            st[0] += nn;
#pragma unroll
            for (int i = 0; i < 6; i++) {
                s1[i] = sc[i] * __uint_as_float(v[1 + i]);
                st[1 + i] += fmaf(nn, dl[i], s1[i]);
            }
            int u = 7;
#pragma unroll
            for (int a = 0; a < 6; a++)
#pragma unroll
                for (int b = a; b < 6; b++, u++)
                    st[u] += fmaf(sc[a] * sc[b], __uint_as_float(v[u]),
                                  fmaf(dl[a], s1[b], fmaf(s1[a], dl[b], nn * dl[a] * dl[b])));
        };
        // Chunk u: (a) B1 and lse2 of chunk u+1 (threads 0..63); (b) the
        // responsibilities of chunk u from MMA1(u); (c) once MMA2(u-1) is done,
        // the statistics of chunk u-1 from D2 and B2 of chunk u+1 (threads
        // 64..127, its stage was MMA2(u-1)'s).  MMA2(u-1) thus runs while (b)
        // computes, instead of the epilogue waiting for it.
        const int64_t nc = cend - cbeg;
        if (nc > 0) {
            load_next(cbeg);
            build(0, 0);
            org0 = nc0;
            if (nc > 1) load_next(cbeg + 1);
        }
        for (int64_t u = 0; u < nc && ok; u++) {
            const int s = (int)(u & 1);
            const int64_t cn = cbeg + u + 1;
            if (cn < cend && tid < 64) build(s ^ 1, (int)((u + 1) % 3));
            ok = __all_sync(0xffffffffu, mbar_wait(&S.bar_d1full[s], (uint32_t)((u >> 1) & 1), flags));
            if (!ok) break;
            fence_after();
            uint32_t v0[32], v1[32];
            const uint32_t tb = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(s * kChunk2);
            tmem_ld32(tb, v0);
            tmem_ld32(tb + 32, v1);
            tmem_wait_ld();
            fence_before();
            mbar_arrive(&S.bar_d1free[s]);
            // r = 2^(l2 - lse2) -> FP16, row m of P (P[s] was last read by
            // MMA2(u-2), waited for in the previous chunk's step (c))
            unsigned char *prow = S.P[s];
            const float4 *l4 = reinterpret_cast<const float4 *>(S.lse2[u % 3]);
#pragma unroll
            for (int g = 0; g < 8; g++) {
                const float4 la = l4[2 * g], lb = l4[2 * g + 1];
                const float lv[8] = {la.x, la.y, la.z, la.w, lb.x, lb.y, lb.z, lb.w};
                float r[8];
#pragma unroll
                for (int e = 0; e < 8; e++) {
                    const int col = g * 8 + e;
                    const uint32_t raw = col < 32 ? v0[col] : v1[col - 32];
                    r[e] = ex2f(fmaf(__uint_as_float(raw), scale, -lv[e]));
                }
                uint32_t ph[4], pl[4];
#pragma unroll
                for (int e = 0; e < 4; e++) H<BF16>::split2(r[2 * e], r[2 * e + 1], ph[e], pl[e]);
                *reinterpret_cast<uint4 *>(prow + p_off(m, g * 8)) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
                *reinterpret_cast<uint4 *>(prow + kPBytes + p_off(m, g * 8)) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
            }
            fence_async_smem();
            mbar_arrive(&S.bar_pfull[s]);
            if (u >= 1) {
                // MMA2(u-1) done: chunk u-1's moments are in D2[s^1], and
                // the B2 stage s^1 is free for chunk u+1
                ok = __all_sync(0xffffffffu, mbar_wait(&S.bar_stfree[s ^ 1], (uint32_t)(((u - 1) >> 1) & 1), flags));
                if (!ok) break;
                fence_after();
                add_d2(s ^ 1);
            }
            if (cn < cend) {
                if (tid >= 64) build(s ^ 1, (int)((u + 1) % 3));
                if (s) org0 = nc0; else org1 = nc0;
                if (cn + 1 < cend) load_next(cn + 1);
            }
        }
        if (ok && nc >= 1) {
            const int sl = (int)((nc - 1) & 1);
            ok = __all_sync(0xffffffffu, mbar_wait(&S.bar_stfree[sl], (uint32_t)(((nc - 1) >> 1) & 1), flags));
            if (ok) {
                fence_after();
                add_d2(sl);
            }
        }
        const int k = j * kCols + m;
        if (k < K) {
            float4 *dst = reinterpret_cast<float4 *>(part + ((size_t)item * kCols + m) * 28);
#pragma unroll
            for (int i = 0; i < 7; i++) dst[i] = make_float4(st[4 * i], st[4 * i + 1], st[4 * i + 2], st[4 * i + 3]);
        }
    } else if (warp == 4 && lane == 0) {
        // ---------------- copy + MMA issuer ----------------
        constexpr uint32_t id1 = idesc_mn<BF16>(128, kChunk2);
        constexpr uint32_t id2 = idesc_mn<BF16>(128, kFeat);
        bool ok = true;
        bool a_loaded = false;
        int n_proc = 0;
        bool any_mma = false;
        int64_t c = next_chunk(cbeg);
        if (c < cend) {
            mbar_expect_tx(&S.bar_a, kTileBytes);
            bulk_g2s(S.A, tiles + (size_t)j * kTileBytes, kTileBytes, &S.bar_a);
            a_loaded = true;
            ok = mbar_wait(&S.bar_a, 0u, flags);
        }
        auto mma1 = [&](int uu) {
            const int s = uu & 1;
            const uint32_t d = tmem + (uint32_t)(s * kChunk2);
            const unsigned char *Ahi = S.A, *Alo = S.A + kOperandBytes;
            const unsigned char *Bh = S.B1[s], *Bl = S.B1[s] + kB1Bytes;
            mma(d, smem_desc_sbo(Ahi, 512), smem_desc_sbo(Bh, 512), id1, 0u);
            mma(d, smem_desc_sbo(Ahi + 256, 512), smem_desc_sbo(Bh + 256, 512), id1, 1u);
            if (!(knobs & VBGS_KNOB_P2_PHI_LO)) {    // the points' features, lo term
                mma(d, smem_desc_sbo(Ahi, 512), smem_desc_sbo(Bl, 512), id1, 1u);
                mma(d, smem_desc_sbo(Ahi + 256, 512), smem_desc_sbo(Bl + 256, 512), id1, 1u);
            }
            if (!(knobs & VBGS_KNOB_P2_C_LO)) {      // the coefficients, lo term
                mma(d, smem_desc_sbo(Alo, 512), smem_desc_sbo(Bh, 512), id1, 1u);
                mma(d, smem_desc_sbo(Alo + 256, 512), smem_desc_sbo(Bh + 256, 512), id1, 1u);
            }
            mma_commit(&S.bar_d1full[s]);
        };
        // MMA1 of the first chunk
        if (ok && c < cend) {
            ok = mbar_wait(&S.bar_b1full[0], 0u, flags);
            if (ok) { fence_after(); mma1(0); any_mma = true; }
        }
        int u = 0;
        while (ok && c < cend) {
            const int s = u & 1;
            const int64_t cn = next_chunk(c + 1);
            if (cn < cend) {
                const int s1 = (u + 1) & 1;
                ok = mbar_wait(&S.bar_b1full[s1], (uint32_t)(((u + 1) >> 1) & 1), flags) &&
                     (u + 1 < 2 || mbar_wait(&S.bar_d1free[s1], (uint32_t)((((u + 1) >> 1) - 1) & 1), flags));
                if (!ok) break;
                fence_after();
                mma1(u + 1);
            }
            ok = mbar_wait(&S.bar_pfull[s], (uint32_t)((u >> 1) & 1), flags) &&
                 mbar_wait(&S.bar_b2full[s], (uint32_t)((u >> 1) & 1), flags);
            if (!ok) break;
            fence_after();
            const unsigned char *Pp = S.P[s];
            const unsigned char *Bh = S.B2[s], *Bl = S.B2[s] + kB2Bytes;
            const uint32_t d2 = tmem + 128u + (uint32_t)(s * kFeat);
            const unsigned char *Pl = Pp + kPBytes;
#pragma unroll
            for (int t = 0; t < kChunk2 / 16; t++) {
                mma(d2, smem_desc_sbo(Pp + 256 * t, 1024), smem_desc_sbo(Bh + 256 * t, 1024), id2, t > 0 ? 1u : 0u);
                if (!(knobs & VBGS_KNOB_P2_S_LO))    // the statistics' features, lo term
                    mma(d2, smem_desc_sbo(Pp + 256 * t, 1024), smem_desc_sbo(Bl + 256 * t, 1024), id2, 1u);
                if (!(knobs & VBGS_KNOB_P2_P_LO))    // the responsibilities, lo term
                    mma(d2, smem_desc_sbo(Pl + 256 * t, 1024), smem_desc_sbo(Bh + 256 * t, 1024), id2, 1u);
            }
            mma_commit(&S.bar_stfree[s]);
            n_proc = u + 1;
            c = cn;
            u++;
        }
        // Drain: last phases of the barriers the copy and the commits arrive on.
        if (a_loaded) mbar_wait(&S.bar_a, 0u, flags, true);
        for (int s = 0; s < 2; s++) {
            const int last = ((n_proc - 1 - s) >= 0) ? s + ((n_proc - 1 - s) / 2) * 2 : -1;
            if (last >= 0) mbar_wait(&S.bar_stfree[s], (uint32_t)((last >> 1) & 1), flags, true);
        }
        if (any_mma) {
            mma_commit(&S.bar_final);
            mbar_wait(&S.bar_final, 0u, flags, true);
        }
        if (pairs && n_proc > 0) atomicAdd(pairs, (unsigned long long)n_proc * kChunk2 * kCols);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256) : "memory");
    }
}

// dS[kperm[p]] = sum over the items of p's tile (in item order) of the
// moments of position p about its component's mean m (FP64 record), shifted
// to raw moments: S1 = S1' + N m, S2 = S2' + m S1'^T + S1' m^T + N m m^T.
// One CTA per (tile, 32 positions): warp w sums the items q = w, w + 4, ...
// of the tile in order; the 4 warp sums are added in warp order.
// nz (nullable): per block, whether its rows of dS were last written nonzero;
// with skip_zero, a block without items whose rows are already zero writes
// nothing (iterations after the first of a frame: same points and order).
// ml.list (nullable): warp 0 also enters its 32 positions into the M-step's
// list (MstepList).
__global__ void __launch_bounds__(128) k_reduce_items(const float *__restrict__ part,
                                                      const int *__restrict__ item_start, int K,
                                                      const double *__restrict__ rec, const int *__restrict__ kperm,
                                                      double *__restrict__ dS, int *__restrict__ nz, bool skip_zero,
                                                      MstepList ml)
{
    pdl_wait();
    __shared__ float sh[4][32][29];
    const int j = blockIdx.x >> 2, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int m = (blockIdx.x & 3) * 32 + lane;
    const int p = j * kCols + m;
    const int q0 = item_start[j], q1 = item_start[j + 1];
    // warp 0, all lanes: position p (zero: its statistics are all zero) into
    // the M-step's list, or its "q = p" hand-off
    auto list_entry = [&](bool zero) {
        if (!ml.list) return;
        bool act = false;
        if (p < K) {
            const size_t k = kperm ? (size_t)kperm[p] : (size_t)p;
            act = !(zero && ml.pc33[k * ml.pc_stride] != 0.0);
            if (!act) {
                double *ks = ml.ks33 + k * ml.ks_stride;
                ks[0] = 0.0;
                ks[1] = 0.0;
            }
        }
        const unsigned b = __ballot_sync(0xffffffffu, act);
        if (b) {
            int base = 0;
            if (lane == 0) base = atomicAdd(ml.count, __popc(b));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (act) ml.list[base + __popc(b & ((1u << lane) - 1u))] = p;
        }
    };
    if (q0 == q1) {
        // no pair of this tile was evaluated: zero statistics
        if (!(skip_zero && nz[blockIdx.x] == 0)) {
            if (w == 0 && p < K) {
                const size_t dst = kperm ? (size_t)kperm[p] : (size_t)p;
                double2 *o = reinterpret_cast<double2 *>(dS + dst * 28);   // 224-byte rows
#pragma unroll
                for (int f = 0; f < 14; f++) o[f] = make_double2(0.0, 0.0);
            }
            if (nz && threadIdx.x == 0) nz[blockIdx.x] = 0;
        }
        if (w == 0) list_entry(true);
        return;
    }
    if (nz && threadIdx.x == 0) nz[blockIdx.x] = 1;
    // The item partials are FP32 sums: they and the four warp sums are added
    // in FP32, then shifted to raw moments in FP64.  An FP64 instruction
    // holds a warp's sub-partition for 64 cycles, so the FP64 part is three
    // FMAs per second moment, spread over the four warps (warp 0: the count
    // and first moments, warps 1-3: seven second moments each), and the
    // FP32 -> FP64 conversions are exact bit manipulations on the integer
    // pipe.
    float t[28];
#pragma unroll
    for (int f = 0; f < 28; f++) t[f] = 0.f;
    if (p < K)
        for (int q = q0 + w; q < q1; q += 4) {
            const float4 *src = reinterpret_cast<const float4 *>(part + ((size_t)q * kCols + m) * 28);
#pragma unroll
            for (int f = 0; f < 7; f++) {
                const float4 v = src[f];
                t[4 * f] += v.x; t[4 * f + 1] += v.y; t[4 * f + 2] += v.z; t[4 * f + 3] += v.w;
            }
        }
#pragma unroll
    for (int f = 0; f < 28; f++) sh[w][lane][f] = t[f];
    __syncthreads();
    auto fsum32 = [&](int f) {   // the four warp sums in warp order
        return (sh[0][lane][f] + sh[1][lane][f]) + (sh[2][lane][f] + sh[3][lane][f]);
    };
    if (w == 0) {
        // the raw moments below are all zero exactly when these sums are
        bool zero = true;
#pragma unroll
        for (int f = 0; f < 28; f++) zero = zero && (__float_as_uint(fsum32(f)) << 1) == 0u;
        list_entry(zero);
    }
    if (p >= K) return;
    auto fsum = [&](int f) { return f2d_exact(fsum32(f)); };
    double d0[7], mk[6];
#pragma unroll
    for (int f = 0; f < 7; f++) d0[f] = fsum(f);
#pragma unroll
    for (int i = 0; i < 6; i++) mk[i] = rec[(size_t)p * VBGS_REC + i];
    const size_t dst = kperm ? (size_t)kperm[p] : (size_t)p;
    double *o = dS + dst * 28;
    if (w == 0) {
        o[0] = d0[0];
#pragma unroll
        for (int i = 0; i < 6; i++) o[1 + i] = fma(d0[0], mk[i], d0[1 + i]);
        return;
    }
    // second moments u = 7 + 7 (w - 1) .. 7 + 7 w - 1 (upper triangle, row-major):
    // S2' + S1'_a m_b + m_a S1'_b + (N' m_a) m_b
    int u = 7;
#pragma unroll
    for (int a = 0; a < 6; a++)
#pragma unroll
        for (int b = a; b < 6; b++, u++)
            if (u >= 7 * w && u < 7 * w + 7)
                o[u] = fma(d0[0] * mk[a], mk[b], fma(mk[a], d0[1 + b], fma(d0[1 + a], mk[b], fsum(u))));
}

} // namespace

size_t tc_tile_bytes(int K) { return (size_t)((K + kCols - 1) / kCols) * kTileBytes; }
size_t tc_hdr_floats(int K) { return (size_t)((K + kCols - 1) / kCols) * 32; }
size_t tc_tmax_floats(int64_t N, int K) { return (size_t)((N + 31) / 32) * (size_t)((K + kCols - 1) / kCols); }

int launch_coef_tiles(const double *rec, const float *rec32, int K, bool bf16, unsigned char *tiles, float *hdr,
                      int *dirty, int epoch, cudaStream_t st, Prof *pf)
{
    const int nt = (K + kCols - 1) / kCols;
    pf->begin(VBGS_PROF_MSTEP, st);
    if (bf16) launch_pdl(k_coef_tiles<true>, nt, 128, 0, st, rec, rec32, K, tiles, hdr, dirty, epoch);
    else      launch_pdl(k_coef_tiles<false>, nt, 128, 0, st, rec, rec32, K, tiles, hdr, dirty, epoch);
    pf->end(st);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}


// Item capacity of pass 2: at least two items per tile.
int tc_item_cap(int K) { return std::max(kItemCap, 2 * ((K + kCols - 1) / kCols)); }
size_t tc_pass2_part_doubles(int K) { return (size_t)tc_item_cap(K) * kCols * 28; }

size_t tc_plan_ints(int64_t N, int K)
{
    const size_t nt = (size_t)((K + kCols - 1) / kCols);
    return nt * (size_t)(1 + (N + kChunk2 - 1) / kChunk2) + (nt + 1) + 3 * (size_t)tc_item_cap(K) + 1;
}

int launch_pass2_tc(const float *Xhl, const float *lse2f, int64_t N, int K, bool bf16, const unsigned char *tiles,
                    const float *hdr, const double *rec, const float *tmax, const float *minlse, int *plan, double *part,
                    size_t part_cap_doubles, const int *kperm, double *dS, int *flags, int num_sms, int splits_override,
                    int *nz, bool skip_zero, cudaStream_t st, Prof *pf, uint32_t knobs, double skip_nats_d,
                    unsigned int *plan_done, const MstepList *ml)
{
    const float skip_nats = (float)skip_nats_d;
    unsigned long long *pairs = pf->on ? pf->d_pairs : nullptr;
    const int ntiles = (K + kCols - 1) / kCols;
    const int64_t nchunks = (N + kChunk2 - 1) / kChunk2;
    // balanced work items: chunks of each tile's list, at least cmin per item
    // (4 unless tuned), as many items as the partial buffer holds (at most
    // kItemCap); one CTA per item slot
    const int cmin = splits_override > 0 ? splits_override : 4;
    const int icap = tc_item_cap(K);
    const int tcap = (int)std::min<size_t>((size_t)icap, part_cap_doubles / ((size_t)kCols * 28));
    if (tcap < ntiles + 1) return -2;
    int *counts = plan, *list = plan + ntiles;
    int *item_start = list + (size_t)ntiles * nchunks;
    int *item_tile = item_start + ntiles + 1, *item_lo = item_tile + icap, *item_hi = item_lo + icap;
    int *nitems = item_hi + icap;
    pf->begin(VBGS_PROF_PLAN, st);
    if (tmax)   // the plan's last block builds the work items
        launch_pdl(k_p2_plan, ntiles, 256, 0, st, tmax, minlse, N, ntiles, counts, list, skip_nats,
                   ItemsArgs{cmin, tcap, item_start, item_tile, item_lo, item_hi, nitems, plan_done,
                             ml ? ml->count : nullptr});
    else
        launch_pdl(k_p2_items, 1, 1024, 0, st, (const int *)nullptr, ntiles, nchunks, cmin, tcap, item_start,
                   item_tile, item_lo, item_hi, nitems, ml ? ml->count : nullptr);
    pf->end(st);
    const size_t smem = sizeof(Smem2) + 128;
    if (tc_set_attributes()) return -1;
    float *fpart = reinterpret_cast<float *>(part);   // item partials: FP32 register sums
    pf->begin(VBGS_PROF_PASS2, st);
    if (bf16)
        launch_pdl(k_pass2_tc<true>, tcap, kThreadsTC, smem, st, Xhl, lse2f, N, K, tiles, hdr, ntiles, tmax ? counts : nullptr,
                                                         list, item_tile, item_lo, item_hi, nitems, rec, fpart, flags,
                                                         pairs, knobs);
    else
        launch_pdl(k_pass2_tc<false>, tcap, kThreadsTC, smem, st, Xhl, lse2f, N, K, tiles, hdr, ntiles, tmax ? counts : nullptr,
                                                          list, item_tile, item_lo, item_hi, nitems, rec, fpart, flags,
                                                         pairs, knobs);
    pf->end(st);
    pf->begin(VBGS_PROF_REDUCE, st);
    launch_pdl(k_reduce_items, ntiles * 4, 128, 0, st, fpart, item_start, K, rec, kperm, dS, nz, skip_zero && nz,
               ml ? *ml : MstepList{});
    pf->end(st);
    return cudaGetLastError() == cudaSuccess ? 3 : -1;
}

// K-splits of pass 1: many small CTAs (two resident per SM) that the hardware
// scheduler balances, with the number of waves close to an integer so the
// last wave is not nearly empty; a mild penalty per split for pipeline fill.
int tc_pass1_auto_splits(int64_t N, int K, int num_sms)
{
    const int ntiles = (K + kCols - 1) / kCols;
    const int ptiles = (int)((N + kRows - 1) / kRows);
    int splits = 1;
    const double slots = 2.0 * num_sms;
    double best = -1.0;
    const int smax = std::max(1, std::min(64, ntiles / 4));
    for (int sp = 1; sp <= smax; sp++) {
        const int tp = (ntiles + sp - 1) / sp;
        const int sreal = (ntiles + tp - 1) / tp;
        const double waves = ptiles * (double)sreal / slots;
        const double eff = waves / std::ceil(waves) - 0.004 * sreal;
        if (eff > best + 1e-9) { best = eff; splits = sreal; }
    }
    return splits;
}

// Shared-memory attributes of the tensor-core kernels (set once, before any
// stream capture).
bool g_tc_attr = false;
int tc_set_attributes()
{
    if (g_tc_attr) return 0;
    const int s1 = (int)(sizeof(Smem) + 1024), s2 = (int)(sizeof(Smem2) + 128);
    if (cudaFuncSetAttribute(k_pass1_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s1) != cudaSuccess ||
        cudaFuncSetAttribute(k_pass1_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s1) != cudaSuccess ||
        cudaFuncSetAttribute(k_pass2_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s2) != cudaSuccess ||
        cudaFuncSetAttribute(k_pass2_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s2) != cudaSuccess)
        return -1;
    g_tc_attr = true;
    return 0;
}

// Points as FP32 hi/lo pairs, 16 floats per point (hi at 0-5, lo at 8-13):
// the tensor-core builders then form differences in FP32 double-float
// arithmetic instead of FP64.
__global__ void k_split_points(const double *__restrict__ X, int64_t N, float *__restrict__ Xhl)
{
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * 8) return;
    const int64_t n = i >> 3;
    const int q = (int)(i & 7);
    float hi = 0.f, lo = 0.f;
    if (q < 6) {
        const double v = X[n * VBGS_XS + q];
        hi = (float)v;
        lo = (float)(v - (double)hi);
    }
    Xhl[n * 16 + q] = hi;
    Xhl[n * 16 + 8 + q] = lo;
}

// lse_n from the item partials of its point tile and, with skipping, the
// seed launch's partial (FP32, log2 units: the partials carry the
// tensor-core pass's FP32 sums), natural-unit lse in FP64, the smallest lse
// per 32 points and per-block FP64 sums of lse.
constexpr int kMergeThreads = 256;
__global__ void __launch_bounds__(kMergeThreads) k_merge_tc(const float2 *__restrict__ part,
                                                            const int *__restrict__ item_start,
                                                            const float2 *__restrict__ spart, int64_t N,
                                                            double *__restrict__ lse, float *__restrict__ lse2f,
                                                            double *__restrict__ lse_part, float *__restrict__ minlse,
                                                            unsigned int *__restrict__ done,
                                                            double *__restrict__ sum_out)
{
    pdl_wait();
    constexpr int kW = kMergeThreads / 32;
    __shared__ double sh[kW];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (n < N) {
        const int64_t P = n >> 7;
        const size_t row = (size_t)(n & 127);
        const int q0 = item_start[P], q1 = item_start[P + 1];
        const float2 sp = spart ? spart[(size_t)n] : make_float2(-INFINITY, 0.f);
        float M = sp.x;
        for (int q = q0; q < q1; q++) M = fmaxf(M, part[(size_t)q * kRows + row].x);
        float sm = sp.y > 0.f ? sp.y * ex2f(sp.x - M) : 0.f;
        for (int q = q0; q < q1; q++) {
            const float2 p = part[(size_t)q * kRows + row];
            if (p.y > 0.f) sm += p.y * ex2f(p.x - M);
        }
        const float l2 = M + __log2f(sm);
        v = (double)l2 * 0.6931471805599453;
        lse[n] = v;
        lse2f[n] = l2;
    }
    float vm = n < N ? (float)v : INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v += __shfl_down_sync(0xffffffffu, v, o);
        vm = fminf(vm, __shfl_down_sync(0xffffffffu, vm, o));
    }
    if (lane == 0) {
        sh[wid] = v;
        const int64_t w = (int64_t)blockIdx.x * kW + wid;
        if (minlse && w * 32 < N) minlse[w] = vm;
    }
    __syncthreads();
    // the block sums, added in block order by the last block to finish (the
    // same sum on every run); it leaves the counter at zero for the next merge
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int i = 0; i < kW; i++) b += sh[i];
        lse_part[blockIdx.x] = b;
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double t = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += __ldcg(lse_part + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    __syncthreads();
    if (lane == 0) sh[wid] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int i = 0; i < kW; i++) tot += sh[i];
        *sum_out = tot;
        *done = 0u;
    }
}

// Pass-1 work items: at most kItemCap1 + point tiles, so item partials of
// 128 (max, sum) pairs fit next to the other scratch.
constexpr int kItemCap1 = 2048;
size_t tc_p1plan_ints(int64_t N, int K)
{
    const size_t pt = (size_t)((N + kRows - 1) / kRows), nt = (size_t)((K + kCols - 1) / kCols);
    // lists, counts, items; the seed launch's items
    return pt * nt + pt + (pt + 1) + 3 * (kItemCap1 + pt) + 1 + 3 * pt + 1;
}
size_t tc_p1ub_floats(int64_t N, int K)
{
    const size_t pt = (size_t)((N + kRows - 1) / kRows);
    // coarse bounds, the point-tile boxes, then the seed launch's partials
    // (128 float2 per point tile) at an even offset
    return pt * (size_t)((K + kCols - 1) / kCols) + 12 * pt + 1 + 2 * (size_t)kRows * pt;
}

int launch_pass1_tc(const double *X, float *Xhl, bool same_points, int64_t N, int K, bool bf16,
                    const unsigned char *tiles, const float *hdr, const float *rec32, double *part_buf,
                    size_t part_cap_doubles, float *tmax, int *p1plan, float *p1ub, int *flags, int num_sms,
                    int tiles_per_item, const int *tile_epoch, int since, const int **item_start_out,
                    const double **seed_part_out, cudaStream_t st, Prof *pf, uint32_t knobs, double skip_nats,
                    unsigned int *plan_done)
{
    float2 *part = reinterpret_cast<float2 *>(part_buf);
    int launches = 0;
    if (N > 0 && !same_points) {
        launches++;
        pf->begin(VBGS_PROF_PLAN, st);
        launch_pdl(k_split_points, (unsigned)((N * 8 + 255) / 256), 256, 0, st, X, N, Xhl);
        pf->end(st);
    }
    const int ntiles = (K + kCols - 1) / kCols;
    const int ptiles = (int)((N + kRows - 1) / kRows);
    unsigned long long *pairs1 = pf->on ? pf->d_pairs + 1 : nullptr;
    const int icap = (int)std::min<size_t>((size_t)kItemCap1 + ptiles, part_cap_doubles / (2 * (size_t)kRows));
    if (icap < ptiles + 1) return -2;
    int *list = p1plan, *counts = list + (size_t)ptiles * ntiles;
    int *item_start = counts + ptiles, *item_tile = item_start + ptiles + 1;
    int *item_lo = item_tile + icap, *item_hi = item_lo + icap, *nitems = item_hi + icap;
    // least tiles per item: tuned, or the K-split decomposition when every
    // tile is evaluated; with skipping, at least 4 (items then follow the
    // lists' total so the grid keeps several waves)
    int tmin = tiles_per_item;
    if (tmin <= 0) {
        if (tmax) tmin = 4;
        else {
            const int splits = tc_pass1_auto_splits(N, K, num_sms);
            tmin = (ntiles + splits - 1) / splits;
        }
    }
    const int target = tmax ? std::min(icap, std::max(ptiles + 1, 8 * num_sms)) : icap;
    const size_t smem = sizeof(Smem) + 1024;
    if (tc_set_attributes()) return -1;
    auto pass1 = [&](int grid, const int *lst, const int *it, const int *il, const int *ih, const int *ni,
                     float2 *out, const float2 *seed, float drop) {
        if (bf16)
            launch_pdl(k_pass1_tc<true>, grid, kThreadsTC, smem, st, Xhl, N, K, tiles, hdr, ntiles, lst, it, il, ih,
                       ni, out, tmax, flags, pairs1, knobs, seed, drop);
        else
            launch_pdl(k_pass1_tc<false>, grid, kThreadsTC, smem, st, Xhl, N, K, tiles, hdr, ntiles, lst, it, il, ih,
                       ni, out, tmax, flags, pairs1, knobs, seed, drop);
    };
    // batches of the main launch below log2 K + 25 of a row's running maximum
    // are left out (see k_pass1_tc)
    const float drop = (float)(std::log2((double)std::max(K, 2)) + 25.0);
    const float2 *seed_rows = nullptr;
    *seed_part_out = nullptr;
    pf->begin(VBGS_PROF_PLAN, st);
    if (tmax) {
        float *boxes = p1ub + (size_t)ptiles * ntiles;
        if (!same_points) {   // the boxes of the previous E-step's points are current
            launch_pdl(k_p1_boxes, ptiles, kRows, 0, st, X, N, boxes);
            launches++;
        }
        // bounds of the tiles rebuilt since the last plan of these points
        const int *te = same_points ? tile_epoch : nullptr;
        launch_pdl(k_p1_ub, dim3(ntiles, (ptiles + kCols - 1) / kCols), kCols, 0, st, (const float *)boxes, ptiles, K,
                   ntiles, rec32, p1ub, te, since);
        int *sitem_tile = nitems + 1, *sitem_lo = sitem_tile + ptiles, *sitem_hi = sitem_lo + ptiles;
        int *snitems = sitem_hi + ptiles;
        // (float2: 8-byte aligned, so an even float offset)
        float2 *spart = reinterpret_cast<float2 *>(p1ub + (((size_t)ptiles * ntiles + 12 * (size_t)ptiles + 1) & ~(size_t)1));
        launch_pdl(k_p1_seed, ptiles, kPlanThreads, 0, st, N, ntiles, ptiles, (const float *)p1ub, list, sitem_tile,
                   sitem_lo, sitem_hi, snitems, tmax);
        pf->end(st);
        // the seed tile of every point tile, on the tensor cores
        pf->begin(VBGS_PROF_PASS1, st);
        pass1(ptiles, list, sitem_tile, sitem_lo, sitem_hi, snitems, spart, nullptr, 0.f);
        seed_rows = spart;
        pf->end(st);
        pf->begin(VBGS_PROF_PLAN, st);
        // its last block builds the main launch's work items
        launch_pdl(k_p1_plan, ptiles, kPlanThreads, 0, st, N, ntiles, (const float2 *)spart, (const float *)p1ub,
                   list, counts, (float)(skip_nats * 1.4426950408889634),
                   ItemsArgs{tmin, target, item_start, item_tile, item_lo, item_hi, nitems, plan_done, nullptr});
        *seed_part_out = reinterpret_cast<const double *>(spart);
    } else {
        launch_pdl(k_p2_items, 1, 1024, 0, st, (const int *)nullptr, ptiles, ntiles, tmin, target, item_start,
                   item_tile, item_lo, item_hi, nitems, (int *)nullptr);
    }
    pf->end(st);
    pf->begin(VBGS_PROF_PASS1, st);
    const int *lst = tmax ? list : nullptr;
    {
        Pass1Launch &L = pf->p1_last;
        L.valid = true;
        L.bf16 = bf16;
        L.grid = target;
        L.smem = smem;
        L.Xhl = Xhl;
        L.N = N;
        L.K = K;
        L.ntiles = ntiles;
        L.tiles = tiles;
        L.hdr = hdr;
        L.list = lst;
        L.item_tile = item_tile;
        L.item_lo = item_lo;
        L.item_hi = item_hi;
        L.nitems = nitems;
        L.part = part;
        L.tmax = tmax;
        L.flags = flags;
        L.knobs = knobs;
        L.seed = seed_rows;
        L.drop = drop;
    }
    pass1(target, lst, item_tile, item_lo, item_hi, nitems, part, seed_rows, drop);
    pf->end(st);
    *item_start_out = item_start;
    return cudaGetLastError() == cudaSuccess ? launches + (tmax ? 5 : 2) : -1;
}

int launch_lse_merge_tc(const double *part_buf, const double *seed_part, int64_t N, const int *item_start, double *lse,
                        float *lse2f, double *lse_part, float *minlse, double *sum_out, unsigned int *done,
                        cudaStream_t st, Prof *pf)
{
    const int mb = (int)((N + kMergeThreads - 1) / kMergeThreads);
    pf->begin(VBGS_PROF_MERGE, st);
    launch_pdl(k_merge_tc, mb, kMergeThreads, 0, st, reinterpret_cast<const float2 *>(part_buf), item_start,
               reinterpret_cast<const float2 *>(seed_part), N, lse, lse2f, lse_part, minlse, done, sum_out);
    pf->end(st);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int tc_replay_pass1(const Pass1Launch &L, int reps, unsigned long long *pairs, cudaStream_t st, float *ms)
{
    if (!L.valid || reps < 1) return -1;
    auto launch = [&](unsigned long long *pc) {
        if (L.bf16)
            return launch_pdl(k_pass1_tc<true>, L.grid, kThreadsTC, L.smem, st, L.Xhl, L.N, L.K, L.tiles, L.hdr,
                              L.ntiles, L.list, L.item_tile, L.item_lo, L.item_hi, L.nitems, L.part, L.tmax, L.flags,
                              pc, L.knobs, L.seed, L.drop);
        return launch_pdl(k_pass1_tc<false>, L.grid, kThreadsTC, L.smem, st, L.Xhl, L.N, L.K, L.tiles, L.hdr,
                          L.ntiles, L.list, L.item_tile, L.item_lo, L.item_hi, L.nitems, L.part, L.tmax, L.flags, pc,
                          L.knobs, L.seed, L.drop);
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1;
    bool ok = launch(pairs) == cudaSuccess && launch(nullptr) == cudaSuccess &&   // counted, then a warm-up
              cudaEventRecord(e0, st) == cudaSuccess;
    for (int r = 0; ok && r < reps; r++) ok = launch(nullptr) == cudaSuccess;
    ok = ok && cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
    float t = 0.f;
    ok = ok && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok) return -1;
    *ms = t / (float)reps;
    return 0;
}

int tc_set_wait_limit(long long cycles)
{
    const long long v = cycles > 0 ? cycles : kSpinCycles;
    return cudaMemcpyToSymbol(g_wait_limit, &v, sizeof v) == cudaSuccess ? 0 : -1;
}

} // namespace vbgs
