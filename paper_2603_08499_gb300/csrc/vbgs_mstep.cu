// vbgs_mstep.cu -- FP64 posterior update (`update_from_statistics`, Alg. 1),
// per-component KL terms of the ELBO and the E-step records they feed.
//
// One thread per component.  From the prior (alpha0, beta0, nu0, m0_k, W0)
// and statistics S = (N_k, S1_k, S2_k) the conjugate Normal-Wishart /
// Dirichlet posterior in raw-moment form is
//   alpha = alpha0 + N, beta = beta0 + N, nu = nu0 + N,
//   beta m = beta0 m0 + S1,  W^-1 = W0^-1 + S2 + beta0 m0 m0^T - beta m m^T.
// The kernel forms it twice per component: the effective prior p from S_past
// (the posterior of all earlier frames, the prior of this frame in the
// continual setting of Alg. 1) and the posterior q from S_past + Delta S.
// It then writes the E-step record of q (m, M = sqrt(nu) L^-1 with
// W^-1 = L L^T, and the constant c of log rho) and KL(q || p).
#include "vbgs_internal.cuh"
#include <math.h>
#include <algorithm>

namespace vbgs {

namespace {

constexpr double kLn2 = 0.69314718055994530942;
constexpr double kLn2Pi = 1.8378770664093454836;
constexpr double kLnPi = 1.1447298858494001741;

// Digamma for x > 0: raise x to >= 10 with psi(x) = psi(x+1) - 1/x, then the
// asymptotic expansion ln x - 1/(2x) - sum_k B_2k / (2k x^2k) through B_16.
__device__ double dg_digamma(double x)
{
    // shift = sum 1/(x + i) accumulated as one fraction num/den; one division
    // gives both shift and 1/x
    double num = 0.0, den = 1.0;
    while (x < 10.0) { num = fma(num, x, den); den *= x; x += 1.0; }
    const double r = 1.0 / (den * x);
    const double shift = num * x * r, ix = den * r;
    const double t = ix * ix;
    // B2/2, B4/4, ..., B16/16
    const double c1 = 1.0 / 12.0, c2 = -1.0 / 120.0, c3 = 1.0 / 252.0, c4 = -1.0 / 240.0;
    const double c5 = 1.0 / 132.0, c6 = -691.0 / 32760.0, c7 = 1.0 / 12.0, c8 = -3617.0 / 8160.0;
    double p = c8;
    p = fma(p, t, c7); p = fma(p, t, c6); p = fma(p, t, c5); p = fma(p, t, c4);
    p = fma(p, t, c3); p = fma(p, t, c2); p = fma(p, t, c1);
    return log(x) - 0.5 * ix - p * t - shift;
}

// psi_6(a) = sum_{i=0..5} psi(a - i/2): two series evaluations (at x = a and
// x = a - 1/2) and the recurrence psi(x - 1) = psi(x) - 1/(x - 1), i.e.
// psi(x) + psi(x-1) + psi(x-2) = 3 psi(x) - (3x - 5) / ((x - 1)(x - 2)).
__device__ double mv_digamma6(double a)
{
    double s = 0.0;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const double x = a - 0.5 * h;
        s += 3.0 * dg_digamma(x) - (3.0 * x - 5.0) / ((x - 1.0) * (x - 2.0));
    }
    return s;
}
// ln Gamma_6(a) = 7.5 ln pi + sum_{i=0..5} lnGamma(a - i/2), with
// lnGamma(x - 1) = lnGamma(x) - ln(x - 1): per half-step x,
// 3 lnGamma(x) - ln((x - 1)^2 (x - 2)).
__device__ double mv_lgamma6(double a)
{
    double s = 7.5 * kLnPi;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const double x = a - 0.5 * h;
        s += 3.0 * lgamma(x) - log((x - 1.0) * (x - 1.0) * (x - 2.0));
    }
    return s;
}

// The split model's two 3-D blocks with the same nu: 2 psi_3(a) and
// 2 ln Gamma_3(a), psi_3(a) = psi(a) + psi(a - 1/2) + psi(a - 1) with
// psi(a - 1) = psi(a) - 1/(a - 1), ln Gamma_3(a) = 1.5 ln pi + lnGamma(a) +
// lnGamma(a - 1/2) + lnGamma(a - 1) with lnGamma(a - 1) = lnGamma(a) - ln(a - 1).
__device__ double mv_digamma_split(double a)
{
    double s = 4.0 * dg_digamma(a) - 2.0 / (a - 1.0);
    s += 2.0 * dg_digamma(a - 0.5);
    return s;
}
__device__ double mv_lgamma_split(double a)
{
    double s = 3.0 * kLnPi;
    s += 4.0 * lgamma(a) - 2.0 * log(a - 1.0);
    s += 2.0 * lgamma(a - 0.5);
    return s;
}

// Largest eigenvalue of a symmetric 3x3 matrix (a00, a01, a02, a11, a12,
// a22) by the trigonometric solution of its characteristic cubic (Smith 1961):
// q = tr/3, p = sqrt(tr((A - qI)^2)/6), r = det((A - qI)/p)/2,
// lambda_max = q + 2 p cos(acos(r)/3).  In FP32: the result is within a few
// 1e-6 of |A| >= lambda_max; callers inflate it by 1e-4.
__device__ float sym3_max_eig(float a00, float a01, float a02, float a11, float a12, float a22)
{
    const float p1 = a01 * a01 + a02 * a02 + a12 * a12;
    if (p1 == 0.f) return fmaxf(a00, fmaxf(a11, a22));
    const float q = (a00 + a11 + a22) * (1.f / 3.f);
    const float b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
    const float p = sqrtf((b00 * b00 + b11 * b11 + b22 * b22 + 2.f * p1) * (1.f / 6.f));
    const float ip = 1.f / p;
    const float c00 = b00 * ip, c11 = b11 * ip, c22 = b22 * ip, c01 = a01 * ip, c02 = a02 * ip, c12 = a12 * ip;
    const float r = 0.5f * (c00 * (c11 * c22 - c12 * c12) - c01 * (c01 * c22 - c12 * c02) + c02 * (c01 * c12 - c11 * c02));
    const float phi = acosf(fminf(1.f, fmaxf(-1.f, r))) * (1.f / 3.f);
    return q + 2.f * p * cosf(phi);
}

// Posterior parameters from prior and statistics; A is W^-1, packed lower
// triangular (A[tri(i, j)], j <= i).  Packed storage keeps the 6 x 6
// matrices of one thread in registers.
__device__ __forceinline__ void nw_from_stats(const MstepParams &P, const double *m0, const double *s,
                              double &alpha, double &beta, double &nu, double m[6], double A[21])
{
    const double N = s[0];
    alpha = P.alpha0 + N;
    beta = P.beta0 + N;
    nu = P.nu0 + N;
    const double ib = 1.0 / beta;
#pragma unroll
    for (int i = 0; i < 6; i++) m[i] = (P.beta0 * m0[i] + s[1 + i]) * ib;
#pragma unroll
    for (int i = 0; i < 6; i++)
#pragma unroll
        for (int j = i; j < 6; j++)
            A[tri(j, i)] = (P.split && i < 3 && j >= 3)   // split model: no position-colour block
                               ? 0.0
                               : P.W0inv[i * 6 + j] + s[upper_index(i, j)] + P.beta0 * m0[i] * m0[j] - beta * m[i] * m[j];
}

// One column of the in-register Cholesky A = L L^T (both packed lower
// triangular); a template so the compiler unrolls every loop and keeps A and
// L in registers.
template <int J>
__device__ __forceinline__ void chol6_col(const double A[21], double L[21], bool &ok)
{
    double d = A[tri(J, J)];
#pragma unroll
    for (int k = 0; k < J; k++) d -= L[tri(J, k)] * L[tri(J, k)];
    ok = ok && (d > 0.0);
    d = fmax(d, 1e-300);
    const double inv = rsqrt(d);
    L[tri(J, J)] = d * inv;
#pragma unroll
    for (int i = J + 1; i < 6; i++) {
        double t = A[tri(i, J)];
#pragma unroll
        for (int k = 0; k < J; k++) t -= L[tri(i, k)] * L[tri(J, k)];
        L[tri(i, J)] = t * inv;
    }
}

// A = L L^T; false if A is not positive definite.
__device__ __forceinline__ bool chol6(const double A[21], double L[21])
{
    bool ok = true;
    chol6_col<0>(A, L, ok);
    chol6_col<1>(A, L, ok);
    chol6_col<2>(A, L, ok);
    chol6_col<3>(A, L, ok);
    chol6_col<4>(A, L, ok);
    chol6_col<5>(A, L, ok);
    return ok;
}

// Inverse of a lower-triangular 6x6 matrix, both packed.
__device__ __forceinline__ void trinv6(const double L[21], double Li[21])
{
#pragma unroll
    for (int c = 0; c < 6; c++) Li[tri(c, c)] = 1.0 / L[tri(c, c)];
#pragma unroll
    for (int c = 0; c < 6; c++) {
#pragma unroll
        for (int i = c + 1; i < 6; i++) {
            double t = 0.0;
#pragma unroll
            for (int k = c; k < i; k++) t += L[tri(i, k)] * Li[tri(k, c)];
            Li[tri(i, c)] = -t * Li[tri(i, i)];
        }
    }
}

// Per-component cache of the effective prior p = prior0 (+) S_past, fixed
// within a frame: alpha, beta, nu, m (6), W^-1 upper (21), ln|W^-1|,
// ln Gamma_6(nu/2), ln Gamma(alpha).
constexpr int kPC = 40;

// Block-level fixed-order sums of 4 values (klk, aq, ap, dN) -> part[block].
__device__ void block_sums4(double v0, double v1, double v2, double v3, double *__restrict__ part)
{
    __shared__ double sh[4][4];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_down_sync(0xffffffffu, v0, o);
        v1 += __shfl_down_sync(0xffffffffu, v1, o);
        v2 += __shfl_down_sync(0xffffffffu, v2, o);
        v3 += __shfl_down_sync(0xffffffffu, v3, o);
    }
    if (lane == 0) { sh[0][w] = v0; sh[1][w] = v1; sh[2][w] = v2; sh[3][w] = v3; }
    __syncthreads();
    if (threadIdx.x < 4) {
        const int q = threadIdx.x;
        part[(size_t)blockIdx.x * 4 + q] = ((sh[q][0] + sh[q][1]) + (sh[q][2] + sh[q][3]));
    }
}

// dS == nullptr: the posterior is the effective prior (frame start): write its
// E-step record and the prior cache; KL terms are zero.  Otherwise: the
// posterior prior0 (+) (S_past + dS), its record, and KL against the cache.
//
// Threads run over record positions p (component k = kperm[p]), so that
// spatial neighbours share a warp.  A component whose frame statistics are
// all exactly zero has q = p bit for bit: when its record already holds p
// (flag cache[33], set by the frame-start call and by any call that wrote p),
// nothing is recomputed and its KL term is exactly zero.
//
// The record (the next E-step's input) is this kernel's job; the KL terms of
// the ELBO are k_mstep_kl_list's, which runs on a second stream beside the
// next E-step: for every recomputed component this kernel leaves in kls[k]
// (kKS doubles) m_q (6), L^-1 of W_q^-1 = L L^T (21, packed lower), alpha_q,
// beta_q, nu_q, ln|W_q^-1|, psi_6(nu_q/2), psi(alpha_q), a flag (1:
// recomputed, 0: q = p) and the frame count Delta N_k; k_mstep_kl_list adds
// the component's KL term as the last double.
constexpr int kKS = 36;

// all 28 frame statistics of component k exactly zero (either sign): an
// integer test of the bit patterns, off the FP64 pipe
__device__ __forceinline__ bool stats_zero(const double *__restrict__ dS, int k)
{
    const longlong2 *v = reinterpret_cast<const longlong2 *>(dS + (size_t)k * 28);   // 224-byte rows
    unsigned long long bits = 0;
#pragma unroll
    for (int f = 0; f < 14; f++) {
        const longlong2 w = v[f];
        bits |= (unsigned long long)w.x | (unsigned long long)w.y;
    }
    return (bits << 1) == 0;
}

// The posterior of component k (record position pos), one thread: record,
// prior cache (dS == nullptr) or KL hand-off (dS), and the next frame's
// prior into the slot cq (nullable).
__device__ __forceinline__ void mstep_thread(const MstepParams &P, const double *__restrict__ m0,
                                             const double *__restrict__ Spast, const double *__restrict__ dS,
                                             int pos, int k, bool zero, double *__restrict__ rec,
                                             float *__restrict__ rec32, double *__restrict__ pc,
                                             double *__restrict__ kls, int *__restrict__ flags,
                                             int *__restrict__ tile_dirty, double *__restrict__ cq)
{
    double *ks = kls + (size_t)k * kKS;
    {
        double st[28], m0k[6], aq;
#pragma unroll
        for (int f = 0; f < 28; f++) st[f] = Spast[(size_t)k * 28 + f] + (dS ? dS[(size_t)k * 28 + f] : 0.0);
#pragma unroll
        for (int i = 0; i < 6; i++) m0k[i] = m0[(size_t)k * 6 + i];
        double bq, nq, mq[6], Aq[21];
        nw_from_stats(P, m0k, st, aq, bq, nq, mq, Aq);
        double Lq[21], Li[21];
        const bool ok = chol6(Aq, Lq);
        if (!ok) atomicCAS(&flags[FL_NONPD], 0, k + 1);
        double dprod = 1.0;   // ln|W^-1| = 2 ln prod_i L_ii
#pragma unroll
        for (int i = 0; i < 6; i++) dprod *= Lq[tri(i, i)];
        const double ldq = 2.0 * log(dprod);
        trinv6(Lq, Li);

        // E-step record: quad = nu |L^-1 (x - m)|^2 = |M (x - m)|^2.
        if (tile_dirty) tile_dirty[pos >> 7] = 1;   // its tensor-core tile must be rebuilt
        const double sn = sqrt(nq);
        double *r = rec + (size_t)pos * VBGS_REC;
        float *r32 = rec32 + (size_t)pos * VBGS_REC;
        const float s2 = 1.2011224087864498f;   // sqrt(log2 e): FP32 record in log2 units
#pragma unroll
        for (int i = 0; i < 6; i++) { r[i] = mq[i]; r32[i] = (float)mq[i]; }
#pragma unroll
        for (int i = 0; i < 6; i++)
#pragma unroll
            for (int j = 0; j <= i; j++) {
                double v = sn * Li[tri(i, j)];
                r[6 + tri(i, j)] = v;
                r32[6 + tri(i, j)] = (float)v * s2;
            }
        const double psi_nu = P.split ? mv_digamma_split(0.5 * nq) : mv_digamma6(0.5 * nq);
        const double psi_a = dg_digamma(aq);
        const double elogdet = psi_nu + 6.0 * kLn2 - ldq;
        const double c = psi_a + 0.5 * elogdet - 3.0 * kLn2Pi - 3.0 / bq;
        r[27] = c;
        r32[27] = (float)(c * 1.4426950408889634);
#pragma unroll
        for (int i = 28; i < 32; i++) { r[i] = 0.0; r32[i] = 0.f; }
        if (P.want_bounds) {
            // Lower bounds (log2 units) of the smallest eigenvalue of the
            // marginal precision of the position block and of the colour
            // block, for the tile-skip bounds of pass 1 and the proposal
            // certificate.  Minimising (x - m)^T nu W (x - m) over the colour
            // part leaves the position part's quadratic form in the inverse
            // of its covariance block (W^-1)_pp / nu, whose smallest
            // eigenvalue is nu / lambda_max((W^-1)_pp); same for colour.
            // (largest eigenvalue of each 3 x 3 block in FP32, inflated by
            // 1e-4 so the bound stays below the exact one)
            // The rest in FP32: a few roundings of 2^-24 each, covered by
            // the 1e-5 deflation.
            const float a0 = (float)Aq[tri(0, 0)], a7 = (float)Aq[tri(1, 1)], a14 = (float)Aq[tri(2, 2)];
            const float a21 = (float)Aq[tri(3, 3)], a28 = (float)Aq[tri(4, 4)], a35 = (float)Aq[tri(5, 5)];
            const float lpp = sym3_max_eig(a0, (float)Aq[tri(1, 0)], (float)Aq[tri(2, 0)], a7, (float)Aq[tri(2, 1)], a14);
            const float lcc = sym3_max_eig(a21, (float)Aq[tri(4, 3)], (float)Aq[tri(5, 3)], a28, (float)Aq[tri(5, 4)], a35);
            const float num = 1.44269504f * (1.f - 1e-5f) * (float)nq;
            r32[28] = num / (lpp * (1.f + 1e-4f));
            r32[29] = num / (lcc * (1.f + 1e-4f));
            // and of the full precision: lambda_min(nu W) >= nu / tr(W^-1)
            r32[30] = num / ((a0 + a7) + (a14 + a21) + (a28 + a35));
        }

        double *cache = pc + (size_t)k * kPC;
        if (!dS) {
            cache[0] = aq; cache[1] = bq; cache[2] = nq;
#pragma unroll
            for (int i = 0; i < 6; i++) cache[3 + i] = mq[i];
            int u = 9;
#pragma unroll
            for (int i = 0; i < 6; i++)
#pragma unroll
                for (int j = i; j < 6; j++, u++) cache[u] = Aq[tri(j, i)];
            cache[30] = ldq;
            cache[33] = 1.0;   // the record holds the effective prior
        } else {
            // the record holds the prior again only if this frame's
            // statistics of the component are all zero
            cache[33] = zero ? 1.0 : 0.0;
#pragma unroll
            for (int i = 0; i < 6; i++) ks[i] = mq[i];
#pragma unroll
            for (int i = 0; i < 6; i++)
#pragma unroll
                for (int j = 0; j <= i; j++) ks[6 + tri(i, j)] = Li[tri(i, j)];
            ks[27] = aq; ks[28] = bq; ks[29] = nq; ks[30] = ldq; ks[31] = psi_nu; ks[32] = psi_a;
            ks[33] = 1.0;
            ks[34] = st[0] - Spast[(size_t)k * 28];
            if (cq) {
                // After the commit S_past + Delta S is bitwise the st above,
                // so q is the next frame's effective prior: its cache entry
                // (the lnGamma terms come from k_mstep_kl_list) and k.
                cq[34] = (double)k;
                cq[0] = aq; cq[1] = bq; cq[2] = nq;
#pragma unroll
                for (int i = 0; i < 6; i++) cq[3 + i] = mq[i];
                int u = 9;
#pragma unroll
                for (int i = 0; i < 6; i++)
#pragma unroll
                    for (int j = i; j < 6; j++, u++) cq[u] = Aq[tri(j, i)];
                cq[30] = ldq;
                cq[33] = 1.0;
            }
        }
    }
}

__global__ void __launch_bounds__(64) k_mstep(MstepParams P, const double *__restrict__ m0,
                                               const double *__restrict__ Spast,
                                               const double *__restrict__ dS,
                                               const int *__restrict__ kperm,
                                               double *__restrict__ rec, float *__restrict__ rec32,
                                               double *__restrict__ pc, double *__restrict__ kls,
                                               int *__restrict__ flags, int *__restrict__ tile_dirty,
                                               double *__restrict__ pcq)
{
    pdl_wait();
    const int pos = blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= P.K) return;
    const int k = kperm ? kperm[pos] : pos;
    bool zero = false;
    if (dS) {
        zero = stats_zero(dS, k);
        if (zero && pc[(size_t)k * kPC + 33] != 0.0) {
            double *ks = kls + (size_t)k * kKS;
            ks[33] = 0.0;
            ks[34] = 0.0;
            return;
        }
    }
    mstep_thread(P, m0, Spast, dS, pos, k, zero, rec, rec32, pc, kls, flags, tile_dirty, nullptr);
}

// ---------------------------------------------------------------------------
// M-step of an iteration (dS given).  Few components change in an iteration
// (a few thousand of 50,000 on the room stream), and an FP64 instruction
// occupies a warp's SM sub-partition for 64 cycles whatever its active lanes,
// so a thread-per-component kernel is bound by the latency of one component's
// serial FP64 chain.  k_mstep_scan compacts the components to recompute into
// a list (the others only hand over q = p); k_mstep_list then computes each
// five listed components with a warp, six lanes each over the rows of its
// 6 x 6 matrices (about 300 FP64 instructions per warp instead of 650 for
// one chain), or, for long lists, one thread per component as k_mstep does.
// k_mstep_list runs one CTA of four warps per SM (its shared-memory request
// keeps a second CTA off the SM), so each sub-partition's FP64 pipe serves
// one warp, and the warps take groups of five from a counter: two busy warps
// never share a pipe while another stands idle.  Every entry is formed by
// the same operations in the same order as in mstep_thread.
constexpr int kListWarpMax = 5 * 1216;   // longest list computed five components to a warp
constexpr int kListSmem = 120 * 1024;    // dynamic shared memory of k_mstep_list: one CTA per SM

__global__ void __launch_bounds__(128) k_mstep_scan(int K, const double *__restrict__ dS, const int *__restrict__ kperm,
                                                    const double *__restrict__ pc, double *__restrict__ kls,
                                                    int *__restrict__ list, int *__restrict__ count)
{
    pdl_wait();
    const int pos = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31;
    bool act = false;
    if (pos < K) {
        const int k = kperm ? kperm[pos] : pos;
        act = !(stats_zero(dS, k) && pc[(size_t)k * kPC + 33] != 0.0);
        if (!act) {   // q = p (also the next frame's prior: its cache entry stays)
            double *ks = kls + (size_t)k * kKS;
            ks[33] = 0.0;
            ks[34] = 0.0;
        }
    }
    const unsigned b = __ballot_sync(0xffffffffu, act);
    if (b) {
        const int leader = __ffs(b) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(count, __popc(b));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (act) list[base + __popc(b & ((1u << lane) - 1u))] = pos;
    }
}

// a ? x : y as a 64-bit bit select the compiler keeps in registers (a chain
// of ternaries over an array is otherwise turned into a local-memory lookup)
__device__ __forceinline__ double sel64(bool a, double x, double y)
{
    unsigned long long r;
    asm("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %3, 0;\n\tselp.b64 %0, %1, %2, p;\n\t}"
        : "=l"(r)
        : "l"(__double_as_longlong(x)), "l"(__double_as_longlong(y)), "r"((unsigned)a));
    return __longlong_as_double((long long)r);
}

// The psi terms of row r of a listed component: psi(alpha_q) on row 0, the
// two halves of psi_6(nu_q / 2) on rows 1, 2 (other rows: unused).
__device__ __forceinline__ double mstep_psi_term(const MstepParams &P, int r, double aq, double nq)
{
    const double xd = r == 1 ? 0.5 * nq - 0.5 * 0 : r == 2 ? 0.5 * nq - 0.5 * 1 : aq;
    const double yd = dg_digamma(xd);
    return r == 0    ? yd
           : !P.split ? 3.0 * yd - (3.0 * xd - 5.0) / ((xd - 1.0) * (xd - 2.0))
           : r == 1   ? 4.0 * yd - 2.0 / (xd - 1.0)   // mv_digamma_split's two parts
                      : 2.0 * yd;
}

// Two warps on different SM sub-partitions sharing one group of components
// (named barrier `id`, 64 threads).
__device__ __forceinline__ void pair_sync(int id) { asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory"); }

// Listed components, five to a warp: lanes 6g..6g+5 hold rows r = 0..5 of
// component g's matrices (lanes 30, 31 idle).  w0r[j] = W0^-1 at
// (min(r, j), max(r, j)), as nw_from_stats reads it.  The inverse L^-1 is kept
// by distance from the diagonal (Lid[s] = (L^-1)[r][r - s]) so that every
// register index stays a compile-time constant.
__device__ __forceinline__ void mstep_group(const MstepParams &P, const double w0r[6], int r, int gb, bool gv,
                                            const double *__restrict__ m0, const double *__restrict__ Spast,
                                            const double *__restrict__ dS, int pos, int k, double *__restrict__ rec,
                                            float *__restrict__ rec32, double *__restrict__ pc,
                                            double *__restrict__ kls, int *__restrict__ flags,
                                            int *__restrict__ tile_dirty, double *__restrict__ cq,
                                            const double *term_src, int bar_id)
{
    constexpr unsigned F = 0xffffffffu;
    auto row = [&](double v, int rr) { return __shfl_sync(F, v, (gb + rr) & 31); };
    const double *Sk = Spast + (size_t)k * 28, *dk = dS + (size_t)k * 28;
    // posterior parameters (nw_from_stats, entry by entry)
    const double st0 = Sk[0] + dk[0];
    const double aq = P.alpha0 + st0, bq = P.beta0 + st0, nq = P.nu0 + st0;
    const double ib = 1.0 / bq;
    const double m0r = m0[(size_t)k * 6 + r];
    const double mr = (P.beta0 * m0r + (Sk[1 + r] + dk[1 + r])) * ib;
    double A[6];   // row r of W_q^-1
#pragma unroll
    for (int j = 0; j < 6; j++) {
        const double mj = row(mr, j), m0j = row(m0r, j);
        const bool lo = r <= j;   // (r, j) is an upper entry (i = r) or a lower one (i = j)
        const int u = lo ? upper_index(r, j) : upper_index(j, r);
        const double mi_ = lo ? mr : mj, mj_ = lo ? mj : mr, m0i_ = lo ? m0r : m0j, m0j_ = lo ? m0j : m0r;
        A[j] = (P.split && ((r < 3) != (j < 3))) ? 0.0 : w0r[j] + (Sk[u] + dk[u]) + P.beta0 * m0i_ * m0j_ - bq * mi_ * mj_;
    }
    // Cholesky by columns (chol6_col's operations and order); row r in Lr
    double Lr[6];
    bool ok = true;
#pragma unroll
    for (int J = 0; J < 6; J++) {
        double t = A[J];
#pragma unroll
        for (int kk = 0; kk < J; kk++) t -= Lr[kk] * row(Lr[kk], J);
        const double dv = row(t, J);
        ok = ok && (dv > 0.0);
        const double d = fmax(dv, 1e-300);
        const double inv = rsqrt(d);
        Lr[J] = (r >= J) ? ((r == J) ? d : t) * inv : 0.0;
    }
    if (gv && r == 0 && !ok) atomicCAS(&flags[FL_NONPD], 0, k + 1);
    double dprod = 1.0;   // ln|W^-1| = 2 ln prod_i L_ii
#pragma unroll
    for (int i = 0; i < 6; i++) dprod *= row(Lr[i], i);
    const double ldq = 2.0 * log(dprod);
    // L^-1 (trinv6's operations and order), by distance from the diagonal
    double Ld[6], Lid[6];
#pragma unroll
    for (int sd = 0; sd < 6; sd++) {
        double v = 0.0;
#pragma unroll
        for (int kk = 0; kk < 6; kk++) v = sel64(kk == r - sd, Lr[kk], v);
        Ld[sd] = v;
        Lid[sd] = 0.0;
    }
    Lid[0] = 1.0 / Ld[0];
#pragma unroll
    for (int d = 1; d < 6; d++) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < d; q++) {
            // entry (r, r - d): L[r][k] (own, k = r - d + q) times (L^-1)[k][r - d] (row k, distance q)
            const int src = r - d + q;
            t += Ld[d - q] * __shfl_sync(F, Lid[q], (gb + (src > 0 ? src : 0)) & 31);
        }
        if (r >= d) Lid[d] = -t * Lid[0];
    }
    // the psi terms: from the partner warp (term_src, after the pair's
    // barrier) or computed here
    double term;
    if (term_src) {
        pair_sync(bar_id);
        term = term_src[threadIdx.x & 31];
    } else {
        term = mstep_psi_term(P, r, aq, nq);
    }
    const double psi_a = row(term, 0);
    double psi_nu = 0.0;
    psi_nu += row(term, 1);
    psi_nu += row(term, 2);
    const double elogdet = psi_nu + 6.0 * kLn2 - ldq;
    const double c = psi_a + 0.5 * elogdet - 3.0 * kLn2Pi - 3.0 / bq;
    // eigenvalue bounds: position block on row 0, colour block on row 1
    const double p00 = row(A[0], 0), p01 = row(A[0], 1), p02 = row(A[0], 2);
    const double p11 = row(A[1], 1), p12 = row(A[1], 2), p22 = row(A[2], 2);
    const double c00 = row(A[3], 3), c01 = row(A[3], 4), c02 = row(A[3], 5);
    const double c11 = row(A[4], 4), c12 = row(A[4], 5), c22 = row(A[5], 5);
    const bool colr = r == 1;
    const float eig = sym3_max_eig((float)(colr ? c00 : p00), (float)(colr ? c01 : p01), (float)(colr ? c02 : p02),
                                   (float)(colr ? c11 : p11), (float)(colr ? c12 : p12), (float)(colr ? c22 : p22));
    const float lpp = (float)__shfl_sync(F, eig, gb & 31), lcc = (float)__shfl_sync(F, eig, (gb + 1) & 31);
    const float trw = ((float)p00 + (float)p11) + ((float)p22 + (float)c00) + ((float)c11 + (float)c22);
    if (!gv) return;
    // E-step record
    const double sn = sqrt(nq);
    double *rr = rec + (size_t)pos * VBGS_REC;
    float *r32 = rec32 + (size_t)pos * VBGS_REC;
    const float s2f = 1.2011224087864498f;   // sqrt(log2 e): FP32 record in log2 units
    rr[r] = mr;
    r32[r] = (float)mr;
    double *ks = kls + (size_t)k * kKS;
    ks[r] = mr;
#pragma unroll
    for (int sd = 0; sd < 6; sd++)
        if (sd <= r) {
            const int e = tri(r, r - sd);
            const double v = sn * Lid[sd];
            rr[6 + e] = v;
            r32[6 + e] = (float)v * s2f;
            ks[6 + e] = Lid[sd];
        }
    if (r == 0) {
        if (tile_dirty) tile_dirty[pos >> 7] = 1;
        rr[27] = c;
        r32[27] = (float)(c * 1.4426950408889634);
#pragma unroll
        for (int i = 28; i < 32; i++) { rr[i] = 0.0; r32[i] = 0.f; }
        if (P.want_bounds) {
            const float num = 1.44269504f * (1.f - 1e-5f) * (float)nq;
            r32[28] = num / (lpp * (1.f + 1e-4f));
            r32[29] = num / (lcc * (1.f + 1e-4f));
            r32[30] = num / trw;
        }
        // KL hand-off and the "record holds the prior" flag
        pc[(size_t)k * kPC + 33] = stats_zero(dS, k) ? 1.0 : 0.0;
        ks[27] = aq; ks[28] = bq; ks[29] = nq; ks[30] = ldq; ks[31] = psi_nu; ks[32] = psi_a;
        ks[33] = 1.0;
        ks[34] = st0 - Sk[0];
    }
    if (cq) {   // the next frame's prior (lnGamma terms from k_mstep_kl_list) and k
        if (r == 0) { cq[0] = aq; cq[1] = bq; cq[2] = nq; cq[30] = ldq; cq[33] = 1.0; cq[34] = (double)k; }
        cq[3 + r] = mr;
#pragma unroll
        for (int j = 0; j < 6; j++)
            if (j >= r) cq[9 + upper_index(r, j) - 7] = A[j];
    }
}

// pcq (nullable): slot e of the list receives the next frame's prior of
// entry e's component (k_mstep_kl_list adds its lnGamma terms).
__global__ void __launch_bounds__(128) k_mstep_list(MstepParams P, const double *__restrict__ m0,
                                                    const double *__restrict__ Spast, const double *__restrict__ dS,
                                                    const int *__restrict__ kperm, const int *__restrict__ list,
                                                    const int *__restrict__ count, double *__restrict__ rec,
                                                    float *__restrict__ rec32, double *__restrict__ pc,
                                                    double *__restrict__ kls, int *__restrict__ flags,
                                                    int *__restrict__ tile_dirty, double *__restrict__ pcq)
{
    pdl_wait();
    const int n = *count;
    if (n <= kListWarpMax) {
        const int lane = threadIdx.x & 31, g = lane / 6, r = lane - 6 * (lane / 6);
        const int rr = g < 5 ? r : 0;
        double w0r[6];   // W0^-1 at (min(rr, j), max(rr, j)), selected without indexing the parameter array
#pragma unroll
        for (int j = 0; j < 6; j++) {
            const int idx = rr <= j ? rr * 6 + j : j * 6 + rr;
            double w = 0.0;
#pragma unroll
            for (int q = 0; q < 36; q++) w = sel64(q == idx, P.W0inv[q], w);
            w0r[j] = w;
        }
        int *next = const_cast<int *>(count) + 1;   // groups handed out (zeroed with the count)
        // Few groups (at most one per warp pair): each pair of warps (on two
        // SM sub-partitions) shares a group, the odd warp computing its psi
        // terms beside the even warp's Cholesky chain.  Otherwise each warp
        // computes whole groups.
        const int pairs = (int)gridDim.x * ((int)blockDim.x / 64);
        if (n <= 5 * pairs) {
            __shared__ int e0_sh[2];
            __shared__ double term_sh[2][32];
            const int w = threadIdx.x >> 5, pr = w >> 1, role = w & 1;
            for (;;) {
                if (role == 0) {
                    int e0 = 0;
                    if (lane == 0) e0 = atomicAdd(next, 5);
                    e0 = __shfl_sync(0xffffffffu, e0, 0);
                    if (lane == 0) e0_sh[pr] = e0;
                }
                pair_sync(1 + pr);
                const int e0 = e0_sh[pr];
                if (e0 >= n) break;   // both warps
                const int e = e0 + g;
                const bool gv = g < 5 && e < n;
                const int pos = list[gv ? e : e0];
                const int k = kperm ? kperm[pos] : pos;
                if (role == 1) {
                    const double st0 = Spast[(size_t)k * 28] + dS[(size_t)k * 28];
                    term_sh[pr][lane] = mstep_psi_term(P, rr, P.alpha0 + st0, P.nu0 + st0);
                    pair_sync(1 + pr);
                } else {
                    mstep_group(P, w0r, rr, 6 * g, gv, m0, Spast, dS, pos, k, rec, rec32, pc, kls, flags, tile_dirty,
                                pcq ? pcq + (size_t)e * kPC : nullptr, term_sh[pr], 1 + pr);
                }
            }
        } else {
            for (;;) {
                int e0 = 0;
                if (lane == 0) e0 = atomicAdd(next, 5);
                e0 = __shfl_sync(0xffffffffu, e0, 0);
                if (e0 >= n) break;   // warp-uniform
                const int e = e0 + g;
                const bool gv = g < 5 && e < n;
                const int pos = list[gv ? e : e0];
                const int k = kperm ? kperm[pos] : pos;
                mstep_group(P, w0r, rr, 6 * g, gv, m0, Spast, dS, pos, k, rec, rec32, pc, kls, flags, tile_dirty,
                            pcq ? pcq + (size_t)e * kPC : nullptr, nullptr, 0);
            }
        }
    } else {
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
            const int pos = list[e];
            const int k = kperm ? kperm[pos] : pos;
            mstep_thread(P, m0, Spast, dS, pos, k, stats_zero(dS, k), rec, rec32, pc, kls, flags, tile_dirty,
                         pcq ? pcq + (size_t)e * kPC : nullptr);
        }
    }
}

// The next frame's prior from the slots of the previous frame's last
// M-step: pc[k] = slot for each listed component (the others kept q = p).
__global__ void k_apply_next(const int *__restrict__ count, const double *__restrict__ slots, double *__restrict__ pc)
{
    pdl_wait();
    const int n = *count;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * 34; i += gridDim.x * blockDim.x) {
        const int e = i / 34, f = i - e * 34;
        const int k = (int)slots[(size_t)e * kPC + 34];
        pc[(size_t)k * kPC + f] = slots[(size_t)e * kPC + f];
    }
}

// Frame start (second stream): the lnGamma terms of the effective prior's
// cache; q = p, so KL = 0.  Block sums of (0, alpha_p, alpha_p, 0) in
// position order.
__global__ void __launch_bounds__(128) k_mstep_kl_prior(int K, bool split, const int *__restrict__ kperm,
                                                        double *__restrict__ pc, double *__restrict__ bpart)
{
    const int pos = blockIdx.x * blockDim.x + threadIdx.x;
    double a = 0.0;
    if (pos < K) {
        double *cache = pc + (size_t)(kperm ? kperm[pos] : pos) * kPC;
        a = cache[0];
        cache[31] = split ? mv_lgamma_split(0.5 * cache[2]) : mv_lgamma6(0.5 * cache[2]);
        cache[32] = lgamma(a);
    }
    block_sums4(0.0, a, a, 0.0, bpart);
}

constexpr int kKlBlocks = 304;   // 1,216 warps: a list of up to 4,864 components in one pass

// KL(NW_q || NW_p) plus the per-component part of KL(Dir(alpha_q) ||
// Dir(alpha_p)) of every listed component (second stream, beside the next
// E-step), from kls and the cache; the psi(sum) and lnGamma(sum) terms of the
// Dirichlet part are added after the cross-component sums.  Eight lanes to a
// component, four components to a warp: lanes r = 0..5 take row r of
// |L^-1 (m_q - m_p)|^2 and of tr(W_p^-1 W_q); lanes 0, 1 and 2 take one
// lnGamma and one log each (the two half-steps of ln Gamma_6(nu_q / 2), then
// ln Gamma(alpha_q) beside ln(beta_q / beta_p)).  An FP64 instruction costs a
// warp the same whatever its active lanes, so spreading the terms over lanes
// shortens the chain each warp issues.  Leaves the KL term in ks[35] and the
// next frame's lnGamma terms in slot e of pcq (nullable).  Split model: the
// two blocks share beta and nu and their matrices are block diagonal, so the
// sum of their two Normal-Wishart KL terms is this form with 2 psi_3 and
// 2 ln Gamma_3 in place of psi_6 and ln Gamma_6.
__global__ void __launch_bounds__(128) k_mstep_kl_list(bool split, const int *__restrict__ kperm, const int *__restrict__ list,
                                                       const int *__restrict__ count, const double *__restrict__ pc,
                                                       double *__restrict__ kls, double *__restrict__ pcq)
{
    const int n = *count;
    const unsigned F = 0xffffffffu;
    const int lane = threadIdx.x & 31, g = lane >> 3, r = lane & 7, gb = lane & ~7;
    const int rr = r < 6 ? r : 5;   // lanes 6, 7 repeat row 5 and are left out of the sums
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int e0 = gw * 4; e0 < n; e0 += nw * 4) {   // warp-uniform
        const int e = e0 + g;
        const bool gv = e < n;   // an empty group repeats entry e0 and writes nothing
        const int pos = list[gv ? e : e0];
        const double *cache = pc + (size_t)(kperm ? kperm[pos] : pos) * kPC;
        double *ks = kls + (size_t)(kperm ? kperm[pos] : pos) * kKS;
        const double *Li = ks + 6;   // L^-1, packed lower
        double d[6];
#pragma unroll
        for (int j = 0; j < 6; j++) d[j] = ks[j] - cache[3 + j];
        // row rr of L^-1 (m_q - m_p)
        double t = 0.0;
#pragma unroll
        for (int j = 0; j < 6; j++)
            if (j <= rr) t += Li[tri(rr, j)] * d[j];
        // row rr of sum_ij (W_p^-1)_ij (W_q)_ij, W_q = L^-T L^-1:
        // (W_q)_ij = sum_{l >= max(i, j)} (L^-1)_li (L^-1)_lj, W_p^-1 upper in the cache
        double tr = 0.0;
#pragma unroll
        for (int j = 0; j < 6; j++)
            if (j >= rr) {
                double w = 0.0;
#pragma unroll
                for (int l = j; l < 6; l++) w += Li[tri(l, rr)] * Li[tri(l, j)];
                tr += (rr == j ? 1.0 : 2.0) * cache[2 + upper_index(rr, j)] * w;
            }
        double maha = r < 6 ? t * t : 0.0;
        tr = r < 6 ? tr : 0.0;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            maha += __shfl_xor_sync(F, maha, o);
            tr += __shfl_xor_sync(F, tr, o);
        }
        const double aq = ks[27], bq = ks[28], nq = ks[29], ldq = ks[30], psi_nu = ks[31], psi_a = ks[32];
        const double ap = cache[0], bp = cache[1], np = cache[2], ldp = cache[30];
        const double x = 0.5 * nq - 0.5 * (r & 1);
        const double y = r < 2 ? x : r == 2 ? aq : 2.0;
        const double z = r < 2 ? (split ? (r == 0 ? x - 1.0 : 1.0) : (x - 1.0) * (x - 1.0) * (x - 2.0))
                         : r == 2 ? bq / bp : 1.0;
        const double lg = lgamma(y), lz = log(z);
        const double lg0 = __shfl_sync(F, lg, gb), lz0 = __shfl_sync(F, lz, gb);
        const double lg1 = __shfl_sync(F, lg, gb + 1), lz1 = __shfl_sync(F, lz, gb + 1);
        const double lgaq = __shfl_sync(F, lg, gb + 2), lbq = __shfl_sync(F, lz, gb + 2);
        double lg6q;   // ln Gamma_6(nu_q / 2) as mv_lgamma6 sums it (split model: mv_lgamma_split)
        if (split) {
            lg6q = 3.0 * kLnPi;
            lg6q += 4.0 * lg0 - 2.0 * lz0;
            lg6q += 2.0 * lg1;
        } else {
            lg6q = 7.5 * kLnPi;
            lg6q += 3.0 * lg0 - lz0;
            lg6q += 3.0 * lg1 - lz1;
        }
        double kl = 0.5 * (6.0 * bp / bq - 6.0 + bp * nq * maha + 6.0 * lbq);
        kl += 0.5 * (nq - np) * psi_nu - 3.0 * nq + 0.5 * nq * tr + 0.5 * np * (ldq - ldp) + cache[31] - lg6q;
        kl += -lgaq + cache[32] + (aq - ap) * psi_a;
        if (gv && r == 0 && ks[33] != 0.0) {
            ks[35] = kl;
            if (pcq) {
                pcq[(size_t)e * kPC + 31] = lg6q;
                pcq[(size_t)e * kPC + 32] = lgaq;
            }
        }
    }
}

// Block sums of (KL, alpha_q, alpha_p, Delta N) in position order: the
// listed components' terms from kls, alpha_q = alpha_p and no KL elsewhere.
__global__ void __launch_bounds__(128) k_mstep_kl_sum(int K, const int *__restrict__ kperm,
                                                      const double *__restrict__ pc, const double *__restrict__ kls,
                                                      double *__restrict__ bpart)
{
    pdl_wait();
    const int pos = blockIdx.x * blockDim.x + threadIdx.x;
    double kl = 0.0, aq = 0.0, ap = 0.0, dn = 0.0;
    if (pos < K) {
        const int k = kperm ? kperm[pos] : pos;
        const double *ks = kls + (size_t)k * kKS;
        ap = pc[(size_t)k * kPC];
        aq = ap;
        if (ks[33] != 0.0) {
            kl = ks[35];
            aq = ks[27];
            dn = ks[34];
        }
    }
    block_sums4(kl, aq, ap, dn, bpart);
}

// One block of four warps: fixed-order sums of the per-block partials, then
// the Dirichlet terms that need the totals, psi(sum alpha_q), lnGamma(sum
// alpha_q) and lnGamma(sum alpha_p) each on its own warp (so on its own SM
// sub-partition, side by side).  scal[SC_PSI_AHAT] = psi(sum alpha_q);
// scal[SC_KL_TOTAL] = sum_k KL_NW,k + KL_Dir.
__global__ void __launch_bounds__(128) k_mstep_finalize(const double *__restrict__ bpart, int nblocks,
                                                        double *__restrict__ scal)
{
    pdl_wait();
    __shared__ double sh[4][4];
    __shared__ double tf[3];
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        s0 += bpart[(size_t)b * 4]; s1 += bpart[(size_t)b * 4 + 1];
        s2 += bpart[(size_t)b * 4 + 2]; s3 += bpart[(size_t)b * 4 + 3];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
        s3 += __shfl_down_sync(0xffffffffu, s3, o);
    }
    if (lane == 0) { sh[0][w] = s0; sh[1][w] = s1; sh[2][w] = s2; sh[3][w] = s3; }
    __syncthreads();
    const double t1 = (sh[1][0] + sh[1][1]) + (sh[1][2] + sh[1][3]);
    const double t2 = (sh[2][0] + sh[2][1]) + (sh[2][2] + sh[2][3]);
    if (lane == 0) {   // warp-uniform branches
        if (w == 0) tf[0] = dg_digamma(t1);
        else if (w == 1) tf[1] = lgamma(t1);
        else if (w == 2) tf[2] = lgamma(t2);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double t0 = (sh[0][0] + sh[0][1]) + (sh[0][2] + sh[0][3]);
        const double t3 = (sh[3][0] + sh[3][1]) + (sh[3][2] + sh[3][3]);
        const double psi = tf[0];
        scal[SC_PSI_AHAT] = psi;
        scal[SC_KL_TOTAL] = t0 + tf[1] - tf[2] - psi * t3;
    }
}

// S_past += Delta S, skipped when anything of the frame failed: a bad point,
// a posterior update, a bounded wait or a consistency check.
__global__ void k_commit(double *__restrict__ Spast, const double *__restrict__ dS, size_t n,
                         const int *__restrict__ flags)
{
    pdl_wait();
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flags[FL_NONPD] == 0 && flags[FL_BAD_POINT] == 0 && flags[FL_TIMEOUT] == 0 &&
        flags[FL_CHECK] == 0)
        Spast[i] += dS[i];
}

// Consistency checks of a frame (one block): every statistic and lse_n
// finite, counts non-negative, and the two conservation laws of Eq. 3 --
// sum_k N_k = N (responsibilities sum to one per point) and
// sum_k S1_k = sum_n x_n -- within a relative tolerance.
__global__ void __launch_bounds__(1024) k_check_frame(const double *__restrict__ dS, int K,
                                                      const double *__restrict__ X, int64_t N,
                                                      const double *__restrict__ lse, double tol,
                                                      int *__restrict__ flags)
{
    pdl_wait();
    __shared__ double sh[32][14];
    __shared__ int bad_sh;
    if (threadIdx.x == 0) bad_sh = 0;
    __syncthreads();
    double acc[14];
#pragma unroll
    for (int q = 0; q < 14; q++) acc[q] = 0.0;
    int bad = 0;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const double *r = dS + (size_t)k * 28;
        for (int q = 0; q < 28; q++) bad |= !isfinite(r[q]);
        bad |= r[0] < 0.0;
#pragma unroll
        for (int q = 0; q < 7; q++) acc[q] += r[q];
    }
    for (int64_t n = threadIdx.x; n < N; n += blockDim.x) {
        const double *x = X + (size_t)n * VBGS_XS;
        acc[7] += 1.0;
#pragma unroll
        for (int q = 0; q < 6; q++) acc[8 + q] += x[q];
        if (lse) bad |= !isfinite(lse[n]);
    }
    if (bad) atomicOr(&bad_sh, 1);
#pragma unroll
    for (int q = 0; q < 14; q++) {
        double v = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][q] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[14];
        for (int q = 0; q < 14; q++) {
            t[q] = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) t[q] += sh[w][q];
        }
        bool ok = !bad_sh && fabs(t[0] - t[7]) <= tol * fmax(t[7], 1.0);
        double d2 = 0.0, n2 = 0.0;
        for (int q = 0; q < 6; q++) {
            d2 += (t[1 + q] - t[8 + q]) * (t[1 + q] - t[8 + q]);
            n2 += t[8 + q] * t[8 + q];
        }
        ok = ok && isfinite(d2) && sqrt(d2) <= tol * fmax(sqrt(n2), 1.0);
        if (!ok) flags[FL_CHECK] = 1;
    }
}

__global__ void k_elbo(double *__restrict__ scal, double N, double *__restrict__ out)
{
    pdl_wait();
    *out = scal[SC_SUM_LSE] - N * scal[SC_PSI_AHAT] - scal[SC_KL_TOTAL];
    scal[SC_PSI_ESTEP] = scal[SC_PSI_AHAT];
}

// Copy N x 6 points into the N x 8 staging layout and flag non-finite input.
__global__ void k_stage(const double *__restrict__ src, int64_t N, double *__restrict__ X,
                        int *__restrict__ flags)
{
    pdl_wait();
    int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    bool bad = false;
#pragma unroll
    for (int i = 0; i < 6; i++) {
        double v = src[n * 6 + i];
        bad |= !isfinite(v);
        X[n * VBGS_XS + i] = v;
    }
    X[n * VBGS_XS + 6] = 0.0;
    X[n * VBGS_XS + 7] = 0.0;
    if (bad) atomicOr(&flags[FL_BAD_POINT], 1);
}

} // namespace

size_t mstep_prior_cache_doubles(int K) { return (size_t)K * kPC; }

size_t mstep_cache_doubles(int K)
{
    // cache, block sums, KL inputs, then the list of components to recompute
    // (K ints, its count and the list kernel's group counter)
    return (size_t)K * kPC + (size_t)((K + 127) / 128) * 4 + (size_t)K * kKS + (size_t)(K + 4) / 2;
}

MstepList mstep_list_view(double *cache, int K)
{
    const int nb = (K + 127) / 128;
    double *kls = cache + (size_t)K * kPC + (size_t)nb * 4;
    int *list = reinterpret_cast<int *>(kls + (size_t)K * kKS);
    return MstepList{cache + 33, kPC, kls + 33, kKS, list, list + K};
}

int launch_mstep(const MstepParams &P, const double *m0, const double *Spast, const double *dS,
                 const int *kperm, double *rec, float *rec32, double *cache, int *flags, double *scal,
                 int *tile_dirty, double *cache_next, cudaStream_t st, cudaStream_t side, cudaEvent_t ev_fork,
                 cudaEvent_t ev_join, Prof *pf, bool listed)
{
    if (!dS) cache_next = nullptr;
    const int K = P.K;
    const int nb = (K + 127) / 128;
    double *bpart = cache + (size_t)K * kPC;
    double *kls = bpart + (size_t)nb * 4;
    int launches = 3;
    if (!dS) {
        pf->begin(VBGS_PROF_MSTEP, st);
        // 64 threads a block: the per-component work is long, so smaller
        // blocks spread it over more SMs
        launch_pdl(k_mstep, (K + 63) / 64, 64, 0, st, P, m0, Spast, dS, kperm, rec, rec32, cache, kls, flags,
                   tile_dirty, cache_next);
        pf->end(st);
    } else {
        int *list = reinterpret_cast<int *>(kls + (size_t)K * kKS), *count = list + K;
        if (!listed) {
            if (cudaMemsetAsync(count, 0, 2 * sizeof(int), st) != cudaSuccess) return -1;
            pf->begin(VBGS_PROF_MSTEP, st);
            launch_pdl(k_mstep_scan, (K + 127) / 128, 128, 0, st, K, dS, kperm, cache, kls, list, count);
            pf->end(st);
        }
        pf->begin(VBGS_PROF_MSTEP, st);
        static bool attr_set = false;
        if (!attr_set) {
            if (cudaFuncSetAttribute(k_mstep_list, cudaFuncAttributeMaxDynamicSharedMemorySize, kListSmem) !=
                cudaSuccess)
                return -1;
            attr_set = true;
        }
        launch_pdl(k_mstep_list, std::max(1, P.num_sms), 128, kListSmem, st, P, m0, Spast, dS, kperm, list, count,
                   rec, rec32, cache, kls, flags, tile_dirty, cache_next);
        pf->end(st);
        launches = listed ? 3 : 4;
    }
    // KL terms and their sums beside the next E-step
    if (cudaEventRecord(ev_fork, st) != cudaSuccess || cudaStreamWaitEvent(side, ev_fork, 0) != cudaSuccess) return -1;
    if (!dS) {
        pf->begin(VBGS_PROF_KL, side);
        k_mstep_kl_prior<<<nb, 128, 0, side>>>(K, P.split != 0, kperm, cache, bpart);
        pf->end(side);
    } else {
        const int *list = reinterpret_cast<const int *>(kls + (size_t)K * kKS), *count = list + K;
        pf->begin(VBGS_PROF_KL, side);
        k_mstep_kl_list<<<kKlBlocks, 128, 0, side>>>(P.split != 0, kperm, list, count, cache, kls, cache_next);
        pf->end(side);
        pf->begin(VBGS_PROF_KL, side);
        launch_pdl(k_mstep_kl_sum, nb, 128, 0, side, K, kperm, (const double *)cache, (const double *)kls, bpart);
        pf->end(side);
        launches++;
    }
    pf->begin(VBGS_PROF_KL, side);
    launch_pdl(k_mstep_finalize, 1, 128, 0, side, (const double *)bpart, nb, scal);
    pf->end(side);
    if (cudaEventRecord(ev_join, side) != cudaSuccess) return -1;
    return cudaGetLastError() == cudaSuccess ? launches : -1;
}

// Records to the positions of a new component order: dst[p] = src[kinv_old[kperm[p]]].
__global__ void k_move_records(const int *__restrict__ kperm, const int *__restrict__ kinv_old, int K,
                               const double *__restrict__ rec, const float *__restrict__ rec32,
                               double *__restrict__ rec_dst, float *__restrict__ rec32_dst)
{
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)K * 16) return;
    const int p = (int)(i >> 4), q = (int)(i & 15);   // 16-byte pieces: 16 of the FP64 record, 8 of the FP32
    const int po = kinv_old[kperm[p]];
    reinterpret_cast<double2 *>(rec_dst + (size_t)p * VBGS_REC)[q] =
        reinterpret_cast<const double2 *>(rec + (size_t)po * VBGS_REC)[q];
    if (q < 8)
        reinterpret_cast<float4 *>(rec32_dst + (size_t)p * VBGS_REC)[q] =
            reinterpret_cast<const float4 *>(rec32 + (size_t)po * VBGS_REC)[q];
}

int launch_apply_next(int K, const double *slots, double *cache, cudaStream_t st, Prof *pf)
{
    const int nb = (K + 127) / 128;
    const int *count = reinterpret_cast<const int *>(cache + (size_t)K * kPC + (size_t)nb * 4 + (size_t)K * kKS) + K;
    pf->begin(VBGS_PROF_MSTEP, st);
    launch_pdl(k_apply_next, 152 * 4, 256, 0, st, count, slots, cache);
    pf->end(st);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_move_records(const int *kperm, const int *kinv_old, int K, const double *rec, const float *rec32,
                        double *rec_dst, float *rec32_dst, cudaStream_t st, Prof *pf)
{
    pf->begin(VBGS_PROF_MSTEP, st);
    launch_pdl(k_move_records, (unsigned)(((int64_t)K * 16 + 255) / 256), 256, 0, st, kperm, kinv_old, K, rec, rec32,
               rec_dst, rec32_dst);
    pf->end(st);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_commit(double *Spast, const double *dS, int K, const int *flags, cudaStream_t st, Prof *pf)
{
    size_t n = (size_t)K * 28;
    pf->begin(VBGS_PROF_MISC, st);
    launch_pdl(k_commit, (unsigned)((n + 255) / 256), 256, 0, st, Spast, dS, n, flags);
    pf->end(st);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_check_frame(const double *dS, int K, const double *X, int64_t N, const double *lse, double tol,
                       int *flags, cudaStream_t st, Prof *pf)
{
    pf->begin(VBGS_PROF_MISC, st);
    launch_pdl(k_check_frame, 1, 1024, 0, st, dS, K, X, N, lse, tol, flags);
    pf->end(st);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_elbo(double *scal, int64_t N, double *elbo_out, cudaStream_t st, Prof *pf)
{
    pf->begin(VBGS_PROF_MISC, st);
    launch_pdl(k_elbo, 1, 1, 0, st, scal, (double)N, elbo_out);
    pf->end(st);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_stage_points(const double *src, int64_t N, double *X, int *flags, cudaStream_t st, Prof *pf)
{
    if (N <= 0) return 0;
    pf->begin(VBGS_PROF_MISC, st);
    launch_pdl(k_stage, (unsigned)((N + 255) / 256), 256, 0, st, src, N, X, flags);
    pf->end(st);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

} // namespace vbgs
