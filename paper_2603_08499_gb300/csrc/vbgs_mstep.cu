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

namespace vbgs {

namespace {

constexpr double kLn2 = 0.69314718055994530942;
constexpr double kLn2Pi = 1.8378770664093454836;
constexpr double kLnPi = 1.1447298858494001741;

// Digamma for x > 0: raise x to >= 10 with psi(x) = psi(x+1) - 1/x, then the
// asymptotic expansion ln x - 1/(2x) - sum_k B_2k / (2k x^2k) through B_16.
__device__ double dg_digamma(double x)
{
    double shift = 0.0;
    while (x < 10.0) { shift += 1.0 / x; x += 1.0; }
    const double t = 1.0 / (x * x);
    // B2/2, B4/4, ..., B16/16
    const double c1 = 1.0 / 12.0, c2 = -1.0 / 120.0, c3 = 1.0 / 252.0, c4 = -1.0 / 240.0;
    const double c5 = 1.0 / 132.0, c6 = -691.0 / 32760.0, c7 = 1.0 / 12.0, c8 = -3617.0 / 8160.0;
    double p = c8;
    p = fma(p, t, c7); p = fma(p, t, c6); p = fma(p, t, c5); p = fma(p, t, c4);
    p = fma(p, t, c3); p = fma(p, t, c2); p = fma(p, t, c1);
    return log(x) - 0.5 / x - p * t - shift;
}

// Sum over i = 1..6 of f(a + (1 - i)/2).
__device__ double mv_digamma6(double a)
{
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 6; i++) s += dg_digamma(a - 0.5 * i);
    return s;
}
__device__ double mv_lgamma6(double a)
{
    double s = 7.5 * kLnPi;   // D(D-1)/4 ln pi with D = 6
#pragma unroll
    for (int i = 0; i < 6; i++) s += lgamma(a - 0.5 * i);
    return s;
}

// Posterior parameters from prior and statistics; A is the full symmetric W^-1.
__device__ void nw_from_stats(const MstepParams &P, const double *m0, const double *s,
                              double &alpha, double &beta, double &nu, double m[6], double A[36])
{
    const double N = s[0];
    alpha = P.alpha0 + N;
    beta = P.beta0 + N;
    nu = P.nu0 + N;
#pragma unroll
    for (int i = 0; i < 6; i++) m[i] = (P.beta0 * m0[i] + s[1 + i]) / beta;
#pragma unroll
    for (int i = 0; i < 6; i++)
#pragma unroll
        for (int j = i; j < 6; j++) {
            double v = P.W0inv[i * 6 + j] + s[upper_index(i, j)]
                     + P.beta0 * m0[i] * m0[j] - beta * m[i] * m[j];
            A[i * 6 + j] = v;
            A[j * 6 + i] = v;
        }
}

// In-register Cholesky A = L L^T (L lower, full 6x6 storage); false if not PD.
__device__ bool chol6(const double A[36], double L[36])
{
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 36; i++) L[i] = 0.0;
#pragma unroll
    for (int j = 0; j < 6; j++) {
        double d = A[j * 6 + j];
#pragma unroll
        for (int k = 0; k < j; k++) d -= L[j * 6 + k] * L[j * 6 + k];
        ok = ok && (d > 0.0);
        d = sqrt(fmax(d, 1e-300));
        L[j * 6 + j] = d;
        const double inv = 1.0 / d;
#pragma unroll
        for (int i = j + 1; i < 6; i++) {
            double t = A[i * 6 + j];
#pragma unroll
            for (int k = 0; k < j; k++) t -= L[i * 6 + k] * L[j * 6 + k];
            L[i * 6 + j] = t * inv;
        }
    }
    return ok;
}

// Inverse of a lower-triangular 6x6 matrix (result lower triangular).
__device__ void trinv6(const double L[36], double Li[36])
{
#pragma unroll
    for (int i = 0; i < 36; i++) Li[i] = 0.0;
#pragma unroll
    for (int c = 0; c < 6; c++) {
        Li[c * 6 + c] = 1.0 / L[c * 6 + c];
#pragma unroll
        for (int i = c + 1; i < 6; i++) {
            double t = 0.0;
#pragma unroll
            for (int k = c; k < i; k++) t += L[i * 6 + k] * Li[k * 6 + c];
            Li[i * 6 + c] = -t / L[i * 6 + i];
        }
    }
}

__global__ void __launch_bounds__(128) k_mstep(MstepParams P, const double *__restrict__ m0,
                                               const double *__restrict__ Spast,
                                               const double *__restrict__ dS,
                                               const int *__restrict__ kinv,
                                               double *__restrict__ rec, float *__restrict__ rec32,
                                               double *__restrict__ klk, double *__restrict__ aq_out,
                                               double *__restrict__ ap_out, double *__restrict__ dN_out,
                                               int *__restrict__ flags)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P.K) return;
    double sp[28], st[28], m0k[6];
#pragma unroll
    for (int f = 0; f < 28; f++) {
        sp[f] = Spast[(size_t)k * 28 + f];
        st[f] = sp[f] + (dS ? dS[(size_t)k * 28 + f] : 0.0);
    }
#pragma unroll
    for (int i = 0; i < 6; i++) m0k[i] = m0[(size_t)k * 6 + i];

    double ap, bp, np, mp[6], Ap[36];
    double aq, bq, nq, mq[6], Aq[36];
    nw_from_stats(P, m0k, sp, ap, bp, np, mp, Ap);
    nw_from_stats(P, m0k, st, aq, bq, nq, mq, Aq);

    double Lq[36], Lp[36], Li[36];
    bool ok = chol6(Aq, Lq);
    ok = chol6(Ap, Lp) && ok;
    if (!ok) atomicCAS(&flags[FL_NONPD], 0, k + 1);
    double ldq = 0.0, ldp = 0.0;   // ln|W^-1|
#pragma unroll
    for (int i = 0; i < 6; i++) { ldq += 2.0 * log(Lq[i * 6 + i]); ldp += 2.0 * log(Lp[i * 6 + i]); }
    trinv6(Lq, Li);

    // E-step record: quad = nu |L^-1 (x - m)|^2 = |M (x - m)|^2.
    const double sn = sqrt(nq);
    const size_t pos = kinv ? (size_t)kinv[k] : (size_t)k;   // record position (processing order)
    double *r = rec + pos * VBGS_REC;
    float *r32 = rec32 + pos * VBGS_REC;
    const float s2 = 1.2011224087864498f;   // sqrt(log2 e): FP32 record in log2 units
#pragma unroll
    for (int i = 0; i < 6; i++) { r[i] = mq[i]; r32[i] = (float)mq[i]; }
#pragma unroll
    for (int i = 0; i < 6; i++)
#pragma unroll
        for (int j = 0; j <= i; j++) {
            double v = sn * Li[i * 6 + j];
            r[6 + tri(i, j)] = v;
            r32[6 + tri(i, j)] = (float)v * s2;
        }
    const double elogdet = mv_digamma6(0.5 * nq) + 6.0 * kLn2 - ldq;
    const double c = dg_digamma(aq) + 0.5 * elogdet - 3.0 * kLn2Pi - 3.0 / bq;
    r[27] = c;
    r32[27] = (float)(c * 1.4426950408889634);
#pragma unroll
    for (int i = 28; i < 32; i++) { r[i] = 0.0; r32[i] = 0.f; }

    // KL(NW_q || NW_p).
    double d[6];
#pragma unroll
    for (int i = 0; i < 6; i++) d[i] = mq[i] - mp[i];
    double maha = 0.0;   // (m_q - m_p)^T W_q (m_q - m_p) = |L^-1 (m_q - m_p)|^2
#pragma unroll
    for (int i = 0; i < 6; i++) {
        double t = 0.0;
#pragma unroll
        for (int j = 0; j <= i; j++) t += Li[i * 6 + j] * d[j];
        maha += t * t;
    }
    // tr(W_p^-1 W_q) with W_q = Li^T Li: sum_i (Li Ap Li^T)_ii.
    double tr = 0.0;
#pragma unroll
    for (int i = 0; i < 6; i++) {
#pragma unroll
        for (int l = 0; l < 6; l++) {
            double b = 0.0;
#pragma unroll
            for (int j = 0; j <= i; j++) b += Li[i * 6 + j] * Ap[j * 6 + l];
            if (l <= i) tr += b * Li[i * 6 + l];
        }
    }
    double kl = 0.5 * (6.0 * bp / bq - 6.0 + bp * nq * maha + 6.0 * log(bq / bp));
    kl += 0.5 * (nq - np) * mv_digamma6(0.5 * nq) - 3.0 * nq + 0.5 * nq * tr
        + 0.5 * np * (ldq - ldp) + mv_lgamma6(0.5 * np) - mv_lgamma6(0.5 * nq);
    // Per-component part of KL(Dir(alpha_q) || Dir(alpha_p)); the psi(sum)
    // and lnGamma(sum) terms are added after the cross-component sums.
    kl += -lgamma(aq) + lgamma(ap) + (aq - ap) * dg_digamma(aq);
    klk[k] = kl;
    aq_out[k] = aq;
    ap_out[k] = ap;
    dN_out[k] = st[0] - sp[0];
}

// One block: deterministic fixed-order sums over components, then the
// Dirichlet terms that need the totals.  scal[SC_PSI_AHAT] = psi(sum alpha_q);
// scal[SC_KL_TOTAL] = sum_k KL_NW,k + KL_Dir.
__global__ void __launch_bounds__(1024) k_mstep_finalize(const double *__restrict__ klk,
                                                         const double *__restrict__ aq,
                                                         const double *__restrict__ ap,
                                                         const double *__restrict__ dN, int K,
                                                         double *__restrict__ scal)
{
    __shared__ double sh[4][32];
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        s0 += klk[k]; s1 += aq[k]; s2 += ap[k]; s3 += dN[k];
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
    if (threadIdx.x == 0) {
        double t0 = 0, t1 = 0, t2 = 0, t3 = 0;
        const int nw = blockDim.x >> 5;
        for (int i = 0; i < nw; i++) { t0 += sh[0][i]; t1 += sh[1][i]; t2 += sh[2][i]; t3 += sh[3][i]; }
        const double psi = dg_digamma(t1);
        scal[SC_PSI_AHAT] = psi;
        scal[SC_KL_TOTAL] = t0 + lgamma(t1) - lgamma(t2) - psi * t3;
    }
}

// S_past += Delta S, skipped when the last posterior update failed.
__global__ void k_commit(double *__restrict__ Spast, const double *__restrict__ dS, size_t n,
                         const int *__restrict__ flags)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flags[FL_NONPD] == 0 && flags[FL_BAD_POINT] == 0) Spast[i] += dS[i];
}

__global__ void k_elbo(double *__restrict__ scal, double N, double *__restrict__ out)
{
    *out = scal[SC_SUM_LSE] - N * scal[SC_PSI_AHAT] - scal[SC_KL_TOTAL];
    scal[SC_PSI_ESTEP] = scal[SC_PSI_AHAT];
}

// Copy N x 6 points into the N x 8 staging layout and flag non-finite input.
__global__ void k_stage(const double *__restrict__ src, int64_t N, double *__restrict__ X,
                        int *__restrict__ flags)
{
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

int launch_mstep(const MstepParams &P, const double *m0, const double *Spast, const double *dS,
                 const int *kinv, double *rec, float *rec32, double *klk, double *aq, double *ap,
                 double *dN, int *flags, double *scal, cudaStream_t st, Prof *pf)
{
    const int K = P.K;
    pf->begin(VBGS_PROF_MSTEP, st);
    k_mstep<<<(K + 127) / 128, 128, 0, st>>>(P, m0, Spast, dS, kinv, rec, rec32, klk, aq, ap, dN, flags);
    pf->end(st);
    pf->begin(VBGS_PROF_MSTEP, st);
    k_mstep_finalize<<<1, 1024, 0, st>>>(klk, aq, ap, dN, K, scal);
    pf->end(st);
    return cudaGetLastError() == cudaSuccess ? 2 : -1;
}

int launch_commit(double *Spast, const double *dS, int K, const int *flags, cudaStream_t st, Prof *pf)
{
    size_t n = (size_t)K * 28;
    pf->begin(VBGS_PROF_MISC, st);
    k_commit<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Spast, dS, n, flags);
    pf->end(st);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_elbo(double *scal, int64_t N, double *elbo_out, cudaStream_t st, Prof *pf)
{
    pf->begin(VBGS_PROF_MISC, st);
    k_elbo<<<1, 1, 0, st>>>(scal, (double)N, elbo_out);
    pf->end(st);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_stage_points(const double *src, int64_t N, double *X, int *flags, cudaStream_t st, Prof *pf)
{
    if (N <= 0) return 0;
    pf->begin(VBGS_PROF_MISC, st);
    k_stage<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(src, N, X, flags);
    pf->end(st);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

} // namespace vbgs
