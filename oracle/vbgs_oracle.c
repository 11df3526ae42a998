/*
 * vbgs_oracle.c -- plain, slow FP64 CPU oracle of the VBGS coordinate-ascent
 * (CAVI) update.  TEST INFRASTRUCTURE ONLY: nothing on the product path may
 * call, link or load this file; only tests/, __graft_entry__.smoke() and the
 * CPU-baseline / reference legs of bench.py use it.
 *
 * What it computes (the paper's Section 2.1.2 model and Algorithm 1 `fit`):
 *   - the VBGS mixture: z ~ Cat(pi), pi ~ Dirichlet(alpha0), and per
 *     component a Gaussian over the joint point x = (position, colour) with a
 *     conjugate Normal-Wishart prior on (mu, Lambda) (Sec. 2.1.2, Fig. 3; the
 *     paper's NIW(m, kappa, V, n) written in precision space:
 *     kappa = beta, V = W^-1, n = nu);
 *   - `compute_elbo_delta`: the expected log-likelihood log rho_nk of every
 *     point under every component, its per-point log-sum-exp lse_n and the
 *     responsibilities r_nk = exp(log rho_nk - lse_n) (Alg. 1);
 *   - `sum_stats_over_samples`: Delta S = R^T S_u with per-point unsummed
 *     statistics S_u = phi(x) = [1, x, upper(x x^T)] (Eq. 3);
 *   - `update_from_statistics`: the closed-form conjugate posterior from the
 *     accumulated statistics (Alg. 1), in raw-moment form;
 *   - the ELBO at the optimal q(z):  sum_n lse_n - sum_k KL(NW_k || NW0_k)
 *     - KL(Dir || Dir0).
 * The paper defers these update equations to the original VBGS work; they are
 * the textbook mean-field updates of a Bayesian Gaussian mixture with
 * Normal-Wishart / Dirichlet priors, written here from the mathematics:
 * the expected log-density uses the factored quadratic form
 * (x-m)^T W (x-m) = |L^-1 (x-m)|^2 with W^-1 = L L^T solved by forward
 * substitution per pair (no expansion into features, no precomputed inverse).
 *
 * Statistics layout (F = 1 + D + D(D+1)/2, 28 for D = 6), per component:
 *   [0]              N_k   = sum_n r_nk
 *   [1 .. D]         S1_k  = sum_n r_nk x_n
 *   [1+D .. F-1]     S2_k  = sum_n r_nk x_n x_n^T, upper triangle, row-major
 *                            (0,0),(0,1)..(0,D-1),(1,1)..(D-1,D-1)
 *
 * Parity: every function here is pinned by tests/test_oracle_pins.py against
 * closed forms (K = 1 conjugate posterior and exact log evidence), brute-force
 * enumeration of hard assignments, Monte Carlo expectations drawn with
 * library samplers, invariants and special function tables.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXD 16
static const double OR_PI = 3.14159265358979323846264338327950288;

static int or_F(int D) { return 1 + D + D * (D + 1) / 2; }

/* Digamma psi(x) for x > 0: recurrence psi(x) = psi(x+1) - 1/x up to x >= 12,
 * then the asymptotic series psi(x) ~ ln x - 1/(2x) - sum_k B_2k / (2k x^2k)
 * (Abramowitz & Stegun 6.3.5 and 6.3.18), Bernoulli numbers B2..B14. */
double or_digamma(double x)
{
    double acc = 0.0;
    while (x < 12.0) { acc -= 1.0 / x; x += 1.0; }
    double x2 = 1.0 / (x * x);
    /* B_2k/(2k): 1/12, -1/120, 1/252, -1/240, 1/132, -691/32760, 1/12 */
    double series = x2 * (1.0 / 12 - x2 * (1.0 / 120 - x2 * (1.0 / 252 - x2 * (1.0 / 240
                  - x2 * (1.0 / 132 - x2 * (691.0 / 32760 - x2 * (1.0 / 12)))))));
    return acc + log(x) - 0.5 / x - series;
}

/* ln Gamma_D(a) = D(D-1)/4 ln pi + sum_{i=1..D} ln Gamma(a + (1-i)/2) */
double or_lmvgamma(int D, double a)
{
    double s = 0.25 * D * (D - 1) * log(OR_PI);
    for (int i = 1; i <= D; i++) s += lgamma(a + 0.5 * (1 - i));
    return s;
}

/* psi_D(a) = sum_{i=1..D} psi(a + (1-i)/2) */
static double or_mvdigamma(int D, double a)
{
    double s = 0.0;
    for (int i = 1; i <= D; i++) s += or_digamma(a + 0.5 * (1 - i));
    return s;
}

/* Cholesky A = L L^T of a symmetric positive-definite D x D matrix (row-major,
 * full storage).  Returns 0, or -1 if A is not positive definite. */
static int or_cholesky(int D, const double *A, double *L)
{
    memset(L, 0, sizeof(double) * D * D);
    for (int j = 0; j < D; j++) {
        double s = A[j * D + j];
        for (int k = 0; k < j; k++) s -= L[j * D + k] * L[j * D + k];
        if (!(s > 0.0)) return -1;
        double d = sqrt(s);
        L[j * D + j] = d;
        for (int i = j + 1; i < D; i++) {
            double t = A[i * D + j];
            for (int k = 0; k < j; k++) t -= L[i * D + k] * L[j * D + k];
            L[i * D + j] = t / d;
        }
    }
    return 0;
}

/* Solve L y = b by forward substitution (L lower triangular). */
static void or_forward(int D, const double *L, const double *b, double *y)
{
    for (int i = 0; i < D; i++) {
        double t = b[i];
        for (int k = 0; k < i; k++) t -= L[i * D + k] * y[k];
        y[i] = t / L[i * D + i];
    }
}

/* W = (L L^T)^-1, full D x D, by solving L L^T W = I column by column. */
static void or_inverse_from_chol(int D, const double *L, double *W)
{
    double e[OR_MAXD], y[OR_MAXD], w[OR_MAXD];
    for (int c = 0; c < D; c++) {
        for (int i = 0; i < D; i++) e[i] = (i == c) ? 1.0 : 0.0;
        or_forward(D, L, e, y);
        /* back substitution L^T w = y */
        for (int i = D - 1; i >= 0; i--) {
            double t = y[i];
            for (int k = i + 1; k < D; k++) t -= L[k * D + i] * w[k];
            w[i] = t / L[i * D + i];
        }
        for (int i = 0; i < D; i++) W[i * D + c] = w[i];
    }
}

/*
 * update_from_statistics (Alg. 1): conjugate Normal-Wishart / Dirichlet
 * posterior from total statistics S (K x F), raw-moment form:
 *   alpha = alpha0 + N_k,  beta = beta0 + N_k,  nu = nu0 + N_k,
 *   beta m = beta0 m0_k + S1_k,
 *   W^-1 = W0^-1 + S2_k + beta0 m0_k m0_k^T - beta m m^T.
 * Outputs alpha, beta, nu (K), m (K x D), Winv (K x D x D, full).
 */
void or_mstep(int K, int D, double alpha0, double beta0, double nu0,
              const double *m0, const double *W0inv, const double *S,
              double *alpha, double *beta, double *nu, double *m, double *Winv)
{
    const int F = or_F(D);
    for (int k = 0; k < K; k++) {
        const double *s = S + (size_t)k * F;
        double Nk = s[0];
        alpha[k] = alpha0 + Nk;
        beta[k] = beta0 + Nk;
        nu[k] = nu0 + Nk;
        for (int i = 0; i < D; i++)
            m[(size_t)k * D + i] = (beta0 * m0[(size_t)k * D + i] + s[1 + i]) / beta[k];
        int u = 1 + D;
        for (int i = 0; i < D; i++)
            for (int j = i; j < D; j++, u++) {
                double v = W0inv[i * D + j] + s[u]
                         + beta0 * m0[(size_t)k * D + i] * m0[(size_t)k * D + j]
                         - beta[k] * m[(size_t)k * D + i] * m[(size_t)k * D + j];
                Winv[(size_t)k * D * D + i * D + j] = v;
                Winv[(size_t)k * D * D + j * D + i] = v;
            }
    }
}

/*
 * Per-component expected log-likelihood constant of compute_elbo_delta:
 *   E[ln pi_k] + 1/2 E[ln|Lambda_k|] - D/2 ln 2pi - D/(2 beta_k),
 *   E[ln pi_k] = psi(alpha_k) - psi(sum alpha),
 *   E[ln|Lambda_k|] = psi_D(nu_k/2) + D ln 2 + ln|W_k|.
 * Also returns the Cholesky factor L_k of W_k^-1 (K x D x D).
 * Returns 0, or -(k+1) for the first component whose W^-1 is not PD.
 */
static int or_estep_prepare(int K, int D, const double *alpha, const double *beta,
                            const double *nu, const double *Winv,
                            double *cst, double *Lfac)
{
    double asum = 0.0;
    for (int k = 0; k < K; k++) asum += alpha[k];
    double psi_sum = or_digamma(asum);
    for (int k = 0; k < K; k++) {
        double *L = Lfac + (size_t)k * D * D;
        if (or_cholesky(D, Winv + (size_t)k * D * D, L)) return -(k + 1);
        double logdet_Winv = 0.0;
        for (int i = 0; i < D; i++) logdet_Winv += 2.0 * log(L[i * D + i]);
        double elogdet = or_mvdigamma(D, 0.5 * nu[k]) + D * log(2.0) - logdet_Winv;
        cst[k] = or_digamma(alpha[k]) - psi_sum + 0.5 * elogdet
               - 0.5 * D * log(2.0 * OR_PI) - 0.5 * D / beta[k];
    }
    return 0;
}

/* log rho_nk = cst_k - nu_k/2 (x_n - m_k)^T W_k (x_n - m_k), the quadratic
 * form as |L_k^-1 (x_n - m_k)|^2 by forward substitution. */
static double or_log_rho_one(int D, const double *x, const double *mk, const double *Lk,
                             double nuk, double cstk)
{
    double d[OR_MAXD], y[OR_MAXD];
    for (int i = 0; i < D; i++) d[i] = x[i] - mk[i];
    or_forward(D, Lk, d, y);
    double q = 0.0;
    for (int i = 0; i < D; i++) q += y[i] * y[i];
    return cstk - 0.5 * nuk * q;
}

/* log rho for all pairs (N x K), for small test cases. */
int or_log_rho(int N, int K, int D, const double *X, const double *alpha, const double *beta,
               const double *nu, const double *m, const double *Winv, double *logrho)
{
    double *cst = malloc(sizeof(double) * K);
    double *Lf = malloc(sizeof(double) * (size_t)K * D * D);
    int rc = or_estep_prepare(K, D, alpha, beta, nu, Winv, cst, Lf);
    if (rc == 0)
        for (int n = 0; n < N; n++)
            for (int k = 0; k < K; k++)
                logrho[(size_t)n * K + k] = or_log_rho_one(D, X + (size_t)n * D, m + (size_t)k * D,
                                                           Lf + (size_t)k * D * D, nu[k], cst[k]);
    free(cst); free(Lf);
    return rc;
}

/*
 * compute_elbo_delta + sum_stats_over_samples (Alg. 1, Eq. 3) for one batch:
 *   lse_n = logsumexp_k log rho_nk,  r_nk = exp(log rho_nk - lse_n),
 *   dS_k  = sum_n r_nk phi(x_n),  phi(x) = [1, x, upper(x x^T)].
 * Outputs lse (N), dS (K x F), and R (N x K) when R != NULL.
 * Points are processed in parallel with per-thread statistics buffers that are
 * summed afterwards.
 */
int or_estep_stats(int N, int K, int D, const double *X, const double *alpha,
                   const double *beta, const double *nu, const double *m,
                   const double *Winv, double *lse, double *dS, double *R)
{
    const int F = or_F(D);
    double *cst = malloc(sizeof(double) * K);
    double *Lf = malloc(sizeof(double) * (size_t)K * D * D);
    int rc = or_estep_prepare(K, D, alpha, beta, nu, Winv, cst, Lf);
    if (rc) { free(cst); free(Lf); return rc; }
    memset(dS, 0, sizeof(double) * (size_t)K * F);
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    double *part = calloc((size_t)nthr * K * F, sizeof(double));
#pragma omp parallel
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        double *my = part + (size_t)t * K * F;
        double *lr = malloc(sizeof(double) * K);
        double phi[1 + OR_MAXD + OR_MAXD * (OR_MAXD + 1) / 2];
#pragma omp for schedule(static)
        for (int n = 0; n < N; n++) {
            const double *x = X + (size_t)n * D;
            double mx = -INFINITY;
            for (int k = 0; k < K; k++) {
                lr[k] = or_log_rho_one(D, x, m + (size_t)k * D, Lf + (size_t)k * D * D, nu[k], cst[k]);
                if (lr[k] > mx) mx = lr[k];
            }
            double s = 0.0;
            for (int k = 0; k < K; k++) s += exp(lr[k] - mx);
            double l = mx + log(s);
            lse[n] = l;
            phi[0] = 1.0;
            for (int i = 0; i < D; i++) phi[1 + i] = x[i];
            int u = 1 + D;
            for (int i = 0; i < D; i++)
                for (int j = i; j < D; j++) phi[u++] = x[i] * x[j];
            for (int k = 0; k < K; k++) {
                double r = exp(lr[k] - l);
                if (R) R[(size_t)n * K + k] = r;
                double *acc = my + (size_t)k * F;
                for (int f = 0; f < F; f++) acc[f] += r * phi[f];
            }
        }
        free(lr);
    }
    for (int t = 0; t < nthr; t++)
        for (size_t i = 0; i < (size_t)K * F; i++) dS[i] += part[(size_t)t * K * F + i];
    free(part); free(cst); free(Lf);
    return 0;
}

/* KL( NW(m, beta, W, nu) || NW(m0, beta0, W0, nu0) ) for one component, with
 * the scale matrices given as inverses Winv = W^-1, W0inv = W0^-1:
 *  1/2 [D beta0/beta - D + beta0 nu (m-m0)^T W (m-m0) + D ln(beta/beta0)]
 *  + (nu-nu0)/2 psi_D(nu/2) - nu D/2 + nu/2 tr(W0^-1 W)
 *  + nu0/2 (ln|W0| - ln|W|) + ln Gamma_D(nu0/2) - ln Gamma_D(nu/2). */
double or_kl_nw(int D, const double *mq, double bq, const double *Winvq, double nq,
                const double *mp, double bp, const double *Winvp, double np)
{
    double Lq[OR_MAXD * OR_MAXD], Lp[OR_MAXD * OR_MAXD], Wq[OR_MAXD * OR_MAXD];
    if (or_cholesky(D, Winvq, Lq) || or_cholesky(D, Winvp, Lp)) return NAN;
    double ldq = 0.0, ldp = 0.0; /* ln|W^-1| */
    for (int i = 0; i < D; i++) { ldq += 2.0 * log(Lq[i * D + i]); ldp += 2.0 * log(Lp[i * D + i]); }
    or_inverse_from_chol(D, Lq, Wq);
    double d[OR_MAXD], y[OR_MAXD];
    for (int i = 0; i < D; i++) d[i] = mq[i] - mp[i];
    or_forward(D, Lq, d, y);
    double maha = 0.0;
    for (int i = 0; i < D; i++) maha += y[i] * y[i];
    double tr = 0.0;
    for (int i = 0; i < D; i++)
        for (int j = 0; j < D; j++) tr += Winvp[i * D + j] * Wq[j * D + i];
    double kl = 0.5 * (D * bp / bq - D + bp * nq * maha + D * log(bq / bp));
    /* ln|W0| - ln|W| = -ldp + ldq */
    kl += 0.5 * (nq - np) * or_mvdigamma(D, 0.5 * nq) - 0.5 * nq * D + 0.5 * nq * tr
        + 0.5 * np * (ldq - ldp) + or_lmvgamma(D, 0.5 * np) - or_lmvgamma(D, 0.5 * nq);
    return kl;
}

/* KL( Dir(alpha) || Dir(alpha0) ) over K components. */
double or_kl_dir(int K, const double *a, const double *a0)
{
    double as = 0.0, a0s = 0.0;
    for (int k = 0; k < K; k++) { as += a[k]; a0s += a0[k]; }
    double psi_as = or_digamma(as);
    double kl = lgamma(as) - lgamma(a0s);
    for (int k = 0; k < K; k++)
        kl += -lgamma(a[k]) + lgamma(a0[k]) + (a[k] - a0[k]) * (or_digamma(a[k]) - psi_as);
    return kl;
}

/* Sum over components of the posterior-vs-effective-prior KL terms. */
static double or_kl_total(int K, int D, const double *aq, const double *bq, const double *nq,
                          const double *mq, const double *Wq, const double *ap, const double *bp,
                          const double *np_, const double *mp, const double *Wp)
{
    double kl = or_kl_dir(K, aq, ap);
    for (int k = 0; k < K; k++)
        kl += or_kl_nw(D, mq + (size_t)k * D, bq[k], Wq + (size_t)k * D * D, nq[k],
                       mp + (size_t)k * D, bp[k], Wp + (size_t)k * D * D, np_[k]);
    return kl;
}

/*
 * One frame of Alg. 1 `fit` with n_iters CAVI iterations:
 *   effective prior  p = prior0 (+) S_past          (update_from_statistics)
 *   q_0 = p
 *   for t in 0..n_iters-1:
 *     E-step under q_t -> lse, dS     (compute_elbo_delta, Eq. 3)
 *     elbo[t] = sum_n lse_n - KL(q_t || p)
 *     q_{t+1} = prior0 (+) (S_past + dS)
 *   S_past += dS   (continual, replay-free accumulation)
 * Inputs: X (N x D), prior0 (alpha0, beta0, nu0 scalars, m0 K x D, W0 D x D).
 * In/out: S_past (K x F).  Outputs: elbo (n_iters, nullable), lse_last (N,
 * nullable: lse of the last E-step), dS_last (K x F, nullable).
 * Returns 0, or a negative code if a W^-1 is not positive definite.
 */
int or_cavi_frame(int N, int K, int D, const double *X, double alpha0, double beta0, double nu0,
                  const double *m0, const double *W0, double *S_past, int n_iters,
                  double *elbo, double *lse_last, double *dS_last)
{
    const int F = or_F(D);
    int rc = 0;
    double W0inv[OR_MAXD * OR_MAXD], L0[OR_MAXD * OR_MAXD];
    if (or_cholesky(D, W0, L0)) return -1000000;
    or_inverse_from_chol(D, L0, W0inv);
    size_t KD = (size_t)K * D, KDD = (size_t)K * D * D;
    double *pa = malloc(8 * K), *pb = malloc(8 * K), *pn = malloc(8 * K), *pm = malloc(8 * KD), *pW = malloc(8 * KDD);
    double *qa = malloc(8 * K), *qb = malloc(8 * K), *qn = malloc(8 * K), *qm = malloc(8 * KD), *qW = malloc(8 * KDD);
    double *dS = calloc((size_t)K * F, 8), *St = malloc(8 * (size_t)K * F);
    double *lse = malloc(8 * (size_t)(N > 0 ? N : 1));
    or_mstep(K, D, alpha0, beta0, nu0, m0, W0inv, S_past, pa, pb, pn, pm, pW);
    memcpy(qa, pa, 8 * K); memcpy(qb, pb, 8 * K); memcpy(qn, pn, 8 * K);
    memcpy(qm, pm, 8 * KD); memcpy(qW, pW, 8 * KDD);
    for (int t = 0; t < n_iters; t++) {
        rc = or_estep_stats(N, K, D, X, qa, qb, qn, qm, qW, lse, dS, NULL);
        if (rc) break;
        double sl = 0.0;
        for (int n = 0; n < N; n++) sl += lse[n];
        if (elbo) elbo[t] = sl - or_kl_total(K, D, qa, qb, qn, qm, qW, pa, pb, pn, pm, pW);
        for (size_t i = 0; i < (size_t)K * F; i++) St[i] = S_past[i] + dS[i];
        or_mstep(K, D, alpha0, beta0, nu0, m0, W0inv, St, qa, qb, qn, qm, qW);
    }
    if (rc == 0) {
        for (size_t i = 0; i < (size_t)K * F; i++) S_past[i] += dS[i];
        if (lse_last) memcpy(lse_last, lse, 8 * (size_t)N);
        if (dS_last) memcpy(dS_last, dS, 8 * (size_t)K * F);
    }
    free(pa); free(pb); free(pn); free(pm); free(pW);
    free(qa); free(qb); free(qn); free(qm); free(qW);
    free(dS); free(St); free(lse);
    return rc;
}

/* ELBO of the posterior prior0 (+) (S_past + S_frame) on points X, against the
 * effective prior prior0 (+) S_past (the bound recorded by or_cavi_frame for
 * the posterior entering an iteration). */
int or_elbo(int N, int K, int D, const double *X, double alpha0, double beta0, double nu0,
            const double *m0, const double *W0, const double *S_past, const double *S_frame,
            double *elbo_out)
{
    const int F = or_F(D);
    double W0inv[OR_MAXD * OR_MAXD], L0[OR_MAXD * OR_MAXD];
    if (or_cholesky(D, W0, L0)) return -1000000;
    or_inverse_from_chol(D, L0, W0inv);
    size_t KD = (size_t)K * D, KDD = (size_t)K * D * D;
    double *pa = malloc(8 * K), *pb = malloc(8 * K), *pn = malloc(8 * K), *pm = malloc(8 * KD), *pW = malloc(8 * KDD);
    double *qa = malloc(8 * K), *qb = malloc(8 * K), *qn = malloc(8 * K), *qm = malloc(8 * KD), *qW = malloc(8 * KDD);
    double *St = malloc(8 * (size_t)K * F), *dS = malloc(8 * (size_t)K * F);
    double *lse = malloc(8 * (size_t)(N > 0 ? N : 1));
    or_mstep(K, D, alpha0, beta0, nu0, m0, W0inv, S_past, pa, pb, pn, pm, pW);
    for (size_t i = 0; i < (size_t)K * F; i++) St[i] = S_past[i] + (S_frame ? S_frame[i] : 0.0);
    or_mstep(K, D, alpha0, beta0, nu0, m0, W0inv, St, qa, qb, qn, qm, qW);
    int rc = or_estep_stats(N, K, D, X, qa, qb, qn, qm, qW, lse, dS, NULL);
    if (rc == 0) {
        double sl = 0.0;
        for (int n = 0; n < N; n++) sl += lse[n];
        *elbo_out = sl - or_kl_total(K, D, qa, qb, qn, qm, qW, pa, pb, pn, pm, pW);
    }
    free(pa); free(pb); free(pn); free(pm); free(pW);
    free(qa); free(qb); free(qn); free(qm); free(qW);
    free(St); free(dS); free(lse);
    return rc;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
