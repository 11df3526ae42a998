// vbgs_proposal.cu -- learned candidate proposal for the E-step.
//
// With many components, nearly every (point, component) responsibility is
// negligible.  A small MLP over the point (x, y, z, r, g, b) proposes the 4
// most likely of G = 1024 component clusters (k-means of the posterior means,
// refreshed after every posterior update); the E-step then scores only the
// components of those clusters.  A certificate bounds, per point and cluster,
// the mass sum_{k in g} exp(l_nk) (tables of per-member bounds, below); the
// candidate pass adds the cluster with the largest bound while the bound mass
// of the other clusters exceeds 1e-3 of the candidates' mass, up to 32
// clusters.  Points still above 1e-3 (and a seeded 1% audit sample) run the
// exact E-step over all components; the audit also scores all components in
// the candidates' FP32 arithmetic to measure the true missed mass.
// The MLP is trained on the GPU by the kernels below (forward, backward, Adam)
// on the cluster masses q_ng = sum_{k in g} r_nk of the exact E-steps.
//
// All logits here are in log2 units (FP32 records: c and M scaled by log2 e),
// and, like every E-step logit of the library, without the -psi(sum alpha)
// term shared by all components (it cancels in every ratio used here).
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

// ------------------------------------------------------- certificate -----
// The logit of component k is l_k(x) = c_k - 1/2 (x - m_k)^T Lam_k (x - m_k).
// Four lower bounds of the quadratic form, each a scale times a squared norm:
//   metric:   mu_k |L^T (x - m_k)|^2 with P = L L^T the cluster's metric and
//             mu_k = lambda_min(L^-1 Lam_k L^-T);
//   position: lp_k |x_p - m_p|^2 (lp_k: smallest eigenvalue of the position
//             block's Schur complement, i.e. of the marginal precision);
//   colour:   lc_k |x_c - m_c|^2;
//   joint:    la_k |x - m|^2 (la_k = lambda_min(Lam_k)).
// With the triangle inequality |x - m_k| >= |x - o| - |m_k - o| in the same
// norm around the cluster centre o, every kind q gives
//   sum_{k in g} exp(l_k(x)) <= T_q(d_q) = sum_k exp(c_k - 1/2 mu_qk (d_q - r_qk)_+^2),
// d_q the distance of x to o and r_qk that of m_k; T_q does not increase
// with d_q.  Each T_q is tabulated (log2 units) at kTJ - 1 grid points and
// at d_last = r_max + sqrt(2 span / mu_min); beyond d_last the tail
//   T_q(d) <= T_q(d_last) - 1/2 mu_min (d - d_last)(d + d_last - 2 r_max)
// holds because every term decays at least that fast once d >= r_max.  The
// bound of a cluster at x is the smallest of the four table look-ups.
constexpr int kTJ = 16;                   // table points per kind
constexpr int kKind = 4;                  // metric, position, colour, joint
constexpr int kKS = kTJ + 5;              // T[kTJ], 1/h, d_last, tail slope, r_max, eps
constexpr int kCP = 28 + kKind * kKS;     // [0..5] centre, [6..26] L (lower), [27] metric valid
constexpr int kMS = 9;                    // per member: c (log2), mu[4], r[4]
constexpr int kCScr = 28;                 // per cluster FP64: centre, L, valid
constexpr double kSpanNats = 30.0;
static_assert(kCP % 4 == 0, "cluster records are staged as float4");

// Upper bound of the largest eigenvalue of a symmetric positive definite 6 x 6
// matrix (lower triangle, tri order): with B = S / tr(S),
// lambda_max(B)^8 <= |B^8|_F, which overestimates by at most 6^(1/16).  The
// three squarings run in FP32: B is positive semi-definite with |B| <= 1, so
// each rounded product is within a relative 6 * 6 * 2^-24 of the exact one in
// norm, the rounding of |B^8|_F stays below 2e-5 relative and its eighth root
// below 3e-6; the result is inflated by 1e-4.
__device__ double lmax_bound6(const double *S)
{
    double t = 0.0;
    for (int i = 0; i < 6; i++) t += S[tri(i, i)];
    if (!(t > 0.0)) return INFINITY;
    const double it = 1.0 / t;
    float B[21], C[21];
#pragma unroll
    for (int q = 0; q < 21; q++) B[q] = (float)(S[q] * it);
#pragma unroll
    for (int rep = 0; rep < 3; rep++) {   // B <- B^2, three times: B^8
#pragma unroll
        for (int i = 0; i < 6; i++)
#pragma unroll
            for (int j = 0; j <= i; j++) {
                float v = 0.f;
#pragma unroll
                for (int l = 0; l < 6; l++)
                    v = fmaf(B[i >= l ? tri(i, l) : tri(l, i)], B[l >= j ? tri(l, j) : tri(j, l)], v);
                C[tri(i, j)] = v;
            }
#pragma unroll
        for (int q = 0; q < 21; q++) B[q] = C[q];
    }
    double f = 0.0;
#pragma unroll
    for (int i = 0; i < 6; i++)
#pragma unroll
        for (int j = 0; j <= i; j++) f += (i == j ? 1.0 : 2.0) * (double)B[tri(i, j)] * (double)B[tri(i, j)];
    return t * pow(sqrt(f), 0.125) * (1.0 + 1e-4);
}

// Cluster centre and metric: o = mean of the member means, P = the average
// member precision weighted by N_k + 1e-3, L = chol(P) rounded to FP32.
__global__ void __launch_bounds__(64) k_cluster_metric(const double *__restrict__ rec, const int *__restrict__ order,
                                                       const int *__restrict__ cstart,
                                                       const double *__restrict__ Spast,
                                                       const double *__restrict__ dS, const int *__restrict__ kperm,
                                                       float *__restrict__ cpar, double *__restrict__ cscr)
{
    __shared__ double sh[28][2];
    const int g = blockIdx.x, t = threadIdx.x;
    const int b = cstart[g], e = cstart[g + 1];
    double acc[28];
#pragma unroll
    for (int q = 0; q < 28; q++) acc[q] = 0.0;
    for (int i = b + t; i < e; i += 64) {
        const int p = order[i];
        const double *r = rec + (size_t)p * VBGS_REC;
        const int k = kperm[p];
        const double w = Spast[(size_t)k * VBGS_F] + (dS ? dS[(size_t)k * VBGS_F] : 0.0) + 1e-3;
#pragma unroll
        for (int q = 0; q < 6; q++) acc[q] += r[q];
        // Lam = M^T M with M lower triangular (tri order at r + 6)
#pragma unroll
        for (int a = 0; a < 6; a++)
#pragma unroll
            for (int c = 0; c <= a; c++) {
                double v = 0.0;
#pragma unroll
                for (int l = a; l < 6; l++) v = fma(r[6 + tri(l, a)], r[6 + tri(l, c)], v);
                acc[6 + tri(a, c)] = fma(w, v, acc[6 + tri(a, c)]);
            }
        acc[27] += w;
    }
#pragma unroll
    for (int q = 0; q < 28; q++) {
        double v = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((t & 31) == 0) sh[q][t >> 5] = v;
    }
    __syncthreads();
    if (t != 0) return;
    float *cp = cpar + (size_t)g * kCP;
    double *cs = cscr + (size_t)g * kCScr;
    const int n = e - b;
    double L[21];
    bool ok = n > 0;
    double o[6];
    for (int q = 0; q < 6; q++) o[q] = n > 0 ? (sh[q][0] + sh[q][1]) / n : 0.0;
    if (ok) {
        const double iw = 1.0 / (sh[27][0] + sh[27][1]);
        for (int q = 0; q < 21; q++) L[q] = (sh[6 + q][0] + sh[6 + q][1]) * iw;
        // in-place Cholesky of P (lower, tri order)
        for (int j = 0; j < 6 && ok; j++) {
            double d = L[tri(j, j)];
            for (int l = 0; l < j; l++) d -= L[tri(j, l)] * L[tri(j, l)];
            if (!(d > 0.0)) { ok = false; break; }
            d = sqrt(d);
            L[tri(j, j)] = d;
            for (int i = j + 1; i < 6; i++) {
                double v = L[tri(i, j)];
                for (int l = 0; l < j; l++) v -= L[tri(i, l)] * L[tri(j, l)];
                L[tri(i, j)] = v / d;
            }
        }
    }
    for (int q = 0; q < 6; q++) {
        const float of = (float)o[q];
        cp[q] = of;
        cs[q] = (double)of;
    }
    for (int q = 0; q < 21; q++) {
        const float lf = ok ? (float)L[q] : 0.f;
        cp[6 + q] = lf;
        cs[6 + q] = (double)lf;
    }
    cp[27] = ok ? 1.f : 0.f;
    cs[27] = ok ? 1.0 : 0.0;
}

__device__ __forceinline__ float f_up(double v)
{
    float f = (float)v;
    if ((double)f < v) f = nextafterf(f, INFINITY);
    return f;
}
__device__ __forceinline__ float f_down(double v)
{
    float f = (float)v;
    if ((double)f > v) f = nextafterf(f, -INFINITY);
    return f;
}

// Per member (sorted position i): constant (log2, rounded up), the four
// scales mu (rounded down) and the four radii r (rounded up).
__global__ void __launch_bounds__(128) k_cluster_members(const double *__restrict__ rec,
                                                         const float *__restrict__ rec32,
                                                         const int *__restrict__ order,
                                                         const unsigned int *__restrict__ skey, int K,
                                                         const double *__restrict__ cscr, float *__restrict__ mscr)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K) return;
    const int p = order[i];
    const int g = (int)skey[i];
    const double *r = rec + (size_t)p * VBGS_REC;
    const double *cs = cscr + (size_t)g * kCScr;
    double M[21], Mi[21];
    for (int q = 0; q < 21; q++) M[q] = r[6 + q];
    // inverse of the lower-triangular M
    for (int j = 0; j < 6; j++) {
        Mi[tri(j, j)] = 1.0 / M[tri(j, j)];
        for (int a = j + 1; a < 6; a++) {
            double v = 0.0;
            for (int l = j; l < a; l++) v = fma(M[tri(a, l)], Mi[tri(l, j)], v);
            Mi[tri(a, j)] = -v / M[tri(a, a)];
        }
    }
    // covariance Sigma = Lam^-1 = Mi Mi^T
    double Sg[21];
    for (int a = 0; a < 6; a++)
        for (int c = 0; c <= a; c++) {
            double v = 0.0;
            for (int l = 0; l <= c; l++) v = fma(Mi[tri(a, l)], Mi[tri(c, l)], v);
            Sg[tri(a, c)] = v;
        }
    const double la = 1.0 / lmax_bound6(Sg);
    // metric kind: lambda_min(L^-1 Lam L^-T) = 1 / lambda_max(L^T Sigma L)
    double mu_m = 0.0;
    const double *L = cs + 6;
    if (cs[27] != 0.0) {
        double Z[36];   // Sigma L
        for (int a = 0; a < 6; a++)
            for (int c = 0; c < 6; c++) {
                double v = 0.0;
                for (int l = c; l < 6; l++) v = fma(Sg[a >= l ? tri(a, l) : tri(l, a)], L[tri(l, c)], v);
                Z[a * 6 + c] = v;
            }
        double A[21];   // L^T Sigma L
        for (int a = 0; a < 6; a++)
            for (int c = 0; c <= a; c++) {
                double v = 0.0;
                for (int l = a; l < 6; l++) v = fma(L[tri(l, a)], Z[l * 6 + c], v);
                A[tri(a, c)] = v;
            }
        mu_m = 1.0 / lmax_bound6(A);
    }
    const double lp = (double)rec32[(size_t)p * VBGS_REC + 28] * 0.6931471805599453 * (1.0 - 1e-6);
    const double lc = (double)rec32[(size_t)p * VBGS_REC + 29] * 0.6931471805599453 * (1.0 - 1e-6);
    double dx[6], rp = 0.0, rc = 0.0, rm = 0.0;
    for (int q = 0; q < 6; q++) dx[q] = r[q] - cs[q];
    for (int q = 0; q < 3; q++) { rp = fma(dx[q], dx[q], rp); rc = fma(dx[3 + q], dx[3 + q], rc); }
    for (int c = 0; c < 6; c++) {
        double y = 0.0;
        for (int a = c; a < 6; a++) y = fma(L[tri(a, c)], dx[a], y);
        rm = fma(y, y, rm);
    }
    float *ms = mscr + (size_t)i * kMS;
    ms[0] = f_up(r[27] * 1.4426950408889634);
    ms[1] = f_down(fmax(mu_m * (1.0 - 1e-9), 0.0));
    ms[2] = f_down(fmax(lp, 0.0));
    ms[3] = f_down(fmax(lc, 0.0));
    ms[4] = f_down(fmax(la * (1.0 - 1e-9), 0.0));
    ms[5] = f_up(sqrt(rm) * (1.0 + 1e-12));
    ms[6] = f_up(sqrt(rp) * (1.0 + 1e-12));
    ms[7] = f_up(sqrt(rc) * (1.0 + 1e-12));
    ms[8] = f_up(sqrt(rp + rc) * (1.0 + 1e-12));
}

// The tables: one block per cluster, thread (q, j) = (kind, table point).
__global__ void __launch_bounds__(64) k_cluster_tables(const float *__restrict__ mscr, const int *__restrict__ cstart,
                                                       float xmax, float *__restrict__ cpar)
{
    const int g = blockIdx.x, t = threadIdx.x, q = t >> 4, j = t & 15;
    const int b = cstart[g], e = cstart[g + 1];
    float *cp = cpar + (size_t)g * kCP;
    float *tq = cp + 28 + q * kKS;
    if (e == b) {
        tq[j] = -INFINITY;
        if (j == 0) { tq[kTJ] = 0.f; tq[kTJ + 1] = INFINITY; tq[kTJ + 2] = 0.f; tq[kTJ + 3] = 0.f; tq[kTJ + 4] = 0.f; }
        return;
    }
    float rmax = 0.f, mumin = INFINITY;
    for (int i = b + j; i < e; i += kTJ) {
        rmax = fmaxf(rmax, mscr[(size_t)i * kMS + 5 + q]);
        mumin = fminf(mumin, mscr[(size_t)i * kMS + 1 + q]);
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
        rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
        mumin = fminf(mumin, __shfl_xor_sync(0xffffffffu, mumin, o));
    }
    float dl = INFINITY, inv_h = 0.f;
    double hd = 0.0;
    if (mumin > 0.f) {
        dl = f_down((double)rmax + sqrt(2.0 * kSpanNats / (double)mumin));
        inv_h = f_down((double)(kTJ - 1) / (double)dl);
        hd = 1.0 / (double)inv_h;
    }
    const float dj = (j < kTJ - 1) ? f_down((double)j * hd) : (mumin > 0.f ? dl : 0.f);
    const float hmu = 0.72134752044448170f;   // log2(e) / 2
    float mx = -INFINITY;
    for (int i = b; i < e; i++) {
        const float *ms = mscr + (size_t)i * kMS;
        const float dd = fmaxf(dj - ms[5 + q], 0.f);
        mx = fmaxf(mx, ms[0] - hmu * ms[1 + q] * dd * dd);
    }
    float s = 0.f;
    for (int i = b; i < e; i++) {
        const float *ms = mscr + (size_t)i * kMS;
        const float dd = fmaxf(dj - ms[5 + q], 0.f);
        s += exp2f(ms[0] - hmu * ms[1 + q] * dd * dd - mx);
    }
    // FP32 rounding of the terms and of the sum: a margin of 1e-3 + 1e-6 |T|
    const float T = mx + log2f(s);
    tq[j] = T + 1e-3f + 1e-6f * fabsf(T);
    if (j == 0) {
        float lf = 1.f;
        if (q == 0) {
            float f2 = 0.f;
            for (int a = 0; a < 21; a++) f2 = fmaf(cp[6 + a], cp[6 + a], f2);
            lf = sqrtf(f2);
        }
        tq[kTJ] = inv_h;
        tq[kTJ + 1] = dl;
        tq[kTJ + 2] = hmu * mumin * (1.f - 1e-6f);
        tq[kTJ + 3] = rmax;
        // rounding of the point, the centre and the distance in FP32
        tq[kTJ + 4] = 1e-6f * (rmax + (mumin > 0.f ? dl : 0.f)) + 1e-6f * lf * xmax;
    }
}

__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Table look-up of one kind at distance d (log2 units).  The 1e-5 relative
// shrink of d covers the error of the approximate square roots.
__device__ __forceinline__ float table_bound(const float *__restrict__ tq, float d)
{
    d = fmaxf(fmaf(d, 1.f - 1e-5f, -tq[kTJ + 4]), 0.f);
    const float dl = tq[kTJ + 1];
    if (d >= dl) return tq[kTJ - 1] - tq[kTJ + 2] * (d - dl) * (d + dl - 2.f * tq[kTJ + 3]);
    const int j = min((int)(d * tq[kTJ] * 0.999999f), kTJ - 2);
    return tq[j];
}

// Bound of every cluster at every point: UB[n][g] (log2 units), one thread
// per point, clusters staged through shared memory kBC at a time; blockIdx.y
// selects one of kBG groups of clusters (more CTAs in flight).
constexpr int kBC = 16;
constexpr int kBG = 4;
__global__ void __launch_bounds__(128) k_bounds(const double *__restrict__ X, int64_t N,
                                                const float *__restrict__ cpar, float *__restrict__ UB)
{
    __shared__ __align__(16) float sp[kBC * kCP];
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = n < N;
    float x[6];
#pragma unroll
    for (int i = 0; i < 6; i++) x[i] = live ? (float)X[n * VBGS_XS + i] : 0.f;
    const int gb = blockIdx.y * (kG / kBG), ge = gb + kG / kBG;
    for (int g0 = gb; g0 < ge; g0 += kBC) {
        __syncthreads();
        const float4 *src = reinterpret_cast<const float4 *>(cpar + (size_t)g0 * kCP);
        for (int i = threadIdx.x; i < kBC * kCP / 4; i += blockDim.x) reinterpret_cast<float4 *>(sp)[i] = src[i];
        __syncthreads();
        float out[kBC];
#pragma unroll
        for (int c = 0; c < kBC; c++) {
            const float *cp = sp + c * kCP;
            float dx[6];
#pragma unroll
            for (int i = 0; i < 6; i++) dx[i] = x[i] - cp[i];
            const float dp2 = fmaf(dx[0], dx[0], fmaf(dx[1], dx[1], dx[2] * dx[2]));
            const float dc2 = fmaf(dx[3], dx[3], fmaf(dx[4], dx[4], dx[5] * dx[5]));
            float dm2 = 0.f;
#pragma unroll
            for (int a = 0; a < 6; a++) {
                float y = 0.f;
#pragma unroll
                for (int l = a; l < 6; l++) y = fmaf(cp[6 + tri(l, a)], dx[l], y);
                dm2 = fmaf(y, y, dm2);
            }
            const float b0 = table_bound(cp + 28, sqrt_approx(dm2));
            const float b1 = table_bound(cp + 28 + kKS, sqrt_approx(dp2));
            const float b2 = table_bound(cp + 28 + 2 * kKS, sqrt_approx(dc2));
            const float b3 = table_bound(cp + 28 + 3 * kKS, sqrt_approx(dp2 + dc2));
            out[c] = fminf(fminf(b0, b1), fminf(b2, b3));
        }
        if (live) {
            float4 *dst = reinterpret_cast<float4 *>(UB + n * kG + g0);
#pragma unroll
            for (int c = 0; c < kBC / 4; c++) dst[c] = make_float4(out[4 * c], out[4 * c + 1], out[4 * c + 2], out[4 * c + 3]);
        }
    }
}

// ------------------------------------------------------------------ MLP -----
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
// Slot of sample i when the samples are dealt round-robin into nb minibatches
// of stride S (minibatch b holds samples b, b + nb, ...: each spans the whole
// frame instead of one region of its Morton order); nb = 1: slot i.
__device__ __forceinline__ int64_t deal_slot(int64_t i, int64_t nb, int64_t S)
{
    return nb > 1 ? (i % nb) * S + i / nb : i;
}

__global__ void k_mlp_inputs(const double *__restrict__ X, const int *__restrict__ rows, int64_t rstride, int64_t n,
                             BoxParams box, int64_t nb, int64_t S, float *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t r = rows ? rows[i] : i * rstride;
    const double *x = X + r * VBGS_XS;
    float *o = out + deal_slot(i, nb, S) * 6;
#pragma unroll
    for (int q = 0; q < 3; q++) o[q] = (float)((x[q] - box.lo[q]) * box.inv_ext[q] * 2.0 - 1.0);
#pragma unroll
    for (int q = 3; q < 6; q++) o[q] = (float)(x[q] * 2.0 - 1.0);
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

// Candidate pass 1, in rounds.  Per point: the candidate clusters
// cand[n][0 .. nc), of which slots [pend, nc) are not scored yet, and the
// running (max, sum) of 2^logit over the scored candidates (log2 units).
// A round scores the pending (cluster, point) pairs cluster-major (k_cand_score:
// a CTA per (cluster, chunk of points), the cluster's member records in
// shared memory, a thread per point) into per-slot partials, then k_cand_select
// (a warp per point) merges them in slot order and evaluates the certificate:
// while the bound mass of the other clusters exceeds thresh times the
// candidates' mass, it adds the clusters with the largest bounds (up to
// kAddMax per round, no more than the bound says are needed), which the next
// round scores.  The last round's select writes the lse, the bound and the
// point's status (0 proposal, 1 fallback, 2 seeded audit).  Every round is
// enqueued without a host read: a round's kernels return at once when the
// round before it added no cluster (prev_added, that round's count, is 0),
// so the rounds after the first that adds nothing change no state.
constexpr int kAddMax = 8;
constexpr int kPB = 128;   // points per work item of the cluster-major kernels

__global__ void __launch_bounds__(256) k_cand_init(const int *__restrict__ top, int64_t N, int *__restrict__ cand,
                                                   int *__restrict__ ncand, int *__restrict__ pend,
                                                   float2 *__restrict__ run, float2 *__restrict__ part)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    for (int t = 0; t < kMaxCand; t++) {
        cand[n * kMaxCand + t] = t < kTop ? top[n * kTop + t] : -1;
        part[n * kMaxCand + t] = make_float2(-INFINITY, 0.f);
    }
    ncand[n] = kTop;
    pend[n] = 0;
    run[n] = make_float2(-INFINITY, 0.f);
}

// (cluster, point * 32 + slot) keys of the pending candidate slots (at most
// kAddMax per point: the top 4, or one round's additions).
__global__ void k_pend_keys(const int *__restrict__ cand, const int *__restrict__ ncand,
                            const int *__restrict__ pend, int64_t N, const unsigned long long *__restrict__ prev_added,
                            unsigned int *__restrict__ key, int *__restrict__ val)
{
    if (prev_added && *prev_added == 0ull) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * kAddMax) return;
    const int64_t n = i / kAddMax;
    const int t = pend[n] + (int)(i % kAddMax);
    const bool p = t < ncand[n];
    key[i] = p ? (unsigned int)cand[n * kMaxCand + t] : (unsigned int)kG;
    val[i] = (int)(n * kMaxCand + (p ? t : 0));
}

constexpr int kSM = 256;   // member records staged per pass of k_cand_score
__global__ void __launch_bounds__(kPB) k_cand_score(const double *__restrict__ X, const float *__restrict__ rec32,
                                                    const int *__restrict__ order, const int *__restrict__ cstart,
                                                    const int *__restrict__ pstart, const int *__restrict__ plist,
                                                    const int *__restrict__ item_start,
                                                    const unsigned long long *__restrict__ prev_added,
                                                    float2 *__restrict__ part)
{
    __shared__ __align__(16) float sr[kSM * 28];
    __shared__ int sg;
    const int item = blockIdx.x;
    // the grid is an upper bound of the item count (item_start[kG])
    if ((prev_added && *prev_added == 0ull) || item >= item_start[kG]) return;
    if (threadIdx.x == 0) {
        int lo = 0, hi = kG;   // largest g with item_start[g] <= item
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (item_start[mid] <= item) lo = mid; else hi = mid;
        }
        sg = lo;
    }
    __syncthreads();
    const int g = sg;
    const int c = item - item_start[g];
    const int b = cstart[g], S = cstart[g + 1] - b;
    const int p0 = pstart[g] + c * kPB, cnt = min(kPB, pstart[g + 1] - p0);
    const int t = threadIdx.x;
    const bool live = t < cnt;
    const int v = live ? plist[p0 + t] : 0;
    float x[6];
#pragma unroll
    for (int q = 0; q < 6; q++) x[q] = live ? (float)X[(int64_t)(v / kMaxCand) * VBGS_XS + q] : 0.f;
    float mx = -INFINITY, sum = 0.f;
    for (int m0 = 0; m0 < S; m0 += kSM) {
        const int ms = min(kSM, S - m0);
        __syncthreads();
        for (int i = t; i < ms * 28; i += blockDim.x) {
            const int mm = i / 28, f = i - mm * 28;
            sr[i] = rec32[(size_t)order[b + m0 + mm] * VBGS_REC + f];
        }
        __syncthreads();
        if (live)
            for (int mm = 0; mm < ms; mm++) {
                const float l = logit32(sr + mm * 28, x);
                if (l > mx) { sum = sum * ex2a(mx - l) + 1.f; mx = l; }
                else sum += ex2a(l - mx);
            }
    }
    if (live) part[v] = make_float2(mx, sum);
}

__global__ void __launch_bounds__(256) k_cand_select(const float *__restrict__ UB, int64_t N,
                                                     const int *__restrict__ cstart, float thresh, int final_round,
                                                     uint32_t audit_seed, uint32_t audit_per_mille,
                                                     int *__restrict__ cand, int *__restrict__ ncand,
                                                     int *__restrict__ pend, float2 *__restrict__ run,
                                                     float2 *__restrict__ part, double *__restrict__ lse_c,
                                                     float *__restrict__ bound, int *__restrict__ exact,
                                                     unsigned long long *__restrict__ counters,
                                                     const unsigned long long *__restrict__ prev_added,
                                                     unsigned long long *__restrict__ added_out)
{
    if (prev_added && *prev_added == 0ull) return;
    const int lane = threadIdx.x & 31;
    const int64_t n = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (n >= N) return;
    int nc = ncand[n];
    const int p = pend[n];
    // a point whose last select added nothing (pend == ncand; never in the
    // first round, which starts from the top 4) has nothing to merge and would
    // write back the bound, lse and status it holds: it is done
    if (p == nc) return;
    // candidate membership: lane l holds clusters 32 j + l
    const int my = lane < nc ? cand[n * kMaxCand + lane] : -1;
    uint32_t mine = 0u;
    for (int t = 0; t < nc; t++) {
        const int g = __shfl_sync(0xffffffffu, my, t);
        if ((g & 31) == lane) mine |= 1u << (g >> 5);
    }
    // merge the new partials in slot order
    float2 r = run[n];
    float mx = r.x, s = r.y;
    const float2 pp = (lane >= p && lane < nc) ? part[n * kMaxCand + lane] : make_float2(-INFINITY, 0.f);
    for (int t = p; t < nc; t++) {
        const float pm = __shfl_sync(0xffffffffu, pp.x, t), ps = __shfl_sync(0xffffffffu, pp.y, t);
        if (pm == -INFINITY) continue;
        if (pm > mx) { s = s * ex2a(mx - pm) + ps; mx = pm; }
        else s += ps * ex2a(pm - mx);
    }
    const float l2 = (mx == -INFINITY) ? -INFINITY : mx + __log2f(s);
    float u[32];
#pragma unroll
    for (int j = 0; j < 32; j++) u[j] = UB[n * kG + j * 32 + lane];
    float ls = 0.f;
#pragma unroll
    for (int j = 0; j < 32; j++)
        if (!(mine & (1u << j))) ls += ex2a(fminf(u[j] - l2, 64.f));
    float mm = warp_sum(ls);
    int added = 0;
    unsigned long long new_pairs = 0;
    if (!final_round) {
        // add the largest-bound clusters while the remaining mass exceeds the
        // threshold (each pick removes its term), at most kAddMax per round
        float rest = mm;
        while (rest > thresh && nc < kMaxCand && added < kAddMax) {
            float lb = -INFINITY;
            int lj = -1;
#pragma unroll
            for (int j = 0; j < 32; j++)
                if (!(mine & (1u << j)) && u[j] > lb) { lb = u[j]; lj = j; }
            int bg = lj >= 0 ? lj * 32 + lane : 0x7fffffff;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ov = __shfl_xor_sync(0xffffffffu, lb, o);
                const int og = __shfl_xor_sync(0xffffffffu, bg, o);
                if (ov > lb || (ov == lb && og < bg)) { lb = ov; bg = og; }
            }
            if (bg == 0x7fffffff || lb == -INFINITY) break;
            if (lane == (bg & 31)) mine |= 1u << (bg >> 5);
            if (lane == 0) {
                cand[n * kMaxCand + nc] = bg;
                part[n * kMaxCand + nc] = make_float2(-INFINITY, 0.f);
            }
            rest -= ex2a(fminf(lb - l2, 64.f));
            new_pairs += (unsigned long long)(cstart[bg + 1] - cstart[bg]);
            nc++;
            added++;
        }
    }
    if (lane == 0) {
        run[n] = make_float2(mx, s);
        pend[n] = ncand[n];
        ncand[n] = nc;
        bound[n] = mm;
        lse_c[n] = (double)l2 * 0.6931471805599453;   // natural units
        if (added) atomicAdd(added_out, (unsigned long long)added);
        atomicAdd(&counters[0], new_pairs);
        if (!added) {
            // seeded audit sample: a hash of (seed, point index)
            uint32_t h = audit_seed ^ (uint32_t)(n * 0x9E3779B9u);
            h ^= h >> 16; h *= 0x7feb352du; h ^= h >> 15; h *= 0x846ca68bu; h ^= h >> 16;
            const bool audit = (h % 1000u) < audit_per_mille;
            exact[n] = !(mm <= thresh) ? 1 : (audit ? 2 : 0);
        }
    }
}

// Final counts of the candidate pass: fallback / audit points, clusters
// added beyond the proposal's top 4, and the scored pairs of the top 4.
__global__ void __launch_bounds__(256) k_cand_count(const int *__restrict__ exact, const int *__restrict__ ncand,
                                                    const int *__restrict__ cand, const int *__restrict__ cstart,
                                                    int64_t N, unsigned long long *__restrict__ counters)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long fb = 0, au = 0, ad = 0, pr = 0;
    if (n < N) {
        fb = exact[n] == 1;
        au = exact[n] == 2;
        ad = (unsigned long long)(ncand[n] - kTop);
        for (int t = 0; t < kTop; t++) {
            const int g = cand[n * kMaxCand + t];
            pr += (unsigned long long)(cstart[g + 1] - cstart[g]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fb += __shfl_xor_sync(0xffffffffu, fb, o);
        au += __shfl_xor_sync(0xffffffffu, au, o);
        ad += __shfl_xor_sync(0xffffffffu, ad, o);
        pr += __shfl_xor_sync(0xffffffffu, pr, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&counters[1], fb);
        atomicAdd(&counters[2], au);
        atomicAdd(&counters[3], ad);
        atomicAdd(&counters[0], pr);
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

// Candidate pass 2.  Work items are (cluster, chunk of up to kPB2 of the
// cluster's proposal points); item_start[g] and the partial base fbase[g]
// come from one scan over the clusters.  An item's CTA stages its points in
// shared memory; each thread owns a member component and accumulates
// r [1, d, upper(d d^T)] about the component's mean (FP32) over the chunk,
// written as the item's partial.  A second kernel sums a member's partials
// in item order (FP64, deterministic), shifts them to raw moments and adds
// them to the component's frame statistics.
__global__ void __launch_bounds__(1024) k_items(const int *__restrict__ pstart, const int *__restrict__ cstart,
                                                int chunk, int *__restrict__ item_start,
                                                long long *__restrict__ fbase)
{
    __shared__ long long sa[kG], sb[kG];
    const int g = threadIdx.x;
    const int cnt = pstart[g + 1] - pstart[g];
    const int S = cstart[g + 1] - cstart[g];
    const long long items = S > 0 ? (cnt + chunk - 1) / chunk : 0;
    sa[g] = items;
    sb[g] = items * S;
    __syncthreads();
    // inclusive Hillis-Steele scans of both columns
    for (int o = 1; o < kG; o <<= 1) {
        const long long a = g >= o ? sa[g - o] : 0, b = g >= o ? sb[g - o] : 0;
        __syncthreads();
        sa[g] += a;
        sb[g] += b;
        __syncthreads();
    }
    item_start[g + 1] = (int)sa[g];
    fbase[g + 1] = sb[g];
    if (g == 0) { item_start[0] = 0; fbase[0] = 0; }
}

constexpr int kPB2 = 512;   // points per work item of candidate pass 2

__global__ void __launch_bounds__(64) k_cand_pass2(const double *__restrict__ X, const double *__restrict__ lse_c,
                                                   const float *__restrict__ rec32, const int *__restrict__ order,
                                                   const int *__restrict__ cstart, const int *__restrict__ pstart,
                                                   const int *__restrict__ plist, const int *__restrict__ item_start,
                                                   const long long *__restrict__ fbase, float *__restrict__ part)
{
    __shared__ float sp[kPB2][8];
    __shared__ int sg;
    const int item = blockIdx.x;
    if (threadIdx.x == 0) {
        int lo = 0, hi = kG;   // largest g with item_start[g] <= item
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (item_start[mid] <= item) lo = mid; else hi = mid;
        }
        sg = lo;
    }
    __syncthreads();
    const int g = sg;
    const int c = item - item_start[g];
    const int b = cstart[g], S = cstart[g + 1] - b;
    const int p0 = pstart[g] + c * kPB2, cnt = min(kPB2, pstart[g + 1] - p0);
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        const int n = plist[p0 + t];
#pragma unroll
        for (int q = 0; q < 6; q++) sp[t][q] = (float)X[(int64_t)n * VBGS_XS + q];
        sp[t][6] = (float)(lse_c[n] * 1.4426950408889634);
    }
    __syncthreads();
    for (int m0 = 0; m0 < S; m0 += blockDim.x) {
        const int ml = m0 + threadIdx.x;
        if (ml >= S) break;
        const int pos = order[b + ml];
        float r[28];
#pragma unroll
        for (int i = 0; i < 28; i++) r[i] = rec32[(size_t)pos * VBGS_REC + i];
        float acc[28];
#pragma unroll
        for (int f = 0; f < 28; f++) acc[f] = 0.f;
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
        float *dst = part + (fbase[g] + (long long)c * S + ml) * VBGS_F;
#pragma unroll
        for (int f = 0; f < 28; f++) dst[f] = acc[f];
    }
}

// One CTA per cluster: lane = member (32 at a time), warp w sums the items
// c = w, w + 4, ... in order; the four warp sums are added in warp order.
__global__ void __launch_bounds__(128) k_cand_reduce(const float *__restrict__ part, const float *__restrict__ rec32,
                                                     const int *__restrict__ order, const int *__restrict__ cstart,
                                                     const int *__restrict__ item_start,
                                                     const long long *__restrict__ fbase,
                                                     const int *__restrict__ kperm, double *__restrict__ dS)
{
    __shared__ double sh[3][32][29];
    const int g = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int b = cstart[g], S = cstart[g + 1] - b;
    const int items = item_start[g + 1] - item_start[g];
    if (items == 0) return;
    for (int m0 = 0; m0 < S; m0 += 32) {
        const int ml = m0 + lane;
        const bool v = ml < S;
        double s[28];
#pragma unroll
        for (int f = 0; f < 28; f++) s[f] = 0.0;
        if (v)
            for (int c = w; c < items; c += 4) {
                const float *src = part + (fbase[g] + (long long)c * S + ml) * VBGS_F;
#pragma unroll
                for (int f = 0; f < 28; f++) s[f] += (double)src[f];
            }
        __syncthreads();
        if (w > 0)
#pragma unroll
            for (int f = 0; f < 28; f++) sh[w - 1][lane][f] = s[f];
        __syncthreads();
        if (w == 0 && v) {
#pragma unroll
            for (int f = 0; f < 28; f++) s[f] += sh[0][lane][f] + sh[1][lane][f] + sh[2][lane][f];
            const int pos = order[b + ml];
            double a[6];
#pragma unroll
            for (int q = 0; q < 6; q++) a[q] = (double)rec32[(size_t)pos * VBGS_REC + q];
            int u = 7;
#pragma unroll
            for (int q = 0; q < 6; q++)
#pragma unroll
                for (int j = q; j < 6; j++, u++) s[u] += a[q] * s[1 + j] + s[1 + q] * a[j] + s[0] * a[q] * a[j];
#pragma unroll
            for (int q = 0; q < 6; q++) s[1 + q] += s[0] * a[q];
            double *dst = dS + (size_t)kperm[pos] * VBGS_F;
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
// clusters whose certificate bound is not below 2^-40 of the point's mass
// (UB row of the point's frame index: rows[i] when the points were gathered).  One warp
// per point: lanes test the clusters, then share the scoring of each kept one.
__global__ void __launch_bounds__(256) k_labels(const double *__restrict__ Xe, const double *__restrict__ lse_e,
                                                const int *__restrict__ rows, int64_t rstride, int64_t ne,
                                                const float *__restrict__ rec32, const int *__restrict__ order,
                                                const int *__restrict__ cstart, const float *__restrict__ UB,
                                                int64_t nb, int64_t S, float *__restrict__ Q)
{
    const int lane = threadIdx.x & 31;
    const int64_t n = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (n >= ne) return;
    float x[6];
#pragma unroll
    for (int i = 0; i < 6; i++) x[i] = (float)Xe[n * rstride * VBGS_XS + i];
    const float l2 = (float)(lse_e[n * rstride] * 1.4426950408889634);
    float *q = Q + deal_slot(n, nb, S) * kG;
    const float *ub = UB + (int64_t)(rows ? rows[n * rstride] : n * rstride) * kG;
    for (int g0 = 0; g0 < kG; g0 += 32) {
        const int g = g0 + lane;
        const bool keep = ub[g] - l2 > -40.f;
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
                                                     const int *__restrict__ erows, int64_t ne)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    lse_c[erows[i]] = lse_e[i];
}

// True missed mass of the proposal on the audit points: every component
// scored in the candidates' FP32 arithmetic, 1 - 2^(lse2_cand - lse2_all).
// Blocks of (kAP exact rows) x (256 components) write per-row partial
// (max, sum) pairs; the final kernel merges them in component-chunk order.
// Rows that are fallbacks (not audits) report 0.
constexpr int kAP = 32;
__global__ void __launch_bounds__(256) k_audit_part(const double *__restrict__ X, const int *__restrict__ erows,
                                                    int64_t ne, const int *__restrict__ exact,
                                                    const float *__restrict__ rec32, int K, float2 *__restrict__ part)
{
    __shared__ float xs[kAP][6];
    __shared__ int live[kAP];
    __shared__ float2 wp[kAP][8];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int64_t i0 = (int64_t)blockIdx.x * kAP;
    if (t < kAP) {
        const int64_t i = i0 + t;
        const bool ok = i < ne && exact[erows[i]] == 2;
        live[t] = ok;
#pragma unroll
        for (int q = 0; q < 6; q++) xs[t][q] = ok ? (float)X[(int64_t)erows[i] * VBGS_XS + q] : 0.f;
    }
    __syncthreads();
    const int k = blockIdx.y * 256 + t;
    const bool kv = k < K;
    float r[28];
#pragma unroll
    for (int q = 0; q < 28; q++) r[q] = kv ? rec32[(size_t)k * VBGS_REC + q] : 0.f;
    for (int p = 0; p < kAP; p++) {
        if (!live[p]) continue;
        float x[6];
#pragma unroll
        for (int q = 0; q < 6; q++) x[q] = xs[p][q];
        const float l = kv ? logit32(r, x) : -INFINITY;
        const float m = warp_max(l);
        const float e = (m == -INFINITY) ? 0.f : warp_sum(ex2a(l - m));
        if (lane == 0) wp[p][w] = make_float2(m, e);
    }
    __syncthreads();
    if (t < kAP) {
        float2 out = make_float2(-INFINITY, 0.f);
        if (live[t]) {
            float m = -INFINITY;
            for (int q = 0; q < 8; q++) m = fmaxf(m, wp[t][q].x);
            float sum = 0.f;
            if (m != -INFINITY)
                for (int q = 0; q < 8; q++) sum += wp[t][q].y * ex2a(wp[t][q].x - m);
            out = make_float2(m, sum);
        }
        if (i0 + t < ne) part[(i0 + t) * gridDim.y + blockIdx.y] = out;
    }
}

__global__ void __launch_bounds__(256) k_audit_final(const float2 *__restrict__ part, int nch,
                                                     const int *__restrict__ erows, int64_t ne,
                                                     const int *__restrict__ exact, const double *__restrict__ lse_c,
                                                     float *__restrict__ audit_missed)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    const int n = erows[i];
    if (exact[n] != 2) { audit_missed[i] = 0.f; return; }
    float m = -INFINITY;
    for (int c = 0; c < nch; c++) m = fmaxf(m, part[i * nch + c].x);
    double s = 0.0;
    for (int c = 0; c < nch; c++)
        if (part[i * nch + c].x != -INFINITY) s += (double)part[i * nch + c].y * (double)ex2a(part[i * nch + c].x - m);
    const double l2 = (double)m + log2(s);
    const double d = lse_c[n] * 1.4426950408889634 - l2;
    audit_missed[i] = (float)fmax(0.0, -expm1(d * 0.6931471805599453));
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
int prop_launch_kmeans(const float *rec32, int K, float csc, float *pts, float *cent, SortBuffers &sb, int *order,
                       unsigned int *skey, int *cstart, int lloyd_iters, cudaStream_t st)
{
    k_means_of_records<<<(K + 255) / 256, 256, 0, st>>>(rec32, K, csc, pts);
    return prop_launch_lloyd(pts, K, cent, sb, order, skey, cstart, lloyd_iters, st);
}

// lloyd_iters rounds of (nearest centroid, centroid = mean of its members),
// then the nearest-centroid assignment of the final centroids: skey / order
// hold the sorted assignment, cstart the cluster boundaries.
int prop_launch_lloyd(const float *pts, int K, float *cent, SortBuffers &sb, int *order, unsigned int *skey,
                      int *cstart, int lloyd_iters, cudaStream_t st)
{
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

int prop_launch_certificate(const double *rec, const float *rec32, const int *order, const unsigned int *skey,
                            const int *cstart, int K, const double *Spast, const double *dS, const int *kperm,
                            float xmax, float *cpar, double *cscr, float *mscr, cudaStream_t st)
{
    k_cluster_metric<<<kG, 64, 0, st>>>(rec, order, cstart, Spast, dS, kperm, cpar, cscr);
    k_cluster_members<<<(K + 127) / 128, 128, 0, st>>>(rec, rec32, order, skey, K, cscr, mscr);
    k_cluster_tables<<<kG, 64, 0, st>>>(mscr, cstart, xmax, cpar);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

void prop_bounds(const double *X, int64_t N, const float *cpar, float *UB, cudaStream_t st)
{
    if (N > 0) k_bounds<<<dim3((unsigned)((N + 127) / 128), kBG), 128, 0, st>>>(X, N, cpar, UB);
}

size_t prop_cpar_floats() { return (size_t)kG * kCP; }
size_t prop_cscr_doubles() { return (size_t)kG * kCScr; }
size_t prop_mscr_floats(int K) { return (size_t)K * kMS; }

int prop_gemm(int M, int N, int K, const float *A, int sam, int sak, const float *B, int sbk, int sbn, bool exact_b,
              float *C, int ldc, const float *bias, bool relu, bool accumulate, float *part, size_t part_floats,
              int *flags, cudaStream_t st)
{
    return mlp_gemm_tc(M, N, K, A, sam, sak, true, B, sbn, sbk, !exact_b, C, ldc, bias, relu, accumulate, part,
                       part_floats, flags, st);
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
                 cudaStream_t st, int64_t nb, int64_t S)
{
    if (n > 0) k_mlp_inputs<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(X, rows, rstride, n, box, nb, S, out);
}

void prop_cand_init(const int *top, int64_t N, int *cand, int *ncand, int *pend, float2 *run, float2 *part,
                    cudaStream_t st)
{
    if (N > 0) k_cand_init<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(top, N, cand, ncand, pend, run, part);
}

int prop_pend_lists(const int *cand, const int *ncand, const int *pend, int64_t N,
                    const unsigned long long *prev_added, SortBuffers &sb, unsigned int *skey, int *plist,
                    int *pstart, cudaStream_t st)
{
    const int64_t n = N * kAddMax;
    k_pend_keys<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(cand, ncand, pend, N, prev_added, sb.keys_in,
                                                            sb.idx_in);
    size_t bytes = sb.temp_bytes;
    if (cub::DeviceRadixSort::SortPairs(sb.temp, bytes, sb.keys_in, skey, sb.idx_in, plist, (int)n, 0, 11, st) !=
        cudaSuccess)
        return -1;
    k_list_bounds<<<(unsigned)((n + 256) / 256), 256, 0, st>>>(skey, n, pstart);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int64_t prop_score_items_max(int64_t N) { return (N * kAddMax + kPB - 1) / kPB + kG + 1; }

void prop_cand_score(const double *X, const float *rec32, const int *order, const int *cstart, const int *pstart,
                     const int *plist, const int *item_start, int64_t N, const unsigned long long *prev_added,
                     float2 *part, cudaStream_t st)
{
    if (N > 0)
        k_cand_score<<<(unsigned)prop_score_items_max(N), kPB, 0, st>>>(X, rec32, order, cstart, pstart, plist,
                                                                        item_start, prev_added, part);
}

void prop_cand_select(const float *UB, int64_t N, const int *cstart, float thresh, bool final_round, uint32_t seed,
                      uint32_t audit_per_mille, int *cand, int *ncand, int *pend, float2 *run, float2 *part,
                      double *lse_c, float *bound, int *exact, unsigned long long *counters,
                      const unsigned long long *prev_added, unsigned long long *added_out, cudaStream_t st)
{
    if (N > 0)
        k_cand_select<<<(unsigned)((N * 32 + 255) / 256), 256, 0, st>>>(UB, N, cstart, thresh, final_round ? 1 : 0,
                                                                          seed, audit_per_mille, cand, ncand, pend,
                                                                          run, part, lse_c, bound, exact, counters,
                                                                          prev_added, added_out);
}

void prop_cand_count(const int *exact, const int *ncand, const int *cand, const int *cstart, int64_t N,
                     unsigned long long *counters, cudaStream_t st)
{
    if (N > 0) k_cand_count<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(exact, ncand, cand, cstart, N, counters);
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

int prop_cand_items(const int *pstart, const int *cstart, bool pass2, int *item_start, long long *fbase,
                    cudaStream_t st)
{
    k_items<<<1, kG, 0, st>>>(pstart, cstart, pass2 ? kPB2 : kPB, item_start, fbase);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

void prop_cand_pass2(const double *X, const double *lse_c, const float *rec32, const int *order, const int *cstart,
                     const unsigned int *skey, int K, const int *pstart, const int *plist, const int *item_start,
                     const long long *fbase, int n_items, float *part, const int *kperm, double *dS, cudaStream_t st)
{
    if (n_items > 0)
        k_cand_pass2<<<(unsigned)n_items, 64, 0, st>>>(X, lse_c, rec32, order, cstart, pstart, plist, item_start,
                                                        fbase, part);
    k_cand_reduce<<<kG, 128, 0, st>>>(part, rec32, order, cstart, item_start, fbase, kperm, dS);
}

void prop_labels(const double *Xe, const double *lse_e, const int *rows, int64_t rstride, int64_t ne,
                 const float *rec32, const int *order, const int *cstart, const float *UB, float *Q, cudaStream_t st,
                 int64_t nb, int64_t S)
{
    if (ne > 0)
        k_labels<<<(unsigned)((ne * 32 + 255) / 256), 256, 0, st>>>(Xe, lse_e, rows, rstride, ne, rec32, order,
                                                                     cstart, UB, nb, S, Q);
}

size_t prop_audit_floats(int64_t ne, int K) { return (size_t)std::max<int64_t>(ne, 1) * ((K + 255) / 256) * 2; }

void prop_audit(const double *X, const int *erows, int64_t ne, const int *exact, const double *lse_c,
                const float *rec32, int K, float *scratch, float *audit_missed, cudaStream_t st)
{
    if (ne <= 0) return;
    const int nch = (K + 255) / 256;
    float2 *part = reinterpret_cast<float2 *>(scratch);
    k_audit_part<<<dim3((unsigned)((ne + kAP - 1) / kAP), (unsigned)nch), 256, 0, st>>>(X, erows, ne, exact, rec32,
                                                                                          K, part);
    k_audit_final<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(part, nch, erows, ne, exact, lse_c, audit_missed);
}

void prop_lse_combine(double *lse_c, const double *lse_e, const int *erows, int64_t ne, cudaStream_t st)
{
    if (ne > 0) k_lse_combine<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(lse_c, lse_e, erows, ne);
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
