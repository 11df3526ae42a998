/*
 * vbgs.h -- C ABI of the GB300 (sm_103a) VBGS coordinate-ascent update.
 *
 * The library implements the data-parallel hot path of Variational Bayes
 * Gaussian Splatting: the `fit` step of Algorithm 1 (Section 2.1.2) for a
 * mixture of K components over joint D = 6 points x = (x, y, z, r, g, b),
 * each component carrying a conjugate Normal-Wishart prior on its mean and
 * precision and the mixture weights a Dirichlet prior (Fig. 3; the paper's
 * NIW(m, kappa, V, n) in precision space: kappa = beta, V = W^-1, n = nu).
 * One CAVI iteration is
 *   - `compute_elbo_delta`: log rho_nk for every (point, component) pair,
 *     the per-point log-sum-exp lse_n, responsibilities r_nk (Alg. 1);
 *   - `sum_stats_over_samples` as the fused contraction Delta S = R^T S_u of
 *     Eq. 3, with S_u = phi(x) = [1, x, upper(x x^T)]: no N x K (or larger)
 *     array is ever stored;
 *   - `update_from_statistics`: the closed-form FP64 posterior (Alg. 1);
 *   - the ELBO  sum_n lse_n - sum_k KL(NW_k || NW0_k) - KL(Dir || Dir0).
 *
 * Conventions for every entry point:
 *   - return VBGS_OK (0) on success, a negative VBGS_E* code on failure; the
 *     message is available from vbgs_last_error(ctx) (or
 *     vbgs_last_error(NULL) for failures before a context exists);
 *   - the caller owns every pointer it passes; the context owns all device
 *     memory it allocates and frees it in vbgs_destroy;
 *   - point arrays are N x D row-major doubles and may live in host or
 *     device memory (detected with cudaPointerGetAttributes); all other
 *     array arguments are host memory;
 *   - all device work is enqueued on the context's CUDA stream; calls that
 *     return host outputs synchronise that stream before returning;
 *   - a context is not thread-safe: one host thread at a time.
 */
#ifndef VBGS_H
#define VBGS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VBGS_OK        0
#define VBGS_EINVAL   -1   /* bad argument: D != 6, K <= 0, N < 0, NULL, non-finite input */
#define VBGS_ENOMEM   -2   /* device or host allocation failed */
#define VBGS_ECUDA    -3   /* a CUDA runtime call failed */
#define VBGS_ENUMERIC -4   /* a posterior W^-1 is not positive definite (component in message) */
#define VBGS_ETIMEOUT -5   /* a bounded device-side wait gave up */
#define VBGS_ECHECK   -6   /* a consistency check of the frame's results failed (options.checks) */
#define VBGS_EIO      -7   /* a state file could not be written or read, or is not a valid state */

/* Statistics per component, F = 1 + D + D(D+1)/2 = 28 doubles for D = 6:
 * [0] N_k, [1..6] S1 = sum r x, [7..27] S2 = sum r x x^T upper triangle,
 * row-major (0,0),(0,1)..(0,5),(1,1)..(5,5).  Always in the caller's frame. */
#define VBGS_D 6
#define VBGS_F 28

/* Arithmetic of the E-step and statistics passes.  The posterior update and
 * the cross-tile statistic reduction are FP64 in every form.
 *   VBGS_FP64:  all FP64 on CUDA cores, factored quadratic form (the plain
 *               form; parity <= 1e-10 against the FP64 oracle).
 *   VBGS_FP32:  FP32 factored quadratic form on CUDA cores, FP64 partials.
 *   VBGS_FP16X3 / VBGS_BF16X3: logits as a tensor-core GEMM of per-point
 *               features [1, x, upper(x x^T)] against per-component
 *               coefficients, operands split hi/lo in FP16 / BF16 with FP32
 *               accumulation (three products), in a per-component-tile local
 *               frame; statistics R^T phi also on the tensor cores. */
typedef enum {
    VBGS_FP64 = 0,
    VBGS_FP16X3 = 1,
    VBGS_BF16X3 = 2,
    VBGS_FP32 = 3
} vbgs_precision;

/* Option flags.  By default points (per frame) and components (by
 * posterior mean, refreshed every fourth frame) are processed in Morton
 * order, and the passes skip the (point tile, component tile) pairs whose
 * responsibilities are all below e^-t by a certified bound (pass 1: a bound
 * of the tile's logits over the points' box against a lower bound of their
 * lse; pass 2: the tile maxima pass 1 measured); a point then loses at most
 * K e^-t of its mass: t = ln K + 37 in the FP64 form (~1e-16) and ln K + 20
 * in the FP32 and tensor-core forms (~2e-9, below FP32 resolution).
 * Neither changes a result beyond the form's rounding.  The plain form sets
 * both flags. */
#define VBGS_FLAG_NO_REORDER 1   /* process in the caller's order */
#define VBGS_FLAG_NO_SKIP    2   /* evaluate every tile in pass 2 */
#define VBGS_FLAG_PROPOSAL   4   /* learned candidate proposal (see vbgs_proposal_report) */
#define VBGS_FLAG_SPLIT      8   /* the split model of Fig. 3 (below) */

/* The split model (VBGS_FLAG_SPLIT; Sec. 2.1.2, Fig. 3): each component has
 * a spatial Gaussian over (x, y, z) and a colour Gaussian over (r, g, b), each
 * with its own Normal-Wishart prior and posterior, and one Dirichlet over the
 * weights; log rho_nk is E[ln pi_k] plus the two blocks' expected
 * log-likelihoods.  The blocks share alpha0, beta0, nu0 (nu0 > 2) and m0;
 * their prior scales are the diagonal 3 x 3 blocks of W0.  The statistics keep
 * the layout above (the position-colour cross moments are accumulated and not
 * used), every W^-1 is block diagonal, and the ELBO's KL is the Dirichlet term
 * plus both blocks' Normal-Wishart terms. */

/* Options of a context (vbgs_init, vbgs_load_state).  A zero-filled struct
 * is the FP64 form on the legacy default stream with every default.
 *   checks: 1 = after every frame, run the consistency checks of the frame's
 *     results on the device (every count, moment and lse_n finite and the
 *     counts non-negative; sum_k Delta N_k = N and sum_k Delta S1_k =
 *     sum_n x_n within the form's tolerance: 1e-9 relative for FP64, 1e-3
 *     otherwise); a failed check returns VBGS_ECHECK and, like every failed
 *     frame, leaves S_past unchanged.  0 = off.
 *   autotune_cache: tensor-core forms only; non-NULL = before the first frame
 *     of each size class (rounded log2 N) pick the work decomposition with
 *     vbgs_autotune on that frame's points, read from / added to this JSON
 *     file; NULL = the automatic decomposition.  The path is copied.
 *   seed: seed of the library's own random draws (the proposal network's
 *     initial weights and its audit sample); 0 = the library's default. */
typedef struct {
    int precision;        /* vbgs_precision */
    int flags;            /* VBGS_FLAG_* */
    void *cuda_stream;    /* cudaStream_t to enqueue on; NULL = legacy default stream */
    int checks;
    const char *autotune_cache;
    uint64_t seed;
} vbgs_options;

/* Prior of every component (Sec. 2.1.2): Dirichlet(alpha0) weights and
 * NW(m0_k, beta0, W0, nu0) per component.  m0 is K x D row-major (host),
 * W0 the D x D Wishart scale in precision space (host, symmetric positive
 * definite).  Both are copied by vbgs_init. */
typedef struct {
    double alpha0, beta0, nu0;
    const double *m0;
    const double *W0;
} vbgs_prior;

typedef struct vbgs_ctx vbgs_ctx;

/* Create a context (Sec. 2.1.2: the model of Fig. 3 under its conjugate prior;
 * Alg. 1 starts from S = 0) for K components of dimension D (must be 6) with the given
 * prior; opt may be NULL (FP64 form, default stream).  The accumulated
 * statistics S_past start at zero, so the model starts at the prior.
 * Errors: VBGS_EINVAL (bad sizes, NULL, nu0 <= D-1 (split model: nu0 <= 2),
 * beta0 <= 0, alpha0 <= 0, W0 not SPD, non-finite m0), VBGS_ENOMEM, VBGS_ECUDA. */
int vbgs_init(vbgs_ctx **out, const vbgs_prior *prior, int K, int D, const vbgs_options *opt);

/* Process one frame X_t (Alg. 1 `fit`): n_iters CAVI iterations over the N
 * points, each an E-step under the current posterior, the fused statistics
 * contraction (Eq. 3) and the FP64 posterior update from S_past + Delta S;
 * then S_past += Delta S (continual, replay-free).  elbo_trace (n_iters
 * doubles, host, may be NULL) receives the ELBO of the posterior entering
 * each iteration, against the effective prior prior0 (+) S_past.  N may be 0.
 * Errors: VBGS_EINVAL (NULL ctx/points with N > 0, N < 0, n_iters < 1,
 * non-finite coordinates; the state is left unchanged: S_past and the
 * posterior.  Without the learned proposal the points are checked while
 * the frame runs, so after such an error the per-call results -- elbo_trace,
 * vbgs_get_lse, vbgs_get_frame_stats -- are undefined), VBGS_ENUMERIC, VBGS_ECUDA,
 * VBGS_ENOMEM. */
int vbgs_update(vbgs_ctx *ctx, const double *points, int64_t N, int n_iters, double *elbo_trace);

/* Alg. 1 `fit` for many independent scenes at once (running them in one launch
 * has no paper counterpart; each scene is its own context, uneven N and K):
 * every scene runs the same frame update as vbgs_update(scenes[i],
 * points[i], N[i], n_iters), all of them as the branches of one CUDA graph
 * launched once, so small scenes fill the SMs that large ones leave idle.
 * The graph's branches are created in decreasing N K (longest first).  The
 * graph is cached by (scenes, N, n_iters, tuning, component-order schedule)
 * and replayed for later frames of the same shapes.  Points are host or
 * device arrays as in vbgs_update; elbo_traces is n_scenes x n_iters (host,
 * may be NULL).  Ordering: the graph starts after the work already queued on
 * every scene's own stream and each scene's stream waits for the graph's
 * end (events, no host wait); inside, the scenes run on the library's own
 * streams (a graph's branches need a stream each).  The call synchronises
 * once, to return the ELBO traces.  Unlike vbgs_update, each frame starts
 * from a posterior recomputed from S_past (a replayed graph cannot take the
 * carried one), which agrees with it bit for bit.
 * Errors as vbgs_update; the message names the scene.  Not thread-safe. */
int vbgs_update_batched(vbgs_ctx *const *scenes, int n_scenes, const double *const *points,
                        const int64_t *N, int n_iters, double *elbo_traces);

/* No paper counterpart (a tuning aid of this library).  Pick the work
 * decomposition of the tensor-core passes (the least number
 * of component tiles per pass-1 work item and of 64-point chunks per pass-2
 * work item; both passes cut their lists of tile pairs not ruled out by the
 * skip bounds into such items, one CTA each) for this context's K and frames
 * of N
 * points, by timing 4 x 4 candidates on `points` (one E-step each; the model
 * state is unchanged).  With cache_path, the choice is read from / added to
 * that JSON file, {"<form>_N2^<log2 N>_K2^<log2 K>_sms<SMs>": [pass-1 tiles,
 * pass-2 chunks], ...} (rounded log2 of N and K; written to path.tmp and
 * renamed over path; VBGS_EIO when that fails).  The
 * CUDA-core forms have nothing to tune (returns VBGS_OK).  vbgs_get_tuning
 * reports the current choice (0 = automatic). */
int vbgs_autotune(vbgs_ctx *ctx, const double *points, int64_t N, const char *cache_path);
int vbgs_get_tuning(const vbgs_ctx *ctx, int *pass1_tiles, int *pass2_chunks);
/* No paper counterpart.  Set the decomposition directly (0 = automatic), e.g. a choice
 * vbgs_autotune made on another context of the same sizes.  Errors:
 * VBGS_EINVAL (NULL ctx, negative values). */
int vbgs_set_tuning(vbgs_ctx *ctx, int pass1_tiles, int pass2_chunks);

/* Learned proposal (VBGS_FLAG_PROPOSAL at vbgs_init).  A small MLP over the
 * point (x, y, z, r, g, b), 6 -> 128 -> 128 -> 1024 with ReLU, BF16-rounded
 * weights and FP32 accumulation, proposes the 4 most likely of 1024
 * component clusters (k-means of the posterior means, 2 Lloyd iterations
 * after every posterior update); the E-step scores only their components.
 * A certified bound of the responsibility mass outside them sends points
 * above 1e-3 to the exact E-step, as does a seeded 1% audit sample, which
 * measures the true missed mass; a frame with more than 20% such points runs
 * exact.  The network is trained on the GPU (forward, backward, Adam lr 3e-3,
 * minibatches of up to 4096 points dealt round-robin from the frame's up to
 * 16,384 labelled points, 8 epochs per frame by default; the GEMMs on the
 * tensor cores, BF16 operands with activations split hi/lo, FP32
 * accumulation) on the cluster masses of the exact E-steps of each frame.
 * vbgs_proposal_report fills out[11]: candidate pairs scored, fallback
 * points, audit points, audit max and mean missed mass, frame ran exact
 * (0/1), mean training loss of the last epoch, frames trained, pairs of the
 * exact E-step, points, clusters added by the certificate (all of the last
 * iteration of the last frame).
 * vbgs_proposal_weights reads (get, 149,504 floats) and/or replaces (set)
 * the FP32 master weights [W1 128x6 | b1 | W2 128x128 | b2 | W3 1024x128 |
 * b3] (setting resets Adam).  vbgs_proposal_grad runs the network on B <=
 * 4096 inputs (B x 6, already mapped to [-1, 1]) and returns the top-4
 * clusters, and with labels (B x 1024) the mean soft cross-entropy and its
 * gradient (host arrays; no update).  vbgs_proposal_clusters refreshes the
 * clusters and returns the centroids (1024 x 6) and each component's
 * cluster (K).  vbgs_proposal_bounds evaluates the certificate of the
 * current posterior (prior (+) accumulated statistics) at N host points
 * (N x 6): ub[n * 1024 + g] (host, N x 1024) is an upper bound, in log2
 * units, of log2 sum_{k in cluster g} exp(l_nk), with l_nk the natural-unit
 * logit of Eq. 1's E-step; cluster_of (K, nullable) receives each
 * component's cluster.  It refreshes the clusters once, like the start of a
 * frame.  The proposal is host-driven (one synchronisation per iteration)
 * and is not available in vbgs_update_batched. */
int vbgs_proposal_report(vbgs_ctx *ctx, double *out);
/* No paper counterpart: the proposal network's training schedule -- epochs
 * over each frame's labelled points (0: the network is not trained; it keeps
 * its initial or loaded weights) and the Adam learning rate.  Defaults: 8
 * epochs, 3e-3.  Errors: VBGS_EINVAL (no proposal, epochs outside 0..1000,
 * learning_rate outside (0, 1)). */
int vbgs_proposal_config(vbgs_ctx *ctx, int epochs, double learning_rate);
int vbgs_proposal_weights(vbgs_ctx *ctx, float *get, const float *set);
int vbgs_proposal_grad(vbgs_ctx *ctx, const float *inputs, const float *labels, int B, float *loss, float *grad,
                       int *top);
int vbgs_proposal_clusters(vbgs_ctx *ctx, float *centroids, int *cluster_of);
int vbgs_proposal_bounds(vbgs_ctx *ctx, const double *points, int64_t N, float *ub, int *cluster_of);

/* No paper counterpart: the clustering step of the learned proposal on
 * caller data.  K points (K x 6 floats, host), G = 1024 centroids (1024 x 6
 * floats, host, in/out: the warm start, replaced by the result), lloyd_iters
 * rounds of Lloyd's algorithm -- each point to its nearest centroid (squared
 * Euclidean distance in FP32, ties to the lower centroid index), then each
 * centroid to the mean of its members (an empty cluster keeps its centroid)
 * -- and cluster_of (K ints, host, may be NULL) receives the nearest-centroid
 * assignment under the returned centroids.  These are the kernels the
 * proposal runs on the posterior means after every posterior update (with
 * lloyd_iters = 2).  Temporary device memory is allocated and freed; the
 * call synchronises.  Errors: VBGS_EINVAL (K < 0, NULL, lloyd_iters outside
 * 0..64, non-finite values), VBGS_ENOMEM, VBGS_ECUDA (message from
 * vbgs_last_error(NULL)). */
int vbgs_kmeans(const float *points, int K, float *centroids, int lloyd_iters, int *cluster_of);

/* Alg. 1 `compute_elbo_delta` and the ELBO of Sec. 2.1.2's model: the ELBO
 * of the points X under the current posterior q = prior0 (+) S_past
 * (the value elbo_trace[0] of a vbgs_update on X would take), without
 * changing the state.  lse_out (N doubles, host, may be NULL) receives the
 * per-point terms lse_n, the per-point ELBO that `reassign` ranks on. */
int vbgs_elbo(vbgs_ctx *ctx, const double *points, int64_t N, double *elbo_out, double *lse_out);

/* reassign (Alg. 1, the step before fit in every frame; Sec. 2.1.2): the
 * per-point ELBO term lse_n of the frame's N points (host or device, N x 6)
 * under the current posterior prior0 (+) S_past, n points sampled toward low
 * ELBO, the n least-used components, and the prior means m0 (position and
 * colour) of those components set to the sampled points.  Nothing else of
 * the prior and nothing of S_past changes; the next vbgs_update starts from
 * the new prior.
 *   Points: the n largest keys g_n - lse_n / tau, ties to the lower index.
 *     gumbel (host, N finite doubles) holds standard Gumbel variates the
 *     caller draws (-ln(-ln u), u uniform on (0, 1)); the n largest keys are
 *     then a sample without replacement with probability proportional to
 *     exp(-lse_n / tau) (Gumbel-top-k).  tau > 0, natural log units.
 *   Components: ascending count N_k of S_past; ties by comp_key (host, K
 *     finite doubles, ascending; NULL: none), then by the lower index.
 *     Components no data has reached (N_k = 0) all tie, so a random
 *     comp_key picks among them at random.
 *   The i-th sampled point (by key rank) becomes the mean of the i-th picked
 *   component.  picked_points (n int64) and picked_comps (n ints), host,
 *   nullable, receive the choices in that order; vbgs_get_lse afterwards
 *   returns the lse_n ranked on.
 * n = 0 changes nothing.  Errors: VBGS_EINVAL (NULL points or gumbel with
 * n > 0, n < 0, n > min(N, K), tau not > 0, a non-finite point, gumbel or
 * comp_key value), VBGS_ENUMERIC, VBGS_ECUDA; on error the prior is
 * unchanged. */
int vbgs_reassign(vbgs_ctx *ctx, const double *points, int64_t N, int n, double tau, const double *gumbel,
                  const double *comp_key, int64_t *picked_points, int *picked_comps);

/* Alg. 1 `update_from_statistics`: the posterior q = prior0 (+) S_past, host
 * arrays allocated by the caller:
 * alpha, beta, nu (K), m (K x D), Winv (K x D x D, full symmetric W^-1).
 * Any pointer may be NULL to skip it. */
int vbgs_get_posterior(vbgs_ctx *ctx, double *alpha, double *beta, double *m,
                       double *Winv, double *nu);

/* Alg. 1's statistics buffer S: the accumulated statistics S_past (K x F, host). */
int vbgs_get_stats(vbgs_ctx *ctx, double *S);

/* Alg. 1's statistics buffer S: replace S_past (K x F, host), e.g. to resume a stream or to evaluate one
 * iteration from a given state.  Errors: VBGS_EINVAL on non-finite input. */
int vbgs_set_stats(vbgs_ctx *ctx, const double *S);

/* Alg. 1's continual state (Sec. 2.1.2: the model M and the statistics
 * buffer S carried from frame to frame) to and from a file.  vbgs_save_state
 * writes everything that determines the context's later results: the prior
 * (alpha0, beta0, nu0, W0 and the current m0, including means `reassign`
 * changed), S_past, the form and flags, the work decomposition, the
 * posterior the last frame's M-step carried into the next frame (records,
 * effective-prior cache, component order, coefficient tiles), and with the
 * learned proposal its network (FP32 master weights, their BF16 copies, the
 * Adam moments and step), the clusters' centroids and the frame counter of
 * its audit sample.  vbgs_load_state creates a new context from such a file
 * (*out, destroy with vbgs_destroy): continuing a stream through it gives
 * the same results, bit for bit, as continuing the saved context.  The form,
 * flags and seed are the saved ones; from opt (may be NULL) only
 * cuda_stream, checks and autotune_cache are taken.  The file is a
 * little-endian binary image with a 64-bit FNV-1a checksum, written to
 * path.tmp and renamed over path; it holds ~1.3 kB per component (plus
 * ~2.4 MB with the proposal).  Both calls synchronise the stream.
 * Errors: VBGS_EINVAL (NULL), VBGS_EIO (cannot write or read the file, bad
 * magic, version, size or checksum), VBGS_ENOMEM, VBGS_ECUDA. */
int vbgs_save_state(vbgs_ctx *ctx, const char *path);
int vbgs_load_state(vbgs_ctx **out, const char *path, const vbgs_options *opt);

/* No paper counterpart: the consistency check that options.checks runs
 * after every frame, on caller data (host arrays): dS (K x 28 statistics),
 * points (N x 6), lse (N, may be NULL).  *ok = 1 when every statistic and
 * lse_n is finite, every count non-negative, |sum_k dS_k0 - N| <= tol
 * max(N, 1) and |sum_k dS_k(1..6) - sum_n x_n| <= tol max(|sum_n x_n|, 1)
 * (Euclidean norms); else *ok = 0.  Temporary device memory is allocated
 * and freed; the call synchronises.  Errors: VBGS_EINVAL, VBGS_ENOMEM,
 * VBGS_ECUDA (message from vbgs_last_error(NULL)). */
int vbgs_check_frame(const double *dS, int K, const double *points, int64_t N, const double *lse, double tol,
                     int *ok);

/* Eq. 3's statistics Delta S (K x F) of the last iteration of the last
 * vbgs_update, and its per-point lse_n (N_last doubles) of Alg. 1's
 * `compute_elbo_delta`. */
int vbgs_get_frame_stats(vbgs_ctx *ctx, double *dS);
int vbgs_get_lse(vbgs_ctx *ctx, double *lse, int64_t N);

/* No paper counterpart: kernel launches issued by the last vbgs_update /
 * vbgs_elbo call. */
int64_t vbgs_last_launch_count(const vbgs_ctx *ctx);

/* No paper counterpart (measurement).  Per-kernel device timing.  When
 * enabled, the library records a CUDA event
 * pair around every kernel it launches on the context's stream and, at the
 * end of each call that synchronises, adds the elapsed times per kernel
 * class.  on: 0 off, 1 every class, otherwise a mask of the classes to time
 * (VBGS_PROF_ONLY(c) | ...): each pair of events serialises its kernel with
 * its neighbours, so timing one class perturbs the rest least.  vbgs_profile_read copies VBGS_PROF_COUNT totals (milliseconds and
 * launch counts) into caller arrays (either may be NULL) and optionally
 * resets them.  vbgs_profile_name(i) names class i. */
enum {
    VBGS_PROF_PASS1 = 0,   /* logits + online log-sum-exp per point */
    VBGS_PROF_MERGE = 1,   /* split merge of lse and fixed-order sums */
    VBGS_PROF_PASS2 = 2,   /* recomputed responsibilities x features (Eq. 3) */
    VBGS_PROF_REDUCE = 3,  /* FP64 cross-split statistic reduction */
    VBGS_PROF_MSTEP = 4,   /* FP64 posterior update, records, coefficient tiles */
    VBGS_PROF_MISC = 5,    /* staging, ELBO, commit */
    VBGS_PROF_PLAN = 6,    /* tensor-core work lists: tile bounds, skip lists, work items */
    VBGS_PROF_KL = 7,      /* KL terms and their sums (second stream, beside the next E-step) */
    VBGS_PROF_COUNT = 8
};
#define VBGS_PROF_ONLY(c) (1 << ((c) + 1))
/* No paper counterpart (measurement): switch the timing described above on
 * or off, and read or reset its totals. */
int vbgs_profile_enable(vbgs_ctx *ctx, int on);
int vbgs_profile_read(vbgs_ctx *ctx, double *ms, int64_t *launches, int reset);
/* No paper counterpart (measurement).  Work counters of the profiled calls
 * since the last reset: pairs scored by
 * pass 1 (every pair in the CUDA-core forms; in the tensor-core forms the
 * pairs of the component tiles its certified bound did not rule out) and
 * pairs pass 2 evaluated (the ones its skip bound did not rule out).
 * Synchronises the stream. */
int vbgs_profile_pairs(vbgs_ctx *ctx, int64_t *pass1_pairs, int64_t *pass2_pairs);
const char *vbgs_profile_name(int i);

/* No paper counterpart (measurement).  The duration of the dominant kernel
 * without its neighbours: the last tensor-core pass-1 launch of the
 * context (the E-step's logits and online log-sum-exp) is launched again,
 * once to count the (point, component) pairs it evaluates and once to warm
 * up, then reps times back to back between two CUDA events on the
 * context's stream; *ms_per_launch receives the mean time per launch,
 * *pairs_per_launch (may be NULL) the pairs and *exp_pairs_per_launch (may be
 * NULL) the pairs whose exponential it takes (the others lie in 64-column
 * batches certified negligible for every row of a warp).  The relaunches
 * rewrite the same partial results, so the context's state is unchanged.
 * Needs a tensor-core context whose buffers have not been reallocated since
 * that launch.  Synchronises.  Errors: VBGS_EINVAL, VBGS_ECUDA,
 * VBGS_ETIMEOUT. */
int vbgs_profile_replay(vbgs_ctx *ctx, int reps, double *ms_per_launch, int64_t *pairs_per_launch,
                        int64_t *exp_pairs_per_launch);

/* No paper counterpart (measurement).  Measure this GPU's arithmetic peaks
 * with short probe kernels (a few
 * milliseconds each, device `device`): out[0] FP64 FMA TFLOP/s, out[1] FP32
 * FMA TFLOP/s, out[2] MUFU ex2.approx.f32 results per second (1e9 units),
 * out[3] SM count.  Used for the ALU rooflines of the CUDA-core kernels. */
int vbgs_probe_peaks(int device, double *out);

/* E-step that allocates no memory.  The paper has no counterpart: this is
 * a deployment variant for callers that cannot call cudaMalloc -- a host
 * runtime that owns all device memory through its own pool, a process held
 * to a fixed device-memory budget, or a frame loop that cannot take an
 * allocation (which may synchronise the device) mid-frame.
 * Under the context's current posterior q = prior0 (+) S_past it writes the
 * per-point lse_n (N doubles) and the frame statistics
 * Delta S = sum_n r_nk [1, x_n, upper(x_n x_n^T)] (K x 28 doubles) into the
 * caller's DEVICE buffers lse_out and dS_out; points is an N x 6 DEVICE
 * array (host pointers are rejected with VBGS_EINVAL before any launch).
 * Arithmetic: an FP64 context runs the FP64 CUDA-core E-step (the values of
 * vbgs_update's first E-step to FP64 rounding); FP32, FP16X3 and BF16X3
 * contexts all run the FP32 CUDA-core E-step (factored quadratic form in FP32,
 * FP64 cross-split sums; not the tensor-core kernels), within the FP32 form's
 * tolerance of the FP64 result.  The posterior and the statistics of the
 * context are not changed (its launch count and last error are).
 * Scratch memory comes from one static device array of
 * VBGS_NOALLOC_SCRATCH_BYTES held by every GPU that loads the library until
 * the process exits; the call fails with VBGS_EINVAL when
 * 32 + 8 N + max(2 N, 28 K) doubles exceed it, e.g.
 * N = 40,000 points with K = 50,000 components fit.  The array's device
 * address is looked up by the first call in each CUDA context (with its
 * device current), so make that first call before any stream capture.  All
 * calls share the array: calls that overlap on the GPU race; calls on one
 * stream are ordered.  Every call validates the points and synchronises the
 * context's stream once to read the result of that check; the results are
 * enqueued on the stream after it without a final sync.
 * Errors: VBGS_EINVAL (NULL, N < 0, a host pointer, sizes beyond the array,
 * non-finite points), VBGS_ECUDA. */
#define VBGS_NOALLOC_SCRATCH_BYTES (24u * 1024u * 1024u)
int vbgs_estep_noalloc(vbgs_ctx *ctx, const double *points, int64_t N, double *lse_out, double *dS_out);

/* The quality metric of the paper (Sec. 5.1, Setup): render
 * the current posterior prior0 (+) S_past at a held-out camera and score it
 * by PSNR = 10 log10(255^2 / MSE), MSE over all pixels and RGB channels on
 * a 0..255 scale.  The paper does not describe its renderer; here every
 * component that data has reached (accumulated count N_k >= 1; the others
 * hold only the prior and are left out) is a splat at its spatial posterior
 * mean with the expected
 * spatial covariance W_s^-1 / (nu - d - 1) of its Wishart posterior (d = 6;
 * 3 for the split model's spatial block), the colour posterior mean clamped
 * to [0, 1] and opacity 0.99, projected by elliptical weighted averaging
 * (perspective Jacobian, +0.3 px^2 on the screen covariance's diagonal;
 * splats nearer than 0.1 m to the camera plane left out) and composited
 * front to back at pixel centres in increasing camera depth (ties by
 * component index): alpha = min(0.99, 0.99 exp(-q / 2)) with q the squared
 * screen-space Mahalanobis distance, alpha < 1/255 skipped, black
 * background.  A pixel stops compositing once its transmittance is below
 * 1e-7.  camera: 13 doubles, host: centre o (3), the camera-to-world
 * rotation Rwc (9, row-major; pixel (u, v) looks along
 * Rwc ((u + 1/2 - width/2) / f, (v + 1/2 - height/2) / f, 1)), focal length
 * f in pixels.  image (height x width x 3 floats, host, may be NULL)
 * receives the rendering; with reference (same layout, host, in [0, 1]) psnr
 * (may be NULL) receives the PSNR against it.  device_ms (may be NULL): the
 * device time of the render's kernels (CUDA events).  The call allocates
 * its buffers on first use (kept by the context) and synchronises.
 * Errors: VBGS_EINVAL (NULL ctx or camera, sizes outside 1..16384, a PSNR
 * without a reference, non-finite camera, f <= 0), VBGS_ECUDA. */
int vbgs_render(vbgs_ctx *ctx, const double *camera, int width, int height, float *image, const float *reference,
                double *psnr, double *device_ms);

/* Per-operation precision of the tensor-core forms, the knobs the
 * mixed-precision search of Sec. 4.2 chooses between (precision_search.py
 * drives it with measured error and latency).  Every product of the passes
 * is a sum of hi*hi, hi*lo and lo*hi terms of FP16 (or BF16) operand pairs;
 * a set bit leaves one lo term out, the operand then carries its hi part
 * alone (11 or 8 significant bits instead of ~22 or ~16):
 *   VBGS_KNOB_P1_PHI_LO  pass 1 (logits): the points' features
 *   VBGS_KNOB_P1_C_LO    pass 1: the components' coefficients
 *   VBGS_KNOB_P2_PHI_LO  pass 2, recomputed logits: the points' features
 *   VBGS_KNOB_P2_C_LO    pass 2, recomputed logits: the coefficients
 *   VBGS_KNOB_P2_P_LO    pass 2, statistics: the responsibilities
 *   VBGS_KNOB_P2_S_LO    pass 2, statistics: the points' features
 * 0 (the default) keeps every term.  The CUDA-core forms ignore the knobs.
 * Errors: VBGS_EINVAL (NULL ctx, unknown bits). */
#define VBGS_KNOB_P1_PHI_LO 1u
#define VBGS_KNOB_P1_C_LO   2u
#define VBGS_KNOB_P2_PHI_LO 4u
#define VBGS_KNOB_P2_C_LO   8u
#define VBGS_KNOB_P2_P_LO   16u
#define VBGS_KNOB_P2_S_LO   32u
#define VBGS_KNOB_ALL       63u
int vbgs_set_precision_knobs(vbgs_ctx *ctx, unsigned int knobs);
unsigned int vbgs_get_precision_knobs(const vbgs_ctx *ctx);

/* No paper counterpart (failure handling).  Set the limit, in SM clock
 * cycles, of the bounded waits between the warp roles of the tensor-core
 * kernels on the current device (default ~2 s; cycles <= 0 restores it).
 * Such a wait that gives up sets the frame's timeout flag: the kernels stop
 * issuing work, wait (with the full limit) for the copies and MMAs already
 * issued, release their tensor memory and return, and the call reports
 * VBGS_ETIMEOUT with S_past unchanged.  A very short limit makes those
 * waits give up as a stalled pipeline would, which is how the timeout path
 * is tested.  Affects every context on the device.  Errors: VBGS_ECUDA. */
int vbgs_set_wait_limit(long long cycles);

/* No paper counterpart.  Message of the last failure on ctx (or of the last failure with no context
 * when ctx is NULL).  Never NULL. */
const char *vbgs_last_error(const vbgs_ctx *ctx);

/* No paper counterpart.  Free every device and host resource of ctx (NULL is a no-op). */
void vbgs_destroy(vbgs_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* VBGS_H */
