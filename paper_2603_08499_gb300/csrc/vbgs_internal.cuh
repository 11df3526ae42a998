// vbgs_internal.cuh -- shared declarations of the GB300 VBGS library.
//
// Device data layout (all resident in HBM for the life of a context):
//   X      : N x 8 doubles, points (x y z r g b) + 2 pad, caller's frame
//   Spast  : K x 28 doubles, accumulated statistics (Alg. 1 buffer S)
//   dS     : K x 28 doubles, statistics of the current frame (Eq. 3)
//   rec    : K x 32 doubles, E-step record of the current posterior:
//            [0..5] m_k, [6..26] M_k = sqrt(nu_k) L_k^-1 packed lower
//            triangle row-major, [27] c_k (constant of log rho_nk without
//            the -psi(sum alpha) term), [28..31] pad
//   rec32  : K x 32 floats, the same record in FP32, log2 units
//   pcache : K x 40 doubles, effective-prior terms of the frame (+ block sums)
//   lse    : N doubles, logsumexp_k of the logits without -psi(sum alpha)
//   scal   : small FP64 scalars (psi(sum alpha), KL total, sum lse, ...)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <utility>
#include <vector>
#include "../../include/vbgs.h"

#define VBGS_REC 32       // doubles (or floats) per E-step record
#define VBGS_PROP_CLUSTERS 1024   // proposal clusters (k-means of the posterior means)
#define VBGS_PROP_TOP 4           // clusters proposed per point
#define VBGS_PROP_MAXCAND 32      // candidate clusters per point after certified expansion
#define VBGS_XS 8         // doubles per staged point

namespace vbgs {

// Programmatic dependent launch.  A kernel launched with launch_pdl is set up
// while the kernel before it in the stream finishes (its CTAs exiting are the
// trigger), which hides most of the launch latency between dependent kernels.
// It calls pdl_wait() as its first statement: that returns once every earlier
// grid of the stream has completed and its writes are visible (a no-op for a
// kernel launched without the attribute).  An explicit early trigger
// (griddepcontrol.launch_dependents at kernel start) measured slower on the
// K = 50,000 room stream: 3.29e12 against 3.74e12 pair updates/s.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Offsets into the packed lower triangle of a 6x6 matrix, row-major i >= j.
__host__ __device__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }
// Offset of (i, j), i <= j, in the statistics upper triangle (after 1 + D).
__host__ __device__ constexpr int upper_index(int i, int j) { return 7 + i * 6 - i * (i - 1) / 2 + (j - i); }

enum ScalarSlot {
    SC_PSI_AHAT = 0,   // psi(sum_k alpha_k) of the posterior
    SC_KL_TOTAL = 1,   // sum_k KL_NW + KL_Dir
    SC_SUM_LSE = 2,    // sum_n lse_n (without -psi term)
    SC_PSI_ESTEP = 3,  // psi(sum alpha) of the posterior the last E-step ran under
    SC_P1_DONE = 4,    // (as an unsigned int) blocks of the pass-1 plan finished; 0 between plans
    SC_P2_DONE = 5,    // (as an unsigned int) blocks of the pass-2 plan finished; 0 between plans
    SC_MERGE_DONE = 7, // (as an unsigned int) blocks of the lse merge finished; 0 between merges
    SC_COUNT = 8
};

enum FlagSlot {
    FL_BAD_POINT = 0,  // a non-finite coordinate was staged
    FL_NONPD = 1,      // index + 1 of a component whose W^-1 is not PD (0 = none)
    FL_TIMEOUT = 2,
    FL_CHECK = 3,      // a consistency check of the frame's results failed
    FL_COUNT = 4
};

// Arguments of the last tensor-core pass-1 launch (vbgs_profile_replay).
struct Pass1Launch {
    bool valid = false, bf16 = false;
    int grid = 0;
    size_t smem = 0;
    int64_t alloc_gen = -1;            // the context's allocation generation at the launch
    const float *Xhl = nullptr;
    int64_t N = 0;
    int K = 0, ntiles = 0;
    const unsigned char *tiles = nullptr;
    const float *hdr = nullptr;
    const int *list = nullptr, *item_tile = nullptr, *item_lo = nullptr, *item_hi = nullptr, *nitems = nullptr;
    float2 *part = nullptr;
    float *tmax = nullptr;
    int *flags = nullptr;
    uint32_t knobs = 0;
    const float2 *seed = nullptr;      // the seed launch's partials (batch skipping), or none
    float drop = 0.f;
};

// Per-kernel event timing (enabled by vbgs_profile_enable).  Launchers call
// begin()/end() around each kernel; collect() runs after a stream sync.
struct Prof {
    Pass1Launch p1_last;
    bool on = false;
    unsigned mask = ~0u;                // classes timed (bit c)
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<int> cat_of_pair;       // class of event pair i (events 2i, 2i+1)
    double ms[VBGS_PROF_COUNT] = {};
    int64_t n[VBGS_PROF_COUNT] = {};
    unsigned long long *d_pairs = nullptr;   // device counters: [0] pass-2 pairs evaluated, [1] tensor-core pass-1 pairs evaluated
    int64_t pass1_pairs = 0;                   // pairs scored by the CUDA-core pass 1 (all of them)
    void begin(int cat, cudaStream_t st)
    {
        if (!on || !((mask >> cat) & 1u) || used + 2 > pool.size()) return;
        cudaEventRecord(pool[used], st);
        cat_of_pair.push_back(cat);
    }
    void end(cudaStream_t st)
    {
        if (!on || cat_of_pair.size() * 2 != used + 2) return;
        cudaEventRecord(pool[used + 1], st);
        used += 2;
    }
    void collect()
    {
        for (size_t i = 0; 2 * i + 1 < used; i++) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, pool[2 * i], pool[2 * i + 1]) == cudaSuccess) {
                ms[cat_of_pair[i]] += t;
                n[cat_of_pair[i]] += 1;
            }
        }
        cudaGetLastError();
        cat_of_pair.clear();
        used = 0;
    }
};

struct MstepParams {
    double alpha0, beta0, nu0;
    double W0inv[36];
    int K;
    int want_bounds;   // write the eigenvalue bounds of the proposal certificate (record floats 28-30)
    int split;         // the split model: W^-1 block diagonal (position, colour), 3-D Wishart terms per block
    int num_sms;       // SMs of the device (grid of the M-step's list kernel)
};

// Box of the Morton codes (positions only).
struct BoxParams {
    double lo[3], inv_ext[3];
};

struct SortBuffers {
    uint32_t *keys_in = nullptr, *keys_out = nullptr;
    int *idx_in = nullptr;
    void *temp = nullptr;
    size_t temp_bytes = 0;
    int64_t cap = 0;
};

// reassign (vbgs_reassign.cu): 64-bit sort keys and indices for up to cap
// points or components, the caller's Gumbel variates (g) and component tie
// keys (v), the sorted points and components, and the picks for the host
// (rows: n x 6 point coordinates; picks: n points, then n components).
struct ReassignBuffers {
    unsigned long long *k_in = nullptr, *k_out = nullptr;
    int *i_in = nullptr, *i_out = nullptr, *pts = nullptr, *comps = nullptr, *picks = nullptr;
    double *g = nullptr, *v = nullptr, *rows = nullptr;
    void *temp = nullptr;
    size_t temp_bytes = 0;
    int64_t cap = 0;
};
struct ReassignArgs {
    const double *lse = nullptr;   // caller order, without -psi
    const double *psi = nullptr;   // device scalar: psi(sum alpha) of the E-step
    const double *X = nullptr;     // staged points, caller order, N x 8
    const double *S = nullptr;     // S_past, K x 28
    double *m0 = nullptr;          // prior means, K x 6 (updated)
    int64_t N = 0;
    int K = 0, n = 0;
    double inv_tau = 1.0;
    bool have_v = false;
};
size_t reassign_temp_bytes(int64_t n);
// Returns the kernel launches issued, or -1.
int launch_reassign(const ReassignArgs &a, ReassignBuffers &rb, cudaStream_t st);

// Skipping: pass 1 leaves out a (point tile, component tile) and pass 2 a
// (point chunk, component tile) when the tile's certified largest logit is
// more than t nats below a lower bound of the points' lse: every left-out
// r_nk < e^-t, so a point loses at most K e^-t of its mass.  t = ln K + 37
// in the FP64 form (at most e^-37 ~ 1e-16, FP64 rounding) and ln K + 20 in
// the FP32 and tensor-core forms (e^-20 ~ 2e-9, below FP32's 6e-8), at
// least 20 nats.
double skip_nats_for(int precision, int K);

// Arguments of one E-step (pass 1 + pass 2) over a staged frame.
struct EstepBuffers {
    const double *X;      // N x 8
    int64_t N;
    int K;
    const double *rec;    // K x 32
    const float *rec32;   // K x 32
    double *lse;          // N
    double *lse_part;     // per-block partial sums of lse (fixed order)
    double *scal;
    double *part;         // scratch for split partials
    size_t part_cap;      // doubles
    double *dS;           // K x 28
    const int *kperm;     // position -> component (nullptr: identity)
    float *tmax;          // pass-1 tile maxima [N/256][K/64] (nullptr: no skipping)
    float *minlse;        // per 256-point block min of lse
    float skip_nats;      // skip threshold t (skip_nats_for)
};

// ---- kernels / launchers (return number of launches, or -1 on error) ----
int launch_stage_points(const double *src, int64_t N, double *X, int *flags, cudaStream_t st, Prof *pf);
// Posterior update.  dS == nullptr: the posterior is the effective prior
// prior0 (+) S_past (frame start), whose per-component terms are cached in
// `cache` (mstep_cache_doubles(K) doubles) for the KL of later iterations.
size_t mstep_cache_doubles(int K);
// The record kernel runs on st; the KL terms and their sums (scal) on side,
// after ev_fork; ev_join completes them (wait on it before reading scal).
// cache_next (nullable, used only with dS): also write the posterior q of
// every recomputed component as an effective-prior cache entry (one slot per
// recomputed component, with its index); after the commit they are the next
// frame's effective prior bit for bit (the last iteration of a frame), the
// other components keep q = p.
// listed: the statistics reduction already built the list of components to
// recompute (MstepList), so the M-step skips its own scan.
int launch_mstep(const MstepParams &P, const double *m0, const double *Spast, const double *dS,
                 const int *kperm, double *rec, float *rec32, double *cache, int *flags, double *scal,
                 int *tile_dirty, double *cache_next, cudaStream_t st, cudaStream_t side, cudaEvent_t ev_fork,
                 cudaEvent_t ev_join, Prof *pf, bool listed = false);
// The M-step's list of components to recompute, as a statistics reduction
// builds it while it writes Delta S: a component is listed unless its frame
// statistics are all zero and its record holds the effective prior
// (pc33[k * pc_stride] != 0); an unlisted component gets the "q = p" hand-off
// (ks33[k * ks_stride] and the next double set to zero).  count[0] (entries)
// and count[1] (the list kernel's group counter) start at zero.
struct MstepList {
    const double *pc33;
    int pc_stride;
    double *ks33;
    int ks_stride;
    int *list, *count;
};
MstepList mstep_list_view(double *cache, int K);
int launch_move_records(const int *kperm, const int *kinv_old, int K, const double *rec, const float *rec32,
                        double *rec_dst, float *rec32_dst, cudaStream_t st, Prof *pf);
size_t mstep_prior_cache_doubles(int K);
// cache: the prior cache of the frame's previous M-steps; slots: the next
// frame's prior of each component the last M-step recomputed.
int launch_apply_next(int K, const double *slots, double *cache, cudaStream_t st, Prof *pf);
size_t sort_temp_bytes(int64_t n);
int launch_point_order(const double *X, int64_t N, const BoxParams &box, SortBuffers &sb, double *Xs,
                       int *pidx, cudaStream_t st, Prof *pf);
int launch_comp_order(const double *m0, const double *Spast, int K, double beta0, const BoxParams &box,
                      SortBuffers &sb, int *kperm, int *kinv, cudaStream_t st, Prof *pf);
int launch_commit(double *Spast, const double *dS, int K, const int *flags, cudaStream_t st, Prof *pf);
int launch_elbo(double *scal, int64_t N, double *elbo_out, cudaStream_t st, Prof *pf);
// Consistency checks of a frame's results (options.checks): sets
// flags[FL_CHECK] unless every count, moment and lse is finite, every count
// non-negative, sum_k dS_k0 = N and sum_k dS_k(1..6) = sum_n x_n within tol
// (relative).  X: staged points (N x 8); lse may be null.
int launch_check_frame(const double *dS, int K, const double *X, int64_t N, const double *lse, double tol,
                       int *flags, cudaStream_t st, Prof *pf);

// E-step of the CUDA-core forms: FP64 (precision == VBGS_FP64) or FP32.
int launch_estep_cuda_core(const EstepBuffers &B, int precision, bool want_stats, cudaStream_t st,
                           Prof *pf);
size_t estep_cuda_core_scratch(int64_t N, int K, int precision);
int launch_lse_merge(const double2 *part, int nsplit, int64_t N, const int *item_start, double *lse,
                     double *lse_part, float *minlse, double *sum_out, cudaStream_t st, Prof *pf);
int launch_pass2_fp32(const EstepBuffers &B, int tpb, int tkc, cudaStream_t st, Prof *pf);

// Tensor-core form (vbgs_estep_tc.cu): coefficient tiles of 128 components
// (FP16/BF16 hi/lo, 16 KB each, in the MMA's shared-memory layout) with a
// 32-float frame header each, and pass 1 on tcgen05 with TMEM accumulators.
size_t tc_tile_bytes(int K);
// Relaunch a recorded pass-1 launch: once with the pair counter (zeroed by
// the caller) to count its pairs, then reps times back to back (programmatic
// dependent launch, as in the stream) between two events; *ms = mean time per
// launch.  The launch is idempotent: it rewrites the same partials.
int tc_replay_pass1(const Pass1Launch &L, int reps, unsigned long long *pairs, cudaStream_t st, float *ms);
// Limit (SM cycles) of the waits between warp roles of the tensor-core
// kernels on the current device; cycles <= 0 restores the default (~2 s).
int tc_set_wait_limit(long long cycles);
size_t tc_hdr_floats(int K);
size_t tc_tmax_floats(int64_t N, int K);
// dirty: ntiles flags (records rewritten since the tile's last build), then
// the epoch of each tile's last build (set to `epoch` for the tiles built).
int launch_coef_tiles(const double *rec, const float *rec32, int K, bool bf16, unsigned char *tiles, float *hdr,
                      int *dirty, int epoch, cudaStream_t st, Prof *pf);
size_t tc_plan_ints(int64_t N, int K);
size_t tc_pass2_part_doubles(int K);
size_t tc_p1plan_ints(int64_t N, int K);
size_t tc_p1ub_floats(int64_t N, int K);
// plan_done: the plan's finished-block counter (zero between plans; its last
// block builds the work items).  ml (nullable): also build the M-step's list
// (MstepList) while reducing.
int launch_pass2_tc(const float *Xhl, const float *lse2f, int64_t N, int K, bool bf16, const unsigned char *tiles,
                    const float *hdr, const double *rec, const float *tmax, const float *minlse, int *plan, double *part,
                    size_t part_cap_doubles, const int *kperm, double *dS, int *flags, int num_sms, int splits_override,
                    int *nz, bool skip_zero, cudaStream_t st, Prof *pf, uint32_t knobs, double skip_nats,
                    unsigned int *plan_done, const MstepList *ml = nullptr);
int tc_pass1_auto_splits(int64_t N, int K, int num_sms);
int tc_set_attributes();
// Pass 1 on the tensor cores over balanced work items (point tile, list of
// component tiles).  With tmax (skipping on): a first launch evaluates each
// point tile's seed tile (the largest certified logit bound); its exact
// log-sums give a lower bound of every point's lse, and the main launch
// evaluates the other component tiles whose certified bound over the point
// tile is within the skip threshold of it; tmax of the tiles left out is
// -inf.  same_points: X and N are the previous call's (its FP32 split Xhl
// and point-tile boxes are reused; tile_epoch / since: only the bounds of
// tiles built after epoch `since` are recomputed).  item_start_out: the item
// table the lse merge reads; seed_part_out: the seed launch's partials
// (nullptr without skipping).
int launch_pass1_tc(const double *X, float *Xhl, bool same_points, int64_t N, int K, bool bf16,
                    const unsigned char *tiles, const float *hdr, const float *rec32, double *part_buf,
                    size_t part_cap_doubles, float *tmax, int *p1plan, float *p1ub, int *flags, int num_sms,
                    int tiles_per_item, const int *tile_epoch, int since, const int **item_start_out,
                    const double **seed_part_out, cudaStream_t st, Prof *pf, uint32_t knobs, double skip_nats,
                    unsigned int *plan_done);
// lse from pass 1's FP32 item partials and the seed launch's (nullable),
// minlse per 32 points, sum of lse.
int launch_lse_merge_tc(const double *part_buf, const double *seed_part, int64_t N, const int *item_start, double *lse,
                        float *lse2f, double *lse_part, float *minlse, double *sum_out, unsigned int *done,
                        cudaStream_t st, Prof *pf);
int launch_block_sum(const double *part, int n, double *sum_out, cudaStream_t st, Prof *pf);

// Learned proposal (vbgs_proposal.cu).
int prop_launch_kmeans(const float *rec32, int K, float csc, float *pts, float *cent, SortBuffers &sb, int *order,
                       unsigned int *skey, int *cstart, int lloyd_iters, cudaStream_t st);
int prop_launch_lloyd(const float *pts, int K, float *cent, SortBuffers &sb, int *order, unsigned int *skey,
                      int *cstart, int lloyd_iters, cudaStream_t st);
int prop_launch_certificate(const double *rec, const float *rec32, const int *order, const unsigned int *skey,
                            const int *cstart, int K, const double *Spast, const double *dS, const int *kperm,
                            float xmax, float *cpar, double *cscr, float *mscr, cudaStream_t st);
void prop_bounds(const double *X, int64_t N, const float *cpar, float *UB, cudaStream_t st);
size_t prop_cpar_floats();
size_t prop_cscr_doubles();
size_t prop_mscr_floats(int K);
// The network's GEMMs: C = act(A B^T + bias) (+ C) on the tensor cores
// (vbgs_mlp_tc.cu); B(n, k) = B[n * sbn + k * sbk]; exact_b: B holds BF16
// values (the weights), else it is split hi/lo like A.  part: split-K
// workspace (mlp_gemm_part_floats).  Returns the launches, -1 on failure.
int prop_gemm(int M, int N, int K, const float *A, int sam, int sak, const float *B, int sbk, int sbn, bool exact_b,
              float *C, int ldc, const float *bias, bool relu, bool accumulate, float *part, size_t part_floats,
              int *flags, cudaStream_t st);
int mlp_gemm_tc(int M, int N, int K, const float *A, int sam, int sak, bool split_a, const float *B, int sbn,
                int sbk, bool split_b, float *C, int ldc, const float *bias, bool relu, bool accumulate, float *part,
                size_t part_floats, int *flags, cudaStream_t st);
size_t mlp_gemm_part_floats(int M, int N, int K);
void prop_colsum(const float *X, int M, int Nc, float *out, cudaStream_t st);
void prop_relu_bwd(float *dH, const float *H, size_t n, cudaStream_t st);
void prop_softmax_top(const float *Z, int B, const float *Q, float *dZ, int *top, float *loss_sum, cudaStream_t st);
void prop_adam(float *w, float *wq, float *m, float *v, const float *g, size_t n, float lr, int step, cudaStream_t st);
// nb, S: deal the samples round-robin into nb minibatches of stride S (1, 0: in order)
void prop_inputs(const double *X, const int *rows, int64_t rstride, int64_t n, const BoxParams &box, float *out,
                 cudaStream_t st, int64_t nb = 1, int64_t S = 0);
void prop_cand_init(const int *top, int64_t N, int *cand, int *ncand, int *pend, float2 *run, float2 *part,
                    cudaStream_t st);
// One candidate round; prev_added (nullable: the first round) is the previous
// round's count of added clusters, and a round after one that added none
// does nothing.  The score grid is an upper bound of the round's items.
int prop_pend_lists(const int *cand, const int *ncand, const int *pend, int64_t N,
                    const unsigned long long *prev_added, SortBuffers &sb, unsigned int *skey, int *plist,
                    int *pstart, cudaStream_t st);
int64_t prop_score_items_max(int64_t N);
void prop_cand_score(const double *X, const float *rec32, const int *order, const int *cstart, const int *pstart,
                     const int *plist, const int *item_start, int64_t N, const unsigned long long *prev_added,
                     float2 *part, cudaStream_t st);
void prop_cand_select(const float *UB, int64_t N, const int *cstart, float thresh, bool final_round, uint32_t seed,
                      uint32_t audit_per_mille, int *cand, int *ncand, int *pend, float2 *run, float2 *part,
                      double *lse_c, float *bound, int *exact, unsigned long long *counters,
                      const unsigned long long *prev_added, unsigned long long *added_out, cudaStream_t st);
void prop_cand_count(const int *exact, const int *ncand, const int *cand, const int *cstart, int64_t N,
                     unsigned long long *counters, cudaStream_t st);
void prop_gather_rows(const double *X, const int *rows, int64_t n, double *Xe, cudaStream_t st);
int prop_cand_lists(const int *cand, const int *exact, int64_t N, SortBuffers &sb, unsigned int *skey, int *plist,
                    int *pstart, cudaStream_t st);
int prop_cand_items(const int *pstart, const int *cstart, bool pass2, int *item_start, long long *fbase,
                    cudaStream_t st);
void prop_cand_pass2(const double *X, const double *lse_c, const float *rec32, const int *order, const int *cstart,
                     const unsigned int *skey, int K, const int *pstart, const int *plist, const int *item_start,
                     const long long *fbase, int n_items, float *part, const int *kperm, double *dS, cudaStream_t st);
void prop_labels(const double *Xe, const double *lse_e, const int *rows, int64_t rstride, int64_t ne,
                 const float *rec32, const int *order, const int *cstart, const float *UB, float *Q, cudaStream_t st,
                 int64_t nb, int64_t S);
size_t prop_audit_floats(int64_t ne, int K);
void prop_audit(const double *X, const int *erows, int64_t ne, const int *exact, const double *lse_c,
                const float *rec32, int K, float *scratch, float *audit_missed, cudaStream_t st);
void prop_lse_combine(double *lse_c, const double *lse_e, const int *erows, int64_t ne, cudaStream_t st);
void prop_sum_lse(const double *v, int64_t n, double *part, int *nparts, cudaStream_t st);
void prop_add(double *a, const double *b, size_t n, cudaStream_t st);
void prop_init_centroids(const float *rec32, int K, float csc, float *cent, cudaStream_t st);
void prop_sum_final(const double *part, int n, double *out, cudaStream_t st);
int prop_exact_rows(const int *exact, int64_t N, SortBuffers &sb, unsigned int *skey, int *erows, cudaStream_t st);

// Splat rendering (vbgs_render.cu): buffers grown on demand, kept by the context.
struct RenderBuffers {
    float4 *sp = nullptr;                       // K splat records of 4 float4
    int4 *rect = nullptr;                       // K tile rectangles
    long long *cnt = nullptr, *off = nullptr;   // K + 1 tile counts and their exclusive sums
    unsigned long long *zkey = nullptr, *zkey_s = nullptr;
    int *zidx = nullptr, *zidx_s = nullptr, *rank = nullptr;
    unsigned long long *ekey = nullptr, *ekey_s = nullptr;   // (tile << 32 | depth rank) per covered tile
    int *eval = nullptr, *eval_s = nullptr;
    int2 *range = nullptr;                      // per tile: [first, last) of its sorted entries
    float *img = nullptr, *ref = nullptr;
    double *part = nullptr, *out = nullptr;
    void *temp = nullptr;
    size_t temp_bytes = 0;
    size_t cap_sp = 0, cap_rect = 0, cap_cnt = 0, cap_off = 0, cap_zkey = 0, cap_zkey_s = 0, cap_zidx = 0,
           cap_zidx_s = 0, cap_rank = 0, cap_ekey = 0, cap_ekey_s = 0, cap_eval = 0, cap_eval_s = 0, cap_range = 0,
           cap_img = 0, cap_ref = 0, cap_part = 0, cap_out = 0;
};
// Render the posterior prior0 (+) S (K components; d = 6 joint, 3 split) at
// the camera (o[3], Rwc[9] row-major camera-to-world, f) into image (host,
// H x W x 3, may be null); with ref (host, H x W x 3) also the PSNR.
// device_ms: event time of the render's kernels.  0 on success, -1 with why.
int render_frame(const double *m0, const double *S, const MstepParams &P, int d, int K, const double *camera,
                 int W, int H, RenderBuffers &B, float *image, const float *ref, double *psnr, double *device_ms,
                 cudaStream_t st, std::string &why);
void render_free(RenderBuffers &B);

} // namespace vbgs

// State of the learned proposal of a context (VBGS_FLAG_PROPOSAL).
struct PropState {
    bool on = false;
    bool centroids_ready = false;
    // clusters (k-means of the posterior means, at record positions)
    float *cent = nullptr, *kpts = nullptr;
    // certificate: per-cluster centre, metric and bound tables; FP64 scratch
    // of the cluster metrics; per-member bound terms; bounds of the frame
    float *cpar = nullptr, *mscr = nullptr, *ub = nullptr;
    double *cscr = nullptr;
    // candidate pass-2 work items and partials; audit partials
    int *item_start = nullptr;
    long long *fbase = nullptr;
    float *part2 = nullptr, *apart = nullptr;
    size_t part2_cap = 0, apart_cap = 0;
    int *order = nullptr, *cstart = nullptr;
    unsigned int *skey = nullptr;
    // network: [W1 128x6 | b1 128 | W2 128x128 | b2 128 | W3 1024x128 | b3 1024]
    size_t nparam = 0;
    float *w = nullptr, *wq = nullptr, *am = nullptr, *av = nullptr, *grad = nullptr;
    float *gpart = nullptr;          // split-K partials of the GEMMs
    size_t gpart_cap = 0;
    int step = 0;
    int64_t frames_trained = 0;
    int epochs = 8;                  // training epochs per frame (0: the network is not trained)
    float lr = 3e-3f;                // Adam learning rate
    int64_t lab_nb = 1, lab_S = 0;   // minibatches of the frame's labelled points and their slot stride
    // per frame
    int64_t ncap = 0;
    int *top = nullptr, *cand = nullptr, *exact = nullptr, *erows = nullptr, *plist = nullptr, *pstart = nullptr;
    unsigned int *pkey = nullptr, *ekey = nullptr;
    double *lse_c = nullptr, *Xe = nullptr, *lse_e = nullptr, *lsum = nullptr;
    float *bound = nullptr, *audit = nullptr;
    unsigned long long *counters = nullptr;   // [0] candidate pairs, [1] fallback, [2] audit, [3] added, [8 + r] added in round r
    int *ncand = nullptr, *pend = nullptr;    // candidate count and first unscored slot per point
    float2 *run = nullptr, *cpart = nullptr;  // running (max, sum) per point; per-slot partials
    bool frame_exact = false;
    uint64_t frame = 0;
    // training set of the current frame and minibatch buffers
    int64_t lab_cap = 0, n_lab = 0;
    float *Xin = nullptr, *Q = nullptr;
    float *h1 = nullptr, *h2 = nullptr, *z = nullptr, *dz = nullptr, *dh2 = nullptr, *dh1 = nullptr, *loss = nullptr;
    // report of the last frame
    double rep[11] = {};
};

struct vbgs_ctx {
    int K = 0, D = 6;
    int precision = VBGS_FP64;
    int flags = 0;
    int checks = 0;                            // options.checks: consistency checks after every frame
    uint64_t seed = 0;                         // options.seed (0: the library's default)
    std::string autotune_cache;                // options.autotune_cache (empty: automatic decomposition)
    std::vector<std::pair<int, std::pair<int, int>>> tuned;   // size class -> work decomposition from the cache
    double W0_h[36] = {};                      // the prior's Wishart scale as given
    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr;               // KL terms of the M-step, beside the next E-step
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool side_pending = false;                 // KL work launched on side and not yet joined
    bool mstep_listed = false;                 // the last E-step built the M-step's list (MstepList)
    // The last M-step of the previous frame wrote d_pcache_next and the
    // commit made it the effective prior of the next frame bit for bit; the
    // records hold the same posterior (at the positions of d_kinv).
    bool next_prior_ready = false;
    bool next_written = false;                 // this frame's last M-step wrote d_pcache_next
    double *d_pcache_next = nullptr;           // K x 40: the next frame's effective-prior cache
    double *d_rec_alt = nullptr;               // record buffers for a new component order
    float *d_rec32_alt = nullptr;
    int *d_kinv_alt = nullptr;
    vbgs::BoxParams box{};
    vbgs::SortBuffers sb;
    vbgs::ReassignBuffers ra;
    vbgs::RenderBuffers rb;
    int *d_kperm = nullptr, *d_kinv = nullptr, *d_pidx = nullptr;
    double *d_Xs = nullptr;          // staged points in Morton order
    float *d_tmax = nullptr, *d_minlse = nullptr;
    unsigned char *d_tc_tiles = nullptr;   // tensor-core coefficient tiles
    int *d_plan = nullptr;                 // pass-2 work list (counts + chunk lists per tile)
    size_t plan_cap = 0;
    int *d_p1plan = nullptr;               // pass-1 tile lists and work items
    float *d_p1ub = nullptr;               // pass-1 logit bounds per (point tile, component tile)
    float *d_Xhl = nullptr;                // points as FP32 hi/lo pairs (tensor-core builders)
    float *d_lse2f = nullptr;              // lse in log2 units, FP32 (tensor-core pass 2)
    int64_t xhl_cap = 0;
    size_t p1plan_cap = 0;
    float *d_tc_hdr = nullptr;
    // per 128-position tile: a record changed since its last coefficient
    // build; the epoch of the tile's last build; then per quarter tile
    // whether its rows of dS were last written nonzero (tensor-core reduce)
    int *d_tile_dirty = nullptr;
    int coef_epoch = 0;                    // coefficient-tile builds so far
    int plan_epoch = 0;                    // coef_epoch at the last pass-1 plan
    int num_sms = 152;
    int tune_p1 = 0, tune_p2 = 0;          // work decomposition of the tensor-core passes (0 = automatic)
    uint32_t tc_knobs = 0;                 // VBGS_KNOB_*: lo terms left out of the tensor-core products
    int64_t frame_count = 0;               // frames processed (schedule of the components' Morton order)
    double skip_nats = 50.0;               // skip threshold (skip_nats_for)
    int64_t alloc_gen = 0;                 // bumped by every (re)allocation: cached graphs check it
    size_t tmax_cap = 0;
    bool last_sorted = false;
    vbgs::MstepParams mp{};
    std::vector<double> m0_h;
    double *d_m0 = nullptr, *d_Spast = nullptr, *d_dS = nullptr, *d_zero = nullptr;
    double *d_rec = nullptr;
    float *d_rec32 = nullptr;
    double *d_pcache = nullptr;
    double *d_scal = nullptr, *d_elbo = nullptr;
    int *d_flags = nullptr;
    int elbo_cap = 0;
    int64_t ncap = 0;
    double *d_X = nullptr, *d_lse = nullptr, *d_lse_part = nullptr;
    size_t part_cap = 0;
    double *d_part = nullptr;
    int64_t last_N = 0;
    int64_t launches = 0;
    vbgs::Prof prof;
    PropState prop;
    std::string err;
};
