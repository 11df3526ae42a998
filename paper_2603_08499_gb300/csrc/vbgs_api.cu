// vbgs_api.cu -- host runtime behind the C ABI of include/vbgs.h.
//
// A context owns every device buffer of one mixture model and the CUDA
// stream its work is enqueued on.  vbgs_update drives Algorithm 1's `fit`
// for one frame: stage the points, form the posterior entering the frame
// (prior0 (+) S_past), then per CAVI iteration the E-step passes, the ELBO
// of the posterior entering the iteration, and the FP64 posterior update;
// finally S_past += Delta S.  All launches go on one stream; the only host
// synchronisations are the validation of device-resident points and the
// read-back of host outputs.
#include "vbgs_internal.cuh"
#include <math.h>
#include <cmath>
#include <stdio.h>
#include <string.h>
#include <algorithm>
#include <cstdarg>
#include <map>
#include <mutex>
#include <tuple>

using namespace vbgs;

namespace {

thread_local std::string g_err;

int fail(vbgs_ctx *ctx, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    g_err = buf;
    return code;
}

#define CU(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? VBGS_ENOMEM : VBGS_ECUDA, \
                        "%s: %s", #call, cudaGetErrorString(e_));                        \
    } while (0)

// Host Cholesky of a symmetric 6x6 matrix; false if not positive definite.
bool host_chol6(const double *A, double *L)
{
    memset(L, 0, 36 * sizeof(double));
    for (int j = 0; j < 6; j++) {
        double d = A[j * 6 + j];
        for (int k = 0; k < j; k++) d -= L[j * 6 + k] * L[j * 6 + k];
        if (!(d > 0.0)) return false;
        d = sqrt(d);
        L[j * 6 + j] = d;
        for (int i = j + 1; i < 6; i++) {
            double t = A[i * 6 + j];
            for (int k = 0; k < j; k++) t -= L[i * 6 + k] * L[j * 6 + k];
            L[i * 6 + j] = t / d;
        }
    }
    return true;
}

// Inverse of an SPD 6x6 matrix through its Cholesky factor.
bool host_spd_inverse6(const double *A, double *Ainv)
{
    double L[36], Li[36] = {0};
    if (!host_chol6(A, L)) return false;
    for (int c = 0; c < 6; c++) {
        Li[c * 6 + c] = 1.0 / L[c * 6 + c];
        for (int i = c + 1; i < 6; i++) {
            double t = 0.0;
            for (int k = c; k < i; k++) t += L[i * 6 + k] * Li[k * 6 + c];
            Li[i * 6 + c] = -t / L[i * 6 + i];
        }
    }
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++) {
            double s = 0.0;
            for (int k = std::max(i, j); k < 6; k++) s += Li[k * 6 + i] * Li[k * 6 + j];
            Ainv[i * 6 + j] = s;
        }
    return true;
}

bool is_device_pointer(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
int dalloc(vbgs_ctx *ctx, T **p, size_t n)
{
    if (*p) cudaFree(*p);
    *p = nullptr;
    if (ctx) ctx->alloc_gen++;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(ctx, e == cudaErrorMemoryAllocation ? VBGS_ENOMEM : VBGS_ECUDA,
                    "cudaMalloc of %zu bytes failed: %s", n * sizeof(T), cudaGetErrorString(e));
    }
    return VBGS_OK;
}

bool is_tc(const vbgs_ctx *ctx) { return ctx->precision == VBGS_FP16X3 || ctx->precision == VBGS_BF16X3; }

// Make the per-frame buffers large enough for N points.
int ensure_capacity(vbgs_ctx *ctx, int64_t N)
{
    int rc;
    if (N > ctx->ncap) {
        int64_t cap = std::max<int64_t>(N, 1024);
        if ((rc = dalloc(ctx, &ctx->d_X, (size_t)cap * VBGS_XS))) return rc;
        if ((rc = dalloc(ctx, &ctx->d_lse, (size_t)cap))) return rc;
        if ((rc = dalloc(ctx, &ctx->d_lse_part, (size_t)(cap + 63) / 64 + 1))) return rc;
        if ((rc = dalloc(ctx, &ctx->d_Xs, (size_t)cap * VBGS_XS))) return rc;
        if ((rc = dalloc(ctx, &ctx->d_pidx, (size_t)cap))) return rc;
        if ((rc = dalloc(ctx, &ctx->d_minlse, (size_t)(cap + 31) / 32 + 1))) return rc;
        ctx->ncap = cap;
    }
    const int64_t scap = std::max<int64_t>(ctx->prop.on ? ctx->ncap * VBGS_PROP_MAXCAND : ctx->ncap, ctx->K);
    if (scap > ctx->sb.cap) {
        if ((rc = dalloc(ctx, &ctx->sb.keys_in, (size_t)scap)) || (rc = dalloc(ctx, &ctx->sb.keys_out, (size_t)scap)) ||
            (rc = dalloc(ctx, &ctx->sb.idx_in, (size_t)scap)))
            return rc;
        size_t tb = sort_temp_bytes(scap);
        unsigned char *t = nullptr;
        if ((rc = dalloc(ctx, &t, tb))) return rc;
        if (ctx->sb.temp) cudaFree(ctx->sb.temp);
        ctx->sb.temp = t;
        ctx->sb.temp_bytes = tb;
        ctx->sb.cap = scap;
    }
    const size_t tneed = std::max((size_t)((std::max<int64_t>(N, 1) + 255) / 256) * (size_t)((ctx->K + 63) / 64),
                                  tc_tmax_floats(std::max<int64_t>(N, 1), ctx->K));
    if (tneed > ctx->tmax_cap) {
        if ((rc = dalloc(ctx, &ctx->d_tmax, tneed))) return rc;
        ctx->tmax_cap = tneed;
    }
    const size_t pneed = tc_plan_ints(std::max<int64_t>(N, 1), ctx->K);
    if (is_tc(ctx) && pneed > ctx->plan_cap) {
        if ((rc = dalloc(ctx, &ctx->d_plan, pneed))) return rc;
        ctx->plan_cap = pneed;
    }
    if (is_tc(ctx) && ctx->ncap > ctx->xhl_cap) {
        if ((rc = dalloc(ctx, &ctx->d_Xhl, (size_t)ctx->ncap * 16)) || (rc = dalloc(ctx, &ctx->d_lse2f, (size_t)ctx->ncap)))
            return rc;
        ctx->xhl_cap = ctx->ncap;
    }
    const size_t p1need = tc_p1plan_ints(std::max<int64_t>(N, 1), ctx->K);
    if (is_tc(ctx) && p1need > ctx->p1plan_cap) {
        if ((rc = dalloc(ctx, &ctx->d_p1plan, p1need)) ||
            (rc = dalloc(ctx, &ctx->d_p1ub, tc_p1ub_floats(std::max<int64_t>(N, 1), ctx->K))))
            return rc;
        ctx->p1plan_cap = p1need;
    }
    size_t need = estep_cuda_core_scratch(std::max<int64_t>(N, 1), ctx->K, is_tc(ctx) ? VBGS_FP32 : ctx->precision);
    if (is_tc(ctx))   // pass-1 partials of up to 64 K-splits; pass-2 item partials
        need = std::max(need, std::max((size_t)64 * (size_t)std::max<int64_t>(N, 1) * 2, tc_pass2_part_doubles(ctx->K)));
    if (need > ctx->part_cap) {
        if ((rc = dalloc(ctx, &ctx->d_part, need))) return rc;
        ctx->part_cap = need;
    }
    return VBGS_OK;
}

int ensure_elbo(vbgs_ctx *ctx, int n)
{
    if (n <= ctx->elbo_cap) return VBGS_OK;
    int cap = std::max(n, 64);
    int rc = dalloc(ctx, &ctx->d_elbo, (size_t)cap);
    if (rc) return rc;
    ctx->elbo_cap = cap;
    return VBGS_OK;
}

// Buffers of vbgs_reassign for up to n points or components.
int ensure_reassign(vbgs_ctx *ctx, int64_t n)
{
    ReassignBuffers &r = ctx->ra;
    if (n <= r.cap) return VBGS_OK;
    const int64_t cap = std::max<int64_t>(n, 1024);
    int rc;
    if ((rc = dalloc(ctx, &r.k_in, (size_t)cap)) || (rc = dalloc(ctx, &r.k_out, (size_t)cap)) ||
        (rc = dalloc(ctx, &r.i_in, (size_t)cap)) || (rc = dalloc(ctx, &r.i_out, (size_t)cap)) ||
        (rc = dalloc(ctx, &r.pts, (size_t)cap)) || (rc = dalloc(ctx, &r.comps, (size_t)cap)) ||
        (rc = dalloc(ctx, &r.picks, (size_t)cap * 2)) || (rc = dalloc(ctx, &r.g, (size_t)cap)) ||
        (rc = dalloc(ctx, &r.v, (size_t)cap)) || (rc = dalloc(ctx, &r.rows, (size_t)cap * 6)))
        return rc;
    unsigned char *t = nullptr;
    const size_t tb = reassign_temp_bytes(cap);
    if ((rc = dalloc(ctx, &t, tb))) return rc;
    if (r.temp) cudaFree(r.temp);
    r.temp = t;
    r.temp_bytes = tb;
    r.cap = cap;
    return VBGS_OK;
}

// Stage N points (host or device) into d_X and validate them.  defer_check:
// the points go to the device as they are, the staging kernel sets the
// bad-point flag and the frame runs on; the commit of S_past skips on that
// flag and check_flags reports it, so the statistics stay unchanged without
// a synchronisation or a host pass over the points here.  Every
// kernel of a frame is bounded whatever the values (indices come from counts
// and lists, never from coordinates).
int stage_points(vbgs_ctx *ctx, const double *points, int64_t N, bool defer_check = false)
{
    if (N == 0) return VBGS_OK;
    if (is_device_pointer(points)) {
        CU(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int) * FL_COUNT, ctx->stream));
        int l = launch_stage_points(points, N, ctx->d_X, ctx->d_flags, ctx->stream, &ctx->prof);
        if (l < 0) return fail(ctx, VBGS_ECUDA, "point staging launch failed");
        ctx->launches += l;
        if (defer_check) return VBGS_OK;
        int bad = 0;
        CU(cudaMemcpyAsync(&bad, ctx->d_flags + FL_BAD_POINT, sizeof(int), cudaMemcpyDeviceToHost,
                           ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        ctx->prof.collect();
        if (bad) return fail(ctx, VBGS_EINVAL, "non-finite point coordinate");
    } else if (defer_check) {
        // one contiguous copy into scratch (the Morton-sorted buffer, written
        // later in the frame), then the staging kernel checks and pads
        CU(cudaMemcpyAsync(ctx->d_Xs, points, sizeof(double) * 6 * (size_t)N, cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int) * FL_COUNT, ctx->stream));
        int l = launch_stage_points(ctx->d_Xs, N, ctx->d_X, ctx->d_flags, ctx->stream, &ctx->prof);
        if (l < 0) return fail(ctx, VBGS_ECUDA, "point staging launch failed");
        ctx->launches += l;
    } else {
        for (int64_t i = 0; i < N * 6; i++)
            if (!std::isfinite(points[i]))
                return fail(ctx, VBGS_EINVAL, "non-finite point coordinate at point %lld",
                            (long long)(i / 6));
        CU(cudaMemcpy2DAsync(ctx->d_X, VBGS_XS * sizeof(double), points, 6 * sizeof(double),
                             6 * sizeof(double), (size_t)N, cudaMemcpyHostToDevice, ctx->stream));
    }
    return VBGS_OK;
}

// The M-step's KL terms run on ctx->side; the main stream waits for them
// before anything reads their sums (the ELBO) or rewrites their inputs (the
// next M-step), and before a call returns.
int join_side(vbgs_ctx *ctx)
{
    if (!ctx->side_pending) return VBGS_OK;
    const cudaError_t e = cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0);
    if (e != cudaSuccess) return fail(ctx, VBGS_ECUDA, "stream join failed: %s", cudaGetErrorString(e));
    ctx->side_pending = false;
    return VBGS_OK;
}

// dS == nullptr: the posterior entering a frame, prior0 (+) S_past.
// write_next: also write the next frame's effective-prior cache (the last
// iteration of a frame).
int run_mstep(vbgs_ctx *ctx, const double *dS, bool write_next = false)
{
    int rc;
    if ((rc = join_side(ctx))) return rc;
    if (!dS) ctx->next_prior_ready = false;
    // the list the last E-step built belongs to these statistics only
    const bool listed = dS == ctx->d_dS && ctx->mstep_listed;
    ctx->mstep_listed = false;
    int l = launch_mstep(ctx->mp, ctx->d_m0, ctx->d_Spast, dS, ctx->d_kperm, ctx->d_rec, ctx->d_rec32, ctx->d_pcache,
                         ctx->d_flags, ctx->d_scal, is_tc(ctx) ? ctx->d_tile_dirty : nullptr,
                         write_next ? ctx->d_pcache_next : nullptr, ctx->stream, ctx->side, ctx->ev_fork, ctx->ev_join,
                         &ctx->prof, listed);
    if (l < 0) return fail(ctx, VBGS_ECUDA, "posterior update launch failed");
    ctx->side_pending = true;
    ctx->launches += l;
    if (is_tc(ctx)) {
        l = launch_coef_tiles(ctx->d_rec, ctx->d_rec32, ctx->K, ctx->precision == VBGS_BF16X3, ctx->d_tc_tiles,
                              ctx->d_tc_hdr, ctx->d_tile_dirty, ++ctx->coef_epoch, ctx->stream, &ctx->prof);
        if (l < 0) return fail(ctx, VBGS_ECUDA, "coefficient tile launch failed");
        ctx->launches += l;
    }
    return VBGS_OK;
}

// The posterior entering a frame when the previous frame's last M-step left
// it ready (next_prior_ready): the commit made S_past bitwise the statistics
// that M-step used, so its posterior is this frame's effective prior and the
// records already hold it.  Move the records to the new component order
// (kinv_old: the positions before it), take the prior cache, KL = 0; the
// psi(sum alpha) of that M-step stays (equal up to the order of the sum).
int frame_start_from_next(vbgs_ctx *ctx, bool moved, const int *kinv_old)
{
    int l;
    if (moved) {
        l = launch_move_records(ctx->d_kperm, kinv_old, ctx->K, ctx->d_rec, ctx->d_rec32, ctx->d_rec_alt,
                                ctx->d_rec32_alt, ctx->stream, &ctx->prof);
        if (l < 0) return fail(ctx, VBGS_ECUDA, "record move launch failed");
        ctx->launches += l;
        std::swap(ctx->d_rec, ctx->d_rec_alt);
        std::swap(ctx->d_rec32, ctx->d_rec32_alt);
        if (is_tc(ctx)) CU(cudaMemsetAsync(ctx->d_tile_dirty, 0x01, sizeof(int) * ((ctx->K + 127) / 128), ctx->stream));
    }
    l = launch_apply_next(ctx->K, ctx->d_pcache_next, ctx->d_pcache, ctx->stream, &ctx->prof);
    if (l < 0) return fail(ctx, VBGS_ECUDA, "prior cache launch failed");
    ctx->launches += l;
    CU(cudaMemsetAsync(ctx->d_scal + SC_KL_TOTAL, 0, sizeof(double), ctx->stream));
    if (is_tc(ctx)) {
        l = launch_coef_tiles(ctx->d_rec, ctx->d_rec32, ctx->K, ctx->precision == VBGS_BF16X3, ctx->d_tc_tiles,
                              ctx->d_tc_hdr, ctx->d_tile_dirty, ++ctx->coef_epoch, ctx->stream, &ctx->prof);
        if (l < 0) return fail(ctx, VBGS_ECUDA, "coefficient tile launch failed");
        ctx->launches += l;
    }
    return VBGS_OK;
}

constexpr int kResortFrames = 4;   // frames between refreshes of the components' Morton order

// Whether this frame refreshes the components' Morton order.
bool resort_due(const vbgs_ctx *ctx) { return ctx->frame_count % kResortFrames == 0; }

// Morton order of the frame's points (sorted staging copy) and, with comps,
// of the components by their posterior mean at frame start.
int order_frame(vbgs_ctx *ctx, int64_t N, bool points, bool comps = true)
{
    ctx->last_sorted = false;
    if (ctx->flags & VBGS_FLAG_NO_REORDER) return VBGS_OK;
    int l;
    if (comps) {
        l = launch_comp_order(ctx->d_m0, ctx->d_Spast, ctx->K, ctx->mp.beta0, ctx->box, ctx->sb, ctx->d_kperm,
                              ctx->d_kinv, ctx->stream, &ctx->prof);
        if (l < 0) return fail(ctx, VBGS_ECUDA, "component ordering failed");
        ctx->launches += 2;
    }
    if (points && N > 0) {
        l = launch_point_order(ctx->d_X, N, ctx->box, ctx->sb, ctx->d_Xs, ctx->d_pidx, ctx->stream, &ctx->prof);
        if (l < 0) return fail(ctx, VBGS_ECUDA, "point ordering failed");
        ctx->launches += 2;
        ctx->last_sorted = true;
    }
    return VBGS_OK;
}

// Full E-step over N staged points X (N x 8) into lse (N) and ctx->d_dS.
int run_estep_on(vbgs_ctx *ctx, const double *X, int64_t N, double *lse, bool want_stats, bool same_points = false)
{
    if (ctx->prof.on && !is_tc(ctx)) ctx->prof.pass1_pairs += N * (int64_t)ctx->K;   // tensor-core pass 1 counts on the device
    if (N == 0) {
        CU(cudaMemsetAsync(ctx->d_scal + SC_SUM_LSE, 0, sizeof(double), ctx->stream));
        if (want_stats) CU(cudaMemsetAsync(ctx->d_dS, 0, sizeof(double) * ctx->K * VBGS_F, ctx->stream));
        return VBGS_OK;
    }
    EstepBuffers B;
    B.X = X;
    B.N = N;
    B.K = ctx->K;
    B.rec = ctx->d_rec;
    B.rec32 = ctx->d_rec32;
    B.lse = lse;
    B.lse_part = ctx->d_lse_part;
    B.scal = ctx->d_scal;
    B.part = ctx->d_part;
    B.part_cap = ctx->part_cap;
    B.dS = ctx->d_dS;
    B.kperm = ctx->d_kperm;
    const bool skip = want_stats && !(ctx->flags & VBGS_FLAG_NO_SKIP);
    B.tmax = skip ? ctx->d_tmax : nullptr;
    B.minlse = skip ? ctx->d_minlse : nullptr;
    B.skip_nats = (float)ctx->skip_nats;
    if (is_tc(ctx)) {
        const int *item_start = nullptr;
        const double *seed_part = nullptr;
        int l = launch_pass1_tc(B.X, ctx->d_Xhl, same_points, N, ctx->K, ctx->precision == VBGS_BF16X3,
                                ctx->d_tc_tiles, ctx->d_tc_hdr, ctx->d_rec32, ctx->d_part, ctx->part_cap, B.tmax,
                                ctx->d_p1plan, ctx->d_p1ub, ctx->d_flags, ctx->num_sms, ctx->tune_p1,
                                ctx->d_tile_dirty + (ctx->K + 127) / 128, ctx->plan_epoch, &item_start, &seed_part,
                                ctx->stream, &ctx->prof, ctx->tc_knobs, ctx->skip_nats,
                                reinterpret_cast<unsigned int *>(ctx->d_scal + SC_P1_DONE));
        ctx->plan_epoch = ctx->coef_epoch;
        ctx->prof.p1_last.alloc_gen = ctx->alloc_gen;
        if (l < 0) return fail(ctx, VBGS_ECUDA, "tensor-core pass 1 launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        ctx->launches += l;
        l = launch_lse_merge_tc(ctx->d_part, seed_part, N, item_start, lse, ctx->d_lse2f, ctx->d_lse_part,
                                B.tmax ? ctx->d_minlse : nullptr, ctx->d_scal + SC_SUM_LSE,
                                reinterpret_cast<unsigned int *>(ctx->d_scal + SC_MERGE_DONE), ctx->stream, &ctx->prof);
        if (l < 0) return fail(ctx, VBGS_ECUDA, "lse merge launch failed");
        ctx->launches += l;
        if (want_stats) {
            // The reduction also builds the M-step's list, which rewrites the
            // KL hand-off: the KL work of the last M-step (second stream) must
            // be done first.
            int rc;
            if ((rc = join_side(ctx))) return rc;
            const MstepList ml = mstep_list_view(ctx->d_pcache, ctx->K);
            l = launch_pass2_tc(ctx->d_Xhl, ctx->d_lse2f, N, ctx->K, ctx->precision == VBGS_BF16X3, ctx->d_tc_tiles, ctx->d_tc_hdr,
                                ctx->d_rec, B.tmax, B.tmax ? ctx->d_minlse : nullptr, ctx->d_plan, ctx->d_part, ctx->part_cap, ctx->d_kperm,
                                ctx->d_dS, ctx->d_flags, ctx->num_sms, ctx->tune_p2,
                                ctx->d_tile_dirty + 2 * ((ctx->K + 127) / 128), same_points, ctx->stream, &ctx->prof,
                                ctx->tc_knobs, ctx->skip_nats, reinterpret_cast<unsigned int *>(ctx->d_scal + SC_P2_DONE),
                                &ml);
            if (l < 0) return fail(ctx, VBGS_ECUDA, "tensor-core pass 2 launch failed (%d): %s", l,
                                   cudaGetErrorString(cudaGetLastError()));
            ctx->launches += l;
            ctx->mstep_listed = true;
        }
        return VBGS_OK;
    }
    int l = launch_estep_cuda_core(B, ctx->precision, want_stats, ctx->stream, &ctx->prof);
    if (l < 0) return fail(ctx, VBGS_ECUDA, "E-step launch failed (%d): %s", l,
                           cudaGetErrorString(cudaGetLastError()));
    ctx->launches += l;
    return VBGS_OK;
}


// ---------------------------------------------------------------------------
// Learned proposal (host side).  Constants of the method: G = 1024 clusters,
// top-4 proposals, missed-mass threshold 1e-3, 1% audit, a frame with more
// than 20% fallback points runs exact, 2 Lloyd iterations per refresh;
// training by default 8 epochs (Adam, lr 3e-3) of minibatches of up to 4096
// over each frame's labelled points (vbgs_proposal_config).
// ---------------------------------------------------------------------------
constexpr int kPG = VBGS_PROP_CLUSTERS, kPTop = VBGS_PROP_TOP, kMB = 4096, kHid = 128;
constexpr float kPropThresh = 1e-3f;
constexpr uint32_t kAuditPerMille = 10;
constexpr double kExactFrameFrac = 0.2;
constexpr int64_t kPropTrainPoints = 16384;
constexpr int kPropRounds = 6;   // candidate rounds: the top 4, then up to 8 clusters per round; the last adds none
constexpr size_t kOffB1 = 128 * 6, kOffW2 = kOffB1 + 128, kOffB2 = kOffW2 + 128 * 128, kOffW3 = kOffB2 + 128,
                 kOffB3 = kOffW3 + 1024 * 128, kNParam = kOffB3 + 1024;

uint64_t splitmix(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

float bf16_round(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return x;
    u += 0x7fffu + ((u >> 16) & 1u);
    u &= 0xffff0000u;
    float y;
    memcpy(&y, &u, 4);
    return y;
}

int prop_set_weights(vbgs_ctx *ctx, const float *w)
{
    std::vector<float> q(kNParam);
    for (size_t i = 0; i < kNParam; i++) q[i] = bf16_round(w[i]);
    CU(cudaMemcpyAsync(ctx->prop.w, w, sizeof(float) * kNParam, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(ctx->prop.wq, q.data(), sizeof(float) * kNParam, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemsetAsync(ctx->prop.am, 0, sizeof(float) * kNParam, ctx->stream));
    CU(cudaMemsetAsync(ctx->prop.av, 0, sizeof(float) * kNParam, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->prop.step = 0;
    return VBGS_OK;
}

int prop_alloc(vbgs_ctx *ctx)
{
    PropState &P = ctx->prop;
    const int K = ctx->K;
    int rc;
    if ((rc = dalloc(ctx, &P.cent, (size_t)kPG * 6)) || (rc = dalloc(ctx, &P.kpts, (size_t)K * 6)) ||
        (rc = dalloc(ctx, &P.cpar, prop_cpar_floats())) ||
        (rc = dalloc(ctx, &P.cscr, prop_cscr_doubles())) || (rc = dalloc(ctx, &P.mscr, prop_mscr_floats(K))) || (rc = dalloc(ctx, &P.order, (size_t)K)) ||
        (rc = dalloc(ctx, &P.cstart, (size_t)kPG + 1)) || (rc = dalloc(ctx, &P.skey, (size_t)K)) ||
        (rc = dalloc(ctx, &P.w, kNParam)) || (rc = dalloc(ctx, &P.wq, kNParam)) || (rc = dalloc(ctx, &P.am, kNParam)) ||
        (rc = dalloc(ctx, &P.av, kNParam)) || (rc = dalloc(ctx, &P.grad, kNParam)) ||
        (rc = dalloc(ctx, &P.h1, (size_t)kMB * kHid)) || (rc = dalloc(ctx, &P.h2, (size_t)kMB * kHid)) ||
        (rc = dalloc(ctx, &P.dh1, (size_t)kMB * kHid)) || (rc = dalloc(ctx, &P.dh2, (size_t)kMB * kHid)) ||
        (rc = dalloc(ctx, &P.z, (size_t)kMB * kPG)) || (rc = dalloc(ctx, &P.dz, (size_t)kMB * kPG)) ||
        (rc = dalloc(ctx, &P.loss, 2)) || (rc = dalloc(ctx, &P.counters, 16)) ||
        (rc = dalloc(ctx, &P.pstart, (size_t)kPG + 1)) || (rc = dalloc(ctx, &P.item_start, (size_t)kPG + 1)) ||
        (rc = dalloc(ctx, &P.fbase, (size_t)kPG + 1)))
        return rc;
    {
        // split-K partials of the largest GEMMs of a minibatch
        const size_t gneed = std::max({mlp_gemm_part_floats(kPG, kHid, kMB), mlp_gemm_part_floats(kMB, kHid, kPG),
                                       mlp_gemm_part_floats(kHid, kHid, kMB), mlp_gemm_part_floats(kHid, 6, kMB),
                                       mlp_gemm_part_floats(kMB, kHid, kHid), mlp_gemm_part_floats(kMB, kPG, kHid),
                                       mlp_gemm_part_floats(kMB, kHid, 6), (size_t)1});
        if ((rc = dalloc(ctx, &P.gpart, gneed))) return rc;
        P.gpart_cap = gneed;
    }
    P.nparam = kNParam;
    // He-uniform initial weights from a fixed seed, zero biases
    std::vector<float> w(kNParam, 0.f);
    uint64_t seed = ctx->seed ? ctx->seed : 0x5eedF00Dull;
    auto fill = [&](size_t off, int fan_out, int fan_in) {
        const double a = std::sqrt(6.0 / fan_in);
        for (size_t i = 0; i < (size_t)fan_out * fan_in; i++)
            w[off + i] = (float)(a * (2.0 * ((splitmix(seed) >> 11) * (1.0 / 9007199254740992.0)) - 1.0));
    };
    fill(0, 128, 6);
    fill(kOffW2, 128, 128);
    fill(kOffW3, 1024, 128);
    P.on = true;
    return prop_set_weights(ctx, w.data());
}

int prop_ensure_frame(vbgs_ctx *ctx, int64_t N)
{
    PropState &P = ctx->prop;
    int rc;
    if (N > P.ncap) {
        const int64_t cap = std::max<int64_t>(N, 1024);
        if ((rc = dalloc(ctx, &P.top, (size_t)cap * kPTop)) || (rc = dalloc(ctx, &P.exact, (size_t)cap)) ||
            (rc = dalloc(ctx, &P.erows, (size_t)cap)) || (rc = dalloc(ctx, &P.plist, (size_t)cap * VBGS_PROP_MAXCAND)) ||
            (rc = dalloc(ctx, &P.cand, (size_t)cap * VBGS_PROP_MAXCAND)) ||
            (rc = dalloc(ctx, &P.pkey, (size_t)cap * VBGS_PROP_MAXCAND)) || (rc = dalloc(ctx, &P.ekey, (size_t)cap)) ||
            (rc = dalloc(ctx, &P.lse_c, (size_t)cap)) || (rc = dalloc(ctx, &P.Xe, (size_t)cap * VBGS_XS)) ||
            (rc = dalloc(ctx, &P.lse_e, (size_t)cap)) || (rc = dalloc(ctx, &P.lsum, (size_t)cap / 256 + 2)) ||
            (rc = dalloc(ctx, &P.bound, (size_t)cap)) || (rc = dalloc(ctx, &P.ub, (size_t)cap * kPG)) ||
            (rc = dalloc(ctx, &P.ncand, (size_t)cap)) || (rc = dalloc(ctx, &P.pend, (size_t)cap)) ||
            (rc = dalloc(ctx, &P.run, (size_t)cap)) || (rc = dalloc(ctx, &P.cpart, (size_t)cap * VBGS_PROP_MAXCAND)) || (rc = dalloc(ctx, &P.audit, (size_t)cap)) ||
            (rc = dalloc(ctx, &P.Xin, (size_t)std::max<int64_t>(cap, kPropTrainPoints) * 6)) ||
            (rc = dalloc(ctx, &P.Q, (size_t)kPropTrainPoints * kPG)))
            return rc;
        P.ncap = cap;
        P.lab_cap = cap;
    }
    return VBGS_OK;
}

// k-means of the posterior means (warm start) and the certificate tables of
// the current posterior; with_frame: the posterior includes the frame's
// statistics dS (weights of the cluster metrics).
int prop_refresh(vbgs_ctx *ctx, bool with_frame)
{
    PropState &P = ctx->prop;
    // colour weighted against position in the clustering: scaled by a fifth
    // of the largest extent of the position box
    const double ext = 1.0 / std::min(ctx->box.inv_ext[0], std::min(ctx->box.inv_ext[1], ctx->box.inv_ext[2]));
    const float csc = (float)(0.2 * ext);
    double xmax = 1.0;
    for (int q = 0; q < 3; q++)
        xmax = std::max(xmax, std::max(std::fabs(ctx->box.lo[q]), std::fabs(ctx->box.lo[q] + 1.0 / ctx->box.inv_ext[q])));
    if (!ctx->sb.temp || ctx->sb.cap < ctx->K || !ctx->d_rec || !ctx->d_rec32)
        return fail(ctx, VBGS_ECUDA, "proposal refresh before the buffers exist");
    if (!P.centroids_ready) {
        prop_init_centroids(ctx->d_rec32, ctx->K, csc, P.cent, ctx->stream);
        P.centroids_ready = true;
    }
    if (prop_launch_kmeans(ctx->d_rec32, ctx->K, csc, P.kpts, P.cent, ctx->sb, P.order, P.skey, P.cstart, 2, ctx->stream) ||
        prop_launch_certificate(ctx->d_rec, ctx->d_rec32, P.order, P.skey, P.cstart, ctx->K, ctx->d_Spast,
                                with_frame ? ctx->d_dS : nullptr, ctx->d_kperm, (float)(4.0 * xmax), P.cpar, P.cscr,
                                P.mscr, ctx->stream))
        return fail(ctx, VBGS_ECUDA, "proposal cluster refresh failed");
    ctx->launches += 11;
    return VBGS_OK;
}

void mlp_forward(vbgs_ctx *ctx, const float *Xin, int B)
{
    PropState &P = ctx->prop;
    const float *q = P.wq;
    float *gp = P.gpart;
    const size_t gc = P.gpart_cap;
    int *fl = ctx->d_flags;
    ctx->launches += prop_gemm(B, kHid, 6, Xin, 6, 1, q, 1, 6, true, P.h1, kHid, q + kOffB1, true, false, gp, gc, fl,
                               ctx->stream);
    ctx->launches += prop_gemm(B, kHid, kHid, P.h1, kHid, 1, q + kOffW2, 1, kHid, true, P.h2, kHid, q + kOffB2, true,
                               false, gp, gc, fl, ctx->stream);
    ctx->launches += prop_gemm(B, kPG, kHid, P.h2, kHid, 1, q + kOffW3, 1, kHid, true, P.z, kPG, q + kOffB3, false,
                               false, gp, gc, fl, ctx->stream);
}

// dz (= dLoss/dlogits) -> parameter gradients of the minibatch
void mlp_backward(vbgs_ctx *ctx, const float *Xin, int B)
{
    PropState &P = ctx->prop;
    const float *q = P.wq;
    float *g = P.grad;
    float *gp = P.gpart;
    const size_t gc = P.gpart_cap;
    int *fl = ctx->d_flags;
    cudaStream_t st = ctx->stream;
    int l = 0;
    l += prop_gemm(kPG, kHid, B, P.dz, 1, kPG, P.h2, kHid, 1, false, g + kOffW3, kHid, nullptr, false, false, gp, gc,
                   fl, st);
    prop_colsum(P.dz, B, kPG, g + kOffB3, st);
    l += prop_gemm(B, kHid, kPG, P.dz, kPG, 1, q + kOffW3, kHid, 1, true, P.dh2, kHid, nullptr, false, false, gp, gc,
                   fl, st);
    prop_relu_bwd(P.dh2, P.h2, (size_t)B * kHid, st);
    l += prop_gemm(kHid, kHid, B, P.dh2, 1, kHid, P.h1, kHid, 1, false, g + kOffW2, kHid, nullptr, false, false, gp,
                   gc, fl, st);
    prop_colsum(P.dh2, B, kHid, g + kOffB2, st);
    l += prop_gemm(B, kHid, kHid, P.dh2, kHid, 1, q + kOffW2, kHid, 1, true, P.dh1, kHid, nullptr, false, false, gp,
                   gc, fl, st);
    prop_relu_bwd(P.dh1, P.h1, (size_t)B * kHid, st);
    l += prop_gemm(kHid, 6, B, P.dh1, 1, kHid, Xin, 6, 1, false, g, 6, nullptr, false, false, gp, gc, fl, st);
    prop_colsum(P.dh1, B, kHid, g + kOffB1, st);
    ctx->launches += l + 5;
}

// Proposal of the frame: top-4 clusters of every (sorted) point.
int prop_propose(vbgs_ctx *ctx, const double *X, int64_t N)
{
    PropState &P = ctx->prop;
    for (int64_t off = 0; off < N; off += kMB) {
        const int B = (int)std::min<int64_t>(kMB, N - off);
        prop_inputs(X + off * VBGS_XS, nullptr, 1, B, ctx->box, P.Xin, ctx->stream);
        mlp_forward(ctx, P.Xin, B);
        prop_softmax_top(P.z, B, nullptr, nullptr, P.top + off * kPTop, nullptr, ctx->stream);
        ctx->launches += 2;   // inputs and top-4; mlp_forward counts its GEMMs
    }
    return cudaGetLastError() == cudaSuccess ? VBGS_OK : fail(ctx, VBGS_ECUDA, "proposal inference failed");
}

// One epoch over the frame's labelled points.
int prop_train(vbgs_ctx *ctx)
{
    PropState &P = ctx->prop;
    if (P.n_lab <= 0 || P.epochs <= 0) return VBGS_OK;
    CU(cudaMemsetAsync(P.loss, 0, sizeof(float) * 2, ctx->stream));
    for (int epoch = 0; epoch < P.epochs; epoch++) {
        if (epoch == P.epochs - 1) CU(cudaMemsetAsync(P.loss, 0, sizeof(float) * 2, ctx->stream));
        for (int64_t b = 0; b < P.lab_nb; b++) {
            const int64_t off = b * P.lab_S;
            const int B = (int)((P.n_lab - b + P.lab_nb - 1) / P.lab_nb);   // samples b, b + nb, ...
            const float *Xin = P.Xin + off * 6;
            mlp_forward(ctx, Xin, B);
            prop_softmax_top(P.z, B, P.Q + off * kPG, P.dz, nullptr, P.loss, ctx->stream);
            mlp_backward(ctx, Xin, B);
            prop_adam(P.w, P.wq, P.am, P.av, P.grad, kNParam, P.lr, ++P.step, ctx->stream);
            ctx->launches += 2;   // softmax and Adam; the forward and backward count theirs
        }
    }
    P.frames_trained++;
    P.rep[7] = (double)P.frames_trained;
    P.rep[6] = -1.0;   // filled by vbgs_proposal_report from the device
    return cudaGetLastError() == cudaSuccess ? VBGS_OK : fail(ctx, VBGS_ECUDA, "proposal training failed");
}

// Labels of the exact points of the frame (cluster masses) and their inputs:
// at most kPropTrainPoints of them, evenly strided over the (Morton-ordered)
// points so the sample covers the whole frame.  rows: frame index of each
// point when X holds gathered points (null: X is the frame).
void prop_label(vbgs_ctx *ctx, const double *X, const double *lse, int64_t n, const int *rows)
{
    PropState &P = ctx->prop;
    const int64_t stride = std::max<int64_t>((n + kPropTrainPoints - 1) / kPropTrainPoints, 1);
    const int64_t m = (n + stride - 1) / stride;
    // minibatch b takes samples b, b + nb, ...: every minibatch spans the frame
    const int64_t nb = std::max<int64_t>((m + kMB - 1) / kMB, 1), S = (m + nb - 1) / nb;
    prop_labels(X, lse, rows, stride, m, ctx->d_rec32, P.order, P.cstart, P.ub, P.Q, ctx->stream, nb, S);
    prop_inputs(X, nullptr, stride, m, ctx->box, P.Xin, ctx->stream, nb, S);
    P.n_lab = m;
    P.lab_nb = nb;
    P.lab_S = S;
    ctx->launches += 2;
}

// The E-step of one iteration with the proposal.
int prop_estep(vbgs_ctx *ctx, int64_t N, bool last_iter)
{
    PropState &P = ctx->prop;
    const double *X = ctx->last_sorted ? ctx->d_Xs : ctx->d_X;
    int rc;
    if (P.frame_exact) {
        if ((rc = run_estep_on(ctx, X, N, ctx->d_lse, true))) return rc;
        if (last_iter) {
            prop_bounds(X, N, P.cpar, P.ub, ctx->stream);
            prop_label(ctx, X, ctx->d_lse, N, nullptr);
            ctx->launches += 1;
        }
        return VBGS_OK;
    }
    prop_bounds(X, N, P.cpar, P.ub, ctx->stream);
    ctx->launches += 1;
    CU(cudaMemsetAsync(P.counters, 0, sizeof(unsigned long long) * 16, ctx->stream));
    const uint32_t seed = (uint32_t)(P.frame * 0x9E3779B1ull) ^ 0xA5A5A5A5u ^ (uint32_t)(ctx->seed ^ (ctx->seed >> 32));
    // candidate rounds: score the pending candidates cluster-major, then
    // merge and select the next clusters by the certificate.  All rounds are
    // enqueued without a host read; a round after one that added no cluster
    // returns at once on the device (its count, counters[8 + round], is 0).
    prop_cand_init(P.top, N, P.cand, P.ncand, P.pend, P.run, P.cpart, ctx->stream);
    ctx->launches += 1;
    static_assert(8 + kPropRounds <= 16, "per-round counts fit the counter array");
    for (int round = 0; round < kPropRounds; round++) {
        const unsigned long long *prev = round ? P.counters + 8 + round - 1 : nullptr;
        if (prop_pend_lists(P.cand, P.ncand, P.pend, N, prev, ctx->sb, P.pkey, P.plist, P.pstart, ctx->stream) ||
            prop_cand_items(P.pstart, P.cstart, false, P.item_start, P.fbase, ctx->stream))
            return fail(ctx, VBGS_ECUDA, "candidate lists failed");
        prop_cand_score(X, ctx->d_rec32, P.order, P.cstart, P.pstart, P.plist, P.item_start, N, prev, P.cpart,
                        ctx->stream);
        prop_cand_select(P.ub, N, P.cstart, kPropThresh, round == kPropRounds - 1, seed, kAuditPerMille, P.cand,
                         P.ncand, P.pend, P.run, P.cpart, P.lse_c, P.bound, P.exact, P.counters, prev,
                         P.counters + 8 + round, ctx->stream);
        ctx->launches += 7;
    }
    prop_cand_count(P.exact, P.ncand, P.cand, P.cstart, N, P.counters, ctx->stream);
    ctx->launches += 1;
    unsigned long long cnt[4];
    CU(cudaMemcpyAsync(cnt, P.counters, sizeof cnt, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    const int64_t nfb = (int64_t)cnt[1], nau = (int64_t)cnt[2], ne = nfb + nau;
    P.rep[10] = (double)cnt[3];
    P.rep[0] = (double)cnt[0];
    P.rep[1] = (double)nfb;
    P.rep[2] = (double)nau;
    P.rep[9] = (double)N;
    if ((double)nfb > kExactFrameFrac * (double)N) {
        // the proposal misses too much on this frame: run it exact
        P.frame_exact = true;
        P.rep[5] = 1.0;
        P.rep[8] = (double)N * ctx->K;
        if ((rc = run_estep_on(ctx, X, N, ctx->d_lse, true))) return rc;
        if (last_iter) prop_label(ctx, X, ctx->d_lse, N, nullptr);
        return VBGS_OK;
    }
    P.rep[5] = 0.0;
    P.rep[8] = (double)ne * ctx->K;
    // exact E-step over the fallback and audit points
    if (prop_exact_rows(P.exact, N, ctx->sb, P.ekey, P.erows, ctx->stream))
        return fail(ctx, VBGS_ECUDA, "exact-row compaction failed");
    prop_gather_rows(X, P.erows, ne, P.Xe, ctx->stream);
    if ((rc = run_estep_on(ctx, P.Xe, ne, P.lse_e, true))) return rc;
    ctx->mstep_listed = false;   // the candidate statistics are added below
    const size_t aneed = prop_audit_floats(ne, ctx->K);
    if (aneed > P.apart_cap) {
        if ((rc = dalloc(ctx, &P.apart, aneed))) return rc;
        P.apart_cap = aneed;
    }
    if (last_iter)   // the report's true missed mass (the last iteration's)
        prop_audit(X, P.erows, ne, P.exact, P.lse_c, ctx->d_rec32, ctx->K, P.apart, P.audit, ctx->stream);
    prop_lse_combine(P.lse_c, P.lse_e, P.erows, ne, ctx->stream);
    // candidate statistics of the proposal points, added to the exact ones
    if (prop_cand_lists(P.cand, P.exact, N, ctx->sb, P.pkey, P.plist, P.pstart, ctx->stream) ||
        prop_cand_items(P.pstart, P.cstart, true, P.item_start, P.fbase, ctx->stream))
        return fail(ctx, VBGS_ECUDA, "candidate lists failed");
    int n_items = 0;
    long long n_part = 0;
    CU(cudaMemcpyAsync(&n_items, P.item_start + kPG, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(&n_part, P.fbase + kPG, sizeof(long long), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    const size_t pneed = (size_t)n_part * VBGS_F;
    if (pneed > P.part2_cap) {
        if ((rc = dalloc(ctx, &P.part2, pneed + pneed / 4))) return rc;
        P.part2_cap = pneed + pneed / 4;
    }
    prop_cand_pass2(X, P.lse_c, ctx->d_rec32, P.order, P.cstart, P.skey, ctx->K, P.pstart, P.plist, P.item_start,
                    P.fbase, n_items, P.part2, ctx->d_kperm, ctx->d_dS, ctx->stream);
    // lse of every point and its fixed-order sum
    CU(cudaMemcpyAsync(ctx->d_lse, P.lse_c, sizeof(double) * N, cudaMemcpyDeviceToDevice, ctx->stream));
    int nparts = 0;
    prop_sum_lse(P.lse_c, N, P.lsum, &nparts, ctx->stream);
    prop_sum_final(P.lsum, nparts, ctx->d_scal + SC_SUM_LSE, ctx->stream);
    ctx->launches += 15;
    if (last_iter) {
        prop_label(ctx, P.Xe, P.lse_e, ne, P.erows);
        // true missed mass of the audit sample
        std::vector<int> rows((size_t)ne), ex((size_t)N);
        std::vector<float> miss((size_t)ne);
        if (ne > 0) {
            CU(cudaMemcpyAsync(rows.data(), P.erows, sizeof(int) * ne, cudaMemcpyDeviceToHost, ctx->stream));
            CU(cudaMemcpyAsync(miss.data(), P.audit, sizeof(float) * ne, cudaMemcpyDeviceToHost, ctx->stream));
            CU(cudaMemcpyAsync(ex.data(), P.exact, sizeof(int) * N, cudaMemcpyDeviceToHost, ctx->stream));
            CU(cudaStreamSynchronize(ctx->stream));
        }
        double mx = 0.0, sum = 0.0;
        int64_t na = 0;
        for (int64_t i = 0; i < ne; i++)
            if (ex[(size_t)rows[(size_t)i]] == 2) {
                mx = std::max(mx, (double)miss[(size_t)i]);
                sum += miss[(size_t)i];
                na++;
            }
        P.rep[3] = mx;
        P.rep[4] = na ? sum / na : 0.0;
    }
    return VBGS_OK;
}

// same_points: the points are those of the previous E-step of this frame
// (their FP32 split and tile boxes are current).
int run_estep(vbgs_ctx *ctx, int64_t N, bool want_stats, bool last_iter = false, bool same_points = false)
{
    if (ctx->prop.on && want_stats && N > 0) return prop_estep(ctx, N, last_iter);
    return run_estep_on(ctx, ctx->last_sorted ? ctx->d_Xs : ctx->d_X, N, ctx->d_lse, want_stats, same_points);
}

int check_flags(vbgs_ctx *ctx)
{
    int fl[FL_COUNT];
    CU(cudaMemcpyAsync(fl, ctx->d_flags, sizeof fl, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->prof.collect();
    if (fl[FL_BAD_POINT]) return fail(ctx, VBGS_EINVAL, "non-finite point coordinate");
    // a wait that gave up leaves partial statistics behind, which can make a
    // posterior fail too: the timeout is the cause to report
    if (fl[FL_TIMEOUT]) return fail(ctx, VBGS_ETIMEOUT, "a bounded device wait gave up");
    if (fl[FL_NONPD])
        return fail(ctx, VBGS_ENUMERIC, "posterior W^-1 of component %d is not positive definite",
                    fl[FL_NONPD] - 1);
    if (fl[FL_CHECK])
        return fail(ctx, VBGS_ECHECK, "a consistency check of the frame's results failed (non-finite statistics or "
                                      "lse, a negative count, or counts / first moments not conserved)");
    return VBGS_OK;
}

// vbgs_update in three parts: validation, capacity and staging (may
// synchronise); the asynchronous frame itself (stream-capturable); results.
int update_prepare(vbgs_ctx *ctx, const double *points, int64_t N, int n_iters, bool defer_check = false)
{
    if (!ctx) return fail(nullptr, VBGS_EINVAL, "ctx is NULL");
    if (N < 0 || n_iters < 1) return fail(ctx, VBGS_EINVAL, "need N >= 0 and n_iters >= 1");
    if (N > 0 && !points) return fail(ctx, VBGS_EINVAL, "points is NULL");
    ctx->launches = 0;
    int rc;
    // outside any stream capture: finish the M-step work of earlier calls
    if ((rc = join_side(ctx)) || (rc = ensure_capacity(ctx, N)) || (rc = ensure_elbo(ctx, n_iters))) return rc;
    CU(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int) * FL_COUNT, ctx->stream));   // this frame's flags
    return stage_points(ctx, points, N, defer_check);
}

int update_enqueue(vbgs_ctx *ctx, int64_t N, int n_iters, bool carry_prior)
{
    int rc;
    const bool from_next = carry_prior && ctx->next_prior_ready;
    const bool reorder = !(ctx->flags & VBGS_FLAG_NO_REORDER);
    // The components' Morton order is refreshed on every kResortFrames-th
    // frame of the context (their means move little from frame to frame, so
    // the order changes little; any order gives the same results up to the
    // order of sums).  A schedule by frame count alone keeps a batched and a
    // per-scene stream on the same orders.
    const bool resort = reorder && resort_due(ctx);
    ctx->frame_count++;
    ctx->mstep_listed = false;
    ctx->next_prior_ready = false;
    ctx->next_written = false;
    if (from_next && resort) std::swap(ctx->d_kinv, ctx->d_kinv_alt);   // keep the old inverse order
    if ((rc = order_frame(ctx, N, true, resort))) return rc;
    // Posterior entering the frame: the effective prior prior0 (+) S_past.
    if (from_next) {
        if ((rc = frame_start_from_next(ctx, resort, ctx->d_kinv_alt))) return rc;
    } else if ((rc = run_mstep(ctx, nullptr))) return rc;
    const bool prop = ctx->prop.on && N > 0;
    if (prop) {
        ctx->prop.frame_exact = false;
        ctx->prop.n_lab = 0;
        if ((rc = prop_ensure_frame(ctx, N)) || (rc = prop_refresh(ctx, false)) ||
            (rc = prop_propose(ctx, ctx->last_sorted ? ctx->d_Xs : ctx->d_X, N)))
            return rc;
    }
    for (int it = 0; it < n_iters; it++) {
        if ((rc = run_estep(ctx, N, true, it == n_iters - 1, it > 0))) return rc;
        if ((rc = join_side(ctx))) return rc;
        if (launch_elbo(ctx->d_scal, N, ctx->d_elbo + it, ctx->stream, &ctx->prof) < 0)
            return fail(ctx, VBGS_ECUDA, "ELBO launch failed");
        ctx->launches += 1;
        const bool last = it + 1 == n_iters;
        if ((rc = run_mstep(ctx, ctx->d_dS, carry_prior && last))) return rc;
        if (carry_prior && last) ctx->next_written = true;
        if (prop && it + 1 < n_iters && (rc = prop_refresh(ctx, true))) return rc;
    }
    if (ctx->checks) {
        if (launch_check_frame(ctx->d_dS, ctx->K, ctx->d_X, N, prop ? nullptr : ctx->d_lse,
                               ctx->precision == VBGS_FP64 ? 1e-9 : 1e-3, ctx->d_flags, ctx->stream, &ctx->prof) < 0)
            return fail(ctx, VBGS_ECUDA, "check launch failed");
        ctx->launches += 1;
    }
    if (launch_commit(ctx->d_Spast, ctx->d_dS, ctx->K, ctx->d_flags, ctx->stream, &ctx->prof) < 0)
        return fail(ctx, VBGS_ECUDA, "commit launch failed");
    ctx->launches += 1;
    ctx->last_N = N;
    if (prop) {
        if ((rc = prop_train(ctx))) return rc;
        ctx->prop.frame++;
    }
    return join_side(ctx);
}

void free_all(vbgs_ctx *ctx)
{
    void *ptrs[] = {ctx->d_m0, ctx->d_Spast, ctx->d_dS, ctx->d_zero, ctx->d_rec, ctx->d_rec32,
                    ctx->d_pcache, ctx->d_scal, ctx->d_elbo,
                    ctx->d_flags, ctx->d_X, ctx->d_lse, ctx->d_lse_part, ctx->d_part,
                    ctx->d_kperm, ctx->d_kinv, ctx->d_pidx, ctx->d_Xs, ctx->d_tmax, ctx->d_minlse,
                    ctx->sb.keys_in, ctx->sb.keys_out, ctx->sb.idx_in, ctx->sb.temp, ctx->d_tc_tiles, ctx->d_tc_hdr, ctx->d_plan,
                    ctx->d_p1plan, ctx->d_p1ub, ctx->d_tile_dirty, ctx->d_Xhl, ctx->d_lse2f,
                    ctx->d_pcache_next, ctx->d_rec_alt, ctx->d_rec32_alt, ctx->d_kinv_alt,
                    ctx->ra.k_in, ctx->ra.k_out, ctx->ra.i_in, ctx->ra.i_out, ctx->ra.pts, ctx->ra.comps,
                    ctx->ra.picks, ctx->ra.g, ctx->ra.v, ctx->ra.rows, ctx->ra.temp};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    {
        PropState &P = ctx->prop;
        void *pp[] = {P.cent, P.kpts, P.cpar, P.cscr, P.mscr, P.ub, P.order, P.cstart, P.skey, P.w, P.wq, P.am, P.av, P.grad, P.top, P.cand,
                      P.exact, P.erows, P.plist, P.pstart, P.pkey, P.ekey, P.lse_c, P.Xe, P.lse_e, P.lsum, P.bound,
                      P.audit, P.counters, P.Xin, P.Q, P.h1, P.h2, P.z, P.dz, P.dh2, P.dh1, P.loss,
                      P.item_start, P.fbase, P.part2, P.apart, P.ncand, P.pend, P.run, P.cpart, P.gpart};
        for (void *p : pp)
            if (p) cudaFree(p);
    }
    render_free(ctx->rb);
    if (ctx->side) cudaStreamSynchronize(ctx->side);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    ctx->ev_fork = ctx->ev_join = nullptr;
    ctx->side = nullptr;
    for (cudaEvent_t e : ctx->prof.pool) cudaEventDestroy(e);
    ctx->prof.pool.clear();
    if (ctx->prof.d_pairs) cudaFree(ctx->prof.d_pairs);
    ctx->prof.d_pairs = nullptr;
}

} // namespace


// ---------------------------------------------------------------------------
// Batched scenes: one CUDA graph, one branch per scene.
// ---------------------------------------------------------------------------
namespace {

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    std::vector<int64_t> key;
};

struct BatchRuntime {
    std::mutex mu;
    cudaStream_t main = nullptr;
    std::vector<cudaStream_t> pool;
    std::vector<cudaEvent_t> ev, ev_own;
    cudaEvent_t fork = nullptr, done = nullptr;
    std::vector<GraphEntry> cache;   // most recent first, a few entries
    int device = -1;
};
BatchRuntime g_batch;

int batch_streams(int n)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (g_batch.device != dev) {
        g_batch.device = dev;
        g_batch.pool.clear();
        g_batch.ev.clear();
        g_batch.ev_own.clear();
        g_batch.cache.clear();
        g_batch.main = nullptr;
        g_batch.fork = nullptr;
        g_batch.done = nullptr;
    }
    if (!g_batch.main) {
        if (cudaStreamCreateWithFlags(&g_batch.main, cudaStreamNonBlocking) != cudaSuccess) return -1;
        if (cudaEventCreateWithFlags(&g_batch.fork, cudaEventDisableTiming) != cudaSuccess) return -1;
        if (cudaEventCreateWithFlags(&g_batch.done, cudaEventDisableTiming) != cudaSuccess) return -1;
    }
    while ((int)g_batch.pool.size() < n) {
        cudaStream_t st;
        cudaEvent_t e, eo;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return -1;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return -1;
        if (cudaEventCreateWithFlags(&eo, cudaEventDisableTiming) != cudaSuccess) return -1;
        g_batch.pool.push_back(st);
        g_batch.ev.push_back(e);
        g_batch.ev_own.push_back(eo);
    }
    return 0;
}

} // namespace

// Drop cached graphs that reference a context being destroyed.
void batch_forget(const vbgs_ctx *ctx)
{
    std::lock_guard<std::mutex> lock(g_batch.mu);
    for (size_t c = 0; c < g_batch.cache.size();) {
        bool hit = false;
        const auto &k = g_batch.cache[c].key;
        for (size_t i = 1; i + 3 < k.size() + 1; i += 4)
            if (k[i] == (int64_t)(uintptr_t)ctx) hit = true;
        if (hit) {
            cudaGraphExecDestroy(g_batch.cache[c].exec);
            g_batch.cache.erase(g_batch.cache.begin() + c);
        } else {
            c++;
        }
    }
}

extern "C" int vbgs_update_batched(vbgs_ctx *const *scenes, int n_scenes, const double *const *points,
                                   const int64_t *N, int n_iters, double *elbo_traces)
{
    if (!scenes || n_scenes <= 0 || !points || !N || n_iters < 1)
        return fail(nullptr, VBGS_EINVAL, "vbgs_update_batched: bad arguments");
    for (int i = 0; i < n_scenes; i++) {
        if (!scenes[i]) return fail(nullptr, VBGS_EINVAL, "vbgs_update_batched: scene %d is NULL", i);
        if (scenes[i]->prop.on)
            return fail(nullptr, VBGS_EINVAL, "vbgs_update_batched: scene %d uses the proposal (host-driven fallback)", i);
    }
    std::lock_guard<std::mutex> lock(g_batch.mu);
    if (batch_streams(n_scenes) || tc_set_attributes())
        return fail(nullptr, VBGS_ECUDA, "vbgs_update_batched: stream set-up failed");
    vbgs_ctx *ctx = nullptr;   // for CU() error reporting
    // Every scene runs on a stream of the pool for the duration of the call,
    // after the work already queued on its own stream (an event, no host
    // wait); each scene's own stream waits for the graph at the end, so work
    // the caller queues there later is ordered after this call's.
    std::vector<cudaStream_t> own(n_scenes);
    std::vector<bool> prof_on(n_scenes);
    for (int i = 0; i < n_scenes; i++) {
        own[i] = scenes[i]->stream;
        CU(cudaEventRecord(g_batch.ev_own[i], own[i]));
        CU(cudaStreamWaitEvent(g_batch.pool[i], g_batch.ev_own[i], 0));
        scenes[i]->stream = g_batch.pool[i];
        prof_on[i] = scenes[i]->prof.on;
        scenes[i]->prof.on = false;   // no event records inside the graph
    }
    auto restore = [&]() {
        for (int i = 0; i < n_scenes; i++) {
            scenes[i]->stream = own[i];
            scenes[i]->prof.on = prof_on[i];
        }
    };
    int rc = VBGS_OK;
    // 1. validate, size and stage every scene (outside the graph)
    for (int i = 0; i < n_scenes && rc == VBGS_OK; i++) {
        rc = update_prepare(scenes[i], points[i], N[i], n_iters);
        if (rc) g_err = std::string("scene ") + std::to_string(i) + ": " + scenes[i]->err;
    }
    if (rc) { restore(); return rc; }
    for (int i = 0; i < n_scenes; i++) {
        cudaEventRecord(g_batch.ev[i], g_batch.pool[i]);
        cudaStreamWaitEvent(g_batch.main, g_batch.ev[i], 0);
    }
    // 2. the frames of all scenes as one graph (cached by scene, size and iterations)
    std::vector<int64_t> key;
    key.push_back(n_iters);
    for (int i = 0; i < n_scenes; i++) {
        key.push_back((int64_t)(uintptr_t)scenes[i]);
        key.push_back(N[i]);
        key.push_back(scenes[i]->tune_p1 * 1000 + scenes[i]->tune_p2);
        key.push_back(resort_due(scenes[i]) ? 1 : 0);   // the frame's launches include the component order
        key.push_back(scenes[i]->alloc_gen);
    }
    cudaGraphExec_t exec = nullptr;
    for (size_t c = 0; c < g_batch.cache.size(); c++)
        if (g_batch.cache[c].key == key) {
            exec = g_batch.cache[c].exec;
            if (c) std::swap(g_batch.cache[c], g_batch.cache[0]);
            break;
        }
    if (!exec) {
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(g_batch.main, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            restore();
            return fail(nullptr, VBGS_ECUDA, "vbgs_update_batched: capture failed to start");
        }
        cudaEventRecord(g_batch.fork, g_batch.main);
        // branches in decreasing N K (longest processing time first): the
        // largest scenes' kernels are the first ready, the small ones fill in
        std::vector<int> lpt(n_scenes);
        for (int i = 0; i < n_scenes; i++) lpt[i] = i;
        std::stable_sort(lpt.begin(), lpt.end(), [&](int a, int b) {
            return (double)N[a] * scenes[a]->K > (double)N[b] * scenes[b]->K;
        });
        for (int q = 0; q < n_scenes && rc == VBGS_OK; q++) {
            const int i = lpt[q];
            cudaStreamWaitEvent(g_batch.pool[i], g_batch.fork, 0);
            rc = update_enqueue(scenes[i], N[i], n_iters, false);   // graphs replay: no carried prior
            cudaEventRecord(g_batch.ev[i], g_batch.pool[i]);
            cudaStreamWaitEvent(g_batch.main, g_batch.ev[i], 0);
        }
        cudaError_t ce = cudaStreamEndCapture(g_batch.main, &graph);
        if (rc || ce != cudaSuccess || !graph) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            restore();
            return rc ? rc : fail(nullptr, VBGS_ECUDA, "vbgs_update_batched: capture failed: %s", cudaGetErrorString(ce));
        }
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            restore();
            return fail(nullptr, VBGS_ECUDA, "vbgs_update_batched: instantiate failed: %s", cudaGetErrorString(ce));
        }
        GraphEntry e;
        e.exec = exec;
        e.key = key;
        g_batch.cache.insert(g_batch.cache.begin(), e);
        while (g_batch.cache.size() > 4) {
            cudaGraphExecDestroy(g_batch.cache.back().exec);
            g_batch.cache.pop_back();
        }
    }
    if (cudaGraphLaunch(exec, g_batch.main) != cudaSuccess) {
        restore();
        return fail(nullptr, VBGS_ECUDA, "vbgs_update_batched: graph launch failed");
    }
    CU(cudaEventRecord(g_batch.done, g_batch.main));
    for (int i = 0; i < n_scenes; i++) CU(cudaStreamWaitEvent(own[i], g_batch.done, 0));
    // 3. results: ELBO traces and flags of every scene, one synchronisation
    std::vector<int> fl((size_t)n_scenes * FL_COUNT);
    for (int i = 0; i < n_scenes; i++) {
        if (elbo_traces)
            CU(cudaMemcpyAsync(elbo_traces + (size_t)i * n_iters, scenes[i]->d_elbo, sizeof(double) * n_iters,
                               cudaMemcpyDeviceToHost, g_batch.main));
        CU(cudaMemcpyAsync(&fl[(size_t)i * FL_COUNT], scenes[i]->d_flags, sizeof(int) * FL_COUNT,
                           cudaMemcpyDeviceToHost, g_batch.main));
    }
    CU(cudaStreamSynchronize(g_batch.main));
    restore();
    for (int i = 0; i < n_scenes; i++) {
        const int *f = &fl[(size_t)i * FL_COUNT];
        if (f[FL_NONPD])
            return fail(scenes[i], VBGS_ENUMERIC, "scene %d: posterior W^-1 of component %d is not positive definite", i,
                        f[FL_NONPD] - 1);
        if (f[FL_TIMEOUT]) return fail(scenes[i], VBGS_ETIMEOUT, "scene %d: a bounded device wait gave up", i);
    }
    return VBGS_OK;
}

// ---------------------------------------------------------------------------
// Autotuner of the tensor-core work decomposition.
// ---------------------------------------------------------------------------
namespace {

// The autotuner's cache: a JSON object {"size class key": [pass-1 tiles,
// pass-2 chunks], ...}, one entry per line.  The reader accepts exactly that
// shape (what write_tuning_json writes); anything else reads as empty.
std::map<std::string, std::pair<int, int>> read_tuning_json(const char *path)
{
    std::map<std::string, std::pair<int, int>> out;
    FILE *f = fopen(path, "r");
    if (!f) return out;
    std::string text;
    char buf[4096];
    size_t n;
    while ((n = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, n);
    fclose(f);
    size_t i = 0;
    while ((i = text.find('"', i)) != std::string::npos) {
        const size_t j = text.find('"', i + 1);
        if (j == std::string::npos) break;
        const std::string k = text.substr(i + 1, j - i - 1);
        int a = 0, b = 0;
        if (sscanf(text.c_str() + j + 1, " : [ %d , %d ]", &a, &b) == 2 && a >= 0 && b >= 0) out[k] = {a, b};
        i = j + 1;
    }
    return out;
}

bool write_tuning_json(const char *path, const std::map<std::string, std::pair<int, int>> &entries)
{
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return false;
    fprintf(f, "{\n");
    size_t c = 0;
    for (const auto &e : entries)
        fprintf(f, "  \"%s\": [%d, %d]%s\n", e.first.c_str(), e.second.first, e.second.second,
                ++c < entries.size() ? "," : "");
    fprintf(f, "}\n");
    const bool ok = fclose(f) == 0;
    return ok && rename(tmp.c_str(), path) == 0;
}

} // namespace

extern "C" int vbgs_autotune(vbgs_ctx *ctx, const double *points, int64_t N, const char *cache_path)
{
    if (!ctx) return fail(nullptr, VBGS_EINVAL, "ctx is NULL");
    if (N <= 0 || !points) return fail(ctx, VBGS_EINVAL, "vbgs_autotune needs points");
    if (!is_tc(ctx) || ctx->prop.on) return VBGS_OK;   // nothing to tune
    // size class: rounded log2 of N and K
    const int nb = (int)std::lround(std::log2((double)N)), kb = (int)std::lround(std::log2((double)ctx->K));
    char key[96];
    snprintf(key, sizeof key, "form%d_N2^%d_K2^%d_sms%d", ctx->precision, nb, kb, ctx->num_sms);
    std::map<std::string, std::pair<int, int>> entries;
    if (cache_path) {
        entries = read_tuning_json(cache_path);
        auto it = entries.find(key);
        if (it != entries.end()) {
            ctx->tune_p1 = it->second.first;
            ctx->tune_p2 = it->second.second;
            return VBGS_OK;
        }
    }
    int rc;
    if ((rc = update_prepare(ctx, points, N, 1))) return rc;
    if ((rc = order_frame(ctx, N, true)) || (rc = run_mstep(ctx, nullptr))) return rc;
    const int p1c[4] = {2, 4, 8, 16};   // pass 1: least component tiles per work item
    const int p2c[4] = {2, 4, 8, 16};   // pass 2: least chunks per work item
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    const bool pon = ctx->prof.on;
    ctx->prof.on = false;
    float best = 1e30f;
    int b1 = 0, b2 = 0;
    for (int i = 0; i < 4; i++)
        for (int jx = 0; jx < 4; jx++) {
            ctx->tune_p1 = p1c[i];
            ctx->tune_p2 = p2c[jx];
            if ((rc = run_estep(ctx, N, true))) break;   // warm-up
            cudaEventRecord(e0, ctx->stream);
            if ((rc = run_estep(ctx, N, true))) break;
            cudaEventRecord(e1, ctx->stream);
            CU(cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) { best = ms; b1 = p1c[i]; b2 = p2c[jx]; }
        }
    ctx->prof.on = pon;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    ctx->tune_p1 = b1;
    ctx->tune_p2 = b2;
    if ((rc = check_flags(ctx))) return rc;
    if (cache_path) {
        entries = read_tuning_json(cache_path);   // entries other contexts added meanwhile
        entries[key] = {b1, b2};
        if (!write_tuning_json(cache_path, entries))
            return fail(ctx, VBGS_EIO, "vbgs_autotune: cannot write %s", cache_path);
    }
    return VBGS_OK;
}

extern "C" int vbgs_proposal_report(vbgs_ctx *ctx, double *out)
{
    if (!ctx || !out) return fail(ctx, VBGS_EINVAL, "vbgs_proposal_report: NULL argument");
    if (!ctx->prop.on) return fail(ctx, VBGS_EINVAL, "the context has no proposal");
    float loss = 0.f;
    CU(cudaMemcpyAsync(&loss, ctx->prop.loss, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < 11; i++) out[i] = ctx->prop.rep[i];
    out[6] = ctx->prop.n_lab > 0 ? (double)loss / (double)ctx->prop.n_lab : 0.0;
    return VBGS_OK;
}

extern "C" int vbgs_proposal_weights(vbgs_ctx *ctx, float *get, const float *set)
{
    if (!ctx || !ctx->prop.on) return fail(ctx, VBGS_EINVAL, "the context has no proposal");
    if (set) {
        int rc = prop_set_weights(ctx, set);
        if (rc) return rc;
    }
    if (get) {
        CU(cudaMemcpyAsync(get, ctx->prop.w, sizeof(float) * kNParam, cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
    }
    return VBGS_OK;
}

extern "C" int vbgs_proposal_grad(vbgs_ctx *ctx, const float *inputs, const float *labels, int B, float *loss,
                                  float *grad, int *top)
{
    if (!ctx || !ctx->prop.on) return fail(ctx, VBGS_EINVAL, "the context has no proposal");
    if (!inputs || B <= 0 || B > kMB) return fail(ctx, VBGS_EINVAL, "vbgs_proposal_grad: need 1 <= B <= 4096 inputs");
    PropState &P = ctx->prop;
    int rc;
    if ((rc = prop_ensure_frame(ctx, B))) return rc;
    CU(cudaMemcpyAsync(P.Xin, inputs, sizeof(float) * B * 6, cudaMemcpyHostToDevice, ctx->stream));
    mlp_forward(ctx, P.Xin, B);
    if (top) {
        prop_softmax_top(P.z, B, nullptr, nullptr, P.top, nullptr, ctx->stream);
        CU(cudaMemcpyAsync(top, P.top, sizeof(int) * B * kPTop, cudaMemcpyDeviceToHost, ctx->stream));
    }
    if (labels) {
        CU(cudaMemcpyAsync(P.Q, labels, sizeof(float) * B * kPG, cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaMemsetAsync(P.loss, 0, sizeof(float), ctx->stream));
        prop_softmax_top(P.z, B, P.Q, P.dz, nullptr, P.loss, ctx->stream);
        mlp_backward(ctx, P.Xin, B);
        float l = 0.f;
        CU(cudaMemcpyAsync(&l, P.loss, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
        if (grad) CU(cudaMemcpyAsync(grad, P.grad, sizeof(float) * kNParam, cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        if (loss) *loss = l / (float)B;
    }
    CU(cudaStreamSynchronize(ctx->stream));
    return VBGS_OK;
}

extern "C" int vbgs_proposal_config(vbgs_ctx *ctx, int epochs, double learning_rate)
{
    if (!ctx || !ctx->prop.on) return fail(ctx, VBGS_EINVAL, "the context has no proposal");
    if (epochs < 0 || epochs > 1000 || !(learning_rate > 0) || !(learning_rate < 1))
        return fail(ctx, VBGS_EINVAL, "vbgs_proposal_config: need 0 <= epochs <= 1000 and 0 < learning_rate < 1");
    ctx->prop.epochs = epochs;
    ctx->prop.lr = (float)learning_rate;
    return VBGS_OK;
}

extern "C" int vbgs_proposal_clusters(vbgs_ctx *ctx, float *centroids, int *cluster_of)
{
    if (!ctx || !ctx->prop.on) return fail(ctx, VBGS_EINVAL, "the context has no proposal");
    int rc;
    CU(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int) * FL_COUNT, ctx->stream));
    if ((rc = ensure_capacity(ctx, 0)) || (rc = order_frame(ctx, 0, false)) || (rc = run_mstep(ctx, nullptr)) ||
        (rc = prop_refresh(ctx, false)))
        return rc;
    std::vector<int> order(ctx->K), cstart(kPG + 1), kperm(ctx->K);
    if (centroids) CU(cudaMemcpyAsync(centroids, ctx->prop.cent, sizeof(float) * kPG * 6, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(order.data(), ctx->prop.order, sizeof(int) * ctx->K, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(cstart.data(), ctx->prop.cstart, sizeof(int) * (kPG + 1), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(kperm.data(), ctx->d_kperm, sizeof(int) * ctx->K, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (cluster_of)
        for (int g = 0; g < kPG; g++)
            for (int i = cstart[g]; i < cstart[g + 1]; i++) cluster_of[kperm[order[i]]] = g;
    return VBGS_OK;
}

extern "C" int vbgs_kmeans(const float *points, int K, float *centroids, int lloyd_iters, int *cluster_of)
{
    if (K < 0 || (K > 0 && (!points || !centroids)) || lloyd_iters < 0 || lloyd_iters > 64)
        return fail(nullptr, VBGS_EINVAL, "vbgs_kmeans: need K >= 0, points, centroids and 0 <= lloyd_iters <= 64");
    if (K == 0) return VBGS_OK;
    for (size_t i = 0; i < (size_t)K * 6; i++)
        if (!std::isfinite(points[i])) return fail(nullptr, VBGS_EINVAL, "vbgs_kmeans: non-finite point");
    for (int i = 0; i < kPG * 6; i++)
        if (!std::isfinite(centroids[i])) return fail(nullptr, VBGS_EINVAL, "vbgs_kmeans: non-finite centroid");
    // A local context only carries dalloc's error message; release() frees
    // every buffer whatever fails.
    vbgs_ctx tmp_ctx;
    vbgs_ctx *ctx = &tmp_ctx;
    float *d_pts = nullptr, *d_cent = nullptr;
    int *d_order = nullptr, *d_cstart = nullptr;
    unsigned int *d_skey = nullptr;
    SortBuffers sb;
    cudaStream_t st = nullptr;
    auto release = [&]() {
        cudaFree(d_pts); cudaFree(d_cent); cudaFree(d_order); cudaFree(d_cstart); cudaFree(d_skey);
        cudaFree(sb.keys_in); cudaFree(sb.keys_out); cudaFree(sb.idx_in); cudaFree(sb.temp);
        if (st) cudaStreamDestroy(st);
        cudaGetLastError();
    };
    int rc = VBGS_OK;
    const size_t tb = sort_temp_bytes(K);
    unsigned char *temp = nullptr;
    if ((rc = dalloc(ctx, &d_pts, (size_t)K * 6)) || (rc = dalloc(ctx, &d_cent, (size_t)kPG * 6)) ||
        (rc = dalloc(ctx, &d_order, (size_t)K)) || (rc = dalloc(ctx, &d_cstart, (size_t)kPG + 1)) ||
        (rc = dalloc(ctx, &d_skey, (size_t)K)) || (rc = dalloc(ctx, &sb.keys_in, (size_t)K)) ||
        (rc = dalloc(ctx, &sb.keys_out, (size_t)K)) || (rc = dalloc(ctx, &sb.idx_in, (size_t)K)) ||
        (rc = dalloc(ctx, &temp, tb))) {
        sb.temp = temp;
        release();
        return fail(nullptr, rc, "%s", ctx->err.c_str());
    }
    sb.temp = temp;
    sb.temp_bytes = tb;
    sb.cap = K;
    std::vector<int> order(K), cstart(kPG + 1);
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_pts, points, sizeof(float) * K * 6, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_cent, centroids, sizeof(float) * kPG * 6, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && prop_launch_lloyd(d_pts, K, d_cent, sb, d_order, d_skey, d_cstart, lloyd_iters, st))
        e = cudaErrorLaunchFailure;
    if (e == cudaSuccess) e = cudaMemcpyAsync(centroids, d_cent, sizeof(float) * kPG * 6, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(order.data(), d_order, sizeof(int) * K, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cstart.data(), d_cstart, sizeof(int) * (kPG + 1), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    release();
    if (e != cudaSuccess) return fail(nullptr, VBGS_ECUDA, "vbgs_kmeans: %s", cudaGetErrorString(e));
    if (cluster_of)
        for (int g = 0; g < kPG; g++)
            for (int i = cstart[g]; i < cstart[g + 1]; i++) cluster_of[order[i]] = g;
    return VBGS_OK;
}

extern "C" int vbgs_proposal_bounds(vbgs_ctx *ctx, const double *points, int64_t N, float *ub, int *cluster_of)
{
    if (!ctx || !ctx->prop.on) return fail(ctx, VBGS_EINVAL, "the context has no proposal");
    if (N < 0 || (N > 0 && (!points || !ub))) return fail(ctx, VBGS_EINVAL, "vbgs_proposal_bounds: bad arguments");
    PropState &P = ctx->prop;
    int rc;
    if ((rc = ensure_capacity(ctx, N)) || (rc = prop_ensure_frame(ctx, std::max<int64_t>(N, 1))) ||
        (rc = stage_points(ctx, points, N)))
        return rc;
    CU(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int) * FL_COUNT, ctx->stream));
    if ((rc = order_frame(ctx, 0, false)) || (rc = run_mstep(ctx, nullptr)) || (rc = prop_refresh(ctx, false)))
        return rc;
    prop_bounds(ctx->d_X, N, P.cpar, P.ub, ctx->stream);
    if (N > 0)
        CU(cudaMemcpyAsync(ub, P.ub, sizeof(float) * (size_t)N * kPG, cudaMemcpyDeviceToHost, ctx->stream));
    if (cluster_of) {
        std::vector<int> order(ctx->K), cstart(kPG + 1), kperm(ctx->K);
        CU(cudaMemcpyAsync(order.data(), P.order, sizeof(int) * ctx->K, cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaMemcpyAsync(cstart.data(), P.cstart, sizeof(int) * (kPG + 1), cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaMemcpyAsync(kperm.data(), ctx->d_kperm, sizeof(int) * ctx->K, cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        for (int g = 0; g < kPG; g++)
            for (int i = cstart[g]; i < cstart[g + 1]; i++) cluster_of[kperm[order[i]]] = g;
    }
    return check_flags(ctx);
}

extern "C" int vbgs_set_tuning(vbgs_ctx *ctx, int pass1_tiles, int pass2_chunks)
{
    if (!ctx) return fail(nullptr, VBGS_EINVAL, "ctx is NULL");
    if (pass1_tiles < 0 || pass2_chunks < 0) return fail(ctx, VBGS_EINVAL, "vbgs_set_tuning: negative value");
    ctx->tune_p1 = pass1_tiles;
    ctx->tune_p2 = pass2_chunks;
    return VBGS_OK;
}

int vbgs_get_tuning(const vbgs_ctx *ctx, int *pass1_splits, int *pass2_splits)
{
    if (!ctx) return fail(nullptr, VBGS_EINVAL, "ctx is NULL");
    if (pass1_splits) *pass1_splits = ctx->tune_p1;
    if (pass2_splits) *pass2_splits = ctx->tune_p2;
    return VBGS_OK;
}

// ---------------------------------------------------------------------------
// Continual state to and from a file (Alg. 1's model and statistics buffer,
// plus everything the next frame reads, so that a resumed stream continues
// bit for bit).
// ---------------------------------------------------------------------------
namespace {

constexpr char kStateMagic[8] = {'V', 'B', 'G', 'S', 'S', 'T', 'A', 'T'};
constexpr int32_t kStateVersion = 2;

struct StateHeader {
    char magic[8];
    int32_t version, K, D, precision, flags, has_prop, next_prior_ready, coef_epoch, plan_epoch, tune_p1, tune_p2,
        prop_step, prop_centroids_ready, n_sections, prop_epochs;
    float prop_lr;
    uint32_t tc_knobs;
    int64_t frame_count;
    int64_t prop_frames_trained;
    uint64_t prop_frame, seed;
    double alpha0, beta0, nu0, W0[36], box_lo[3], box_inv_ext[3];
};

// One device array of the state: where it lives and its size in bytes.
struct StateSection {
    void *dev;
    size_t bytes;
};

std::vector<StateSection> state_sections(vbgs_ctx *ctx)
{
    const int K = ctx->K;
    const size_t nt = (size_t)(K + 127) / 128;
    std::vector<StateSection> v = {
        {ctx->d_m0, sizeof(double) * K * 6},
        {ctx->d_Spast, sizeof(double) * K * VBGS_F},
        {ctx->d_dS, sizeof(double) * K * VBGS_F},
        {ctx->d_rec, sizeof(double) * K * VBGS_REC},
        {ctx->d_rec32, sizeof(float) * K * VBGS_REC},
        {ctx->d_pcache, sizeof(double) * mstep_cache_doubles(K)},
        {ctx->d_pcache_next, sizeof(double) * mstep_prior_cache_doubles(K)},
        {ctx->d_scal, sizeof(double) * SC_COUNT},
        {ctx->d_kperm, sizeof(int) * K},
        {ctx->d_kinv, sizeof(int) * K},
        {ctx->d_tile_dirty, sizeof(int) * 6 * nt},
        {ctx->d_tc_tiles, tc_tile_bytes(K)},
        {ctx->d_tc_hdr, sizeof(float) * tc_hdr_floats(K)},
    };
    if (ctx->prop.on) {
        const PropState &P = ctx->prop;
        v.push_back({P.cent, sizeof(float) * kPG * 6});
        v.push_back({P.w, sizeof(float) * kNParam});
        v.push_back({P.wq, sizeof(float) * kNParam});
        v.push_back({P.am, sizeof(float) * kNParam});
        v.push_back({P.av, sizeof(float) * kNParam});
    }
    return v;
}

// 64-bit FNV-1a over a byte range, continuing from h.
uint64_t fnv1a(uint64_t h, const void *p, size_t n)
{
    const unsigned char *b = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; i++) {
        h ^= b[i];
        h *= 0x100000001b3ull;
    }
    return h;
}

constexpr uint64_t kFnvBasis = 0xcbf29ce484222325ull;

} // namespace

extern "C" {

int vbgs_init(vbgs_ctx **out, const vbgs_prior *prior, int K, int D, const vbgs_options *opt)
{
    vbgs_ctx *ctx = nullptr;
    if (!out) return fail(nullptr, VBGS_EINVAL, "out is NULL");
    *out = nullptr;
    if (!prior || !prior->m0 || !prior->W0) return fail(nullptr, VBGS_EINVAL, "prior, m0 or W0 is NULL");
    if (D != VBGS_D) return fail(nullptr, VBGS_EINVAL, "D must be 6 (got %d)", D);
    if (K <= 0) return fail(nullptr, VBGS_EINVAL, "K must be positive (got %d)", K);
    const bool split = opt && (opt->flags & VBGS_FLAG_SPLIT);
    const int dof_min = split ? 2 : D - 1;   // nu0 > (dimension of a Wishart block) - 1
    if (!(prior->alpha0 > 0) || !(prior->beta0 > 0) || !(prior->nu0 > dof_min) ||
        !std::isfinite(prior->alpha0) || !std::isfinite(prior->beta0) || !std::isfinite(prior->nu0))
        return fail(nullptr, VBGS_EINVAL, split ? "need alpha0 > 0, beta0 > 0, nu0 > 2 (split model)"
                                                : "need alpha0 > 0, beta0 > 0, nu0 > D - 1");
    int precision = opt ? opt->precision : VBGS_FP64;
    if (precision != VBGS_FP64 && precision != VBGS_FP32 && precision != VBGS_FP16X3 && precision != VBGS_BF16X3)
        return fail(nullptr, VBGS_EINVAL, "unknown precision %d", precision);
    for (size_t i = 0; i < (size_t)K * 6; i++)
        if (!std::isfinite(prior->m0[i])) return fail(nullptr, VBGS_EINVAL, "non-finite m0");
    double W0[36], W0inv[36];
    for (int i = 0; i < 36; i++) W0[i] = prior->W0[i];
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++)
            if (!std::isfinite(W0[i * 6 + j]) || W0[i * 6 + j] != W0[j * 6 + i])
                return fail(nullptr, VBGS_EINVAL, "W0 must be finite and symmetric");
    if (!host_spd_inverse6(W0, W0inv)) return fail(nullptr, VBGS_EINVAL, "W0 is not positive definite");
    if (split) {
        // the blocks' prior scales are W0's diagonal blocks: invert them alone
        // (the inverse of the block-diagonal matrix is block diagonal, zeros exact)
        double Wb[36];
        for (int i = 0; i < 6; i++)
            for (int j = 0; j < 6; j++) Wb[i * 6 + j] = ((i < 3) == (j < 3)) ? W0[i * 6 + j] : 0.0;
        if (!host_spd_inverse6(Wb, W0inv)) return fail(nullptr, VBGS_EINVAL, "W0's diagonal blocks are not SPD");
    }

    ctx = new vbgs_ctx();
    ctx->K = K;
    ctx->precision = precision;
    ctx->flags = opt ? opt->flags : 0;
    ctx->checks = opt ? opt->checks : 0;
    ctx->skip_nats = skip_nats_for(precision, K);
    ctx->seed = opt ? opt->seed : 0;
    if (opt && opt->autotune_cache) ctx->autotune_cache = opt->autotune_cache;
    for (int i = 0; i < 36; i++) ctx->W0_h[i] = W0[i];
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev);
        cudaGetLastError();
        if (ctx->num_sms <= 0) ctx->num_sms = 152;
    }
    {
        // Morton box: bounding box of the prior means, padded by 10%.
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int k = 0; k < K; k++)
            for (int i = 0; i < 3; i++) {
                lo[i] = std::min(lo[i], prior->m0[(size_t)k * 6 + i]);
                hi[i] = std::max(hi[i], prior->m0[(size_t)k * 6 + i]);
            }
        for (int i = 0; i < 3; i++) {
            double pad = 0.1 * (hi[i] - lo[i]) + 1e-6;
            ctx->box.lo[i] = lo[i] - pad;
            ctx->box.inv_ext[i] = 1.0 / (hi[i] - lo[i] + 2 * pad);
        }
    }
    ctx->stream = opt ? (cudaStream_t)opt->cuda_stream : nullptr;
    if (cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        fail(ctx, VBGS_ECUDA, "stream or event creation failed");
        g_err = ctx->err;
        free_all(ctx);
        delete ctx;
        return VBGS_ECUDA;
    }

    ctx->mp.alpha0 = prior->alpha0;
    ctx->mp.beta0 = prior->beta0;
    ctx->mp.nu0 = prior->nu0;
    ctx->mp.K = K;
    ctx->mp.want_bounds = 1;   // eigenvalue bounds: pass-1 tile lists and the proposal certificate
    for (int i = 0; i < 36; i++) ctx->mp.W0inv[i] = W0inv[i];
    ctx->mp.split = split ? 1 : 0;
    ctx->mp.num_sms = ctx->num_sms;
    ctx->m0_h.assign(prior->m0, prior->m0 + (size_t)K * 6);

    int rc = VBGS_OK;
    const size_t KF = (size_t)K * VBGS_F;
    if ((rc = dalloc(ctx, &ctx->d_m0, (size_t)K * 6)) || (rc = dalloc(ctx, &ctx->d_Spast, KF)) ||
        (rc = dalloc(ctx, &ctx->d_dS, KF)) || (rc = dalloc(ctx, &ctx->d_rec, (size_t)K * VBGS_REC)) ||
        (rc = dalloc(ctx, &ctx->d_rec32, (size_t)K * VBGS_REC)) ||
        (rc = dalloc(ctx, &ctx->d_pcache, mstep_cache_doubles(K))) || (rc = dalloc(ctx, &ctx->d_scal, (size_t)SC_COUNT)) ||
        (rc = dalloc(ctx, &ctx->d_flags, (size_t)FL_COUNT)) || (rc = ensure_elbo(ctx, 64)) ||
        (rc = dalloc(ctx, &ctx->d_kperm, (size_t)K)) || (rc = dalloc(ctx, &ctx->d_kinv, (size_t)K)) ||
        (rc = dalloc(ctx, &ctx->d_tc_tiles, tc_tile_bytes(K))) || (rc = dalloc(ctx, &ctx->d_tc_hdr, tc_hdr_floats(K))) ||
        (rc = dalloc(ctx, &ctx->d_tile_dirty, 6 * (size_t)((K + 127) / 128))) ||
        (rc = dalloc(ctx, &ctx->d_pcache_next, mstep_prior_cache_doubles(K))) ||
        (rc = dalloc(ctx, &ctx->d_rec_alt, (size_t)K * VBGS_REC)) ||
        (rc = dalloc(ctx, &ctx->d_rec32_alt, (size_t)K * VBGS_REC)) || (rc = dalloc(ctx, &ctx->d_kinv_alt, (size_t)K))) {
        g_err = ctx->err;
        free_all(ctx);
        delete ctx;
        return rc;
    }
    auto init_fail = [&](int code) {
        g_err = ctx->err;
        free_all(ctx);
        delete ctx;
        return code;
    };
#undef CU
#define CU(call)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            fail(ctx, VBGS_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));        \
            return init_fail(VBGS_ECUDA);                                          \
        }                                                                          \
    } while (0)
    CU(cudaMemcpyAsync(ctx->d_m0, prior->m0, sizeof(double) * K * 6, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemsetAsync(ctx->d_Spast, 0, sizeof(double) * KF, ctx->stream));
    CU(cudaMemsetAsync(ctx->d_dS, 0, sizeof(double) * KF, ctx->stream));
    CU(cudaMemsetAsync(ctx->d_pcache, 0, sizeof(double) * mstep_cache_doubles(K), ctx->stream));
    CU(cudaMemsetAsync(ctx->d_tile_dirty, 0, 6 * sizeof(int) * ((K + 127) / 128), ctx->stream));
    CU(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int) * FL_COUNT, ctx->stream));
    CU(cudaMemsetAsync(ctx->d_scal, 0, sizeof(double) * SC_COUNT, ctx->stream));
    {
        std::vector<int> ident(K);
        for (int k = 0; k < K; k++) ident[k] = k;
        CU(cudaMemcpyAsync(ctx->d_kperm, ident.data(), sizeof(int) * K, cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaMemcpyAsync(ctx->d_kinv, ident.data(), sizeof(int) * K, cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
    }
    if ((rc = run_mstep(ctx, nullptr)) || (rc = join_side(ctx))) return init_fail(rc);
    if ((ctx->flags & VBGS_FLAG_PROPOSAL) && (rc = prop_alloc(ctx))) return init_fail(rc);
    CU(cudaStreamSynchronize(ctx->stream));
#undef CU
#define CU(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? VBGS_ENOMEM : VBGS_ECUDA, \
                        "%s: %s", #call, cudaGetErrorString(e_));                        \
    } while (0)
    *out = ctx;
    return VBGS_OK;
}

int vbgs_update(vbgs_ctx *ctx, const double *points, int64_t N, int n_iters, double *elbo_trace)
{
    int rc;
    if (ctx && !ctx->autotune_cache.empty() && is_tc(ctx) && !ctx->prop.on && N > 0 && points && n_iters >= 1) {
        // the work decomposition of this size class: tuned (or read from the
        // cache file) on the first frame of the class, reused after
        const int cls = (int)std::lround(std::log2((double)N));
        auto it = std::find_if(ctx->tuned.begin(), ctx->tuned.end(), [&](const auto &e) { return e.first == cls; });
        if (it == ctx->tuned.end()) {
            if ((rc = vbgs_autotune(ctx, points, N, ctx->autotune_cache.c_str()))) return rc;
            ctx->tuned.push_back({cls, {ctx->tune_p1, ctx->tune_p2}});
        } else {
            ctx->tune_p1 = it->second.first;
            ctx->tune_p2 = it->second.second;
        }
    }
    // points are checked during the frame (the proposal's training must not
    // see bad ones, so with the proposal they are checked first)
    if ((rc = update_prepare(ctx, points, N, n_iters, ctx && !ctx->prop.on))) return rc;
    if ((rc = update_enqueue(ctx, N, n_iters, true))) return rc;
    if (elbo_trace)
        CU(cudaMemcpyAsync(elbo_trace, ctx->d_elbo, sizeof(double) * n_iters, cudaMemcpyDeviceToHost,
                           ctx->stream));
    if ((rc = check_flags(ctx))) return rc;
    ctx->next_prior_ready = ctx->next_written;   // the commit ran: the carried prior is exact
    return VBGS_OK;
}

int vbgs_elbo(vbgs_ctx *ctx, const double *points, int64_t N, double *elbo_out, double *lse_out)
{
    if (!ctx) return fail(nullptr, VBGS_EINVAL, "ctx is NULL");
    if (N < 0 || !elbo_out) return fail(ctx, VBGS_EINVAL, "need N >= 0 and elbo_out");
    if (N > 0 && !points) return fail(ctx, VBGS_EINVAL, "points is NULL");
    ctx->launches = 0;
    int rc;
    if ((rc = ensure_capacity(ctx, N)) || (rc = ensure_elbo(ctx, 1))) return rc;
    if ((rc = stage_points(ctx, points, N))) return rc;
    CU(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int) * FL_COUNT, ctx->stream));
    ctx->last_sorted = false;
    if ((rc = run_mstep(ctx, nullptr))) return rc;
    if ((rc = run_estep(ctx, N, false))) return rc;
    if ((rc = join_side(ctx))) return rc;
    if (launch_elbo(ctx->d_scal, N, ctx->d_elbo, ctx->stream, &ctx->prof) < 0)
        return fail(ctx, VBGS_ECUDA, "ELBO launch failed");
    ctx->launches += 1;
    ctx->last_N = N;
    CU(cudaMemcpyAsync(elbo_out, ctx->d_elbo, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if ((rc = check_flags(ctx))) return rc;
    if (lse_out && N > 0) return vbgs_get_lse(ctx, lse_out, N);
    return VBGS_OK;
}

int vbgs_reassign(vbgs_ctx *ctx, const double *points, int64_t N, int n, double tau, const double *gumbel,
                  const double *comp_key, int64_t *picked_points, int *picked_comps)
{
    if (!ctx) return fail(nullptr, VBGS_EINVAL, "ctx is NULL");
    const int K = ctx->K;
    if (n < 0 || N < 0 || n > N || n > K) return fail(ctx, VBGS_EINVAL, "need 0 <= n <= min(N, K)");
    if (N > (int64_t)INT_MAX) return fail(ctx, VBGS_EINVAL, "reassign takes at most %d points", INT_MAX);
    if (!(tau > 0.0) || !std::isfinite(tau)) return fail(ctx, VBGS_EINVAL, "tau must be finite and > 0");
    if (n == 0) return VBGS_OK;
    if (!points || !gumbel) return fail(ctx, VBGS_EINVAL, "points and gumbel are required");
    for (int64_t i = 0; i < N; i++)
        if (!std::isfinite(gumbel[i])) return fail(ctx, VBGS_EINVAL, "non-finite gumbel value at %lld", (long long)i);
    if (comp_key)
        for (int k = 0; k < K; k++)
            if (!std::isfinite(comp_key[k])) return fail(ctx, VBGS_EINVAL, "non-finite comp_key value at %d", k);
    ctx->launches = 0;
    int rc;
    // the per-point ELBO term under the current posterior, as vbgs_elbo
    if ((rc = ensure_capacity(ctx, N)) || (rc = ensure_elbo(ctx, 1)) ||
        (rc = ensure_reassign(ctx, std::max<int64_t>(N, K))))
        return rc;
    if ((rc = stage_points(ctx, points, N))) return rc;
    CU(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int) * FL_COUNT, ctx->stream));
    ctx->last_sorted = false;
    if ((rc = run_mstep(ctx, nullptr))) return rc;
    if ((rc = run_estep(ctx, N, false))) return rc;
    if ((rc = join_side(ctx))) return rc;
    if (launch_elbo(ctx->d_scal, N, ctx->d_elbo, ctx->stream, &ctx->prof) < 0)
        return fail(ctx, VBGS_ECUDA, "ELBO launch failed");
    ctx->launches += 1;
    ctx->last_N = N;
    if ((rc = check_flags(ctx))) return rc;   // before the prior changes
    ReassignBuffers &rb = ctx->ra;
    CU(cudaMemcpyAsync(rb.g, gumbel, sizeof(double) * (size_t)N, cudaMemcpyHostToDevice, ctx->stream));
    if (comp_key) CU(cudaMemcpyAsync(rb.v, comp_key, sizeof(double) * (size_t)K, cudaMemcpyHostToDevice, ctx->stream));
    ReassignArgs a;
    a.lse = ctx->d_lse;   // the E-step above ran on d_X, in caller order
    a.psi = ctx->d_scal + SC_PSI_ESTEP;
    a.X = ctx->d_X;
    a.S = ctx->d_Spast;
    a.m0 = ctx->d_m0;
    a.N = N;
    a.K = K;
    a.n = n;
    a.inv_tau = 1.0 / tau;
    a.have_v = comp_key != nullptr;
    const int l = launch_reassign(a, rb, ctx->stream);
    if (l < 0) return fail(ctx, VBGS_ECUDA, "reassign launch failed");
    ctx->launches += l;
    std::vector<int> picks((size_t)n * 2);
    std::vector<double> rows((size_t)n * 6);
    CU(cudaMemcpyAsync(picks.data(), rb.picks, sizeof(int) * picks.size(), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(rows.data(), rb.rows, sizeof(double) * rows.size(), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    // the host copy of the prior means follows the device's
    for (int i = 0; i < n; i++)
        for (int d = 0; d < 6; d++) ctx->m0_h[(size_t)picks[(size_t)n + i] * 6 + d] = rows[(size_t)i * 6 + d];
    if (picked_points)
        for (int i = 0; i < n; i++) picked_points[i] = picks[i];
    if (picked_comps)
        for (int i = 0; i < n; i++) picked_comps[i] = picks[(size_t)n + i];
    ctx->next_prior_ready = false;   // the next frame starts from the new prior
    return VBGS_OK;
}

int vbgs_get_lse(vbgs_ctx *ctx, double *lse, int64_t N)
{
    if (!ctx) return fail(nullptr, VBGS_EINVAL, "ctx is NULL");
    if (!lse || N != ctx->last_N) return fail(ctx, VBGS_EINVAL, "lse needs N == points of the last call");
    if (N == 0) return VBGS_OK;
    double psi = 0.0;
    CU(cudaMemcpyAsync(lse, ctx->d_lse, sizeof(double) * N, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(&psi, ctx->d_scal + SC_PSI_ESTEP, sizeof(double), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    // The device keeps lse without the -psi(sum alpha) shared by every logit,
    // in processing order.
    if (ctx->last_sorted) {
        std::vector<int> pidx((size_t)N);
        std::vector<double> tmp(lse, lse + N);
        CU(cudaMemcpyAsync(pidx.data(), ctx->d_pidx, sizeof(int) * N, cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        for (int64_t i = 0; i < N; i++) lse[pidx[(size_t)i]] = tmp[(size_t)i];
    }
    for (int64_t n = 0; n < N; n++) lse[n] -= psi;
    return VBGS_OK;
}

int vbgs_get_frame_stats(vbgs_ctx *ctx, double *dS)
{
    if (!ctx) return fail(nullptr, VBGS_EINVAL, "ctx is NULL");
    if (!dS) return fail(ctx, VBGS_EINVAL, "dS is NULL");
    CU(cudaMemcpyAsync(dS, ctx->d_dS, sizeof(double) * ctx->K * VBGS_F, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return VBGS_OK;
}

int vbgs_get_stats(vbgs_ctx *ctx, double *S)
{
    if (!ctx) return fail(nullptr, VBGS_EINVAL, "ctx is NULL");
    if (!S) return fail(ctx, VBGS_EINVAL, "S is NULL");
    CU(cudaMemcpyAsync(S, ctx->d_Spast, sizeof(double) * ctx->K * VBGS_F, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return VBGS_OK;
}

int vbgs_set_stats(vbgs_ctx *ctx, const double *S)
{
    if (!ctx) return fail(nullptr, VBGS_EINVAL, "ctx is NULL");
    if (!S) return fail(ctx, VBGS_EINVAL, "S is NULL");
    for (size_t i = 0; i < (size_t)ctx->K * VBGS_F; i++)
        if (!std::isfinite(S[i])) return fail(ctx, VBGS_EINVAL, "non-finite statistic at %zu", i);
    CU(cudaMemcpyAsync(ctx->d_Spast, S, sizeof(double) * ctx->K * VBGS_F, cudaMemcpyHostToDevice,
                       ctx->stream));
    CU(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int) * FL_COUNT, ctx->stream));
    int rc = run_mstep(ctx, nullptr);
    if (rc) return rc;
    return check_flags(ctx);
}

int vbgs_get_posterior(vbgs_ctx *ctx, double *alpha, double *beta, double *m, double *Winv, double *nu)
{
    if (!ctx) return fail(nullptr, VBGS_EINVAL, "ctx is NULL");
    const int K = ctx->K;
    std::vector<double> S((size_t)K * VBGS_F);
    int rc = vbgs_get_stats(ctx, S.data());
    if (rc) return rc;
    const MstepParams &P = ctx->mp;
    for (int k = 0; k < K; k++) {
        const double *s = &S[(size_t)k * VBGS_F];
        const double *m0 = &ctx->m0_h[(size_t)k * 6];
        const double N = s[0], b = P.beta0 + N;
        double mk[6];
        for (int i = 0; i < 6; i++) mk[i] = (P.beta0 * m0[i] + s[1 + i]) / b;
        if (alpha) alpha[k] = P.alpha0 + N;
        if (beta) beta[k] = b;
        if (nu) nu[k] = P.nu0 + N;
        if (m)
            for (int i = 0; i < 6; i++) m[(size_t)k * 6 + i] = mk[i];
        if (Winv)
            for (int i = 0; i < 6; i++)
                for (int j = i; j < 6; j++) {
                    double v = (P.split && i < 3 && j >= 3)
                                   ? 0.0
                                   : P.W0inv[i * 6 + j] + s[upper_index(i, j)] + P.beta0 * m0[i] * m0[j] - b * mk[i] * mk[j];
                    Winv[(size_t)k * 36 + i * 6 + j] = v;
                    Winv[(size_t)k * 36 + j * 6 + i] = v;
                }
    }
    return VBGS_OK;
}

int64_t vbgs_last_launch_count(const vbgs_ctx *ctx) { return ctx ? ctx->launches : 0; }

int vbgs_profile_enable(vbgs_ctx *ctx, int on)
{
    if (!ctx) return fail(nullptr, VBGS_EINVAL, "ctx is NULL");
    if (on && ctx->prof.pool.empty()) {
        ctx->prof.pool.resize(4096);
        for (auto &e : ctx->prof.pool) CU(cudaEventCreate(&e));
        CU(cudaMalloc(&ctx->prof.d_pairs, 3 * sizeof(unsigned long long)));
        CU(cudaMemsetAsync(ctx->prof.d_pairs, 0, 3 * sizeof(unsigned long long), ctx->stream));
    }
    ctx->prof.on = on != 0;
    ctx->prof.mask = on == 1 ? ~0u : (unsigned)on >> 1;
    return VBGS_OK;
}

int vbgs_profile_read(vbgs_ctx *ctx, double *ms, int64_t *launches, int reset)
{
    if (!ctx) return fail(nullptr, VBGS_EINVAL, "ctx is NULL");
    for (int i = 0; i < VBGS_PROF_COUNT; i++) {
        if (ms) ms[i] = ctx->prof.ms[i];
        if (launches) launches[i] = ctx->prof.n[i];
        if (reset) { ctx->prof.ms[i] = 0; ctx->prof.n[i] = 0; }
    }
    if (reset && ctx->prof.d_pairs) {
        CU(cudaMemsetAsync(ctx->prof.d_pairs, 0, 3 * sizeof(unsigned long long), ctx->stream));
        ctx->prof.pass1_pairs = 0;
    }
    return VBGS_OK;
}

int vbgs_profile_pairs(vbgs_ctx *ctx, int64_t *pass1_pairs, int64_t *pass2_pairs)
{
    if (!ctx) return fail(nullptr, VBGS_EINVAL, "ctx is NULL");
    unsigned long long p[2] = {0, 0};
    if (ctx->prof.d_pairs) {
        CU(cudaMemcpyAsync(p, ctx->prof.d_pairs, sizeof p, cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
    }
    if (pass1_pairs) *pass1_pairs = ctx->prof.pass1_pairs + (int64_t)p[1];
    if (pass2_pairs) *pass2_pairs = (int64_t)p[0];
    return VBGS_OK;
}

const char *vbgs_profile_name(int i)
{
    static const char *names[VBGS_PROF_COUNT] = {"pass1", "merge", "pass2", "reduce", "mstep", "misc", "plan", "kl"};
    return (i >= 0 && i < VBGS_PROF_COUNT) ? names[i] : "?";
}

int vbgs_save_state(vbgs_ctx *ctx, const char *path)
{
    if (!ctx) return fail(nullptr, VBGS_EINVAL, "ctx is NULL");
    if (!path) return fail(ctx, VBGS_EINVAL, "vbgs_save_state: path is NULL");
    int rc;
    if ((rc = join_side(ctx))) return rc;
    CU(cudaStreamSynchronize(ctx->stream));
    StateHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, kStateMagic, 8);
    h.version = kStateVersion;
    h.K = ctx->K;
    h.D = ctx->D;
    h.precision = ctx->precision;
    h.flags = ctx->flags;
    h.has_prop = ctx->prop.on ? 1 : 0;
    h.next_prior_ready = ctx->next_prior_ready ? 1 : 0;
    h.coef_epoch = ctx->coef_epoch;
    h.plan_epoch = ctx->plan_epoch;
    h.tune_p1 = ctx->tune_p1;
    h.tune_p2 = ctx->tune_p2;
    h.prop_step = ctx->prop.step;
    h.prop_centroids_ready = ctx->prop.centroids_ready ? 1 : 0;
    h.prop_epochs = ctx->prop.epochs;
    h.tc_knobs = ctx->tc_knobs;
    h.frame_count = ctx->frame_count;
    h.prop_lr = ctx->prop.lr;
    h.prop_frames_trained = ctx->prop.frames_trained;
    h.prop_frame = ctx->prop.frame;
    h.seed = ctx->seed;
    h.alpha0 = ctx->mp.alpha0;
    h.beta0 = ctx->mp.beta0;
    h.nu0 = ctx->mp.nu0;
    for (int i = 0; i < 36; i++) h.W0[i] = ctx->W0_h[i];
    for (int i = 0; i < 3; i++) {
        h.box_lo[i] = ctx->box.lo[i];
        h.box_inv_ext[i] = ctx->box.inv_ext[i];
    }
    const std::vector<StateSection> secs = state_sections(ctx);
    h.n_sections = (int32_t)secs.size();
    size_t total = 0;
    for (const auto &q : secs) total += q.bytes;
    std::vector<unsigned char> buf(total);
    size_t off = 0;
    for (const auto &q : secs) {
        CU(cudaMemcpyAsync(buf.data() + off, q.dev, q.bytes, cudaMemcpyDeviceToHost, ctx->stream));
        off += q.bytes;
    }
    CU(cudaStreamSynchronize(ctx->stream));
    std::vector<uint64_t> sizes;
    for (const auto &q : secs) sizes.push_back((uint64_t)q.bytes);
    uint64_t sum = fnv1a(kFnvBasis, &h, sizeof h);
    sum = fnv1a(sum, sizes.data(), sizeof(uint64_t) * sizes.size());
    sum = fnv1a(sum, buf.data(), buf.size());
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "wb");
    if (!f) return fail(ctx, VBGS_EIO, "vbgs_save_state: cannot open %s for writing", tmp.c_str());
    bool ok = fwrite(&h, sizeof h, 1, f) == 1 &&
              fwrite(sizes.data(), sizeof(uint64_t), sizes.size(), f) == sizes.size() &&
              fwrite(buf.data(), 1, buf.size(), f) == buf.size() && fwrite(&sum, sizeof sum, 1, f) == 1;
    ok = (fclose(f) == 0) && ok;
    if (!ok || rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        return fail(ctx, VBGS_EIO, "vbgs_save_state: writing %s failed", path);
    }
    return VBGS_OK;
}

int vbgs_load_state(vbgs_ctx **out, const char *path, const vbgs_options *opt)
{
    if (!out) return fail(nullptr, VBGS_EINVAL, "out is NULL");
    *out = nullptr;
    if (!path) return fail(nullptr, VBGS_EINVAL, "vbgs_load_state: path is NULL");
    FILE *f = fopen(path, "rb");
    if (!f) return fail(nullptr, VBGS_EIO, "vbgs_load_state: cannot open %s", path);
    std::vector<unsigned char> file;
    {
        unsigned char chunk[1 << 16];
        size_t n;
        while ((n = fread(chunk, 1, sizeof chunk, f)) > 0) file.insert(file.end(), chunk, chunk + n);
        fclose(f);
    }
    StateHeader h;
    if (file.size() < sizeof h + sizeof(uint64_t)) return fail(nullptr, VBGS_EIO, "vbgs_load_state: %s is too short", path);
    memcpy(&h, file.data(), sizeof h);
    if (memcmp(h.magic, kStateMagic, 8) != 0 || h.version != kStateVersion)
        return fail(nullptr, VBGS_EIO, "vbgs_load_state: %s is not a state file of this version", path);
    if (h.K <= 0 || h.D != VBGS_D || h.n_sections <= 0 || h.n_sections > 64)
        return fail(nullptr, VBGS_EIO, "vbgs_load_state: bad header in %s", path);
    const size_t sizes_off = sizeof h, data_off = sizes_off + sizeof(uint64_t) * h.n_sections;
    if (file.size() < data_off + sizeof(uint64_t)) return fail(nullptr, VBGS_EIO, "vbgs_load_state: %s is truncated", path);
    std::vector<uint64_t> sizes(h.n_sections);
    memcpy(sizes.data(), file.data() + sizes_off, sizeof(uint64_t) * h.n_sections);
    uint64_t total = 0;
    for (uint64_t b : sizes) total += b;
    if (file.size() != data_off + total + sizeof(uint64_t))
        return fail(nullptr, VBGS_EIO, "vbgs_load_state: %s has the wrong size", path);
    uint64_t sum_file;
    memcpy(&sum_file, file.data() + data_off + total, sizeof sum_file);
    if (fnv1a(kFnvBasis, file.data(), data_off + total) != sum_file)
        return fail(nullptr, VBGS_EIO, "vbgs_load_state: checksum mismatch in %s", path);
    // The prior as it stands (m0 from the first section) and the saved form.
    if (sizes[0] != sizeof(double) * (size_t)h.K * 6) return fail(nullptr, VBGS_EIO, "vbgs_load_state: bad m0 section");
    std::vector<double> m0((size_t)h.K * 6);
    memcpy(m0.data(), file.data() + data_off, sizes[0]);
    vbgs_prior pr;
    pr.alpha0 = h.alpha0;
    pr.beta0 = h.beta0;
    pr.nu0 = h.nu0;
    pr.m0 = m0.data();
    pr.W0 = h.W0;
    vbgs_options o;
    memset(&o, 0, sizeof o);
    o.precision = h.precision;
    o.flags = h.flags;
    o.seed = h.seed;
    if (opt) {
        o.cuda_stream = opt->cuda_stream;
        o.checks = opt->checks;
        o.autotune_cache = opt->autotune_cache;
    }
    vbgs_ctx *ctx = nullptr;
    int rc = vbgs_init(&ctx, &pr, h.K, h.D, &o);
    if (rc) return rc;
    const std::vector<StateSection> secs = state_sections(ctx);
    if ((int)secs.size() != h.n_sections) {
        vbgs_destroy(ctx);
        return fail(nullptr, VBGS_EIO, "vbgs_load_state: %s has %d sections, the context %zu", path, h.n_sections,
                    secs.size());
    }
    size_t off = data_off;
    for (size_t i = 0; i < secs.size(); i++) {
        if (sizes[i] != secs[i].bytes) {
            vbgs_destroy(ctx);
            return fail(nullptr, VBGS_EIO, "vbgs_load_state: section %zu of %s has the wrong size", i, path);
        }
        const cudaError_t e = cudaMemcpyAsync(secs[i].dev, file.data() + off, secs[i].bytes, cudaMemcpyHostToDevice,
                                              ctx->stream);
        if (e != cudaSuccess) {
            vbgs_destroy(ctx);
            return fail(nullptr, VBGS_ECUDA, "vbgs_load_state: %s", cudaGetErrorString(e));
        }
        off += secs[i].bytes;
    }
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        vbgs_destroy(ctx);
        return fail(nullptr, VBGS_ECUDA, "vbgs_load_state: copy to the device failed");
    }
    ctx->m0_h = m0;
    ctx->next_prior_ready = h.next_prior_ready != 0;
    ctx->coef_epoch = h.coef_epoch;
    ctx->plan_epoch = h.plan_epoch;
    ctx->tune_p1 = h.tune_p1;
    ctx->tune_p2 = h.tune_p2;
    ctx->tc_knobs = h.tc_knobs;
    ctx->frame_count = h.frame_count;
    for (int i = 0; i < 3; i++) {
        ctx->box.lo[i] = h.box_lo[i];
        ctx->box.inv_ext[i] = h.box_inv_ext[i];
    }
    if (ctx->prop.on) {
        ctx->prop.step = h.prop_step;
        ctx->prop.centroids_ready = h.prop_centroids_ready != 0;
        ctx->prop.epochs = h.prop_epochs;
        ctx->prop.lr = h.prop_lr;
        ctx->prop.frames_trained = h.prop_frames_trained;
        ctx->prop.rep[7] = (double)h.prop_frames_trained;
        ctx->prop.frame = h.prop_frame;
    }
    *out = ctx;
    return VBGS_OK;
}

int vbgs_check_frame(const double *dS, int K, const double *points, int64_t N, const double *lse, double tol,
                     int *ok)
{
    if (!dS || K <= 0 || N < 0 || (N > 0 && !points) || !ok || !(tol >= 0))
        return fail(nullptr, VBGS_EINVAL, "vbgs_check_frame: need dS, K > 0, N >= 0, points, ok and tol >= 0");
    vbgs_ctx tmp_ctx;
    double *d_dS = nullptr, *d_X = nullptr, *d_lse = nullptr;
    int *d_flags = nullptr;
    auto release = [&]() {
        cudaFree(d_dS); cudaFree(d_X); cudaFree(d_lse); cudaFree(d_flags);
        cudaGetLastError();
    };
    int rc;
    if ((rc = dalloc(&tmp_ctx, &d_dS, (size_t)K * VBGS_F)) || (rc = dalloc(&tmp_ctx, &d_X, (size_t)std::max<int64_t>(N, 1) * VBGS_XS)) ||
        (rc = dalloc(&tmp_ctx, &d_lse, (size_t)std::max<int64_t>(N, 1))) || (rc = dalloc(&tmp_ctx, &d_flags, (size_t)FL_COUNT))) {
        release();
        return fail(nullptr, rc, "%s", tmp_ctx.err.c_str());
    }
    std::vector<double> X((size_t)std::max<int64_t>(N, 1) * VBGS_XS, 0.0);
    for (int64_t n = 0; n < N; n++)
        for (int q = 0; q < 6; q++) X[(size_t)n * VBGS_XS + q] = points[(size_t)n * 6 + q];
    int fl[FL_COUNT] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpy(d_dS, dS, sizeof(double) * K * VBGS_F, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_X, X.data(), sizeof(double) * X.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && lse && N > 0) e = cudaMemcpy(d_lse, lse, sizeof(double) * N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(d_flags, 0, sizeof(int) * FL_COUNT);
    Prof off;
    if (e == cudaSuccess &&
        launch_check_frame(d_dS, K, d_X, N, lse && N > 0 ? d_lse : nullptr, tol, d_flags, nullptr, &off) < 0)
        e = cudaErrorLaunchFailure;
    if (e == cudaSuccess) e = cudaMemcpy(fl, d_flags, sizeof fl, cudaMemcpyDeviceToHost);
    release();
    if (e != cudaSuccess) return fail(nullptr, VBGS_ECUDA, "vbgs_check_frame: %s", cudaGetErrorString(e));
    *ok = fl[FL_CHECK] == 0;
    return VBGS_OK;
}

int vbgs_render(vbgs_ctx *ctx, const double *camera, int width, int height, float *image, const float *reference,
                double *psnr, double *device_ms)
{
    if (!ctx) return fail(nullptr, VBGS_EINVAL, "ctx is NULL");
    if (!camera || width <= 0 || height <= 0 || width > 16384 || height > 16384 || (psnr && !reference))
        return fail(ctx, VBGS_EINVAL, "vbgs_render: need a camera, 0 < width, height <= 16384, and a reference "
                                      "image for the PSNR");
    for (int i = 0; i < 13; i++)
        if (!std::isfinite(camera[i])) return fail(ctx, VBGS_EINVAL, "vbgs_render: non-finite camera");
    if (!(camera[12] > 0)) return fail(ctx, VBGS_EINVAL, "vbgs_render: the focal length must be positive");
    int rc;
    if ((rc = join_side(ctx))) return rc;
    std::string why;
    if (render_frame(ctx->d_m0, ctx->d_Spast, ctx->mp, ctx->mp.split ? 3 : 6, ctx->K, camera, width, height, ctx->rb,
                     image, reference, psnr, device_ms, ctx->stream, why))
        return fail(ctx, VBGS_ECUDA, "vbgs_render: %s", why.c_str());
    return VBGS_OK;
}

int vbgs_profile_replay(vbgs_ctx *ctx, int reps, double *ms_per_launch, int64_t *pairs_per_launch,
                        int64_t *exp_pairs_per_launch)
{
    if (!ctx) return fail(nullptr, VBGS_EINVAL, "ctx is NULL");
    if (reps < 1 || !ms_per_launch) return fail(ctx, VBGS_EINVAL, "vbgs_profile_replay: need reps >= 1 and an output");
    const Pass1Launch &L = ctx->prof.p1_last;
    if (!is_tc(ctx) || !L.valid || L.alloc_gen != ctx->alloc_gen)
        return fail(ctx, VBGS_EINVAL, "vbgs_profile_replay: no tensor-core pass-1 launch on the current buffers");
    int rc;
    if ((rc = join_side(ctx))) return rc;
    unsigned long long *d_cnt = nullptr;   // pairs evaluated, pairs exponentiated
    CU(cudaMalloc(&d_cnt, 2 * sizeof(unsigned long long)));
    CU(cudaMemsetAsync(d_cnt, 0, 2 * sizeof(unsigned long long), ctx->stream));
    float ms = 0.f;
    const int r = tc_replay_pass1(L, reps, d_cnt, ctx->stream, &ms);
    unsigned long long cnt[2] = {0, 0};
    const cudaError_t e = cudaMemcpy(cnt, d_cnt, sizeof cnt, cudaMemcpyDeviceToHost);
    cudaFree(d_cnt);
    if (r || e != cudaSuccess) return fail(ctx, VBGS_ECUDA, "vbgs_profile_replay: replay failed");
    *ms_per_launch = ms;
    if (pairs_per_launch) *pairs_per_launch = (int64_t)cnt[0];
    if (exp_pairs_per_launch) *exp_pairs_per_launch = (int64_t)cnt[1];
    return check_flags(ctx);
}

int vbgs_set_precision_knobs(vbgs_ctx *ctx, unsigned int knobs)
{
    if (!ctx) return fail(nullptr, VBGS_EINVAL, "ctx is NULL");
    if (knobs & ~(unsigned)VBGS_KNOB_ALL) return fail(ctx, VBGS_EINVAL, "vbgs_set_precision_knobs: unknown bits");
    ctx->tc_knobs = knobs;
    return VBGS_OK;
}

unsigned int vbgs_get_precision_knobs(const vbgs_ctx *ctx) { return ctx ? ctx->tc_knobs : 0u; }

int vbgs_set_wait_limit(long long cycles)
{
    if (tc_set_wait_limit(cycles)) return fail(nullptr, VBGS_ECUDA, "vbgs_set_wait_limit: cudaMemcpyToSymbol failed");
    return VBGS_OK;
}

const char *vbgs_last_error(const vbgs_ctx *ctx)
{
    if (ctx) return ctx->err.c_str();
    return g_err.c_str();
}

void vbgs_destroy(vbgs_ctx *ctx)
{
    if (!ctx) return;
    batch_forget(ctx);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    free_all(ctx);
    delete ctx;
}

} // extern "C"
