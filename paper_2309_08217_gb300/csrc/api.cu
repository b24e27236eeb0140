// api.cu -- the C ABI of libgenga (declared in include/genga.h): argument
// checks, workspace, and the order of kernels for each entry point.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "internal.cuh"

using namespace genga;

namespace {

struct DeviceGuard {  // run on the context's device, restore the caller's afterwards
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

inline bool is_fin(double v) { return isfinite(v) != 0; }

// The most recent CUDA error an entry point of this thread turned into
// GENGA_ERR_CUDA (genga_last_cuda_error, genga_measure.h).
thread_local cudaError_t g_last_cuda_error = cudaSuccess;

inline genga_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return GENGA_OK;
    g_last_cuda_error = e;
    return GENGA_ERR_CUDA;
}

inline bool is_fp32(int precision) {
    return precision == GENGA_FP32 || precision == GENGA_FP32_HILO || precision == GENGA_FP32_BLOCKREL;
}
// variant family of an FP32 precision mode: 0 all variants, 1 one-sided, 2 mutual
inline int family_of(int precision) {
    return precision == GENGA_FP32_HILO ? 1 : precision == GENGA_FP32_BLOCKREL ? 2 : 0;
}

genga_status check_params(const genga_params *p) {
    if (!p) return GENGA_ERR_INVALID_ARG;
    if (!is_fin(p->G) || p->G < 0.0) return GENGA_ERR_INVALID_ARG;
    if (!is_fin(p->Mstar) || p->Mstar <= 0.0) return GENGA_ERR_INVALID_ARG;
    if (!is_fin(p->dt) || !is_fin(p->n1) || !is_fin(p->n2) || p->n1 < 0.0 || p->n2 < 0.0)
        return GENGA_ERR_INVALID_ARG;
    if (p->rcrit_mode != GENGA_RCRIT_EQ1 && p->rcrit_mode != GENGA_RCRIT_MUTUAL_HILL) return GENGA_ERR_INVALID_ARG;
    if (p->changeover != GENGA_K_CHAMBERS && p->changeover != GENGA_K_QUINTIC) return GENGA_ERR_INVALID_ARG;
    if (p->precision != GENGA_FP64 && !is_fp32(p->precision)) return GENGA_ERR_INVALID_ARG;
    if (p->precision == GENGA_FP32_BLOCKREL && p->n_big >= 0) return GENGA_ERR_INVALID_ARG;  // no mode-2 mutual pass
    if (p->kepler_max_iter < 1) return GENGA_ERR_INVALID_ARG;
    if (p->n_big < -1) return GENGA_ERR_INVALID_ARG;
    // bs_tol: 0 (off) or >= 1e-14 -- below that the error estimate of a member's
    // state is at the rounding of its FP64 heliocentric coordinates and the
    // sub-steps shrink to the floor without converging
    if (!is_fin(p->bs_tol) || p->bs_tol < 0.0 || (p->bs_tol > 0.0 && p->bs_tol < 1e-14)) return GENGA_ERR_INVALID_ARG;
    if (!is_fin(p->r_in) || !is_fin(p->r_out)) return GENGA_ERR_INVALID_ARG;
    if (p->n_levels < 0 || p->n_levels > GENGA_MAX_LEVELS) return GENGA_ERR_INVALID_ARG;
    if (p->n_levels > 0 && (p->bs_tol <= 0.0 || p->n_sub < 2 || p->n_sub > 16)) return GENGA_ERR_INVALID_ARG;
    return GENGA_OK;
}

// Kernels one drift launches: momentum, drift, momentum, central-body drift,
// and with the close-encounter level the grouping kernel and the levels.
int drift_launches(const genga_params &p) {
    if (p.bs_tol <= 0.0) return 4;
    return 5 + level_launches(p.n_levels, p.n_levels > 0 ? p.n_sub : 1);
}

genga_status check_system(const genga_ctx *c, const genga_system *s) {
    if (!c || !s) return GENGA_ERR_INVALID_ARG;
    if (s->N < 0 || s->N > c->max_N) return GENGA_ERR_INVALID_ARG;
    if (s->N > 0 && (!s->x || !s->y || !s->z || !s->vx || !s->vy || !s->vz || !s->m)) return GENGA_ERR_INVALID_ARG;
    return GENGA_OK;
}

inline int npad_of(int N) { return (N + GENGA_PAD - 1) / GENGA_PAD * GENGA_PAD; }

inline int size_bucket(int N) {
    int b = 0;
    for (int v = npad_of(N); v > 1; v >>= 1) b++;
    return b < 32 ? b : 31;
}

PassArgs base_args(genga_ctx *c, const genga_system &sys, const genga_params &p) {
    PassArgs a;
    a.hi = c->pk_hi;
    a.hit = c->pk_t;
    a.hid = c->pk_d;
    a.rel = c->pk_r;
    a.rell = c->pk_rl;
    a.gctr = c->gctr;
    a.mp = MutualPlan{};
    a.wait_ns_log2 = c->test_wait_log2;
    a.hold = c->test_hold;
    a.lo = c->pk_lo;
    a.p64 = c->pk64;
    a.scr = c->scr;
    a.gbox_lo = c->gbox_lo;
    a.gbox_hi = c->gbox_hi;
    a.gflag = c->gflag;
    a.n_big = p.n_big;
    a.perm = c->perm;
    a.a_osc = c->a_osc;
    a.rc_eq1 = c->rc_eq1;
    a.m = sys.m;
    a.partial = c->partial;
    a.enc = c->enc;
    a.enc_count = c->enc_count;
    // the close-encounter level's groups also take the pairs predicted to
    // enter r_crit within the drift: screening widened to PREDICT_RANGE r_crit
    a.pred = c->pred;
    a.predict = p.bs_tol > 0.0 ? 1 : 0;
    a.pred_dt = p.dt;
    a.vx = sys.vx;
    a.vy = sys.vy;
    a.vz = sys.vz;
    a.enc_cap = c->enc_cap;
    a.status = c->status;
    a.N = sys.N;
    a.npad = npad_of(sys.N);
    a.ntiles = 0;
    a.split = 1;
    a.Mstar = p.Mstar;
    a.n1 = p.n1;
    a.rcrit_mode = p.rcrit_mode;
    a.changeover = p.changeover;
    a.list_only = 0;
    a.work = c->work;
    a.tp_b0 = 0;
    a.tp_t0 = 0;
    a.tp_rows_end = 0;
    a.ntier = 1;
    a.excess = 0;
    a.tier_len[0] = 1;
    a.tier_n[0] = 1;
    return a;
}

inline int num_all_variants() { return num_fp32_variants() + num_mutual_variants(); }
inline bool is_mutual(int v) { return v >= num_fp32_variants(); }

// Launches the pass of FP32 variant v (one-sided or mutual) with the work plan
// for a.N bodies; *mp gets the mutual plan (the combine needs it).  False when
// a mutual plan cannot be had (built during a capture): nothing launched.
bool launch_fp32_variant(genga_ctx *c, PassArgs a, int v, cudaStream_t s, MutualPlan *mp, int *split,
                         int *one_row, cudaError_t *err) {
    *err = cudaSuccess;
    if (is_mutual(v)) {
        if (!mutual_plan(c, a.N, v - num_fp32_variants(), s, mp)) return false;
        a.partial = c->partial;  // a mutual plan may have enlarged (reallocated) the partial rows
        a.mp = *mp;
        *split = 0;
        *one_row = 0;
        *err = launch_pass_mutual(a, v - num_fp32_variants(), c->sm_count, s);
        return true;
    }
    int grid = 1;
    a.partial = c->partial;  // the rows may have been reallocated since `a` was filled (tuning)
    plan_pass(a.N, GENGA_FP32, v, c->sm_count, c->partial_cap, &a, &grid);
    *split = a.split;
    *one_row = a.tp_rows_end;
    *err = launch_pass(a, GENGA_FP32, v, grid, s);
    return true;
}

// FP64 pass variants: 0 = the one-sided pass, 1 .. = the mutual FP64 pass.
inline int num_f64_variants() { return 1 + num_mutual64_variants(); }

// Launches FP64 pass variant v; as launch_fp32_variant.
bool launch_fp64_variant(genga_ctx *c, PassArgs a, int v, cudaStream_t s, MutualPlan *mp, int *split, int *one_row,
                         cudaError_t *err) {
    *err = cudaSuccess;
    if (v > 0) {
        if (!mutual64_plan(c, a.N, v - 1, s, mp)) return false;
        a.partial = c->partial;
        a.mp = *mp;
        *split = 0;
        *one_row = 0;
        *err = launch_pass_mutual64(a, v - 1, c->sm_count, s);
        return true;
    }
    int grid = 1;
    a.partial = c->partial;
    plan_pass(a.N, GENGA_FP64, 0, c->sm_count, c->partial_cap, &a, &grid);
    *split = a.split;
    *one_row = a.tp_rows_end;
    *err = launch_pass(a, GENGA_FP64, 0, grid, s);
    return true;
}

// mutual: 0 = the rows of a one-sided pass, 1 = mutual FP32, 2 = mutual FP64.
cudaError_t launch_combine_any(genga_ctx *c, int mutual, const MutualPlan &mp, int split, int one_row, int N,
                               int fp64_rows, double tau, double *acc, const genga_system &sys, cudaStream_t s) {
    if (mutual == 2)
        return launch_combine_mutual64(c->partial, mp, N, npad_of(N), c->perm, tau, acc, sys.vx, sys.vy, sys.vz,
                                       c->status, s);
    if (mutual)
        return launch_combine_mutual(c->partial, mp, N, npad_of(N), c->perm, tau, acc, sys.vx, sys.vy, sys.vz,
                                     c->status, s);
    return launch_combine(c->partial, split, one_row, N, npad_of(N), fp64_rows, c->perm, tau, acc, sys.vx, sys.vy,
                          sys.vz, c->status, s);
}

// Times one variant for the autotuner: pass + combine (no kick applied, no
// output) `reps` times on the packed state, clearing the encounter list after
// each run; the fastest run after the first, 3e38 if a run failed.
template <class Launch>
float time_variant(genga_ctx *c, int N, int reps, int kind, int fp64_rows, cudaStream_t s, cudaEvent_t e0,
                   cudaEvent_t e1, Launch launch) {
    float ms = 3.0e38f;
    for (int rep = 0; rep < reps; rep++) {
        MutualPlan mp{};
        int split = 1, one_row = 0;
        cudaError_t e = cudaSuccess;
        cudaEventRecord(e0, s);
        if (!launch(&mp, &split, &one_row, &e)) break;
        genga_system none{};
        none.N = N;
        if (e == cudaSuccess) e = launch_combine_any(c, kind, mp, split, one_row, N, fp64_rows, 0.0, nullptr, none, s);
        cudaEventRecord(e1, s);
        cudaMemsetAsync(c->enc_count, 0, 2 * sizeof(int32_t), s);
        if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) break;
        float t = 3.0e38f;
        cudaEventElapsedTime(&t, e0, e1);
        if (rep > 0 && t < ms) ms = t;
        if (rep > 0 && t > 20.f) break;  // long passes: one timed run is enough
    }
    return ms;
}

bool can_tune(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
}

// The FP32 pass variant for this size: forced, already tuned, or tuned now.
// Tuning runs every variant's pass and combine (with no kick applied) four
// times on the packed state (the encounter list is cleared after each run)
// and keeps the variant with the fastest of its last three runs; it
// synchronises the stream, so it is skipped while the stream is captured.
// The precision mode sets the family of variants: GENGA_FP32 all of them,
// GENGA_FP32_HILO the one-sided pass (hi/lo split), GENGA_FP32_BLOCKREL the
// mutual pass (group-centred offsets); each family has its own table, and a
// variant already timed for the bucket is not timed again.  Test-particle
// mode 2 has its own table over the one-sided variants (the mutual pass does
// not implement it).  A forced variant outside the family is not used.
int fp32_variant(genga_ctx *c, const PassArgs &base, int N, int precision, cudaStream_t s) {
    const bool tp2 = base.n_big >= 0;
    const int fam = tp2 ? 1 : family_of(precision);
    auto in_family = [&](int v) { return fam == 0 || (fam == 1) == !is_mutual(v); };
    const int first = fam == 2 ? num_fp32_variants() : 0;
    if (c->forced_variant >= 0 && in_family(c->forced_variant)) return c->forced_variant;
    const int b = size_bucket(N);
    int8_t *table = tp2 ? c->f32_variant_tp : c->f32_variant[fam];
    if (table[b] >= 0) return table[b];
    if (!can_tune(s)) return first;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return 0;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return 0;
    }
    int best = first;
    float best_ms = 3.0e38f;
    for (int v = 0; v < num_all_variants(); v++) {
        if (!in_family(v)) continue;
        const bool known = !tp2 && v < GENGA_MAX_VARIANTS && c->tune_ms[b][v] > 0.f;
        const float ms = known ? c->tune_ms[b][v]
                               : time_variant(c, N, 4, is_mutual(v) ? 1 : 0, 0, s, e0, e1,
                                              [&](MutualPlan *mp, int *split, int *one_row, cudaError_t *e) {
                                                  return launch_fp32_variant(c, base, v, s, mp, split, one_row, e);
                                              });
        if (!tp2 && !known && v < GENGA_MAX_VARIANTS) c->tune_ms[b][v] = ms < 3.0e38f ? ms : 0.f;
        if (ms < best_ms) {
            best_ms = ms;
            best = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    table[b] = (int8_t)best;
    return best;
}

// The FP64 pass variant for this size, chosen the same way (test-particle
// mode 2 always takes the one-sided pass, variant 0).
int fp64_variant(genga_ctx *c, const PassArgs &base, int N, cudaStream_t s) {
    if (base.n_big >= 0) return 0;
    if (c->forced_f64 >= 0) return c->forced_f64;
    const int b = size_bucket(N);
    if (c->f64_variant[b] >= 0) return c->f64_variant[b];
    if (!can_tune(s)) return 0;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return 0;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return 0;
    }
    int best = 0;
    float best_ms = 3.0e38f;
    for (int v = 0; v < num_f64_variants(); v++) {
        const float ms = time_variant(c, N, 4, v > 0 ? 2 : 0, 1, s, e0, e1,
                                      [&](MutualPlan *mp, int *split, int *one_row, cudaError_t *e) {
                                          return launch_fp64_variant(c, base, v, s, mp, split, one_row, e);
                                      });
        if (v < GENGA_MAX_VARIANTS) c->tune64_ms[b][v] = ms < 3.0e38f ? ms : 0.f;
        if (ms < best_ms) {
            best_ms = ms;
            best = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->f64_variant[b] = (int8_t)best;
    return best;
}

// Result of a long-range pass: where its partial sums are and how to combine them.
struct PassOut {
    int split = 1, one_row = 0;
    int mutual = 0;  // 0 one-sided rows, 1 mutual FP32, 2 mutual FP64
    MutualPlan mp{};
};

// Long-range pass over the current state: momentum (and list reset), the
// spatial order (skipped when the positions are those of the previous pass),
// prep, pass, and the sort of the encounter list.  Leaves the partial sums in
// c->partial, indexed by position in the spatial order.
cudaError_t run_pass(genga_ctx *c, const genga_system &sys, const genga_params &p, int precision, bool reorder,
                     PassOut *out, cudaStream_t s, bool momentum_valid = false) {
    // momentum_valid: c->mom already holds P of this state (genga_step after a drift)
    cudaError_t e = momentum_valid ? cudaMemsetAsync(c->enc_count, 0, 2 * sizeof(int32_t), s)
                                   : launch_momentum(sys.vx, sys.vy, sys.vz, sys.m, sys.N, c->mom, c->enc_count, s);
    if (e != cudaSuccess) return e;
    c->launches += momentum_valid ? 0 : 1;
    if (reorder || c->ordered_N != sys.N || c->ordered_nbig != p.n_big) {
        if ((e = launch_order(sys, p.Mstar, p.n_big, c, s)) != cudaSuccess) return e;
        c->ordered_N = sys.N;
        c->ordered_nbig = p.n_big;
        c->steps_since_order = 0;
        c->launches += 11;  // extent, keys, 3 x (histogram, scan, scatter)
    }
    if ((e = launch_prep(sys, p, c, s)) != cudaSuccess) return e;
    c->launches += 1;
    PassArgs a = base_args(c, sys, p);
    *out = PassOut{};
    profile_before_pass(c, s);
    if (is_fp32(precision)) {
        int variant = fp32_variant(c, a, sys.N, precision, s);
        if (is_mutual(variant) && p.n_big >= 0) variant = 0;
        out->mutual = is_mutual(variant) ? 1 : 0;
        if (!launch_fp32_variant(c, a, variant, s, &out->mp, &out->split, &out->one_row, &e)) {
            // no mutual plan now: the one-sided default, except where the
            // caller asked for the group-centred form
            if (precision == GENGA_FP32_BLOCKREL) {
                profile_after_pass(c, s);
                return cudaErrorMemoryAllocation;
            }
            out->mutual = 0;
            launch_fp32_variant(c, a, 0, s, &out->mp, &out->split, &out->one_row, &e);
        }
    } else {
        const int variant = fp64_variant(c, a, sys.N, s);
        out->mutual = variant > 0 ? 2 : 0;
        if (!launch_fp64_variant(c, a, variant, s, &out->mp, &out->split, &out->one_row, &e)) {
            out->mutual = 0;
            launch_fp64_variant(c, a, 0, s, &out->mp, &out->split, &out->one_row, &e);
        }
    }
    profile_after_pass(c, s);
    if (e != cudaSuccess) return e;
    c->launches += 1;
    c->enc_sorted = false;  // sorted when the list is read
    return cudaSuccess;
}

cudaError_t run_kick(genga_ctx *c, const genga_system &sys, const genga_params &p, double tau, double *acc,
                     bool reorder, cudaStream_t s, bool momentum_valid = false) {
    PassOut po;
    cudaError_t e = run_pass(c, sys, p, p.precision, reorder, &po, s, momentum_valid);
    if (e != cudaSuccess) return e;
    c->launches += 1;
    return launch_combine_any(c, po.mutual, po.mp, po.split, po.one_row, sys.N, p.precision == GENGA_FP64 ? 1 : 0,
                              tau, acc, sys, s);
}

// ------------------------------------------------------------ batched mode
bool check_offsets(const genga_ctx *c, const genga_system *all, const int32_t *offsets, int D) {
    if (!c || !all || !offsets || D < 1 || D > GENGA_MAX_DISCS) return false;
    if (offsets[0] != 0 || offsets[D] != all->N) return false;
    for (int d = 0; d < D; d++)
        if (offsets[d + 1] < offsets[d]) return false;
    long long np = 0;
    for (int d = 0; d < D; d++) np += npad_of(offsets[d + 1] - offsets[d]) * (offsets[d + 1] > offsets[d] ? 1 : 0);
    return np <= c->npad_max;
}

unsigned long long offsets_hash(const int32_t *offsets, int D) {
    unsigned long long h = 1469598103934665603ull;
    for (int d = 0; d <= D; d++) {
        h ^= (unsigned long long)(uint32_t)offsets[d];
        h *= 1099511628211ull;
    }
    return h ^ (unsigned long long)D;
}

BatchBodies batch_bodies(const int32_t *offsets, int D) {
    BatchBodies bb;
    memset(&bb, 0, sizeof(bb));
    bb.D = D;
    bb.N_total = offsets[D];
    int p = 0;
    for (int d = 0; d < D; d++) {
        bb.off[d] = offsets[d];
        bb.poff[d] = p;
        const int n = offsets[d + 1] - offsets[d];
        p += n > 0 ? npad_of(n) : 0;
    }
    bb.off[D] = offsets[D];
    bb.poff[D] = p;
    bb.npad_total = p;
    return bb;
}

// Work items of the FP32 pass over a batch: system d gets a share of about
// 96 items per SM proportional to npad_d^2 (its pair count), cut
// into j-chunks per i-block; systems are handed out largest item first.
// False if the partial sums would not fit.
bool plan_batch(const genga_ctx *c, const BatchBodies &bb, int variant, BatchItems *bi, int *grid) {
    memset(bi, 0, sizeof(*bi));
    const int IB = fp32_variant_ib(variant), minb = fp32_variant_minb(variant);
    double total = 0.0;
    for (int d = 0; d < bb.D; d++) {
        const double np = bb.poff[d + 1] - bb.poff[d];
        total += np * np;
    }
    for (int target = 96 * c->sm_count; target >= 1; target /= 2) {
        long long pbase = 0;
        for (int d = 0; d < bb.D; d++) {
            const int np = bb.poff[d + 1] - bb.poff[d];
            bi->pbase[d] = pbase;
            if (np == 0) {
                bi->nchunks[d] = bi->blen[d] = bi->iblocks[d] = 0;
                continue;
            }
            const int iblocks = (np + IB - 1) / IB, ntiles = np / 256;
            const double want = target * ((double)np * np / total);
            int nch = (int)((want + iblocks - 1) / iblocks);
            nch = nch < 1 ? 1 : (nch > ntiles ? ntiles : nch);
            const int ct = (ntiles + nch - 1) / nch;
            nch = (ntiles + ct - 1) / ct;
            bi->iblocks[d] = iblocks;
            bi->blen[d] = ct;
            bi->nchunks[d] = nch;
            pbase += (long long)nch * 3 * np;
        }
        if ((size_t)pbase > c->partial_cap) continue;
        // handout order: larger items (more tiles per chunk) first, then by index
        for (int d = 0; d < bb.D; d++) bi->order[d] = d;
        for (int a = 1; a < bb.D; a++) {  // insertion sort, D <= 256
            const int v = bi->order[a];
            int b = a - 1;
            while (b >= 0 && bi->blen[bi->order[b]] < bi->blen[v]) {
                bi->order[b + 1] = bi->order[b];
                b--;
            }
            bi->order[b + 1] = v;
        }
        int q = 0;
        for (int r = 0; r < bb.D; r++) {
            bi->item0[r] = q;
            const int d = bi->order[r];
            q += bi->iblocks[d] * bi->nchunks[d];
        }
        bi->item0[bb.D] = q;
        bi->items_total = q;
        const int slots = minb * c->sm_count;
        *grid = q < slots ? (q > 0 ? q : 1) : slots;
        return true;
    }
    return false;
}

// Launches the batched pass of FP32 variant v (one-sided: its BatchItems
// plan; mutual: the plan over the batch's systems) and its combine.  False
// when a mutual plan cannot be had (built during a capture, or none fits):
// nothing launched.
bool launch_batched_variant(genga_ctx *c, PassArgs a, const BatchBodies &bb, unsigned long long key, int v,
                            double tau, double *acc, const genga_system &all, cudaStream_t s, bool profile,
                            cudaError_t *err) {
    *err = cudaSuccess;
    if (is_mutual(v)) {
        MutualPlan mp;
        if (!mutual_plan_batched(c, bb, key, v - num_fp32_variants(), s, &mp)) return false;
        a.partial = c->partial;  // the plan may have enlarged (reallocated) the partial rows
        a.mp = mp;
        if (profile) profile_before_pass(c, s);
        *err = launch_pass_mutual(a, v - num_fp32_variants(), c->sm_count, s);
        if (profile) profile_after_pass(c, s);
        if (*err == cudaSuccess)
            *err = launch_combine_mutual(c->partial, mp, bb.N_total, bb.npad_total, c->perm, tau, acc, all.vx,
                                         all.vy, all.vz, c->status, s);
        return true;
    }
    BatchItems bi;
    int grid = 1;
    if (!plan_batch(c, bb, v, &bi, &grid)) {
        *err = cudaErrorInvalidValue;
        return true;
    }
    a.partial = c->partial;
    if (profile) profile_before_pass(c, s);
    *err = launch_pass_batched(a, bb, bi, v, grid, s);
    if (profile) profile_after_pass(c, s);
    if (*err == cudaSuccess)
        *err = launch_combine_batched(bb, bi, c->partial, c->perm, tau, acc, all.vx, all.vy, all.vz, c->status, s);
    return true;
}

// The FP32 variant of a batch: forced (within the precision mode's family),
// already tuned for this batch layout and family, or tuned now: every
// variant of the family (one-sided in test-particle mode 2 and for
// GENGA_FP32_HILO, mutual for GENGA_FP32_BLOCKREL, both for GENGA_FP32) run
// three times -- batched pass and combine, no kick applied -- on the packed
// state, the fastest of the last two kept.  The context remembers
// GENGA_BATCH_LAYOUTS (layout, family) pairs (the oldest is replaced).
// Tuning synchronises the stream, so it is skipped during a capture (the
// family's first variant).
int batch_variant(genga_ctx *c, const PassArgs &a, const BatchBodies &bb, unsigned long long key, int precision,
                  cudaStream_t s, bool tune = true) {
    const int fam = a.n_big >= 0 ? 1 : family_of(precision);
    auto in_family = [&](int v) { return fam == 0 || (fam == 1) == !is_mutual(v); };
    const int first = fam == 2 ? num_fp32_variants() : 0;
    if (c->forced_variant >= 0 && in_family(c->forced_variant)) return c->forced_variant;
    const unsigned long long fkey = key ^ (0x9e3779b97f4a7c15ull * (unsigned long long)(fam + 1));
    for (int q = 0; q < GENGA_BATCH_LAYOUTS; q++)
        if (c->bt_var[q] >= 0 && c->bt_key[q] == fkey) return c->bt_var[q];
    if (!tune || !can_tune(s)) return first;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return first;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return first;
    }
    const int slot = c->bt_next;
    c->bt_next = (c->bt_next + 1) % GENGA_BATCH_LAYOUTS;
    genga_system none{};
    none.N = bb.N_total;
    int best = first;
    float best_ms = 3.0e38f;
    for (int v = 0; v < num_all_variants() && v < GENGA_MAX_VARIANTS; v++) {
        c->bt_ms[slot][v] = 0.f;
        if (!in_family(v)) continue;
        float ms = 3.0e38f;
        for (int rep = 0; rep < 3; rep++) {
            cudaError_t e = cudaSuccess;
            cudaEventRecord(e0, s);
            if (!launch_batched_variant(c, a, bb, key, v, 0.0, nullptr, none, s, false, &e)) break;
            cudaEventRecord(e1, s);
            cudaMemsetAsync(c->enc_count, 0, 2 * sizeof(int32_t), s);
            if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) break;
            float t = 3.0e38f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0 && t < ms) ms = t;
        }
        c->bt_ms[slot][v] = ms < 3.0e38f ? ms : 0.f;
        if (ms < best_ms) {
            best_ms = ms;
            best = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->bt_key[slot] = fkey;
    c->bt_var[slot] = (int8_t)best;
    return best;
}

// One batched kick: momenta (list reset), spatial order (when asked or when
// the batch layout changed), prep, FP32 pass, list sort, combine.
cudaError_t run_kick_batched(genga_ctx *c, const genga_system &all, const int32_t *offsets, int D,
                             const genga_params &p, double tau, double *acc, bool reorder, bool momentum_valid,
                             cudaStream_t s) {
    const BatchBodies bb = batch_bodies(offsets, D);
    const unsigned long long key = offsets_hash(offsets, D);
    cudaError_t e = momentum_valid ? cudaMemsetAsync(c->enc_count, 0, 2 * sizeof(int32_t), s)
                                   : launch_momentum_batched(all, bb, c->Pd, c->enc_count, s);
    if (e != cudaSuccess) return e;
    c->launches += momentum_valid ? 0 : 1;
    if (reorder || c->ordered_N != -2 || c->ordered_key != key) {
        if ((e = launch_order_batched(all, bb, p.Mstar, p.n_big, c, s)) != cudaSuccess) return e;
        c->ordered_N = -2;  // the order belongs to a batch
        c->ordered_key = key;
        c->steps_since_order = 0;
        c->launches += 14;  // extent, keys, 4 x (histogram, scan, scatter)
    }
    if ((e = launch_prep_batched(all, bb, p, c, s)) != cudaSuccess) return e;
    c->launches += 1;
    PassArgs a = base_args(c, all, p);
    a.npad = bb.npad_total;
    const int variant = batch_variant(c, a, bb, key, p.precision, s);
    if (!launch_batched_variant(c, a, bb, key, variant, tau, acc, all, s, true, &e)) {
        // no mutual plan now: the one-sided default, except where the caller
        // asked for the group-centred form
        if (p.precision == GENGA_FP32_BLOCKREL) return cudaErrorMemoryAllocation;
        launch_batched_variant(c, a, bb, key, 0, tau, acc, all, s, true, &e);
    }
    if (e != cudaSuccess) return e;
    c->enc_sorted = false;
    c->launches += 2;
    return cudaSuccess;
}

// ------------------------------------------------------------ step graphs
// genga_step and genga_step_batched replay a CUDA graph of GENGA_REORDER_STEPS
// steps -- one rebuild of the spatial order per block, so every block leaves
// the context as it found it -- once the order has just been rebuilt and the
// FP32 variant is tuned.  The graph is captured on an internal stream the
// first time and whenever the key (arrays, N, batch layout, parameters,
// variant) changes, and launched on the caller's stream.  Profiling
// (genga_measure.h) keeps the step-by-step path, whose events are per pass.

unsigned long long mix(unsigned long long h, unsigned long long v) {
    h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    return h;
}

unsigned long long step_key(const genga_system &sys, const genga_params &p, int variant, unsigned long long layout) {
    unsigned long long h = 1469598103934665603ull;
    const double *arrs[7] = {sys.x, sys.y, sys.z, sys.vx, sys.vy, sys.vz, sys.m};
    for (const double *a : arrs) h = mix(h, (unsigned long long)(uintptr_t)a);
    h = mix(h, (unsigned long long)sys.N);
    const double dv[6] = {p.G, p.Mstar, p.dt, p.n1, p.n2, p.bs_tol};  // fields, not the struct's padding
    for (double d : dv) {
        unsigned long long bits;
        memcpy(&bits, &d, sizeof(bits));
        h = mix(h, bits);
    }
    const int32_t iv[7] = {p.rcrit_mode, p.changeover, p.precision, p.kepler_max_iter, p.n_big, p.n_levels,
                           p.n_levels > 0 ? p.n_sub : 0};
    for (int32_t v : iv) h = mix(h, (unsigned long long)(uint32_t)v);
    h = mix(h, (unsigned long long)(variant + 1));
    return mix(h, layout);
}

bool graphs_usable(const genga_ctx *c) { return c->step_graphs && c->cap_stream && !(c->prof && c->prof->enabled); }

// The graph for `key`, capturing `block(stream)` if needed; false (nothing
// captured, state unchanged) when capture is not possible.
template <class Block>
bool step_graph(genga_ctx *c, unsigned long long key, Block block) {
    if (c->step_exec && c->step_key == key) return true;
    if (c->step_exec) {
        cudaGraphExecDestroy(c->step_exec);
        c->step_exec = nullptr;
    }
    const long long l0 = c->launches;
    const int since0 = c->steps_since_order;
    if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
    const cudaError_t eb = block(c->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &graph);
    const long long per = c->launches - l0;
    c->launches = l0;  // nothing ran yet
    c->steps_since_order = since0;
    cudaGraphExec_t exec = nullptr;
    if (eb != cudaSuccess || ee != cudaSuccess || !graph || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();  // clear a capture error; the caller runs step by step
        return false;
    }
    cudaGraphDestroy(graph);
    c->step_exec = exec;
    c->step_key = key;
    c->step_launches = (int32_t)per;
    return true;
}

bool fp64_tuned(const genga_ctx *c, int N, int n_big) {
    return n_big >= 0 || c->forced_f64 >= 0 || c->f64_variant[size_bucket(N)] >= 0;
}

bool fp32_tuned(const genga_ctx *c, int N, int n_big, int precision) {
    const int fam = n_big >= 0 ? 1 : family_of(precision);
    const bool forced_ok = c->forced_variant >= 0 && (fam == 0 || (fam == 1) == !is_mutual(c->forced_variant));
    return forced_ok || (n_big >= 0 ? c->f32_variant_tp : c->f32_variant[fam])[size_bucket(N)] >= 0;
}

template <class T>
cudaError_t alloc(T **p, size_t n) {
    return cudaMalloc((void **)p, n * sizeof(T) > 0 ? n * sizeof(T) : 16);
}

// The group sets of levels 2 .. L + 1, allocated on first use (before any
// launch or capture of the call): per set three per-body arrays, five
// per-slot arrays and a pair list of 8 slots + 4096 pairs.
cudaError_t ensure_levels(genga_ctx *c, int L) {
    cudaError_t e = cudaSuccess;
    const size_t np = (size_t)c->npad_max, slots = (size_t)c->bs_slots;
    for (int k = 0; k < L && k < GENGA_MAX_LEVELS && e == cudaSuccess; k++) {
        LevelSet &l = c->lv[k];
        if (l.grp) continue;
        l.pair_cap = (int32_t)(8 * slots + 4096);
        if (e == cudaSuccess) e = alloc(&l.grp, np);
        if (e == cudaSuccess) e = alloc(&l.gmark, np);
        if (e == cudaSuccess) e = alloc(&l.gslot, np);
        if (e == cudaSuccess) e = alloc(&l.gbody, slots);
        if (e == cudaSuccess) e = alloc(&l.gmem, slots);
        if (e == cudaSuccess) e = alloc(&l.gstart, slots);
        if (e == cudaSuccess) e = alloc(&l.gsize, slots);
        if (e == cudaSuccess) e = alloc(&l.gcur, slots);
        if (e == cudaSuccess) e = alloc(&l.gof, slots);
        if (e == cudaSuccess) e = alloc(&l.gcount, 1);
        if (e == cudaSuccess) e = alloc(&l.pairs, (size_t)l.pair_cap);
        if (e == cudaSuccess) e = alloc(&l.pair_count, 2);
        if (e == cudaSuccess) e = cudaMemset(l.grp, 0xff, sizeof(int32_t) * np);
        if (e == cudaSuccess) e = cudaMemset(l.gmark, 0, sizeof(int32_t) * np);
        if (e == cudaSuccess) e = cudaMemset(l.gcount, 0, sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMemset(l.pair_count, 0, 2 * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {  // a set is complete or absent, never half allocated
            void *lb[] = {l.grp,  l.gmark,  l.gslot, l.gbody, l.gmem,      l.gstart,
                          l.gsize, l.gcur,  l.gof,   l.gcount, l.pairs, l.pair_count};
            for (void *b : lb)
                if (b) cudaFree(b);
            l = LevelSet{};
        }
    }
    return e;
}

}  // namespace

extern "C" {

const char *genga_status_string(genga_status s) {
    switch (s) {
        case GENGA_OK: return "ok";
        case GENGA_ERR_INVALID_ARG: return "invalid argument";
        case GENGA_ERR_CUDA: return "CUDA runtime error";
        case GENGA_ERR_CAPACITY: return "encounter list overflow (list truncated)";
        case GENGA_ERR_KEPLER: return "Kepler solver did not converge for at least one body";
        case GENGA_ERR_NONFINITE: return "non-finite acceleration";
        case GENGA_ERR_TIMEOUT: return "bounded device wait timed out";
        case GENGA_ERR_BS: return "close-encounter level: forced Bulirsch-Stoer sub-step or groups over capacity";
    }
    return "unknown status";
}

void genga_destroy(genga_ctx *c) {
    if (!c) return;
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();
    profile_free(c);
    free_mutual_cache(c);
    if (c->step_exec) cudaGraphExecDestroy(c->step_exec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    void *bufs[] = {c->pk_r,        c->pk_rl,       c->gctr,
                    c->pk_hi,       c->pk_t,        c->pk_d,        c->pk_lo,       c->pk64,        c->scr,      c->gbox_lo,    c->gbox_hi,    c->gflag,
                    c->perm,        c->ord_keys[0], c->ord_keys[1], c->ord_vals[0], c->ord_vals[1], c->ord_hist,
                    c->ord_rbits,   c->a_osc,       c->rc_eq1,      c->partial,  c->mom,        c->enc,
                    c->enc_count,   c->status,      c->energy_part, c->work,   c->Pd,         c->Pd_part,
                    c->grp,         c->gmark,       c->gslot,       c->iperm,  c->gbody,      c->gmem,
                    c->gstart,      c->gsize,       c->gcur,        c->gcount, c->gof,        c->bs_tp,      c->bs_work,
                    c->pred};
    for (void *b : bufs)
        if (b) cudaFree(b);
    for (LevelSet &l : c->lv) {
        void *lb[] = {l.grp,  l.gmark,  l.gslot, l.gbody, l.gmem,      l.gstart,
                      l.gsize, l.gcur,  l.gof,   l.gcount, l.pairs, l.pair_count};
        for (void *b : lb)
            if (b) cudaFree(b);
    }
    delete c;
}

genga_status genga_create(genga_ctx **out, int32_t max_N, int32_t device) {
    if (!out) return GENGA_ERR_INVALID_ARG;
    *out = nullptr;
    if (max_N < 0 || max_N > (1 << 28)) return GENGA_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) return GENGA_ERR_CUDA;
    if (device < 0 || device >= ndev) return GENGA_ERR_INVALID_ARG;
    DeviceGuard g(device);
    if (!g.ok) return GENGA_ERR_CUDA;
    genga_ctx *c = new (std::nothrow) genga_ctx();
    if (!c) return GENGA_ERR_CUDA;
    memset(c, 0, sizeof(*c));
    c->device = device;
    c->max_N = max_N;
    for (int b = 0; b < 32; b++) c->f32_variant[0][b] = c->f32_variant[1][b] = c->f32_variant[2][b] = c->f32_variant_tp[b] = -1;
    c->forced_variant = -1;
    for (int b = 0; b < 32; b++) c->f64_variant[b] = -1;
    for (int q = 0; q < GENGA_BATCH_LAYOUTS; q++) c->bt_var[q] = -1;
    c->bt_next = 0;
    c->forced_f64 = -1;
    c->ordered_N = -1;
    c->step_graphs = 1;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete c;
        return GENGA_ERR_CUDA;
    }
    c->sm_count = prop.multiProcessorCount;
    const int np = npad_of(max_N > 0 ? max_N : 1);
    c->npad_max = np;
    // partial sums: split * 3 * npad doubles; the plans stay near 96 items per
    // SM of up to 512 bodies, i.e. split * npad <~ 96 * SMs * 512 (plan_pass
    // clamps larger i-blocks to this)
    c->partial_cap = 3 * ((size_t)np * 4 + (size_t)96 * c->sm_count * 512 + 4096);
    long long ecap = 4096;
    while (ecap < 16LL * max_N) ecap <<= 1;
    c->enc_cap = (int32_t)ecap;
    c->energy_blocks = np / 256;
    cudaError_t e = init_pass_kernels();
    if (e == cudaSuccess) e = init_mutual_kernels();
    if (e == cudaSuccess) e = init_bs_kernel(c->sm_count);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = alloc(&c->pk_hi, np);
    if (e == cudaSuccess) e = alloc(&c->pk_lo, np);
    if (e == cudaSuccess) e = alloc(&c->pk_t, 4 * (size_t)np);
    if (e == cudaSuccess) e = alloc(&c->pk_d, 2 * (size_t)np);
    if (e == cudaSuccess) e = alloc(&c->pk_r, np);
    if (e == cudaSuccess) e = alloc(&c->pk_rl, np);
    if (e == cudaSuccess) e = alloc(&c->gctr, np / 64);
    if (e == cudaSuccess) e = alloc(&c->pk64, np);
    if (e == cudaSuccess) e = alloc(&c->scr, np);
    if (e == cudaSuccess) e = alloc(&c->gbox_lo, np / 64);
    if (e == cudaSuccess) e = alloc(&c->gbox_hi, np / 64);
    if (e == cudaSuccess) e = alloc(&c->gflag, np / 64);
    if (e == cudaSuccess) e = alloc(&c->perm, np);
    for (int q = 0; q < 2; q++) {
        if (e == cudaSuccess) e = alloc(&c->ord_keys[q], np);
        if (e == cudaSuccess) e = alloc(&c->ord_vals[q], np);
    }
    if (e == cudaSuccess) e = alloc(&c->ord_hist, order_hist_entries(np));
    if (e == cudaSuccess) e = alloc(&c->ord_rbits, 1);
    if (e == cudaSuccess) e = alloc(&c->a_osc, np);
    if (e == cudaSuccess) e = alloc(&c->rc_eq1, np);
    if (e == cudaSuccess) e = alloc(&c->partial, c->partial_cap);
    if (e == cudaSuccess) e = alloc(&c->work, 1);
    if (e == cudaSuccess) e = alloc(&c->Pd, 3 * GENGA_MAX_DISCS);
    if (e == cudaSuccess) e = alloc(&c->Pd_part, 3 * GENGA_MAX_DISCS);
    if (e == cudaSuccess) e = alloc(&c->mom, 256);   // P, block partials, ticket
    if (e == cudaSuccess) e = cudaMemset(c->mom, 0, 256 * sizeof(double));
    if (e == cudaSuccess) e = alloc(&c->enc, (size_t)c->enc_cap);
    if (e == cudaSuccess) e = alloc(&c->enc_count, 2);   // [0] encounter pairs, [1] predicted entries
    if (e == cudaSuccess) e = alloc(&c->pred, (size_t)c->enc_cap);
    if (e == cudaSuccess) e = alloc(&c->status, 1);
    if (e == cudaSuccess) e = alloc(&c->energy_part, (size_t)4 * c->energy_blocks);
    // close-encounter level: labels and marks start cleared (-1 / 0) and are
    // cleared again by the level-1 kernel for every member it moves
    c->bs_slots = np < GENGA_BS_MAX_SLOTS ? np : GENGA_BS_MAX_SLOTS;
    if (e == cudaSuccess) e = alloc(&c->grp, np);
    if (e == cudaSuccess) e = alloc(&c->gmark, np);
    if (e == cudaSuccess) e = alloc(&c->gslot, np);
    if (e == cudaSuccess) e = alloc(&c->iperm, np);
    if (e == cudaSuccess) e = alloc(&c->gbody, c->bs_slots);
    if (e == cudaSuccess) e = alloc(&c->gmem, c->bs_slots);
    if (e == cudaSuccess) e = alloc(&c->gstart, c->bs_slots);
    if (e == cudaSuccess) e = alloc(&c->gsize, c->bs_slots);
    if (e == cudaSuccess) e = alloc(&c->gcur, c->bs_slots);
    if (e == cudaSuccess) e = alloc(&c->gcount, 1);
    if (e == cudaSuccess) e = alloc(&c->gof, c->bs_slots);
    if (e == cudaSuccess) e = alloc(&c->bs_tp, c->bs_slots);
    if (e == cudaSuccess) e = alloc(&c->bs_work, (size_t)GENGA_BS_FIELDS * c->bs_slots);
    if (e == cudaSuccess) e = cudaMemset(c->grp, 0xff, sizeof(int32_t) * (size_t)np);
    if (e == cudaSuccess) e = cudaMemset(c->gmark, 0, sizeof(int32_t) * (size_t)np);
    if (e == cudaSuccess) e = cudaMemset(c->gcount, 0, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(c->enc_count, 0, 2 * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(c->status, 0, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        genga_destroy(c);
        return cuda_status(e);
    }
    *out = c;
    return GENGA_OK;
}

genga_status genga_kick(genga_ctx *c, const genga_system *sys, const genga_params *p, double tau, double *acc,
                        void *stream) {
    genga_status st;
    if ((st = check_system(c, sys)) != GENGA_OK) return st;
    if ((st = check_params(p)) != GENGA_OK) return st;
    if (!is_fin(tau)) return GENGA_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (sys->N == 0) return cuda_status(cudaMemsetAsync(c->enc_count, 0, 2 * sizeof(int32_t), s));
    return cuda_status(run_kick(c, *sys, *p, tau, acc, true, s));
}

genga_status genga_drift(genga_ctx *c, genga_system *sys, const genga_params *p, double dt, void *stream) {
    genga_status st;
    if ((st = check_system(c, sys)) != GENGA_OK) return st;
    if ((st = check_params(p)) != GENGA_OK) return st;
    if (!is_fin(dt)) return GENGA_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    genga_system s2 = *sys;
    if (const cudaError_t e_ = ensure_levels(c, p->n_levels); e_ != cudaSuccess) return cuda_status(e_);
    if (sys->N > 0) c->launches += drift_launches(*p);
    return cuda_status(launch_drift(s2, *p, dt, c, (cudaStream_t)stream));
}

genga_status genga_last_encounters(genga_ctx *c, int32_t *pairs, int32_t capacity, int32_t *count, void *stream) {
    if (!c || capacity < 0 || !count || (capacity > 0 && !pairs)) return GENGA_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (!c->enc_sorted) {  // the list is in discovery order until first read
        if (const cudaError_t e_ = launch_sort_pairs(c->enc, c->enc_cap, c->enc_count, s); e_ != cudaSuccess) return cuda_status(e_);
        c->enc_sorted = true;
        c->launches += 1;
    }
    c->launches += 1;
    return launch_copy_pairs(c->enc, c->enc_count, c->enc_cap, pairs, capacity, count, c->status, s) == cudaSuccess
               ? GENGA_OK
               : GENGA_ERR_CUDA;
}

genga_status genga_encounters(genga_ctx *c, const genga_system *sys, const genga_params *p, int32_t *pairs,
                              int32_t capacity, int32_t *count, void *stream) {
    genga_status st;
    if ((st = check_system(c, sys)) != GENGA_OK) return st;
    if ((st = check_params(p)) != GENGA_OK) return st;
    if (capacity < 0 || !count || (capacity > 0 && !pairs)) return GENGA_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (sys->N == 0) {
        if (const cudaError_t e_ = cudaMemsetAsync(c->enc_count, 0, 2 * sizeof(int32_t), s); e_ != cudaSuccess) return cuda_status(e_);
        c->enc_sorted = true;
    } else {
        PassOut po;
        if (const cudaError_t e_ = run_pass(c, *sys, *p, GENGA_FP32_HILO, true, &po, s); e_ != cudaSuccess) return cuda_status(e_);
    }
    return genga_last_encounters(c, pairs, capacity, count, stream);
}

genga_status genga_step(genga_ctx *c, genga_system *sys, const genga_params *p, int32_t nsteps, void *stream) {
    genga_status st;
    if ((st = check_system(c, sys)) != GENGA_OK) return st;
    if ((st = check_params(p)) != GENGA_OK) return st;
    if (nsteps < 0) return GENGA_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (sys->N == 0 || nsteps == 0) return GENGA_OK;
    if (const cudaError_t e_ = ensure_levels(c, p->n_levels); e_ != cudaSuccess) return cuda_status(e_);
    genga_system s2 = *sys;
    const double h = 0.5 * p->dt;
    genga_params p_close = *p;  // the closing kick of a step: no predicted entries
    p_close.bs_tol = 0.0;
    // The spatial order is a performance device (every pass classifies tiles
    // from the current positions; any order gives the same sum up to
    // rounding), so genga_step rebuilds it every GENGA_REORDER_STEPS drifts,
    // counted across calls, and whenever N changes.  The drift leaves P of the
    // new state in c->mom, which the closing kick reuses.
    auto one_step = [&](cudaStream_t q) -> cudaError_t {
        cudaError_t e = run_kick(c, s2, *p, h, nullptr, false, q);
        if (e == cudaSuccess) e = launch_drift(s2, *p, p->dt, c, q);
        c->launches += drift_launches(*p);
        c->steps_since_order++;
        const bool reorder = c->steps_since_order >= GENGA_REORDER_STEPS;
        // the closing kick needs no predicted entries (the next step's first
        // kick lists them again), so it screens at r_crit only
        if (e == cudaSuccess) e = run_kick(c, s2, p_close, h, nullptr, reorder, q, true);
        return e;
    };
    int k = 0;
    auto aligned = [&]() {
        return c->steps_since_order == 0 && c->ordered_N == s2.N && c->ordered_nbig == p->n_big &&
               (is_fp32(p->precision) ? fp32_tuned(c, s2.N, p->n_big, p->precision) : fp64_tuned(c, s2.N, p->n_big));
    };
    for (; k < nsteps && !(aligned() && nsteps - k >= GENGA_REORDER_STEPS); k++)
        if (const cudaError_t e_ = one_step(s); e_ != cudaSuccess) return cuda_status(e_);
    if (k < nsteps && graphs_usable(c)) {
        int variant = -1;
        if (is_fp32(p->precision)) {
            PassArgs pa = base_args(c, s2, *p);
            variant = fp32_variant(c, pa, s2.N, p->precision, s);  // tuned already (aligned() holds)
            if (is_mutual(variant) && p->n_big < 0) {
                MutualPlan mp;  // the plan is built outside the capture
                if (!mutual_plan(c, s2.N, variant - num_fp32_variants(), s, &mp)) {
                    if (p->precision == GENGA_FP32_BLOCKREL) return GENGA_ERR_CUDA;
                    variant = 0;
                }
            }
        } else {
            PassArgs pa = base_args(c, s2, *p);
            variant = fp64_variant(c, pa, s2.N, s);  // tuned already (aligned() holds)
            if (variant > 0) {
                MutualPlan mp;  // the plan is built outside the capture
                if (!mutual64_plan(c, s2.N, variant - 1, s, &mp)) variant = 0;
            }
            variant += 1000;  // FP64 variants apart from FP32 ones in the graph key
        }
        const unsigned long long key = step_key(s2, *p, variant, 0);
        const bool ok = step_graph(c, key, [&](cudaStream_t q) {
            for (int b = 0; b < GENGA_REORDER_STEPS; b++) {
                const cudaError_t e = one_step(q);
                if (e != cudaSuccess) return e;
            }
            return cudaSuccess;
        });
        if (ok) {
            for (; nsteps - k >= GENGA_REORDER_STEPS; k += GENGA_REORDER_STEPS) {
                if (const cudaError_t e_ = cudaGraphLaunch(c->step_exec, s); e_ != cudaSuccess) return cuda_status(e_);
                c->launches += c->step_launches;
            }
            c->enc_sorted = false;
        }
    }
    for (; k < nsteps; k++)
        if (const cudaError_t e_ = one_step(s); e_ != cudaSuccess) return cuda_status(e_);
    return GENGA_OK;
}

genga_status genga_kick_batched(genga_ctx *c, const genga_system *all, const int32_t *offsets, int32_t D,
                                const genga_params *p, double tau, double *acc, void *stream) {
    genga_status st;
    if ((st = check_system(c, all)) != GENGA_OK) return st;
    if ((st = check_params(p)) != GENGA_OK) return st;
    if (!is_fp32(p->precision) || !is_fin(tau) ||
        !check_offsets(c, all, offsets, D))
        return GENGA_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (all->N == 0) return cuda_status(cudaMemsetAsync(c->enc_count, 0, 2 * sizeof(int32_t), s));
    const cudaError_t e = run_kick_batched(c, *all, offsets, D, *p, tau, acc, true, false, s);
    if (e == cudaErrorInvalidValue) return GENGA_ERR_INVALID_ARG;
    return cuda_status(e);
}

genga_status genga_step_batched(genga_ctx *c, genga_system *all, const int32_t *offsets, int32_t D,
                                const genga_params *p, int32_t nsteps, void *stream) {
    genga_status st;
    if ((st = check_system(c, all)) != GENGA_OK) return st;
    if ((st = check_params(p)) != GENGA_OK) return st;
    if (!is_fp32(p->precision) || nsteps < 0 ||
        !check_offsets(c, all, offsets, D))
        return GENGA_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (all->N == 0 || nsteps == 0) return GENGA_OK;
    if (const cudaError_t e_ = ensure_levels(c, p->n_levels); e_ != cudaSuccess) return cuda_status(e_);
    genga_system a2 = *all;
    const BatchBodies bb = batch_bodies(offsets, D);
    const unsigned long long layout = offsets_hash(offsets, D);
    const double h = 0.5 * p->dt;
    genga_params p_close = *p;  // the closing kick of a step: no predicted entries
    p_close.bs_tol = 0.0;
    auto one_step = [&](cudaStream_t q) -> cudaError_t {
        cudaError_t e = run_kick_batched(c, a2, offsets, D, *p, h, nullptr, false, false, q);
        if (e == cudaSuccess) e = launch_drift_batched(a2, bb, *p, p->dt, c, q);
        c->launches += drift_launches(*p);
        c->steps_since_order++;
        const bool reorder = c->steps_since_order >= GENGA_REORDER_STEPS;
        if (e == cudaSuccess) e = run_kick_batched(c, a2, offsets, D, p_close, h, nullptr, reorder, true, q);
        return e;
    };
    auto status_of = [](cudaError_t e) {
        return e == cudaErrorInvalidValue ? GENGA_ERR_INVALID_ARG : GENGA_ERR_CUDA;
    };
    auto aligned = [&]() { return c->steps_since_order == 0 && c->ordered_N == -2 && c->ordered_key == layout; };
    int k = 0;
    for (; k < nsteps && !(aligned() && nsteps - k >= GENGA_REORDER_STEPS); k++) {
        const cudaError_t e = one_step(s);
        if (e != cudaSuccess) return status_of(e);
    }
    if (k < nsteps && graphs_usable(c)) {
        PassArgs pa = base_args(c, a2, *p);
        int variant = batch_variant(c, pa, bb, layout, p->precision, s, false);  // tuned by the steps above
        if (is_mutual(variant)) {
            MutualPlan mp;  // the plan is built outside the capture
            if (!mutual_plan_batched(c, bb, layout, variant - num_fp32_variants(), s, &mp)) {
                if (p->precision == GENGA_FP32_BLOCKREL) return GENGA_ERR_CUDA;
                variant = 0;
            }
        }
        const unsigned long long key = step_key(a2, *p, variant, mix(layout, 0xba7c4ull));
        const bool ok = step_graph(c, key, [&](cudaStream_t q) {
            for (int b = 0; b < GENGA_REORDER_STEPS; b++) {
                const cudaError_t e = one_step(q);
                if (e != cudaSuccess) return e;
            }
            return cudaSuccess;
        });
        if (ok) {
            for (; nsteps - k >= GENGA_REORDER_STEPS; k += GENGA_REORDER_STEPS) {
                if (const cudaError_t e_ = cudaGraphLaunch(c->step_exec, s); e_ != cudaSuccess) return cuda_status(e_);
                c->launches += c->step_launches;
            }
            c->enc_sorted = false;
        }
    }
    for (; k < nsteps; k++) {
        const cudaError_t e = one_step(s);
        if (e != cudaSuccess) return status_of(e);
    }
    return GENGA_OK;
}

genga_status genga_batched_tuning(genga_ctx *c, const int32_t *offsets, int32_t D, int32_t *variant, float *ms,
                                  int32_t n) {
    if (!c || !offsets || !variant || D < 1 || D > GENGA_MAX_DISCS || n < 0 || (n > 0 && !ms))
        return GENGA_ERR_INVALID_ARG;
    // the entry of the autotuned mode (GENGA_FP32, family 0) for this layout
    const unsigned long long key = offsets_hash(offsets, D) ^ 0x9e3779b97f4a7c15ull;
    *variant = -1;
    for (int q = 0; q < n; q++) ms[q] = 0.f;
    for (int k = 0; k < GENGA_BATCH_LAYOUTS; k++) {
        if (c->bt_var[k] < 0 || c->bt_key[k] != key) continue;
        *variant = c->bt_var[k];
        for (int q = 0; q < n && q < GENGA_MAX_VARIANTS && q < num_all_variants(); q++) ms[q] = c->bt_ms[k][q];
    }
    return GENGA_OK;
}

genga_status genga_energy(genga_ctx *c, const genga_system *sys, const genga_params *p, double *E_L, void *stream) {
    genga_status st;
    if ((st = check_system(c, sys)) != GENGA_OK) return st;
    if ((st = check_params(p)) != GENGA_OK) return st;
    if (!E_L) return GENGA_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    for (int k = 0; k < 4; k++) E_L[k] = 0.0;
    if (sys->N == 0) return GENGA_OK;
    if (const cudaError_t e_ = launch_energy(*sys, *p, c, s); e_ != cudaSuccess) return cuda_status(e_);
    if (launch_momentum(sys->vx, sys->vy, sys->vz, sys->m, sys->N, c->mom, nullptr, s) != cudaSuccess)
        return GENGA_ERR_CUDA;
    const int nb = (sys->N + 255) / 256;
    double *host = (double *)malloc(sizeof(double) * (4 * (size_t)nb + 3));
    if (!host) return GENGA_ERR_CUDA;
    cudaError_t e = cudaMemcpyAsync(host, c->energy_part, sizeof(double) * 4 * nb, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host + 4 * nb, c->mom, sizeof(double) * 3, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        free(host);
        return GENGA_ERR_CUDA;
    }
    // host: block partials in index order, compensated
    for (int q = 0; q < 4; q++) {
        double sum = 0.0, comp = 0.0;
        const double *P = host + 4 * nb;
        double terms_extra = (q == 0) ? (P[0] * P[0] + P[1] * P[1] + P[2] * P[2]) / (2.0 * p->Mstar) : 0.0;
        for (int b = 0; b <= nb; b++) {
            const double v = (b < nb) ? host[4 * b + q] : terms_extra;
            const double t = sum + v;
            comp += (fabs(sum) >= fabs(v)) ? ((sum - t) + v) : ((v - t) + sum);
            sum = t;
        }
        E_L[q] = sum + comp;
    }
    free(host);
    return GENGA_OK;
}

genga_status genga_compact(genga_ctx *c, genga_system *sys, int32_t *id, void *stream) {
    genga_status st;
    if ((st = check_system(c, sys)) != GENGA_OK) return st;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (sys->N == 0) return GENGA_OK;
    genga_system s2 = *sys;
    cudaError_t e = launch_compact(c, s2, id, c->gcount, s);
    int32_t n = sys->N;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&n, c->gcount, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    c->launches += 4;
    if (n != sys->N) {  // the order, the list and the step graph belong to the old arrays
        c->ordered_N = -1;
        cudaMemsetAsync(c->enc_count, 0, 2 * sizeof(int32_t), s);
        c->enc_sorted = true;
    }
    sys->N = n;
    return GENGA_OK;
}

genga_status genga_tune_levels(genga_ctx *c, const genga_system *sys, const genga_params *p, const int32_t *n_levels,
                               const int32_t *n_sub, int32_t ncand, int32_t trial_steps, int32_t *best, float *ms,
                               int32_t *codes, void *stream) {
    genga_status st;
    if ((st = check_system(c, sys)) != GENGA_OK) return st;
    if ((st = check_params(p)) != GENGA_OK) return st;
    if (!n_levels || !n_sub || !best || ncand < 1 || ncand > 64 || trial_steps < 1) return GENGA_ERR_INVALID_ARG;
    for (int k = 0; k < ncand; k++) {
        genga_params q = *p;
        q.n_levels = n_levels[k];
        q.n_sub = n_sub[k];
        if ((st = check_params(&q)) != GENGA_OK) return st;
    }
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t N = (size_t)sys->N, nf = sys->radius ? 8 : 7;
    double *copy = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    // the caller's status bits are kept aside; each trial's bits are read and cleared
    uint32_t bits_before = 0, bits_failed = 0;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&bits_before, c->status, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(c->status, 0, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc((void **)&copy, sizeof(double) * (N > 0 ? nf * N : 1));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const double *src[8] = {sys->x, sys->y, sys->z, sys->vx, sys->vy, sys->vz, sys->m, sys->radius};
    genga_system t = *sys;
    double **dst[8] = {&t.x, &t.y, &t.z, &t.vx, &t.vy, &t.vz, &t.m, &t.radius};
    for (size_t f = 0; f < nf; f++) *dst[f] = copy + f * N;
    auto reset = [&]() {
        for (size_t f = 0; f < nf && e == cudaSuccess; f++)
            e = cudaMemcpyAsync(*dst[f], src[f], sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
    };
    float best_ms = 0.0f, fastest_ms = 0.0f;
    int fastest = 0;
    bool any_ok = false;
    *best = 0;
    for (int k = 0; k < ncand && e == cudaSuccess && st == GENGA_OK; k++) {
        genga_params q = *p;
        q.n_levels = n_levels[k];
        q.n_sub = n_sub[k];
        reset();  // one untimed step (allocation, graph capture, tuning of the pass), then the trial
        if (e == cudaSuccess && (st = genga_step(c, &t, &q, 1, stream)) != GENGA_OK) break;
        reset();
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        if (e == cudaSuccess && (st = genga_step(c, &t, &q, trial_steps, stream)) != GENGA_OK) break;
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t_ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t_ms, e0, e1);
        t_ms /= (float)trial_steps;
        if (ms) ms[k] = t_ms;
        uint32_t bits = 0;  // this candidate's status: a candidate that raised one is not chosen
        if (e == cudaSuccess) e = cudaMemcpy(&bits, c->status, sizeof(uint32_t), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemset(c->status, 0, sizeof(uint32_t));
        int code = 0;
        for (int b = 1; b <= 7 && !code; b++)
            if (bits & GENGA_BIT(b)) code = b;
        if (codes) codes[k] = code;
        bits_failed |= bits;
        if (k == 0 || t_ms < fastest_ms) {
            fastest_ms = t_ms;
            fastest = k;
        }
        if (!code && (!any_ok || t_ms < best_ms)) {
            best_ms = t_ms;
            *best = k;
            any_ok = true;
        }
    }
    if (!any_ok) *best = fastest;  // every candidate raised a status: the fastest, and its bits stay raised
    const uint32_t restore = bits_before | (any_ok ? 0u : bits_failed);
    if (e == cudaSuccess) e = cudaMemcpy(c->status, &restore, sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (copy) {
        cudaStreamSynchronize(s);
        cudaFree(copy);
    }
    c->ordered_N = -1;  // the order and the step graph were built on the copy
    if (st != GENGA_OK) return st;
    return cuda_status(e);
}

const char *genga_last_cuda_error(void) { return cudaGetErrorName(g_last_cuda_error); }

genga_status genga_get_status(genga_ctx *c, void *stream) {
    if (!c) return GENGA_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t bits = 0;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&bits, c->status, sizeof(bits), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(c->status, 0, sizeof(bits));
    if (e != cudaSuccess) return cuda_status(e);
    for (int code = 1; code <= 7; code++)
        if (bits & GENGA_BIT(code)) return (genga_status)code;
    return GENGA_OK;
}

}  // extern "C"
