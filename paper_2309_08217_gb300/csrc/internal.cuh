// internal.cuh -- context layout, launch helpers and PTX wrappers shared by
// the libgenga translation units (sm_103a only).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/genga.h"

// ---------------------------------------------------------------- status bits
// Sticky device status word: bit (code - 1) for each genga_status error code.
#define GENGA_BIT(code) (1u << ((code) - 1))

// Spin-wait limit for mbarrier waits: 2 s of %globaltimer (nanoseconds).
#define GENGA_WAIT_LIMIT_NS 2000000000ull

// ------------------------------------------------------------- tile geometry
// Bodies are padded to a multiple of GENGA_PAD so that every j-tile and every
// i-block is full; padded bodies have zero mass and sit far away.
#define GENGA_PAD 1024
#define GENGA_PAD_POS 1.0e6f
// Largest number of systems in one batched call (the disc index takes the top
// 8 bits of the 32-bit Morton sort key).
#define GENGA_MAX_DISCS GENGA_MAX_BATCH

// genga_step rebuilds the spatial order of the bodies every this many steps.
#define GENGA_REORDER_STEPS 4
// Bodies heavier than this fraction of the central mass are ordered after the
// others (their large r_crit bound would make a group of planetesimals NEAR).
#define GENGA_HEAVY_MASS 1e-7
// Group flags (test-particle mode 2): the group holds a body that is not a
// test particle / a test particle.
#define GENGA_GROUP_BIG 1
#define GENGA_GROUP_TP 2

// Bodies per tile of the tile-blocked FP32 copy (pk_t).
#define GENGA_TILE_T 256

// Close-encounter level: doubles of level-1 workspace per group member
// (encounter.cu), and the most members one drift can integrate.
#define GENGA_BS_FIELDS 239
// Pairs outside r_crit,ij but within this multiple of it whose straight-line
// relative motion over the drift enters r_crit,ij join the level's groups.
#define GENGA_PREDICT_RANGE 1.5
#define GENGA_BS_MAX_SLOTS (1 << 18)

namespace genga {
struct Profile {                // CUDA event pairs around pass launches
    static constexpr int CAP = 65536;
    cudaEvent_t *ev = nullptr;  // [2 * CAP]
    int created = 0;
    int n = 0;
    bool enabled = false;
};
}  // namespace genga

#define GENGA_BATCH_LAYOUTS 8  // batch layouts whose tuned FP32 variant a context remembers
#define GENGA_MAX_VARIANTS 16  // FP32 pass variants the context records tuning times for
#define GENGA_MAX_TIERS 8      // chunk-length tiers of an FP32 pass plan
#define GENGA_MUTUAL_MAX_ITEMS 65536  // work items of one mutual pass plan

namespace genga {
// Work plan of the mutual (symmetric) passes over one or more independent
// systems (a batch), each a range of 64-body groups cut into i-blocks of gpb
// groups (i-tiles of NP groups, one per consumer warp).  Pairs inside a block
// are evaluated one-sided by its diagonal items: every warp takes its i-tile
// against a range of the block's own groups (each ordered pair once, i-side
// only).  Pairs between blocks of a system are evaluated once, for both
// bodies, by the strip items of the earlier block: chunks of the system's
// groups after it.  Item q of the table is {block, first group, end group,
// i-row}: the partial row the item writes for the block's bodies (rows of a
// system are 3 x np entries -- double-float pairs or doubles -- from its
// pbase): diagonal items rows 0 .. cnt.x - 1, strip chunks rows
// S .. S + cnt.y - 1 (S = the most diagonal items of any block of the
// system); strip items of the system's block b also write j-row irows + b for
// the groups they cover.  A body of the system's block b sums i-rows
// [0, cnt.x), [S, S + cnt.y) and j-rows irows + [0, b).
struct MSys {
    int32_t poff, np;           // first packed position (a multiple of 64), packed length (its rows' length)
    int32_t N, off;             // bodies, first caller index (perm[off + k] is packed position poff + k)
    int32_t irows, S;           // first j-row, diagonal rows of its blocks
    int32_t g1, blk0;           // end of its groups holding bodies (a global group index), its first block
    long long pbase;            // first 8-byte entry of its partial rows
};
struct MutualPlan {
    int32_t nb, gpb, items, nsys;
    int32_t nreal;              // > 0: the bodies of system 0 (a single-system plan, built for the padded length)
    const int4 *item;           // [items] {block, first group, end group, i-row}: global blocks and groups
    const int2 *blk;            // [nb] {diagonal items, strip chunks} of each block
    const int32_t *bsys;        // [nb] the system of each block
    const MSys *sys;            // [nsys]
};
struct MutualCache;             // host plans per (N, variant), mutual.cu
}  // namespace genga

namespace genga {
// The groups of one level: the layout the grouping kernel writes (members of
// group g at gmem[gstart[g] ..], gsize[g] of them; grp / gmark per body) and
// the pair list they are formed from.
struct LevelSet {
    int32_t *grp, *gmark, *gslot;               // [npad_max]
    int32_t *gbody, *gmem, *gstart, *gsize, *gcur;  // [bs_slots]
    int32_t *gof;                               // [bs_slots] group of each member slot (levels.cu)
    int32_t *gcount;                            // [1]
    int2 *pairs;                                // [pair_cap] pairs of the level above inside this level's radius
    int32_t *pair_count;                        // [2]: pairs, 0 (the grouping kernel's second list)
    int32_t pair_cap;
};
}  // namespace genga

struct genga_ctx {
    int device;
    int sm_count;
    int32_t max_N;
    int32_t npad_max;          // roundup(max_N, GENGA_PAD)
    // packed per-body data, rebuilt at every kick (prep kernel)
    float4 *pk_hi;             // [npad] {x_hi, y_hi, z_hi, G m (fp32)}
    float4 *pk_lo;             // [npad] {x - x_hi, y - y_hi, z - z_hi, 0}
    float *pk_t;               // [4 npad] tile-blocked {x_hi}, {y_hi}, {z_hi}, {G m} per 256 bodies
    float4 *pk_d;              // [2 npad] duplicated pairs {x_hi, x_hi, y_hi, y_hi}, {z_hi, z_hi, G m, G m}
    float4 *pk_r;              // [npad] group-centred {X, Y, Z, G m}, X = fl32(x - c_group)
    float4 *pk_rl;             // [npad] their residuals {x - c - X, y - c - Y, z - c - Z, test particle}
    float4 *gctr;              // [npad / 64] group centre c (FP32) and the precision distance of the group
    double4_32a *pk64;             // [npad] {x, y, z, G m}
    float2 *scr;               // [npad] screening bound factors {H_i, A_i} (rounded up)
    float4 *gbox_lo;           // [npad / 64] per 64-body group: {min x, min y, min z, max H}
    float4 *gbox_hi;           // [npad / 64]                    {max x, max y, max z, max A}
    int32_t *gflag;            // [npad / 64] GENGA_GROUP_BIG | GENGA_GROUP_TP (test-particle mode 2)
    uint32_t *perm;            // [npad] body at position k of the spatial order
    uint32_t *ord_keys[2];     // [npad] radix sort keys (ping-pong)
    uint32_t *ord_vals[2];     // [npad] radix sort values
    uint32_t *ord_hist;        // digit histograms / offsets
    unsigned *ord_rbits;       // [1] extent of the positions (float bits)
    double *a_osc;             // [npad] osculating semi-major axis (Eq. 1 input)
    double *rc_eq1;            // [npad] per-body Eq. 1 radius
    double *partial;           // [split][3][npad] FP64 partial accelerations
    double *mom;               // [256] P (3 doubles), momentum block partials, ticket
    // encounter list of the most recent pass
    int2 *enc;                 // [enc_cap] unsorted during the pass, sorted after
    int32_t enc_cap;           // power of two
    int32_t *enc_count;        // [2]: encounter pairs, predicted entries (pred)
    int2 *pred;                // [enc_cap] pairs predicted to enter r_crit within the drift (bs_tol > 0)
    bool enc_sorted;           // the list has been sorted since the pass that built it
    uint32_t *status;          // [1] sticky bits
    double *energy_part;       // [energy_blocks][4]
    int32_t energy_blocks;
    genga::Profile *prof;      // measurement hooks (genga_measure.h), NULL when unused
    int32_t *work;             // [1] work-item counter of the persistent pass
    int8_t f32_variant[3][32]; // autotuned FP32 pass variant per family (all, one-sided, mutual) and log2(npad) bucket, -1 = not tuned
    int8_t f32_variant_tp[32]; // the same for test-particle mode 2 (one-sided variants only)
    int32_t test_wait_log2;    // test hook: bounded waits of the pipelined passes give up after 2^this ns (0: 2 s)
    int32_t test_hold;         // test hook: the pipelined passes' producers withhold their first stage
    float tune_ms[32][GENGA_MAX_VARIANTS];  // the autotuner's time of each variant per bucket
    int32_t forced_variant;    // >= 0: use this FP32 variant (genga_set_kernel_variant)
    int8_t f64_variant[32];    // autotuned FP64 pass variant per bucket (0 one-sided, 1.. mutual), -1 = not tuned
    float tune64_ms[32][GENGA_MAX_VARIANTS];  // the autotuner's time of each FP64 variant per bucket
    int32_t forced_f64;        // >= 0: use this FP64 variant (genga_set_fp64_variant)
    // batched mode: the tuned FP32 variant of the last GENGA_BATCH_LAYOUTS batch layouts
    unsigned long long bt_key[GENGA_BATCH_LAYOUTS];  // layout hash (offsets)
    int8_t bt_var[GENGA_BATCH_LAYOUTS];              // -1: empty
    float bt_ms[GENGA_BATCH_LAYOUTS][GENGA_MAX_VARIANTS];  // batched pass time of each one-sided variant
    int32_t bt_next;                                 // slot the next tuned layout replaces
    int32_t steps_since_order; // genga_step: drifts since the spatial order was built
    int32_t ordered_N;         // N of the system the spatial order was built for (-1: none, -2: a batch)
    unsigned long long ordered_key;  // layout hash of the batch the order was built for
    int32_t ordered_nbig;      // genga_params.n_big the order was built for (mode 2 needs big bodies last)
    // captured graph of GENGA_REORDER_STEPS steps (genga_step / genga_step_batched)
    cudaStream_t cap_stream;   // internal stream the graphs are captured on
    cudaGraphExec_t step_exec; // NULL until captured
    unsigned long long step_key;  // arrays, sizes, layout, parameters and variant it was captured for
    int32_t step_launches;     // kernels one replay launches
    int32_t step_graphs;       // 1: use step graphs (default), 0: always launch step by step
    int64_t launches;          // kernels this context has launched (measurement hook)
    // close-encounter level (encounter.cu): groups of the most recent kick's pairs
    int32_t bs_slots;          // members one drift can hold: min(npad_max, GENGA_BS_MAX_SLOTS)
    int32_t *grp;              // [npad_max] group label of each body (smallest member), -1: none
    int32_t *gmark;            // [npad_max] 1 while the body is a member
    int32_t *gslot;            // [npad_max] group number of each group's smallest member
    uint32_t *iperm;           // [npad_max] packed position of each body (written by prep)
    int32_t *gbody;            // [bs_slots] members in discovery order, then sorted per group
    int32_t *gmem;             // [bs_slots] members grouped
    int32_t *gstart, *gsize, *gcur;  // [bs_slots] per group: first slot, members, placement cursor
    int32_t *gcount;           // [1] number of groups
    int32_t *gof;              // [bs_slots] group of each member slot (intermediate levels)
    int32_t *bs_tp;            // [bs_slots] member is a test particle (mode 2)
    double *bs_work;           // [GENGA_BS_FIELDS * bs_slots] level-1 integration state
    // intermediate levels (levels.cu): groups of level 2 .. GENGA_MAX_LEVELS + 1, allocated on
    // first use (genga_params.n_levels > 0); level 1 uses the arrays above
    genga::LevelSet lv[GENGA_MAX_LEVELS];
    double *Pd;                // [3 * GENGA_MAX_DISCS] momentum of each system (batched mode)
    double *Pd_part;           // [3 * GENGA_MAX_DISCS] scratch
    size_t partial_cap;        // doubles in `partial`
    genga::MutualCache *mcache;  // plans of the mutual FP32 pass (mutual.cu), NULL until first used
};

// -------------------------------------------------------------- launchers
namespace genga {

// Batched mode: D independent systems stored one after another in the
// caller's arrays.  Both tables are built on the host for every call and
// passed to the kernels by value (kernel parameters), so a batched call needs
// no host-to-device copy.
struct BatchBodies {
    int32_t D, N_total, npad_total, pad_;
    int32_t off[GENGA_MAX_DISCS + 1];   // first body of system d in the caller's arrays; off[D] = N_total
    int32_t poff[GENGA_MAX_DISCS + 1];  // first packed position of system d (multiple of GENGA_PAD)
};

struct BatchItems {                     // work items of the FP32 pass over all systems
    int32_t items_total;
    int32_t order[GENGA_MAX_DISCS];     // system handed out at rank r (largest items first)
    int32_t item0[GENGA_MAX_DISCS + 1]; // first item of rank r
    int32_t nchunks[GENGA_MAX_DISCS];   // j-chunks per i-block of system d
    int32_t blen[GENGA_MAX_DISCS];      // tiles per chunk (the first one shorter by nchunks * blen - tiles)
    int32_t iblocks[GENGA_MAX_DISCS];   // i-blocks of system d
    int64_t pbase[GENGA_MAX_DISCS];     // first partial double of system d
};

#ifdef __CUDACC__
// Largest d in [0, D) with arr[d] <= v (arr non-decreasing, arr[0] <= v).
__device__ __forceinline__ int find_segment(const int32_t *arr, int D, int v) {
    int lo = 0, hi = D - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (arr[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
#endif

struct PassArgs {               // one long-range pass
    const float4 *hi, *lo;
    const float *hit;           // tile-blocked copy of hi
    const float4 *hid;          // duplicated-pair copy of hi (two float4 per body)
    const float4 *rel;          // group-centred copy (mutual pass): {X, Y, Z, G m} per body
    const float4 *rell;         // residuals of the group-centred copy (mutual pass)
    const float4 *gctr;         // group centres and precision distances (mutual pass)
    const double4_32a *p64;
    const float2 *scr;
    const float4 *gbox_lo, *gbox_hi;
    const int32_t *gflag;       // per 64-body group: GENGA_GROUP_BIG | GENGA_GROUP_TP
    int32_t n_big;              // test-particle mode 2 (genga_params.n_big)
    const uint32_t *perm;
    const double *a_osc, *rc_eq1, *m;
    double *partial;            // [split][3][npad]
    int2 *enc;
    int32_t *enc_count;         // [0] encounter pairs, [1] predicted entries
    int32_t enc_cap;            // capacity of enc and of pred
    int2 *pred;                 // predicted entries (written when predict)
    int32_t predict;            // 1: widen the screening, record predicted entries
    double pred_dt;             // length of the coming drift
    const double *vx, *vy, *vz; // velocities of the state (predicted entries)
    uint32_t *status;
    int32_t N, npad;
    int32_t ntiles;             // npad / tile
    int32_t split;
    double Mstar, n1;
    int32_t rcrit_mode, changeover;
    int32_t list_only;          // 1: encounter list only (no force accumulation needed)
    int32_t *work;              // [1] dynamic work-item counter (zeroed before each launch)
    // FP32: the j-chunks of every i-block in tiers (see plan_pass): tier t has
    // tier_n[t] chunks of tier_len[t] tiles, the first chunk being `excess`
    // tiles shorter; split = sum of tier_n = partial rows per body
    int32_t ntier, excess;
    // test-particle mode 2 plan (tp_b0 > 0): i-blocks 0..tp_b0-1 hold test
    // particles only and get one item over tiles tp_t0.. (those with big
    // bodies, ordered last), writing partial row 0 only; the others get the
    // tiered chunks of every tile
    int32_t tp_b0, tp_t0;
    int32_t tp_rows_end;        // packed positions below it have one partial row (tp_b0 i-blocks)
    int32_t tier_len[GENGA_MAX_TIERS], tier_n[GENGA_MAX_TIERS];
    MutualPlan mp;              // mutual FP32 pass (variants of kind mutual)
    int32_t wait_ns_log2;       // > 0: bounded waits give up after 2^this ns (test hook); 0: GENGA_WAIT_LIMIT_NS
    int32_t hold;               // test hook: the producer withholds its first stage (no copy issued)
};

struct GroupArgs {              // grouping of the encounter pairs (one CTA)
    const int2 *enc, *pred;     // encounter pairs and predicted entries
    const int32_t *enc_count;   // [0], [1]: their counts
    int32_t enc_cap, N, slots;
    int32_t *grp, *gmark, *gslot, *gbody, *gmem, *gstart, *gsize, *gcur, *gcount;
    uint32_t *status;
};

struct BSArgs {                 // level-1 integration of the groups (one warp per group)
    double *x, *y, *z, *vx, *vy, *vz;
    double *m;                  // written back only by mergers
    const uint32_t *iperm;      // packed position of each body: a_osc, rc_eq1, lo.w (test particle)
    const double *a_osc, *rc_eq1;
    const float4 *lo;
    const int32_t *gcount, *gstart, *gsize, *gmem;
    int32_t *gbody, *grp, *gmark, *tpf;  // tpf per slot: 1 test particle, 2 ghost
    double *radius;             // physical radii (NULL: no mergers)
    double *bs;                 // GENGA_BS_FIELDS fields of `slots` doubles
    int32_t slots;
    double G, Mstar, n1, dt, tol;
    int32_t rcrit_mode, changeover;
    int32_t nlev;               // intermediate levels above this one: the pair weight is prod_{k<=nlev} (1 - K_k)
    double nsub;                // their sub-step factor s (r_crit,k = r_crit / s^k)
    double snl;                 // s^nlev (exact; 1 without levels)
    uint32_t *status;
};

struct LevelArgs {              // one intermediate level (levels.cu): its groups and the next level's
    double *x, *y, *z, *vx, *vy, *vz;
    const double *m;
    const uint32_t *iperm;
    const double *a_osc, *rc_eq1;
    const float4 *lo;
    const int32_t *gcount, *gstart, *gsize, *gmem;
    int32_t *gbody;             // members sorted by body index per group (written by the sort)
    int32_t *gof;               // group of each member slot (written by the sort)
    int32_t *grp, *gmark;       // this level's marks (cleared at the end of the level)
    const int32_t *next_grp;    // the next level's labels (members with one move there)
    int2 *next_pairs;           // the next level's pair list
    int32_t *next_count;
    int32_t next_cap;
    double G, Mstar, n1;
    int32_t rcrit_mode, changeover;
    int32_t level, nlev;        // l (1 .. nlev)
    double nsub;                // s
    double sl;                  // s^l (exact)
    int32_t max_iter;
    uint32_t *status;
};

int level_launches(int n_levels, int n_sub);
cudaError_t launch_level_sort(const LevelArgs &a, int sm_count, cudaStream_t s);
cudaError_t launch_level_kick(const LevelArgs &a, double tau, bool zero_next, int sm_count, cudaStream_t s);
cudaError_t launch_level_scan(const LevelArgs &a, double h, int sm_count, cudaStream_t s);
cudaError_t launch_level_drift(const LevelArgs &a, double h, int sm_count, cudaStream_t s);
cudaError_t launch_level_clear(const LevelArgs &a, int sm_count, cudaStream_t s);

cudaError_t launch_groups(const GroupArgs &g, cudaStream_t s);
cudaError_t launch_removal(genga_system &sys, const genga_params &p, cudaStream_t s);
cudaError_t launch_compact(genga_ctx *c, genga_system &sys, int32_t *id, int32_t *count, cudaStream_t s);
cudaError_t launch_bs(const BSArgs &b, int sm_count, cudaStream_t s);
cudaError_t init_bs_kernel(int sm_count);  // the level-1 kernel's resident clusters (at context creation)
cudaError_t launch_momentum(const double *vx, const double *vy, const double *vz, const double *m,
                            int N, double *P, int32_t *zero_me, cudaStream_t s);
cudaError_t launch_prep(const genga_system &sys, const genga_params &p, genga_ctx *c, cudaStream_t s);
cudaError_t launch_order(const genga_system &sys, double Mstar, int n_big, genga_ctx *c, cudaStream_t s);
size_t order_hist_entries(int nmax);
cudaError_t init_pass_kernels();
cudaError_t launch_pass(const PassArgs &a, int precision, int variant, int grid, cudaStream_t s);
int num_fp32_variants();               // one-sided FP32 pass variants (kick.cu)
// mutual FP32 pass (mutual.cu): variants numbered after the one-sided ones
int num_mutual_variants();
void fp32_variant_shape(int variant, int *cw, int *bpt, int *ctas_per_sm);
void mutual_variant_shape(int v, int *cw, int *bpt);
bool mutual_plan(genga_ctx *c, int N, int v, cudaStream_t s, MutualPlan *P);
// the plan of FP32 mutual variant v over the systems of a batch (layout hash key)
bool mutual_plan_batched(genga_ctx *c, const BatchBodies &bb, unsigned long long key, int v, cudaStream_t s,
                         MutualPlan *P);
// FP64 mutual pass (mutual.cu): FP64 pass variants 1 .. (variant 0 is the one-sided FP64 pass)
int num_mutual64_variants();
void fp64_pass_shape(int *warps, int *bpt);  // the one-sided FP64 pass (kick.cu)
void mutual64_variant_shape(int v, int *cw, int *bpt);
bool mutual64_plan(genga_ctx *c, int N, int v, cudaStream_t s, MutualPlan *P);
cudaError_t launch_pass_mutual64(const PassArgs &a, int v, int sm_count, cudaStream_t s);
cudaError_t launch_combine_mutual64(const double *partial, const MutualPlan &P, int N, int npad, const uint32_t *perm,
                                    double tau, double *acc, double *vx, double *vy, double *vz, uint32_t *status,
                                    cudaStream_t s);
void free_mutual_cache(genga_ctx *c);
cudaError_t init_mutual_kernels();
cudaError_t launch_pass_mutual(const PassArgs &a, int v, int sm_count, cudaStream_t s);
cudaError_t launch_combine_mutual(const double *partial, const MutualPlan &P, int N, int npad, const uint32_t *perm,
                                  double tau, double *acc, double *vx, double *vy, double *vz, uint32_t *status,
                                  cudaStream_t s);
void plan_pass(int N, int precision, int variant, int sm_count, size_t partial_cap, PassArgs *a, int *grid);
cudaError_t launch_combine(const double *partial, int split, int one_row_end, int N, int npad, int fp64_rows,
                           const uint32_t *perm,
                           double tau, double *acc, double *vx, double *vy, double *vz, uint32_t *status,
                           cudaStream_t s);
cudaError_t launch_sort_pairs(int2 *enc, int32_t cap, const int32_t *count, cudaStream_t s);
cudaError_t launch_copy_pairs(const int2 *enc, const int32_t *count, int32_t enc_cap, int32_t *pairs,
                              int32_t capacity, int32_t *count_out, uint32_t *status, cudaStream_t s);
cudaError_t launch_drift(genga_system &sys, const genga_params &p, double dt, genga_ctx *c, cudaStream_t s);
cudaError_t launch_energy(const genga_system &sys, const genga_params &p, genga_ctx *c, cudaStream_t s);
// batched mode (batch.cu helpers live next to their single-system versions)
cudaError_t launch_momentum_batched(const genga_system &all, const BatchBodies &bb, double *Pd, int32_t *zero_me,
                                    cudaStream_t s);
cudaError_t launch_order_batched(const genga_system &all, const BatchBodies &bb, double Mstar, int n_big,
                                 genga_ctx *c, cudaStream_t s);
cudaError_t launch_prep_batched(const genga_system &all, const BatchBodies &bb, const genga_params &p, genga_ctx *c,
                                cudaStream_t s);
cudaError_t launch_pass_batched(const PassArgs &a, const BatchBodies &bb, const BatchItems &bi, int variant, int grid,
                                cudaStream_t s);
cudaError_t launch_combine_batched(const BatchBodies &bb, const BatchItems &bi, const double *partial,
                                   const uint32_t *perm, double tau, double *acc, double *vx, double *vy, double *vz,
                                   uint32_t *status, cudaStream_t s);
cudaError_t launch_drift_batched(genga_system &all, const BatchBodies &bb, const genga_params &p, double dt,
                                 genga_ctx *c, cudaStream_t s);
int fp32_variant_ib(int variant);       // i-bodies per work item of an FP32 variant
int fp32_variant_minb(int variant);     // resident CTAs per SM of an FP32 variant
void profile_before_pass(genga_ctx *c, cudaStream_t s);
void profile_after_pass(genga_ctx *c, cudaStream_t s);
void profile_free(genga_ctx *c);

}  // namespace genga

// ------------------------------------------------------------ PTX wrappers
#ifdef __CUDACC__
namespace genga {

// 1/sqrt(x) in FP64: the approximate FP64 reciprocal square root of the SFU
// as seed y0 (relative error ~1e-7), then the third-order correction
// y = y0 (1 + e/2 + 3e^2/8), e = 1 - x y0^2, from the binomial series of
// (1 - e)^(-1/2); the truncation error is O(e^3) ~ 1e-21.
__device__ __forceinline__ double rsqrt_fp64(double x) {
    double y0;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y0) : "d"(x));
    const double t = x * y0;
    const double e = fma(-t, y0, 1.0);
    const double p = fma(e, 0.375, 0.5);
    return fma(y0 * e, p, y0);
}

// x^(-3/2) in FP64 (the inverse cube of r from r^2): the SFU seed
// y0 ~ x^(-1/2) as above, e = 1 - x y0^2, then x^(-3/2) = y0^3 (1 - e)^(-3/2)
// ~ y0^3 (1 + 3e/2 + 15e^2/8) from the binomial series; truncation error
// O(e^3).  Six FP64 operations where 1/sqrt and two products take seven.
__device__ __forceinline__ double rsqrt3_fp64(double x) {
    double y0;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y0) : "d"(x));
    const double y2 = y0 * y0;
    const double y3 = y2 * y0;
    const double e = fma(-x, y2, 1.0);
    const double p = fma(e, 1.875, 1.5);
    return fma(y3 * e, p, y3);
}

// 1/x in FP64 (x normal): the approximate FP64 reciprocal of the SFU as seed
// y0, then the third-order correction y = y0 (1 + e + e^2), e = 1 - x y0,
// from the geometric series of 1 / (1 - e); truncation error O(e^3).
__device__ __forceinline__ double rcp_fp64(double x) {
    double y0;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y0) : "d"(x));
    const double e = fma(-x, y0, 1.0);
    return fma(y0, fma(e, e, e), y0);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// One-dimensional bulk copy global -> shared, completion signalled on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of `bar`, at most `limit_ns` (GENGA_WAIT_LIMIT_NS
// by default).  Returns false (and sets the TIMEOUT bit) when the limit is
// reached.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t *status,
                                                  uint64_t limit_ns = GENGA_WAIT_LIMIT_NS) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_timer_ns() - t0 > limit_ns) {
            atomicOr(status, GENGA_BIT(GENGA_ERR_TIMEOUT));
            return false;
        }
    }
    return true;
}

// The wait limit of a pass: GENGA_WAIT_LIMIT_NS, or 2^wait_ns_log2 ns when the
// test hook of genga_measure.h has set a short one.
__device__ __forceinline__ uint64_t pass_wait_limit(int wait_ns_log2) {
    return wait_ns_log2 > 0 ? (1ull << wait_ns_log2) : GENGA_WAIT_LIMIT_NS;
}

}  // namespace genga
#endif
