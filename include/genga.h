/*
 * genga.h -- C ABI of libgenga: the long-range kick path of the GENGA hybrid
 * symplectic step, on one NVIDIA GB300 (sm_103a).
 *
 * Paper: R. Brasser, S. L. Grimm, P. Hatalova, J. G. Stadel (2023),
 * "Speeding up the GENGA N-body integrator on consumer-grade graphics
 * cards", A&A.  The paper's subject is computing the mutual long-range
 * forces of the N bodies in single precision while the Kepler drift and
 * close-encounter forces stay in double precision (Sect. 1); this library
 * exposes exactly that path.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Coordinates are democratic-heliocentric: heliocentric positions (au),
 *   barycentric velocities (au/day), masses in solar masses.  The central
 *   body is not an array element; it enters through genga_params.Mstar.
 * - All per-body arrays are caller-owned DEVICE memory on the context's
 *   device, float64, structure-of-arrays, length N, 8-byte aligned.  The
 *   library never frees or reallocates them.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Every call is asynchronous on that stream except where
 *   stated; argument errors are detected on the host and returned at once,
 *   before anything is enqueued.
 * - Errors found on the device (Kepler solver did not converge, encounter
 *   list overflow, non-finite accelerations, a bounded wait that gave up, a
 *   forced close-encounter sub-step) are sticky bits in the context, read
 *   and cleared by genga_get_status.
 * - No entry point aborts, traps, prints or allocates device memory, except
 *   genga_create/genga_destroy (workspace).
 * - The first FP32 pass a context runs for a new size bucket (a power of two
 *   of the padded N) times the FP32 kernel variants and keeps the fastest;
 *   that call synchronises its stream (genga_measure.h can pin a variant).
 * - Results are bitwise reproducible for the same sequence of calls on a
 *   context: no floating-point atomics, every reduction has a fixed order.
 * - A context is not re-entrant: one host thread and one stream at a time.
 */
#ifndef GENGA_H
#define GENGA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GENGA_OK = 0,
    GENGA_ERR_INVALID_ARG = 1, /* bad pointer, size or parameter (host check) */
    GENGA_ERR_CUDA = 2,        /* a CUDA runtime call failed */
    GENGA_ERR_CAPACITY = 3,    /* encounter list overflow: list truncated, count is the true total */
    GENGA_ERR_KEPLER = 4,      /* the f/g solver hit kepler_max_iter for at least one body */
    GENGA_ERR_NONFINITE = 5,   /* a NaN or Inf acceleration was produced */
    GENGA_ERR_TIMEOUT = 6,     /* a bounded device wait gave up (the kernel returned early) */
    GENGA_ERR_BS = 7           /* close-encounter level: a group's Bulirsch-Stoer integration
                                  needed a forced sub-step, or the groups did not fit the
                                  workspace (those bodies then got the Kepler drift) */
} genga_status;

/* Precision of the long-range kick (Sect. 1; "Do Kick in single precision", Sect. 4).
 *   GENGA_FP64           every pair term in FP64.
 *   GENGA_FP32_HILO      FP32 pair terms from the hi/lo split x = x_hi + x_lo of the FP64
 *                        positions (x_hi = fl32(x)); where every pair of a 32-body warp
 *                        tile and a 64-body group is farther apart than 0.025 max|x| the
 *                        lo parts are dropped (offset error <= ~5e-6 relative).  The
 *                        one-sided pass: each ordered pair from its i-body's side.
 *   GENGA_FP32_BLOCKREL  FP32 pair terms from block-relative offsets: X = fl32(x - c), the
 *                        FP64 difference rounded, c the centre of the j-body's 64-body
 *                        group; closer than a tenth of the group's half-diagonal (or the
 *                        r_crit bound) the rounding residuals x - c - X are added back.
 *                        The mutual pass: each unordered pair once, its terms added to
 *                        both bodies.  Not with test-particle mode 2 (n_big >= 0):
 *                        GENGA_ERR_INVALID_ARG.
 *   GENGA_FP32           either FP32 form, whichever the autotuner finds faster for the
 *                        size bucket (genga_measure.h).
 * In every FP32 mode: r^2, rsqrt (SFU) and the pair terms in FP32, per-body sums in
 * double-float (about 48 bits), close-encounter pairs exactly in FP64 with K. */
enum { GENGA_FP64 = 0, GENGA_FP32_HILO = 1, GENGA_FP32_BLOCKREL = 2, GENGA_FP32 = 3 };

/* Pair critical radius r_crit,ij (Eq. 1 gives the per-body radius):
 *   GENGA_RCRIT_EQ1         max(r_crit,i, r_crit,j), r_crit,i = max(n1 R_H,i, n2 dt v_i)
 *   GENGA_RCRIT_MUTUAL_HILL n1 ((m_i + m_j) / 3 M*)^(1/3) (a_i + a_j) / 2            */
enum { GENGA_RCRIT_EQ1 = 0, GENGA_RCRIT_MUTUAL_HILL = 1 };

/* Changeover weight K(y), y = (r_ij / r_crit,ij - 0.1) / 0.9, K = 0 for y <= 0 and
 * 1 for y >= 1 (the smooth switch of the hybrid integrator, Sect. 1):
 *   GENGA_K_CHAMBERS  y^2 / (2y^2 - 2y + 1)        GENGA_K_QUINTIC  10y^3 - 15y^4 + 6y^5 */
enum { GENGA_K_CHAMBERS = 0, GENGA_K_QUINTIC = 1 };

typedef struct {
    double G;                /* gravitational constant (au^3 Msun^-1 day^-2 for Gaussian units) */
    double Mstar;            /* central mass, > 0 */
    double dt;               /* step length (enters Eq. 1's velocity term and genga_step) */
    double n1, n2;           /* Eq. 1 constants; the paper's typical values are 3 and 0.4 */
    int32_t rcrit_mode;      /* GENGA_RCRIT_* */
    int32_t changeover;      /* GENGA_K_* */
    int32_t precision;       /* GENGA_FP64, GENGA_FP32_HILO, GENGA_FP32_BLOCKREL or GENGA_FP32 */
    int32_t kepler_max_iter; /* iteration cap of the f/g solver, >= 1 (50 is ample) */
    int32_t n_big;           /* test-particle mode 2 (the giant-planet runs of Sect. 3): with
                                n_big >= 0, bodies n_big..N-1 (of each system in batched mode)
                                are test particles that feel bodies 0..n_big-1 but not each
                                other, while those feel everything -- a pair of two test
                                particles has no force, no encounter and no potential energy;
                                -1: every pair interacts */
    double bs_tol;           /* close-encounter level (level 1 of the hybrid integrator, Sect. 1):
                                > 0: genga_drift / genga_step integrate every group of
                                encounter pairs of the preceding kick with a Bulirsch-Stoer
                                method at this relative tolerance (1e-12 is typical, >= 1e-14:
                                smaller tolerances sit at the rounding of FP64 heliocentric
                                coordinates and cannot be met); 0: off, every body gets the
                                Kepler drift */
    double r_in, r_out;      /* removal radii (Sect. 2): after every drift a body closer than
                                r_in to, or farther than r_out from, the central body is removed
                                (see "ghosts" below); <= 0 switches each test off */
    int32_t n_levels;        /* intermediate levels of the changeover (Sect. 1), 0 .. GENGA_MAX_LEVELS,
                                with bs_tol > 0: level l (1 <= l <= n_levels) moves its groups in
                                n_sub kick-drift-kick sub-steps of dt / n_sub^l with the pair radius
                                r_crit,l = r_crit,ij / n_sub^l; the pair force splits into
                                W_l = K_l prod_{k<l} (1 - K_k) for the kicks of levels 0 .. n_levels
                                and prod_{k<=n_levels} (1 - K_k) for the Bulirsch-Stoer level, with
                                K_l(r) = K((r / r_crit,l - 0.1) / 0.9).  A level-l sub-step forms
                                subgroups from the member pairs inside r_crit,l (and those whose
                                straight-line motion enters it within the sub-step, from within
                                1.5 r_crit,l), drifts the other members on Kepler orbits and moves
                                each subgroup on level l + 1 (Bulirsch-Stoer below the last).
                                0: the groups go to the Bulirsch-Stoer level directly */
    int32_t n_sub;           /* sub-steps per level, 2 .. 16 (ignored when n_levels = 0) */
} genga_params;

#define GENGA_MAX_LEVELS 3

typedef struct {
    int32_t N;                           /* number of non-central bodies, 0 <= N <= max_N */
    double *x, *y, *z;                   /* heliocentric positions, device [N] */
    double *vx, *vy, *vz;                /* barycentric velocities, device [N] */
    double *m;                           /* masses, device [N], >= 0 */
    double *radius;                      /* physical radii (au), device [N], optional: with bs_tol > 0
                                            overlapping members of a close-encounter group merge
                                            (perfect mergers, Sect. 2); NULL: no collisions */
} genga_system;

/*
 * Ghosts.  A body that merged into another one or crossed a removal radius
 * stays in the arrays as a ghost until genga_compact: its mass is set to
 * -0.0 (numerically zero; the sign bit is the mark) and its radius to 0, it
 * exerts no force, is never an encounter pair and never merges again; it
 * still moves (massless).  A caller may also mark bodies this way.
 */

typedef struct genga_ctx genga_ctx;

/* Create a context on `device` with workspace for systems of up to max_N bodies
 * (about 270 bytes per body, plus 1.9 KB per body for the first 262,144 bodies:
 * the close-encounter workspace, plus the encounter buffer).  *ctx is NULL on error. */
genga_status genga_create(genga_ctx **ctx, int32_t max_N, int32_t device);

/* Free the context's workspace (synchronises its device first). NULL is a no-op. */
void genga_destroy(genga_ctx *ctx);

/*
 * Long-range kick (Sect. 1):  a_i = sum_{j != i} G m_j K(y_ij) (x_j - x_i) / r_ij^3,
 * with r_crit evaluated from the current state, then v_i += a_i * tau.
 *   tau   kick length (tau = 0: accelerations only, velocities untouched)
 *   acc   optional device [3*N] float64 output, layout acc[c*N + i] (c = x, y, z);
 *         NULL to skip.
 * params->precision selects the FP64 kick or the FP32 kick (FP32 pair offsets
 * and inverse cubes from FP64 positions, FP64 per-body accumulation); pairs
 * inside r_crit are always evaluated in FP64 with K (Sect. 1, last paragraph).
 * The encounter list of this state is rebuilt as a by-product (see
 * genga_last_encounters).
 */
genga_status genga_kick(genga_ctx *ctx, const genga_system *sys, const genga_params *params,
                        double tau, double *acc, void *stream);

/*
 * Drift of the step: central-body momentum drift x_i += (dt/2) P / M*
 * (P = sum_j m_j v_j), then the Kepler drift of every body about mu = G M* for
 * dt (always FP64, universal-variable f and g functions, Sect. 1), then the
 * momentum drift again with the updated P.  Bodies whose solver hits
 * kepler_max_iter set GENGA_ERR_KEPLER (they are still advanced).
 *
 * With params->bs_tol > 0 the close-encounter level replaces the Kepler drift
 * for the members of every group: the connected components of the encounter
 * pairs of the most recent kick on this context (genga_kick, genga_step,
 * genga_encounters) and of the pairs that kick (when it ran with bs_tol > 0)
 * predicted to come inside r_crit within dt: outside r_crit,ij but within
 * 1.5 r_crit,ij, entering it along their straight-line relative motion.  Each group is integrated over dt in FP64 by a
 * Bulirsch-Stoer method (modified midpoint rule with 2, 4, ..., 16 steps,
 * polynomial extrapolation, relative tolerance bs_tol on each member's |x|
 * and |v|) under the central body and the (1 - K) part of the members' pair
 * forces, with r_crit,ij of that kick, so the kick and this level together
 * apply the whole pair force.  Pair lists of another system are ignored
 * where their indices exceed N.
 */
genga_status genga_drift(genga_ctx *ctx, genga_system *sys, const genga_params *params,
                         double dt, void *stream);

/*
 * Close-encounter pairs of the current state: all (i, j), i < j, with
 * r_ij < r_crit,ij (the changeover region of Sect. 1), sorted by (i, j).
 *   pairs     device int32 [2*capacity]: pairs[2k] = i, pairs[2k+1] = j
 *   capacity  number of pairs `pairs` holds, >= 0
 *   count     device int32 [1]: the true number of pairs, even when it
 *             exceeds capacity (then only `capacity` of them are written and
 *             GENGA_ERR_CAPACITY is raised)
 * Cost: one long-range pass in FP32 screening precision (the decision itself
 * is taken in FP64).
 */
genga_status genga_encounters(genga_ctx *ctx, const genga_system *sys, const genga_params *params,
                              int32_t *pairs, int32_t capacity, int32_t *count, void *stream);

/* Copy the encounter list built by the most recent kick (same format as
 * genga_encounters) without another pass over the pairs. */
genga_status genga_last_encounters(genga_ctx *ctx, int32_t *pairs, int32_t capacity,
                                   int32_t *count, void *stream);

/*
 * nsteps steps of the hybrid symplectic integrator (Sect. 1): kick(dt/2),
 * drift(dt), kick(dt/2).  With params->bs_tol > 0 the drift integrates the
 * groups of encounter pairs of the step's first kick on the close-encounter
 * level (see genga_drift); with bs_tol = 0 every body gets the Kepler drift
 * and pairs inside r_crit keep only their K-weighted force (exact for
 * systems without encounters).  The encounter list of the last kick stays
 * readable through genga_last_encounters (the closing kick of a step lists
 * the encounter pairs only; each step's first kick also predicts the entries
 * its drift integrates, see genga_drift).  The spatial order of the bodies
 * (a performance device of the FP32 pass) is rebuilt every few steps,
 * counted across calls on the context.
 */
genga_status genga_step(genga_ctx *ctx, genga_system *sys, const genga_params *params,
                        int32_t nsteps, void *stream);

/*
 * Batched mode: D independent systems, each a central mass with its own bodies,
 * stored one after another in `all` (system d = bodies offsets[d] ..
 * offsets[d+1]-1 of the seven arrays) and sharing `params`.  Ensembles of
 * independent runs are how the paper's experiments are made (Sect. 2); here
 * they share one launch per kernel.
 *   offsets  HOST int32 [D+1], offsets[0] = 0, non-decreasing, offsets[D] = all->N
 *   D        1 .. GENGA_MAX_BATCH (256)
 * The context's max_N must cover the padded total sum_d roundup(N_d, 1024).
 * params->precision must be one of the FP32 modes (the batched pass is the FP32
 * kick: one-sided for GENGA_FP32_HILO, mutual over each system's pairs for
 * GENGA_FP32_BLOCKREL, the faster of the two -- tuned per batch layout -- for
 * GENGA_FP32).
 * genga_kick_batched: the kick of every system (acc layout acc[c*all->N + i],
 * or NULL), the encounter list of every system with indices into `all`.
 * genga_step_batched: nsteps level-0 steps of every system.
 */
#define GENGA_MAX_BATCH 256
genga_status genga_kick_batched(genga_ctx *ctx, const genga_system *all, const int32_t *offsets, int32_t D,
                                const genga_params *params, double tau, double *acc, void *stream);
genga_status genga_step_batched(genga_ctx *ctx, genga_system *all, const int32_t *offsets, int32_t D,
                                const genga_params *params, int32_t nsteps, void *stream);

/*
 * Energy and angular momentum (Sect. 3.1 diagnostics), FP64, synchronous:
 *   E_L[0] = sum m v^2/2 + |P|^2/(2 M*) - sum G M* m_i / r_i - sum_{i<j} G m_i m_j / r_ij
 *   E_L[1..3] = L = sum m_i x_i cross v_i
 * E_L is HOST memory [4].  The call synchronises `stream`.
 */
genga_status genga_energy(genga_ctx *ctx, const genga_system *sys, const genga_params *params,
                          double *E_L, void *stream);

/*
 * Remove the ghosts (bodies of mass -0.0: merged away or removed by the
 * radii) from the arrays of `sys`: the other bodies keep their order and
 * move to the front of x..m and radius, and of `id` (optional device int32
 * [N] of body labels, moved along; NULL to skip).  Device-side stable
 * compaction; synchronises `stream` and sets sys->N to the new count.  The
 * spatial order and the encounter list are rebuilt by the next kick.
 */
genga_status genga_compact(genga_ctx *ctx, genga_system *sys, int32_t *id, void *stream);

/*
 * Self-tuning of the intermediate levels (Sect. 1: the best number of levels
 * and sub-steps depends on the number of bodies, their surface density and
 * the GPU, so configurations are timed before a run and the fastest is
 * kept).  Each candidate k, params with n_levels = n_levels[k] and n_sub =
 * n_sub[k] (HOST int32 [ncand], each valid for genga_step), runs
 * `trial_steps` steps (>= 1, after one untimed step) from a device copy of
 * the current state of `sys`, timed with events on `stream`; the caller's
 * state is not changed.
 *   best   HOST int32 [1]: index of the fastest candidate whose trial raised
 *          no status (a forced Bulirsch-Stoer acceptance, say, when a dense
 *          group exhausts the level's sub-step or time limits); if every
 *          trial raised one, the fastest of all, and its status bits stay set
 *   ms     HOST float [ncand] or NULL: each candidate's time per step (ms)
 *   codes  HOST int32 [ncand] or NULL: each candidate's status (lowest code)
 * Synchronous.  The context's status bits from before the call are kept; the
 * trials leave the step graph and the spatial order as a genga_step on the
 * copy would.  ncand = 1 .. 64.
 */
genga_status genga_tune_levels(genga_ctx *ctx, const genga_system *sys, const genga_params *params,
                               const int32_t *n_levels, const int32_t *n_sub, int32_t ncand,
                               int32_t trial_steps, int32_t *best, float *ms, int32_t *codes, void *stream);

/* Synchronise `stream`, return the sticky device status (lowest set code) and
 * clear it.  Also returns GENGA_ERR_CUDA if the stream reports an error. */
genga_status genga_get_status(genga_ctx *ctx, void *stream);

/* Static description of a status code. */
const char *genga_status_string(genga_status s);

#ifdef __cplusplus
}
#endif

#endif /* GENGA_H */
