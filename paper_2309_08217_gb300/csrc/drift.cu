// drift.cu -- the drift of the hybrid step, always in FP64 (Sect. 1):
//
//   x_i += (dt/2) P / M*               central-body momentum drift, P = sum m v
//   (x_i, v_i) <- Kepler(mu = G M*, dt) two-body drift of every body outside
//                                      the close-encounter groups (those move
//                                      on level 1, encounter.cu, when enabled)
//   x_i += (dt/2) P' / M*              with the momentum after the drift
//
// The Kepler drift (universal variables, Laguerre-Conway) is in kepler.cuh.
#include "kepler.cuh"

namespace genga {

namespace {

// x += (h / M*) P, then the Kepler drift over dt, except for members of a
// close-encounter group (grp[i] >= 0; grp may be NULL), which the
// close-encounter level moves instead.
__global__ void drift_kernel(double *__restrict__ x, double *__restrict__ y, double *__restrict__ z,
                             double *__restrict__ vx, double *__restrict__ vy, double *__restrict__ vz, int N,
                             const double *__restrict__ P, double hM, double mu, double dt,
                             int max_iter, uint32_t *__restrict__ status, const int32_t *__restrict__ grp) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double xi = fma(hM, P[0], x[i]);
    double yi = fma(hM, P[1], y[i]);
    double zi = fma(hM, P[2], z[i]);
    if (grp && grp[i] >= 0) {
        x[i] = xi; y[i] = yi; z[i] = zi;
        return;
    }
    double ui = vx[i], vi = vy[i], wi = vz[i];
    if (!kepler_drift(mu, dt, max_iter, xi, yi, zi, ui, vi, wi)) atomicOr(status, GENGA_BIT(GENGA_ERR_KEPLER));
    x[i] = xi; y[i] = yi; z[i] = zi;
    vx[i] = ui; vy[i] = vi; vz[i] = wi;
}

// Removal radii (Sect. 2): a live body with |x|^2 < r_in^2 or |x|^2 > r_out^2
// (a test off when its radius is <= 0) becomes a ghost: m = -0.0, R = 0.
__global__ void removal_kernel(const double *__restrict__ x, const double *__restrict__ y,
                               const double *__restrict__ z, double *__restrict__ m, double *__restrict__ radius,
                               int N, double rin2, double rout2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N || signbit(m[i])) return;
    const double r2 = x[i] * x[i] + y[i] * y[i] + z[i] * z[i];
    if ((rin2 > 0.0 && r2 < rin2) || (rout2 > 0.0 && r2 > rout2)) {
        m[i] = -0.0;
        if (radius) radius[i] = 0.0;
    }
}

__global__ void hc_kernel(double *__restrict__ x, double *__restrict__ y, double *__restrict__ z, int N,
                          const double *__restrict__ P, double hM) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    x[i] = fma(hM, P[0], x[i]);
    y[i] = fma(hM, P[1], y[i]);
    z[i] = fma(hM, P[2], z[i]);
}

// Batched: body i of system d (segment of i in off) drifts with P of its system.
__global__ void drift_batched_kernel(double *__restrict__ x, double *__restrict__ y, double *__restrict__ z,
                                     double *__restrict__ vx, double *__restrict__ vy, double *__restrict__ vz,
                                     const double *__restrict__ Pd, double hM, double mu, double dt,
                                     int max_iter, uint32_t *__restrict__ status,
                                     const int32_t *__restrict__ grp, const __grid_constant__ BatchBodies bb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= bb.N_total) return;
    const double *P = Pd + 3 * find_segment(bb.off, bb.D, i);
    double xi = fma(hM, P[0], x[i]);
    double yi = fma(hM, P[1], y[i]);
    double zi = fma(hM, P[2], z[i]);
    if (grp && grp[i] >= 0) {
        x[i] = xi; y[i] = yi; z[i] = zi;
        return;
    }
    double ui = vx[i], vi = vy[i], wi = vz[i];
    if (!kepler_drift(mu, dt, max_iter, xi, yi, zi, ui, vi, wi)) atomicOr(status, GENGA_BIT(GENGA_ERR_KEPLER));
    x[i] = xi; y[i] = yi; z[i] = zi;
    vx[i] = ui; vy[i] = vi; vz[i] = wi;
}

__global__ void hc_batched_kernel(double *__restrict__ x, double *__restrict__ y, double *__restrict__ z,
                                  const double *__restrict__ Pd, double hM,
                                  const __grid_constant__ BatchBodies bb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= bb.N_total) return;
    const double *P = Pd + 3 * find_segment(bb.off, bb.D, i);
    x[i] = fma(hM, P[0], x[i]);
    y[i] = fma(hM, P[1], y[i]);
    z[i] = fma(hM, P[2], z[i]);
}

}  // namespace

// The close-encounter level around the Kepler drift: groups before it (so
// that it skips their members), the level-1 integration after it.  N bodies
// of the caller's arrays `sys` (all systems of a batch).
namespace {

// Level 1's groups live in the context's arrays, formed from the step's
// encounter pairs and predicted entries.
LevelSet base_set(genga_ctx *c) {
    LevelSet l;
    l.grp = c->grp;
    l.gmark = c->gmark;
    l.gslot = c->gslot;
    l.gbody = c->gbody;
    l.gmem = c->gmem;
    l.gstart = c->gstart;
    l.gsize = c->gsize;
    l.gcur = c->gcur;
    l.gcount = c->gcount;
    l.gof = c->gof;
    l.pairs = c->enc;
    l.pair_count = c->enc_count;
    l.pair_cap = c->enc_cap;
    return l;
}

GroupArgs group_args(const genga_system &sys, genga_ctx *c, const LevelSet &l, const int2 *pred) {
    GroupArgs g;
    g.enc = l.pairs;
    g.pred = pred;
    g.enc_count = l.pair_count;
    g.enc_cap = l.pair_cap;
    g.N = sys.N;
    g.slots = c->bs_slots;
    g.grp = l.grp;
    g.gmark = l.gmark;
    g.gslot = l.gslot;
    g.gbody = l.gbody;
    g.gmem = l.gmem;
    g.gstart = l.gstart;
    g.gsize = l.gsize;
    g.gcur = l.gcur;
    g.gcount = l.gcount;
    g.status = c->status;
    return g;
}

// The Bulirsch-Stoer integration of the groups of `l` over dt, below nlev
// intermediate levels.
BSArgs bs_args(genga_system &sys, const genga_params &p, double dt, genga_ctx *c, const LevelSet &l, int nlev) {
    BSArgs b;
    b.x = sys.x; b.y = sys.y; b.z = sys.z;
    b.vx = sys.vx; b.vy = sys.vy; b.vz = sys.vz;
    b.m = sys.m;
    b.iperm = c->iperm;
    b.a_osc = c->a_osc;
    b.rc_eq1 = c->rc_eq1;
    b.lo = c->pk_lo;
    b.gcount = l.gcount;
    b.gstart = l.gstart;
    b.gsize = l.gsize;
    b.gmem = l.gmem;
    b.gbody = l.gbody;
    b.grp = l.grp;
    b.gmark = l.gmark;
    b.tpf = c->bs_tp;
    b.radius = sys.radius;
    b.bs = c->bs_work;
    b.slots = c->bs_slots;
    b.G = p.G;
    b.Mstar = p.Mstar;
    b.n1 = p.n1;
    b.dt = dt;
    b.tol = p.bs_tol;
    b.rcrit_mode = p.rcrit_mode;
    b.changeover = p.changeover;
    b.nlev = nlev;
    b.nsub = nlev > 0 ? (double)p.n_sub : 1.0;
    b.snl = 1.0;
    for (int k = 0; k < nlev; k++) b.snl *= b.nsub;
    b.status = c->status;
    return b;
}

LevelArgs level_args(genga_system &sys, const genga_params &p, genga_ctx *c, const LevelSet &l, const LevelSet &next,
                     int level) {
    LevelArgs a;
    a.x = sys.x; a.y = sys.y; a.z = sys.z;
    a.vx = sys.vx; a.vy = sys.vy; a.vz = sys.vz;
    a.m = sys.m;
    a.iperm = c->iperm;
    a.a_osc = c->a_osc;
    a.rc_eq1 = c->rc_eq1;
    a.lo = c->pk_lo;
    a.gcount = l.gcount;
    a.gstart = l.gstart;
    a.gsize = l.gsize;
    a.gmem = l.gmem;
    a.gbody = l.gbody;
    a.gof = l.gof;
    a.grp = l.grp;
    a.gmark = l.gmark;
    a.next_grp = next.grp;
    a.next_pairs = next.pairs;
    a.next_count = next.pair_count;
    a.next_cap = next.pair_cap;
    a.G = p.G;
    a.Mstar = p.Mstar;
    a.n1 = p.n1;
    a.rcrit_mode = p.rcrit_mode;
    a.changeover = p.changeover;
    a.level = level;
    a.nlev = p.n_levels;
    a.nsub = (double)p.n_sub;
    a.sl = 1.0;
    for (int k = 0; k < level; k++) a.sl *= a.nsub;
    a.max_iter = p.kepler_max_iter;
    a.status = c->status;
    return a;
}

// Level `level` (1 .. n_levels) moves its groups over T in n_sub sub-steps
// (see levels.cu); the next level's groups are formed in every sub-step.
cudaError_t run_level(genga_system &sys, const genga_params &p, genga_ctx *c, int level, double T, cudaStream_t s) {
    const LevelSet l = level == 1 ? base_set(c) : c->lv[level - 2];
    const LevelSet &next = c->lv[level - 1];
    const LevelArgs a = level_args(sys, p, c, l, next, level);
    const double h = T / p.n_sub;
    cudaError_t e = launch_level_sort(a, c->sm_count, s);
    for (int k = 0; k < p.n_sub && e == cudaSuccess; k++) {
        // the closing half kick of sub-step k - 1 and the opening one of
        // sub-step k act at the same positions with the same weights: one
        // kick of h (h / 2 for the first), which also empties the next
        // level's pair list for this sub-step's scan
        e = launch_level_kick(a, k == 0 ? 0.5 * h : h, true, c->sm_count, s);
        if (e == cudaSuccess) e = launch_level_scan(a, h, c->sm_count, s);
        if (e == cudaSuccess) e = launch_groups(group_args(sys, c, next, next.pairs), s);
        if (e == cudaSuccess) e = launch_level_drift(a, h, c->sm_count, s);
        if (e == cudaSuccess)
            e = level < p.n_levels ? run_level(sys, p, c, level + 1, h, s)
                                   : launch_bs(bs_args(sys, p, h, c, next, p.n_levels), c->sm_count, s);
    }
    if (e == cudaSuccess) e = launch_level_kick(a, 0.5 * h, false, c->sm_count, s);  // the last closing half kick
    if (e == cudaSuccess) e = launch_level_clear(a, c->sm_count, s);
    return e;
}

}  // namespace

cudaError_t launch_level1_groups(const genga_system &sys, genga_ctx *c, cudaStream_t s) {
    return launch_groups(group_args(sys, c, base_set(c), c->pred), s);
}

cudaError_t launch_level1(genga_system &sys, const genga_params &p, double dt, genga_ctx *c, cudaStream_t s) {
    if (p.n_levels > 0) return run_level(sys, p, c, 1, dt, s);
    return launch_bs(bs_args(sys, p, dt, c, base_set(c), 0), c->sm_count, s);
}

// Kernels one drift launches for the close-encounter levels beyond the
// grouping kernel: the Bulirsch-Stoer kernel, or with L levels of s
// sub-steps, per level-l sub-step kick, scan, groups, drift, the level below
// and kick, and one sort and one clear per level.
int level_launches(int n_levels, int n_sub) {
    int below = 1;  // the Bulirsch-Stoer kernel
    // per sub-step kick, scan, groups, drift and the level below; sort, the
    // last closing kick and clear once per level
    for (int l = n_levels; l >= 1; l--) below = n_sub * (4 + below) + 3;
    return below;
}

cudaError_t launch_removal(genga_system &sys, const genga_params &p, cudaStream_t s) {
    if (sys.N <= 0 || (p.r_in <= 0.0 && p.r_out <= 0.0)) return cudaSuccess;
    const double rin2 = p.r_in > 0.0 ? p.r_in * p.r_in : 0.0, rout2 = p.r_out > 0.0 ? p.r_out * p.r_out : 0.0;
    removal_kernel<<<(sys.N + 255) / 256, 256, 0, s>>>(sys.x, sys.y, sys.z, sys.m, sys.radius, sys.N, rin2, rout2);
    return cudaGetLastError();
}

cudaError_t launch_drift_batched(genga_system &all, const BatchBodies &bb, const genga_params &p, double dt,
                                 genga_ctx *c, cudaStream_t s) {
    const int N = bb.N_total;
    if (N <= 0) return cudaSuccess;
    const bool level1 = p.bs_tol > 0.0;
    cudaError_t e = launch_momentum_batched(all, bb, c->Pd, nullptr, s);
    if (e == cudaSuccess && level1) e = launch_level1_groups(all, c, s);
    if (e != cudaSuccess) return e;
    drift_batched_kernel<<<(N + 127) / 128, 128, 0, s>>>(all.x, all.y, all.z, all.vx, all.vy, all.vz, c->Pd,
                                                         0.5 * dt / p.Mstar, p.G * p.Mstar, dt, p.kepler_max_iter, c->status,
                                                         level1 ? c->grp : nullptr, bb);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (level1 && (e = launch_level1(all, p, dt, c, s)) != cudaSuccess) return e;
    e = launch_momentum_batched(all, bb, c->Pd, nullptr, s);
    if (e != cudaSuccess) return e;
    hc_batched_kernel<<<(N + 255) / 256, 256, 0, s>>>(all.x, all.y, all.z, c->Pd, 0.5 * dt / p.Mstar, bb);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_removal(all, p, s);
}

cudaError_t launch_drift(genga_system &sys, const genga_params &p, double dt, genga_ctx *c, cudaStream_t s) {
    const int N = sys.N;
    if (N <= 0) return cudaSuccess;
    const bool level1 = p.bs_tol > 0.0;
    cudaError_t e = launch_momentum(sys.vx, sys.vy, sys.vz, sys.m, N, c->mom, nullptr, s);
    if (e == cudaSuccess && level1) e = launch_level1_groups(sys, c, s);
    if (e != cudaSuccess) return e;
    const int nb = (N + 127) / 128;
    drift_kernel<<<nb, 128, 0, s>>>(sys.x, sys.y, sys.z, sys.vx, sys.vy, sys.vz, N, c->mom,
                                    0.5 * dt / p.Mstar, p.G * p.Mstar, dt, p.kepler_max_iter, c->status,
                                    level1 ? c->grp : nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (level1 && (e = launch_level1(sys, p, dt, c, s)) != cudaSuccess) return e;
    e = launch_momentum(sys.vx, sys.vy, sys.vz, sys.m, N, c->mom, nullptr, s);
    if (e != cudaSuccess) return e;
    hc_kernel<<<(N + 255) / 256, 256, 0, s>>>(sys.x, sys.y, sys.z, N, c->mom, 0.5 * dt / p.Mstar);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_removal(sys, p, s);
}

}  // namespace genga
