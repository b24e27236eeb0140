// drift.cu -- the drift of the hybrid step, always in FP64 (Sect. 1):
//
//   x_i += (dt/2) P / M*               central-body momentum drift, P = sum m v
//   (x_i, v_i) <- Kepler(mu = G M*, dt) two-body drift of every body outside
//                                      the close-encounter groups (those move
//                                      on level 1, encounter.cu, when enabled)
//   x_i += (dt/2) P' / M*              with the momentum after the drift
//
// The Kepler drift uses universal variables: Kepler's equation in the
// universal anomaly s,
//   F(s) = r0 G1(s) + eta0 G2(s) + mu G3(s) - dt = 0,  G_k = s^k c_k(beta s^2),
// beta = 2 mu / r0 - v0^2, eta0 = x0 . v0, solved by the Laguerre-Conway
// iteration (order 5, Conway 1986) from a second-order estimate of s, followed
// by the f and g functions.  The Stumpff functions c_k(z) come from their Taylor series for
// |z| < 1 and from the trigonometric / hyperbolic closed forms otherwise
// (with the half-angle form of c2, which does not cancel).
#include "internal.cuh"

namespace genga {

namespace {

// c2(z) = sum_k (-z)^k / (2k+2)!,  c3(z) = sum_k (-z)^k / (2k+3)!, the
// first NT terms (10 terms reach rounding level for |z| < 1, 6 for
// |z| < 0.1: the next terms are below 2^-53 of the sums)
template <int NT>
__device__ __forceinline__ void stumpff_series(double z, double &c2, double &c3) {
    constexpr double a2[10] = {1.0 / 2.0,
                               1.0 / 24.0,
                               1.0 / 720.0,
                               1.0 / 40320.0,
                               1.0 / 3628800.0,
                               1.0 / 479001600.0,
                               1.0 / 87178291200.0,
                               1.0 / 20922789888000.0,
                               1.0 / 6402373705728000.0,
                               1.0 / 2432902008176640000.0};
    constexpr double a3[10] = {1.0 / 6.0,
                               1.0 / 120.0,
                               1.0 / 5040.0,
                               1.0 / 362880.0,
                               1.0 / 39916800.0,
                               1.0 / 6227020800.0,
                               1.0 / 1307674368000.0,
                               1.0 / 355687428096000.0,
                               1.0 / 121645100408832000.0,
                               1.0 / 51090942171709440000.0};
    const double w = -z;
    double p2 = a2[NT - 1], p3 = a3[NT - 1];
#pragma unroll
    for (int k = NT - 2; k >= 0; k--) {
        p2 = fma(p2, w, a2[k]);
        p3 = fma(p3, w, a3[k]);
    }
    c2 = p2;
    c3 = p3;
}

__device__ __forceinline__ void stumpff(double z, double &c0, double &c1, double &c2, double &c3) {
    if (fabs(z) < 0.1) {  // the usual case: dt small against the orbital period
        stumpff_series<6>(z, c2, c3);
        c0 = 1.0 - z * c2;
        c1 = 1.0 - z * c3;
    } else if (fabs(z) < 1.0) {
        stumpff_series<10>(z, c2, c3);
        c0 = 1.0 - z * c2;
        c1 = 1.0 - z * c3;
    } else if (z > 0.0) {
        const double q = sqrt(z);
        double sn, cs, sh, ch;
        sincos(q, &sn, &cs);
        sincos(0.5 * q, &sh, &ch);
        c0 = cs;
        c1 = sn / q;
        c2 = 2.0 * sh * sh / z;
        c3 = (q - sn) / (z * q);
    } else {
        const double q = sqrt(-z);
        const double sn = sinh(q), cs = cosh(q), sh = sinh(0.5 * q);
        c0 = cs;
        c1 = sn / q;
        c2 = 2.0 * sh * sh / (-z);
        c3 = (sn - q) / (-z * q);
    }
}

// Returns true when the iteration met |ds| <= 1e-12 |s| within max_iter steps.
__device__ bool kepler_drift(double mu, double dt, int max_iter, double &x, double &y, double &z, double &u,
                             double &v, double &w) {
    // FP64 divisions and square roots as series-corrected SFU seeds (the
    // FP64 pipe is the slow one on this GPU)
    const double rr = x * x + y * y + z * z;
    const double ir0 = rsqrt_fp64(rr);
    const double r0 = rr * ir0;
    const double v2 = u * u + v * v + w * w;
    const double eta = x * u + y * v + z * w;
    const double beta = 2.0 * mu * ir0 - v2;
    // start from the second-order expansion of s(t) = int dt / r,
    // s ~ dt / r0 - eta dt^2 / (2 r0^3), which saves about one iteration on
    // near-circular orbits; plain dt / r0 where the correction is not small
    const double q = dt * ir0;
    const double corr = 0.5 * eta * q * ir0;
    double s = fabs(corr) < 0.25 ? q * (1.0 - corr) : q;
    double c0, c1, c2, c3;
    bool ok = false;
    for (int it = 0; it < max_iter; it++) {
        stumpff(beta * s * s, c0, c1, c2, c3);
        const double G1 = s * c1, G2 = s * s * c2, G3 = s * s * s * c3;
        const double F = fma(r0, G1, fma(eta, G2, mu * G3)) - dt;
        const double dF = fma(r0, c0, fma(eta, G1, mu * G2));
        const double ddF = fma(eta, c0, (mu - beta * r0) * G1);
        // Laguerre-Conway step, order n = 5
        const double rad = sqrt(fabs(16.0 * dF * dF - 20.0 * F * ddF));
        const double ds = -5.0 * F * rcp_fp64(dF + copysign(rad, dF));
        s += ds;
        if (fabs(ds) <= 1e-12 * fabs(s)) {
            ok = true;
            break;
        }
    }
    stumpff(beta * s * s, c0, c1, c2, c3);
    const double G1 = s * c1, G2 = s * s * c2;
    const double r = fma(r0, c0, fma(eta, G1, mu * G2));
    const double ir = rcp_fp64(r);
    const double f = 1.0 - mu * G2 * ir0;
    const double g = fma(r0, G1, eta * G2);
    const double fd = -mu * G1 * ir * ir0;
    const double gd = 1.0 - mu * G2 * ir;
    const double nx = f * x + g * u, ny = f * y + g * v, nz = f * z + g * w;
    const double nu = fd * x + gd * u, nv = fd * y + gd * v, nw = fd * z + gd * w;
    x = nx; y = ny; z = nz;
    u = nu; v = nv; w = nw;
    return ok;
}

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
cudaError_t launch_level1_groups(const genga_system &sys, genga_ctx *c, cudaStream_t s) {
    GroupArgs g;
    g.enc = c->enc;
    g.pred = c->pred;
    g.enc_count = c->enc_count;
    g.enc_cap = c->enc_cap;
    g.N = sys.N;
    g.slots = c->bs_slots;
    g.grp = c->grp;
    g.gmark = c->gmark;
    g.gslot = c->gslot;
    g.gbody = c->gbody;
    g.gmem = c->gmem;
    g.gstart = c->gstart;
    g.gsize = c->gsize;
    g.gcur = c->gcur;
    g.gcount = c->gcount;
    g.status = c->status;
    return launch_groups(g, s);
}

cudaError_t launch_level1(genga_system &sys, const genga_params &p, double dt, genga_ctx *c, cudaStream_t s) {
    BSArgs b;
    b.x = sys.x; b.y = sys.y; b.z = sys.z;
    b.vx = sys.vx; b.vy = sys.vy; b.vz = sys.vz;
    b.m = sys.m;
    b.iperm = c->iperm;
    b.a_osc = c->a_osc;
    b.rc_eq1 = c->rc_eq1;
    b.lo = c->pk_lo;
    b.gcount = c->gcount;
    b.gstart = c->gstart;
    b.gsize = c->gsize;
    b.gmem = c->gmem;
    b.gbody = c->gbody;
    b.grp = c->grp;
    b.gmark = c->gmark;
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
    b.status = c->status;
    return launch_bs(b, c->sm_count, s);
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
