// kepler.cuh -- the universal-variable Kepler drift in FP64 (Sect. 1: the
// Kepler solver is always double precision), shared by the drift kernels and
// the close-encounter level.
//
// Kepler's equation in the universal anomaly s,
//   F(s) = r0 G1(s) + eta0 G2(s) + mu G3(s) - dt = 0,  G_k = s^k c_k(beta s^2),
// beta = 2 mu / r0 - v0^2, eta0 = x0 . v0, solved by the Laguerre-Conway
// iteration (order 5, Conway 1986) from a second-order estimate of s, followed
// by the f and g functions.  The Stumpff functions c_k(z) come from their
// Taylor series for |z| < 1 and from the trigonometric / hyperbolic closed
// forms otherwise (with the half-angle form of c2, which does not cancel).
#pragma once

#include "internal.cuh"

namespace genga {
namespace {  // a private copy in every translation unit, as the functions were inside drift.cu

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

}  // namespace
}  // namespace genga
