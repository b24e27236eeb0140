// pass_common.cuh -- device helpers shared by the long-range pass kernels
// (kick.cu: one-sided passes; mutual.cu: the symmetric FP32 pass): packed
// two-lane FP32 arithmetic, the changeover weight, the exact FP64 treatment
// of screened pairs, the screening threshold, bounding-box tests and the
// double-float accumulator.  Everything here is TU-local (unnamed namespace).
#pragma once

#include "internal.cuh"

namespace genga {
namespace {

__device__ __forceinline__ float rsqrt_sfu(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Two FP32 lanes in one 64-bit register, driven by the packed f32x2
// instructions of sm_100-class GPUs: one issue slot carries two FP32 ops,
// each rounded to nearest exactly like its scalar counterpart.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk2(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void up2(f32x2 v, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Changeover weight K(y) (Sect. 1): 0 for y <= 0, 1 for y >= 1.
__device__ __forceinline__ double changeover_K(double y, int form) {
    if (y <= 0.0) return 0.0;
    if (y >= 1.0) return 1.0;
    if (form == GENGA_K_CHAMBERS) {
        const double y2 = y * y;
        return y2 / (2.0 * y2 - 2.0 * y + 1.0);
    }
    return y * y * y * (10.0 + y * (6.0 * y - 15.0));
}

// Exact FP64 treatment of one screened pair (packed positions i, j of one
// system whose packed range starts at poff, with Nd bodies that start at
// body `off` of the caller's arrays): the K-weighted acceleration of i due to
// j; records the encounter unless one of the two is a ghost (merged away or
// removed: mass -0.0, so its force is zero anyway).
__device__ __noinline__ double3 screened_pair(const PassArgs &a, int i, int j, int poff, int Nd, int off) {
    double3 f = make_double3(0.0, 0.0, 0.0);
    if (i - poff >= Nd || j - poff >= Nd || i == j) return f;
    if (a.n_big >= 0 && a.lo[i].w != 0.f && a.lo[j].w != 0.f) return f;  // two test particles (mode 2)
    const double4_32a pi = a.p64[i], pj = a.p64[j];
    const double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
    const double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 == 0.0) return f;  // coincident bodies: no direction, no force
    const double r = sqrt(r2);
    const int oi = (int)a.perm[off + i - poff], oj = (int)a.perm[off + j - poff];
    double rc;
    if (a.rcrit_mode == GENGA_RCRIT_EQ1) {
        rc = fmax(a.rc_eq1[i], a.rc_eq1[j]);
    } else {
        rc = a.n1 * cbrt((a.m[oi] + a.m[oj]) / (3.0 * a.Mstar)) * 0.5 * (a.a_osc[i] + a.a_osc[j]);
    }
    double K = 1.0;
    if (r < rc) {
        if (oi < oj && !(signbit(a.m[oi]) || signbit(a.m[oj]))) {  // ghosts (m = -0) are never encounter pairs
            const int pos = atomicAdd(a.enc_count, 1);
            if (pos < a.enc_cap) a.enc[pos] = make_int2(oi, oj);
        }
        K = changeover_K((r / rc - 0.1) / 0.9, a.changeover);
    } else if (a.predict && oi < oj && r < GENGA_PREDICT_RANGE * rc && !(signbit(a.m[oi]) || signbit(a.m[oj]))) {
        // a pair outside r_crit whose straight-line relative motion over the
        // coming drift enters it joins the close-encounter groups (rounded
        // products as written, no contraction)
        const double ux = a.vx[oj] - a.vx[oi], uy = a.vy[oj] - a.vy[oi], uz = a.vz[oj] - a.vz[oi];
        const double uu = __dadd_rn(__dadd_rn(__dmul_rn(ux, ux), __dmul_rn(uy, uy)), __dmul_rn(uz, uz));
        const double du = __dadd_rn(__dadd_rn(__dmul_rn(dx, ux), __dmul_rn(dy, uy)), __dmul_rn(dz, uz));
        double t = uu > 0.0 ? -du / uu : 0.0;
        const double tlo = a.pred_dt < 0.0 ? a.pred_dt : 0.0, thi = a.pred_dt < 0.0 ? 0.0 : a.pred_dt;
        t = fmin(fmax(t, tlo), thi);
        const double px = __dadd_rn(dx, __dmul_rn(ux, t)), py = __dadd_rn(dy, __dmul_rn(uy, t));
        const double pz = __dadd_rn(dz, __dmul_rn(uz, t));
        if (__dadd_rn(__dadd_rn(__dmul_rn(px, px), __dmul_rn(py, py)), __dmul_rn(pz, pz)) < __dmul_rn(rc, rc)) {
            const int pos = atomicAdd(a.enc_count + 1, 1);
            if (pos < a.enc_cap) a.pred[pos] = make_int2(oi, oj);
        }
    }
    if (K == 0.0) return f;
    const double s = pj.w * K / (r2 * r);
    f.x = s * dx;
    f.y = s * dy;
    f.z = s * dz;
    return f;
}

// Screening threshold (squared, FP32) of an i-body against one tile:
// r_crit,ij^2 <= (max(H_i, Hmax) max(A_i, Amax))^2, with a 2^-10 margin for
// the FP32 rounding of r^2 and a floor that always catches r = 0.
__device__ __forceinline__ float screen_threshold(float H, float A, float Hm, float Am) {
    const float b = fmaxf(H, Hm) * fmaxf(A, Am);
    return fmaxf(b * b * (1.0f + 0x1p-10f), 1e-30f);
}

struct Box {      // bounding box of FP32 positions; w components: max H (lo), max A (hi)
    float4 lo, hi;
};

template <int NG>
__device__ __forceinline__ Box group_box(const float4 *__restrict__ glo, const float4 *__restrict__ ghi, int g0) {
    Box b = {glo[g0], ghi[g0]};
#pragma unroll
    for (int q = 1; q < NG; q++) {
        const float4 l = glo[g0 + q], h = ghi[g0 + q];
        b.lo = make_float4(fminf(b.lo.x, l.x), fminf(b.lo.y, l.y), fminf(b.lo.z, l.z), fmaxf(b.lo.w, l.w));
        b.hi = make_float4(fmaxf(b.hi.x, h.x), fmaxf(b.hi.y, h.y), fmaxf(b.hi.z, h.z), fmaxf(b.hi.w, h.w));
    }
    return b;
}

// True when every pair between the two boxes has K = 1 and (if fp32) offsets
// that FP32-rounded positions give to better than ~5e-6 relative.
__device__ __forceinline__ bool far_pair_of_boxes(const Box &u, const Box &v, bool fp32) {
    const bool empty_u = u.lo.x > u.hi.x, empty_v = v.lo.x > v.hi.x;
    if (empty_u || empty_v) return true;
    const float gx = fmaxf(0.f, fmaxf(v.lo.x - u.hi.x, u.lo.x - v.hi.x));
    const float gy = fmaxf(0.f, fmaxf(v.lo.y - u.hi.y, u.lo.y - v.hi.y));
    const float gz = fmaxf(0.f, fmaxf(v.lo.z - u.hi.z, u.lo.z - v.hi.z));
    const float gap2 = gx * gx + gy * gy + gz * gz;
    float need = fmaxf(u.lo.w, v.lo.w) * fmaxf(u.hi.w, v.hi.w) * (1.0f + 0x1p-10f);  // r_crit bound
    if (fp32) {
        const float X = fmaxf(fmaxf(fmaxf(fabsf(u.lo.x), fabsf(u.hi.x)), fmaxf(fabsf(u.lo.y), fabsf(u.hi.y))),
                              fmaxf(fmaxf(fabsf(u.lo.z), fabsf(u.hi.z)),
                                    fmaxf(fmaxf(fmaxf(fabsf(v.lo.x), fabsf(v.hi.x)),
                                                fmaxf(fabsf(v.lo.y), fabsf(v.hi.y))),
                                          fmaxf(fabsf(v.lo.z), fabsf(v.hi.z)))));
        need = fmaxf(need, 0.025f * X);
    }
    return gap2 > need * need;
}

// Double-float accumulator: value = hi + lo, |lo| <= ulp(hi) / 2, about 48
// significant bits from FP32 arithmetic alone (Knuth's two-sum followed by
// a fast-two-sum renormalisation).  The FP32 pass accumulates and stores its
// per-body sums this way: this GPU's FP64 pipe runs at 1/64 of its FP32 rate.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_add(DF a, float bh, float bl) {  // a + (bh + bl)
    const float s = a.hi + bh;
    const float bp = s - a.hi;
    const float e = (a.hi - (s - bp)) + (bh - bp);
    const float l = (a.lo + bl) + e;
    const float h = s + l;
    return DF{h, l - (h - s)};
}

__device__ __forceinline__ DF df_of_double(double x) {
    const float h = __double2float_rn(x);
    return DF{h, __double2float_rn(x - (double)h)};
}

}  // namespace
}  // namespace genga
