// levels.cu -- the intermediate levels of the changeover (Sect. 1: between
// the symplectic step and the Bulirsch-Stoer integrator, further symplectic
// steps with smaller time steps, so that Bulirsch-Stoer is left to the
// closest pairs).
//
// With L levels of s sub-steps, level l (1 <= l <= L) has the step dt / s^l
// and the pair radius r_crit,l = r_crit,ij / s^l, and K_l(r) = K((r /
// r_crit,l - 0.1) / 0.9).  The pair force splits into K_0 for the step's
// kick, W_l = K_l prod_{k<l} (1 - K_k) for the kicks of level l and
// prod_{k<=L} (1 - K_k) for the Bulirsch-Stoer level (encounter.cu); the
// shares add up to 1.  A group of level l moves over the step of level l - 1
// in s sub-steps of h, each
//   kick(h/2)   v_i += h/2 sum_{j in group} G m_j W_l(r_ij) (x_j - x_i) / r_ij^3
//   scan        subgroups for level l + 1: the member pairs inside r_crit,l
//               and those whose straight-line motion over h enters it from
//               within 1.5 r_crit,l (the predicted entries of the step's
//               kick, one level down)
//   groups      the grouping kernel of encounter.cu on those pairs
//   drift       members outside every subgroup: Kepler drift over h
//   level l+1   the subgroups (Bulirsch-Stoer below level L)
//   kick(h/2)
// The host issues these launches level by level (all groups of a level share
// the time grid), so a step's launch count grows with s^L; the whole
// sequence is part of the captured step graph.  The kick and the scan run
// one warp per member (lanes over its partners), so a large group spreads
// over many FP64 pipes (on GB300 one FP64 warp instruction holds an SMSP's
// pipe ~64 cycles whatever the active lanes); the sort, drift and clear one
// warp per group.  FP64 throughout (Sect. 1: close-encounter forces in
// double precision).  The subgroup decision is taken with correctly rounded
// operations as written (no contraction), the oracle's arithmetic.
#include "changeover.cuh"
#include "kepler.cuh"

namespace genga {

namespace {

constexpr int LV_WARPS = 4;  // warps per CTA (each takes one group or one member at a time)

// W_l at separation q with inv9 = 1 / (0.9 r_crit,ij): prod_{k<l} (1 - K_k) * K_l.
__device__ __forceinline__ double level_kick_weight(double q, double inv9, int l, double s, int form) {
    double w = 1.0, f = inv9;
    for (int k = 0; k < l; k++) {
        w *= keep_weight(fma(q, f, -1.0 / 9.0), form);
        f *= s;
    }
    return w * (1.0 - keep_weight(fma(q, f, -1.0 / 9.0), form));
}

struct Body {
    double m, a, rc;
    int tp;
};

__device__ __forceinline__ Body body(const LevelArgs &a, int v) {
    const int k = (int)a.iperm[v];
    return Body{a.m[v], a.a_osc[k], a.rc_eq1[k], a.lo[k].w != 0.f ? 1 : 0};
}

__device__ __forceinline__ double pair_rc(const LevelArgs &a, const Body &i, const Body &j) {
    return pair_rcrit(a.rcrit_mode, a.n1, a.Mstar, i.m, j.m, i.a, j.a, i.rc, j.rc);
}

// The members of every group sorted by body index into gbody (the order of
// every sum) and the group of every member slot into gof; once per level,
// after the grouping kernel formed it.  One warp per group.
__global__ void __launch_bounds__(32 * LV_WARPS) level_sort_kernel(const __grid_constant__ LevelArgs a) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * LV_WARPS + (threadIdx.x >> 5), nw = gridDim.x * LV_WARPS;
    const int ng = *a.gcount;
    for (int g = gw; g < ng; g += nw) {
        const int s0 = a.gstart[g], n = a.gsize[g];
        for (int q = lane; q < n; q += 32) {
            const int v = a.gmem[s0 + q];
            int rank = 0;
            for (int r = 0; r < n; r++) rank += (a.gmem[s0 + r] < v) ? 1 : 0;
            a.gbody[s0 + rank] = v;
            a.gof[s0 + q] = g;
        }
    }
}

// Member slots of all groups: the groups are stored one after another.
__device__ __forceinline__ int member_slots(const LevelArgs &a) {
    const int ng = *a.gcount;
    return ng > 0 ? a.gstart[ng - 1] + a.gsize[ng - 1] : 0;
}

// Warp sum in a fixed butterfly order (every lane ends with the same value).
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// kick(tau) of every member by the level's share of the other members' pair
// forces: one warp per member (a group of n members occupies n warps, so a
// large group spreads over the SMs' FP64 pipes), lanes over its partners in
// body order, a fixed-order warp sum.  Positions are only read, so the
// members' velocities are updated in place.
__global__ void __launch_bounds__(32 * LV_WARPS) level_kick_kernel(const __grid_constant__ LevelArgs a, double tau,
                                                                   int zero_next) {
    const int lane = threadIdx.x & 31;
    // the next level's pair list starts empty for the scan that follows this kick
    if (zero_next && blockIdx.x == 0 && threadIdx.x < 2) a.next_count[threadIdx.x] = 0;
    const int gw = blockIdx.x * LV_WARPS + (threadIdx.x >> 5), nw = gridDim.x * LV_WARPS;
    const int ns = member_slots(a);
    for (int item = gw; item < ns; item += nw) {
        const int g = a.gof[item], s0 = a.gstart[g], n = a.gsize[g];
        const int vi = a.gbody[item];
        const Body bi = body(a, vi);
        if (signbit(bi.m)) continue;  // a ghost: no level force (warp-uniform)
        const double xi = a.x[vi], yi = a.y[vi], zi = a.z[vi];
        double ax = 0.0, ay = 0.0, az = 0.0;
        for (int t = lane; t < n; t += 32) {
            const int vj = a.gbody[s0 + t];
            if (vj == vi) continue;
            const Body bj = body(a, vj);
            if (signbit(bj.m) || (bi.tp && bj.tp)) continue;
            const double dx = a.x[vj] - xi, dy = a.y[vj] - yi, dz = a.z[vj] - zi;
            const double q2 = dx * dx + dy * dy + dz * dz;
            if (q2 == 0.0) continue;
            const double rc = pair_rc(a, bi, bj);
            if (q2 >= rc * rc) continue;  // outside r_crit,0 the step's kick has it all
            const double iq = rsqrt_fp64(q2);
            const double w = level_kick_weight(q2 * iq, 1.0 / (0.9 * rc), a.level, a.nsub, a.changeover);
            const double f = a.G * bj.m * w * (iq * iq * iq);
            ax = fma(f, dx, ax);
            ay = fma(f, dy, ay);
            az = fma(f, dz, az);
        }
        ax = warp_sum(ax);
        ay = warp_sum(ay);
        az = warp_sum(az);
        if (lane == 0) {
            a.vx[vi] = fma(tau, ax, a.vx[vi]);
            a.vy[vi] = fma(tau, ay, a.vy[vi]);
            a.vz[vi] = fma(tau, az, a.vz[vi]);
        }
    }
}

// The member pairs of every group that form the next level's subgroups for a
// drift of h (list appended; its count was zeroed before the launch): one
// warp per member i, lanes over its partners j after it in body order.
__global__ void __launch_bounds__(32 * LV_WARPS) level_scan_kernel(const __grid_constant__ LevelArgs a, double h) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * LV_WARPS + (threadIdx.x >> 5), nw = gridDim.x * LV_WARPS;
    const int ns = member_slots(a);
    const double tlo = h < 0.0 ? h : 0.0, thi = h < 0.0 ? 0.0 : h;
    for (int item = gw; item < ns; item += nw) {
        const int g = a.gof[item], s0 = a.gstart[g], n = a.gsize[g];
        const int vi = a.gbody[item];
        const Body bi = body(a, vi);
        if (signbit(bi.m)) continue;
        for (int t = item - s0 + 1 + lane; t < n; t += 32) {
            const int vj = a.gbody[s0 + t];
            const Body bj = body(a, vj);
            if (signbit(bj.m) || (bi.tp && bj.tp)) continue;
            const double dx = __dsub_rn(a.x[vj], a.x[vi]), dy = __dsub_rn(a.y[vj], a.y[vi]);
            const double dz = __dsub_rn(a.z[vj], a.z[vi]);
            const double q2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            const double rcl = __ddiv_rn(pair_rc(a, bi, bj), a.sl);
            const double rcl2 = __dmul_rn(rcl, rcl), rout = __dmul_rn(1.5, rcl);
            bool in = q2 < rcl2;
            if (!in && q2 < __dmul_rn(rout, rout)) {  // straight-line entry within h
                const double ux = __dsub_rn(a.vx[vj], a.vx[vi]), uy = __dsub_rn(a.vy[vj], a.vy[vi]);
                const double uz = __dsub_rn(a.vz[vj], a.vz[vi]);
                const double uu = __dadd_rn(__dadd_rn(__dmul_rn(ux, ux), __dmul_rn(uy, uy)), __dmul_rn(uz, uz));
                const double du = __dadd_rn(__dadd_rn(__dmul_rn(dx, ux), __dmul_rn(dy, uy)), __dmul_rn(dz, uz));
                double t_c = uu > 0.0 ? __ddiv_rn(-du, uu) : 0.0;
                t_c = t_c < tlo ? tlo : t_c;
                t_c = t_c > thi ? thi : t_c;
                const double px = __dadd_rn(dx, __dmul_rn(ux, t_c)), py = __dadd_rn(dy, __dmul_rn(uy, t_c));
                const double pz = __dadd_rn(dz, __dmul_rn(uz, t_c));
                in = __dadd_rn(__dadd_rn(__dmul_rn(px, px), __dmul_rn(py, py)), __dmul_rn(pz, pz)) < rcl2;
            }
            if (!in) continue;
            const int k = atomicAdd(a.next_count, 1);
            if (k < a.next_cap) a.next_pairs[k] = make_int2(vi, vj);
            else atomicOr(a.status, GENGA_BIT(GENGA_ERR_BS));  // the subgroups would miss the pair
        }
    }
}

// Kepler drift over h of every member outside the next level's subgroups
// (ghosts included: they have no level force).
__global__ void __launch_bounds__(32 * LV_WARPS) level_drift_kernel(const __grid_constant__ LevelArgs a, double h) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * LV_WARPS + (threadIdx.x >> 5), nw = gridDim.x * LV_WARPS;
    const int ng = *a.gcount;
    const double mu = a.G * a.Mstar;
    for (int g = gw; g < ng; g += nw) {
        const int s0 = a.gstart[g], n = a.gsize[g];
        for (int q = lane; q < n; q += 32) {
            const int v = a.gmem[s0 + q];
            if (a.next_grp[v] >= 0) continue;
            double x = a.x[v], y = a.y[v], z = a.z[v], u = a.vx[v], vv = a.vy[v], w = a.vz[v];
            if (!kepler_drift(mu, h, a.max_iter, x, y, z, u, vv, w)) atomicOr(a.status, GENGA_BIT(GENGA_ERR_KEPLER));
            a.x[v] = x; a.y[v] = y; a.z[v] = z;
            a.vx[v] = u; a.vy[v] = vv; a.vz[v] = w;
        }
    }
}

// The level's marks back to "no group" once its groups have moved.
__global__ void __launch_bounds__(32 * LV_WARPS) level_clear_kernel(const __grid_constant__ LevelArgs a) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * LV_WARPS + (threadIdx.x >> 5), nw = gridDim.x * LV_WARPS;
    const int ng = *a.gcount;
    for (int g = gw; g < ng; g += nw) {
        const int s0 = a.gstart[g], n = a.gsize[g];
        for (int q = lane; q < n; q += 32) {
            const int v = a.gmem[s0 + q];
            a.grp[v] = -1;
            a.gmark[v] = 0;
        }
    }
}

}  // namespace

cudaError_t launch_level_sort(const LevelArgs &a, int sm_count, cudaStream_t s) {
    level_sort_kernel<<<2 * sm_count, 32 * LV_WARPS, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_level_kick(const LevelArgs &a, double tau, bool zero_next, int sm_count, cudaStream_t s) {
    level_kick_kernel<<<2 * sm_count, 32 * LV_WARPS, 0, s>>>(a, tau, zero_next ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_level_scan(const LevelArgs &a, double h, int sm_count, cudaStream_t s) {
    level_scan_kernel<<<2 * sm_count, 32 * LV_WARPS, 0, s>>>(a, h);
    return cudaGetLastError();
}

cudaError_t launch_level_drift(const LevelArgs &a, double h, int sm_count, cudaStream_t s) {
    level_drift_kernel<<<2 * sm_count, 32 * LV_WARPS, 0, s>>>(a, h);
    return cudaGetLastError();
}

cudaError_t launch_level_clear(const LevelArgs &a, int sm_count, cudaStream_t s) {
    level_clear_kernel<<<2 * sm_count, 32 * LV_WARPS, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace genga
