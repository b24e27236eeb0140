// encounter.cu -- the close-encounter level of the hybrid step (Sect. 1:
// level 1, the Bulirsch-Stoer integrator that takes over from the Kepler
// drift for bodies in close encounters; the changeover function splits each
// pair force between the kick and this level).
//
//   groups     the connected components of the encounter pairs of the step's
//              first kick and of the pairs that kick predicted to enter
//              r_crit within the drift (one CTA: hook-and-compress union-find
//              over the pairs, then the members of each group stored
//              contiguously)
//   level 1    every group is integrated over the drift by one warp: each
//              member moves about the central body (mu = G M*) and feels the
//              other members through the (1 - K) part of their pair force,
//                dv_i/dt = -mu x_i/|x_i|^3
//                          + sum_{j in group} G m_j (1 - K(y_ij)) (x_j - x_i)/r_ij^3,
//              with r_crit,ij from the a_i, r_crit,i of that kick, so kick +
//              level 1 = the whole Newtonian pair force.  The integrator is
//              Gragg's modified midpoint rule with 2, 4, ..., 16 steps and
//              Aitken-Neville extrapolation in H^2 (Stoer & Bulirsch), step
//              halving and doubling as described at bs_kernel.
//   mergers    with physical radii, overlapping members merge after every
//              accepted sub-step (Sect. 2: collisions are perfect mergers);
//              the absorbed body becomes a ghost of mass -0.0
//
// The drift kernel skips the members (grp[i] >= 0): they get the central-
// body momentum drift only, and this level moves them over dt in between
// the two momentum drifts.  With intermediate levels (levels.cu) this kernel
// integrates the subgroups of the last level over its sub-step, with the
// pair share prod_{k=0}^{L} (1 - K_k) in place of 1 - K.  Everything here is FP64 (Sect. 1, last paragraph:
// close-encounter forces are always double precision).
#include <algorithm>
#include <cooperative_groups.h>

#include "changeover.cuh"
#include "kepler.cuh"

namespace genga {

namespace {

constexpr int GROUP_THREADS = 1024;
constexpr int GROUP_MAX_ROUNDS = 256;  // hook-and-compress rounds (a chain of n bodies needs about log2 n)

constexpr int BS_KMAX = 8;             // extrapolation columns: midpoint step counts 2, 4, ..., 16
constexpr int BS_GROW_COL = 2;         // a sub-step accepted by column <= 2 doubles the next one
constexpr double BS_MIN_FRAC = 0x1p-30;  // smallest sub-step, as a fraction of the drift
constexpr int BS_MAX_ATTEMPTS = 4096;  // sub-step attempts per group and drift
constexpr int BS_WARPS = 4;            // groups in flight per CTA (one warp each)
// Groups of more than BS_TEAM_MIN members are integrated by a whole cluster of
// BS_TEAM_CTAS CTAs (32 warps on 32 SMSPs) instead of one warp.
constexpr int BS_TEAM_CTAS = 8;
constexpr int BS_TEAM_MIN = 24;
// Wall-clock bound of one launch of the level-1 kernel (counted per warp from
// the launch); past it every group still integrating drifts the rest of the
// step on Kepler orbits (GENGA_ERR_BS).
constexpr unsigned long long BS_TIME_LIMIT_NS = 2000000000ull;

__device__ __forceinline__ int ld_cg(const int32_t *p) { return __ldcg(p); }

// Inclusive block scan (GROUP_THREADS threads) of v; returns the scan and
// sets *total to the block sum.
__device__ int block_scan(int v, int *warp_sums, int *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) warp_sums[w] = v;
    __syncthreads();
    if (w == 0) {
        int s = warp_sums[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        warp_sums[lane] = s;  // inclusive over warps
    }
    __syncthreads();
    const int r = v + (w > 0 ? warp_sums[w - 1] : 0);
    *total = warp_sums[31];
    __syncthreads();
    return r;
}

// The p-th pair of the grouping: the encounter pairs, then the predicted entries.
__device__ __forceinline__ int2 group_pair(const GroupArgs &a, int p, int ne) {
    return p < ne ? a.enc[p] : a.pred[p - ne];
}

// One CTA.  In: the encounter pairs and the pairs predicted to enter r_crit
// within the drift (body indices < N).  Out: gcount groups;
// group g has gsize[g] members gmem[gstart[g] ..] (in no particular order),
// grp[v] = the smallest body of v's group for every member (-1 elsewhere),
// gmark[v] = 1 for every member.  More members than `slots`: no groups, the
// marks are cleared again and GENGA_ERR_BS is raised (the bodies then get the
// plain Kepler drift).
__global__ void __launch_bounds__(GROUP_THREADS) group_kernel(const __grid_constant__ GroupArgs a) {
    __shared__ int s_flag, s_nmem, s_ngroups;
    __shared__ int warp_sums[32];
    const int tid = threadIdx.x;
    const int ne = min(a.enc_count[0], a.enc_cap);
    const int np = ne + min(a.enc_count[1], a.enc_cap);
    if (tid == 0) {
        s_nmem = 0;
        s_ngroups = 0;
    }
    // 1. every body of a pair starts as its own group
    for (int p = tid; p < np; p += GROUP_THREADS) {
        const int2 e = group_pair(a, p, ne);
        if (e.x < 0 || e.y < 0 || e.x >= a.N || e.y >= a.N) continue;  // a list of another system
        a.grp[e.x] = e.x;
        a.grp[e.y] = e.y;
    }
    __syncthreads();
    // 2. hook and compress until no pair joins two labels.  Invariant: grp[v]
    //    is a body of v's component and grp[v] <= v; both steps only lower
    //    labels, so the rounds end, and at the end every component carries
    //    its smallest body as label.
    for (int round = 0;; round++) {
        if (tid == 0) s_flag = 0;
        __syncthreads();
        for (int p = tid; p < np; p += GROUP_THREADS) {
            const int2 e = group_pair(a, p, ne);
            if (e.x < 0 || e.y < 0 || e.x >= a.N || e.y >= a.N) continue;
            const int li = ld_cg(a.grp + e.x), lj = ld_cg(a.grp + e.y);
            if (li != lj) {
                atomicMin(a.grp + max(li, lj), min(li, lj));
                s_flag = 1;
            }
        }
        __syncthreads();
        for (int p = tid; p < np; p += GROUP_THREADS) {
            const int2 e = group_pair(a, p, ne);
            if (e.x < 0 || e.y < 0 || e.x >= a.N || e.y >= a.N) continue;
#pragma unroll
            for (int side = 0; side < 2; side++) {
                const int v = side ? e.y : e.x;
                const int l = ld_cg(a.grp + v), ll = ld_cg(a.grp + l);
                if (ll < l) {
                    atomicMin(a.grp + v, ll);
                    s_flag = 1;
                }
            }
        }
        __syncthreads();
        const int f = s_flag;
        __syncthreads();
        if (!f) break;
        if (round + 1 >= GROUP_MAX_ROUNDS) {
            if (tid == 0) atomicOr(a.status, GENGA_BIT(GENGA_ERR_BS));
            break;
        }
    }
    // 3. the distinct members, in discovery order
    for (int p = tid; p < np; p += GROUP_THREADS) {
        const int2 e = group_pair(a, p, ne);
        if (e.x < 0 || e.y < 0 || e.x >= a.N || e.y >= a.N) continue;
#pragma unroll
        for (int side = 0; side < 2; side++) {
            const int v = side ? e.y : e.x;
            if (atomicExch(a.gmark + v, 1) == 0) {
                const int slot = atomicAdd(&s_nmem, 1);
                if (slot < a.slots) a.gbody[slot] = v;
            }
        }
    }
    __syncthreads();
    const int nmem = s_nmem;
    if (nmem > a.slots) {  // the workspace holds fewer members: leave everyone to the Kepler drift
        for (int p = tid; p < np; p += GROUP_THREADS) {
            const int2 e = group_pair(a, p, ne);
            if (e.x < 0 || e.y < 0 || e.x >= a.N || e.y >= a.N) continue;
            a.grp[e.x] = -1;
            a.grp[e.y] = -1;
            a.gmark[e.x] = 0;
            a.gmark[e.y] = 0;
        }
        if (tid == 0) {
            *a.gcount = 0;
            atomicOr(a.status, GENGA_BIT(GENGA_ERR_BS));
        }
        return;
    }
    // 4. a group number for every root, group sizes, offsets, placement
    for (int q = tid; q < nmem; q += GROUP_THREADS) {
        const int v = a.gbody[q];
        if (ld_cg(a.grp + v) == v) {
            const int g = atomicAdd(&s_ngroups, 1);
            a.gslot[v] = g;
            a.gsize[g] = 0;
        }
    }
    __syncthreads();
    const int ng = s_ngroups;
    for (int q = tid; q < nmem; q += GROUP_THREADS) {
        const int v = a.gbody[q];
        atomicAdd(a.gsize + ld_cg(a.gslot + ld_cg(a.grp + v)), 1);
    }
    __syncthreads();
    int carry = 0;
    for (int base = 0; base < ng; base += GROUP_THREADS) {
        const int g = base + tid;
        const int sz = g < ng ? ld_cg(a.gsize + g) : 0;
        int total;
        const int incl = block_scan(sz, warp_sums, &total);
        if (g < ng) {
            a.gstart[g] = carry + incl - sz;
            a.gcur[g] = carry + incl - sz;
        }
        carry += total;
    }
    __syncthreads();
    for (int q = tid; q < nmem; q += GROUP_THREADS) {
        const int v = a.gbody[q];
        const int pos = atomicAdd(a.gcur + ld_cg(a.gslot + ld_cg(a.grp + v)), 1);
        a.gmem[pos] = v;
    }
    if (tid == 0) *a.gcount = ng;
}

// Scratch fields of the level-1 workspace, each `slots` doubles (slot = the
// member's position in gmem/gbody):
constexpr int BS_PAIR_TAB = 16;    // groups of up to this many members keep their pair radii
enum : int {
    F_Y = 0,                              // accepted state x, y, z, vx, vy, vz
    F_F0 = F_Y + 6,                       // acceleration at the accepted state
    F_ISC = F_F0 + 3,                     // 1/|x|, 1/|v| of the sub-step (error scales)
    F_M = F_ISC + 2,                      // mass
    F_A = F_M + 1,                        // osculating a of the first kick
    F_RC = F_A + 1,                       // Eq. 1 radius of the first kick
    F_RAD = F_RC + 1,                     // physical radius (mergers)
    F_Z = F_RAD + 1,                      // per column k: three rotating midpoint states (18 fields)
    F_T = F_Z + 18 * BS_KMAX,             // per column k: the smoothed midpoint result T[k][0] (6 fields)
    F_PR2 = F_T + 6 * BS_KMAX,            // (r_crit,ij / s^nlev)^2 with the first BS_PAIR_TAB members
    F_PIN = F_PR2 + BS_PAIR_TAB,          // 1 / (0.9 r_crit,ij)
    F_COUNT = F_PIN + BS_PAIR_TAB
};
static_assert(F_COUNT == GENGA_BS_FIELDS, "level-1 workspace fields");

struct Work {  // field f of slot s: base[f * stride + s]
    double *base;
    size_t stride;
    __device__ __forceinline__ double *f(int field) const { return base + (size_t)field * stride; }
    __device__ __forceinline__ double &operator()(int field, int s) const { return base[(size_t)field * stride + s]; }
};

// Aitken-Neville coefficients n_{k-j}^2 / (n_k^2 - n_{k-j}^2), n_k = 2 (k + 1),
// at [k * BS_KMAX + j] (correctly rounded quotients of integers).
struct NevilleTable {
    double c[BS_KMAX * BS_KMAX];
    constexpr NevilleTable() : c() {
        for (int k = 0; k < BS_KMAX; k++)
            for (int j = 1; j <= k; j++) {
                const double nk = 2.0 * (k + 1), nkj = 2.0 * (k - j + 1);
                c[k * BS_KMAX + j] = (nkj * nkj) / (nk * nk - nkj * nkj);
            }
    }
};
__constant__ NevilleTable c_neville = NevilleTable();

// Pair radius r_crit,ij of two members (the kick's rule, Eq. 1 inputs of that kick).
__device__ __forceinline__ double pair_radius(const BSArgs &a, double mi, double mj, double ai, double aj, double rci,
                                              double rcj) {
    return pair_rcrit(a.rcrit_mode, a.n1, a.Mstar, mi, mj, ai, aj, rci, rcj);
}

// Share of the pair force this level integrates, at separation q, inv9 =
// 1 / (0.9 r_crit,ij): prod_{k=0}^{nlev} (1 - K_k) with K_k the changeover
// at r_crit,ij / s^k (Sect. 1's intermediate levels take the K_k parts);
// 1 - K_0 without levels.
__device__ __noinline__ double deeper_keep(const BSArgs &a, double q, double inv9) {  // prod_{k=1}^{nlev} (1 - K_k)
    double w = 1.0, f = inv9;
    for (int k = 1; k <= a.nlev; k++) {
        f *= a.nsub;
        w *= keep_weight(fma(q, f, -1.0 / 9.0), a.changeover);
    }
    return w;
}

__device__ __forceinline__ double bs_weight(const BSArgs &a, double q, double inv9) {
    const double w = keep_weight(fma(q, inv9, -1.0 / 9.0), a.changeover);
    return a.nlev > 0 ? w * deeper_keep(a, q, inv9) : w;
}

// Level-1 acceleration of the member in slot s with positions in fields
// (p, p+1, p+2); members in slots [s0, s0 + n).  FP64 throughout; the square
// root and the reciprocals come from series-corrected SFU seeds (the FP64 pipe
// of this GPU takes about 64 cycles per warp instruction, whatever the number
// of active lanes, so the instruction count is the cost).
__device__ void level1_acc(const BSArgs &a, const Work &W, int s, int s0, int n, int p, bool tab, double &ax,
                           double &ay, double &az) {
    const double *__restrict__ px = W.f(p);
    const double *__restrict__ py = W.f(p + 1);
    const double *__restrict__ pz = W.f(p + 2);
    const double xi = px[s], yi = py[s], zi = pz[s];
    const double ir = rsqrt_fp64(xi * xi + yi * yi + zi * zi);
    const double c = -a.G * a.Mstar * (ir * ir * ir);
    ax = c * xi;
    ay = c * yi;
    az = c * zi;
    const int fi = a.tpf[s];
    if (fi & 2) return;  // a ghost feels the central body only
    const double *__restrict__ M = W.f(F_M);
    for (int t = s0; t < s0 + n; t++) {
        const int ft = a.tpf[t];
        if (t == s || (ft & 2) || ((fi & 1) && (ft & 1))) continue;  // self, ghost, two test particles
        const double dx = px[t] - xi, dy = py[t] - yi, dz = pz[t] - zi;
        const double q2 = dx * dx + dy * dy + dz * dz;
        if (q2 == 0.0) continue;
        double rc2, inv9;
        if (tab) {
            rc2 = W(F_PR2 + (t - s0), s);
            inv9 = W(F_PIN + (t - s0), s);
        } else {
            const double rc = pair_radius(a, W(F_M, s), M[t], W(F_A, s), W(F_A, t), W(F_RC, s), W(F_RC, t));
            const double rcl = rc / a.snl;
            rc2 = rcl * rcl;
            inv9 = 1.0 / (0.9 * rc);
        }
        if (q2 >= rc2) continue;  // K = 1 (or K_nlev = 1): the kicks have all of it
        const double iq = rsqrt_fp64(q2);
        const double w = bs_weight(a, q2 * iq, inv9);
        const double f = a.G * M[t] * w * (iq * iq * iq);
        ax = fma(f, dx, ax);
        ay = fma(f, dy, ay);
        az = fma(f, dz, az);
    }
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// One warp per group.  Sub-steps are fractions of dt (exact binary values);
// each runs the modified midpoint rule with n_k = 2 (k + 1) steps for all
// BS_KMAX columns k at once -- the columns are independent, so lane
// 8 q' + k integrates column k for the members q', q' + 4, ... and one
// sub-step costs 2 BS_KMAX force evaluations in sequence instead of their sum:
//   z_0 = y, z_1 = z_0 + H f(z_0), z_{m+1} = z_{m-1} + 2H f(z_m),
//   T[k][0] = (z_n + z_{n-1} + H f(z_n)) / 2,
// then the Aitken-Neville table
//   T[k][j] = T[k][j-1] + (T[k][j-1] - T[k-1][j-1]) n_{k-j}^2 / (n_k^2 - n_{k-j}^2)
// per member and component.  The first column k >= 1 with
// max |T[k][k] - T[k][k-1]| <= tol |x| (positions) and tol |v| (velocities)
// over all members is accepted -- the same values and the same choice as
// building the columns one after another.  No accepted column: the sub-step
// is halved; accepted by column <= BS_GROW_COL: the next one is doubled.  At
// BS_MIN_FRAC the last column is accepted anyway; after BS_MAX_ATTEMPTS
// attempts or past BS_TIME_LIMIT_NS the members drift the rest of dt on
// Kepler orbits; both raise GENGA_ERR_BS.
__device__ __forceinline__ double shfl_d(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// Largest binary fraction f of |dt| with (f |dt|)^2 v2 <= r2 (a pair crosses at
// most its separation in the first sub-step); rounded products as written,
// no contraction, so the decision is the oracle's.
__device__ __forceinline__ double first_frac(double dx, double dy, double dz, double ux, double uy, double uz,
                                             double adt) {
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    const double v2 = __dadd_rn(__dadd_rn(__dmul_rn(ux, ux), __dmul_rn(uy, uy)), __dmul_rn(uz, uz));
    double f = 1.0;
    for (int it = 0; it < 40 && f > BS_MIN_FRAC; it++) {
        const double h = __dmul_rn(f, adt);
        if (!(__dmul_rn(__dmul_rn(h, h), v2) > r2)) break;
        f *= 0.5;
    }
    return f;
}

// Warp minimum of non-negative doubles, compared as integers.
__device__ __forceinline__ double warp_min_nonneg(double v) {
    long long b = __double_as_longlong(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long t = __shfl_xor_sync(0xffffffffu, b, o);
        b = t < b ? t : b;
    }
    return __longlong_as_double(b);
}

// Warp maximum of non-negative doubles, compared as integers (their bit
// patterns order like the values), off the FP64 pipe.
__device__ __forceinline__ double warp_max_nonneg(double v) {
    long long b = __double_as_longlong(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long t = __shfl_xor_sync(0xffffffffu, b, o);
        b = t > b ? t : b;
    }
    return __longlong_as_double(b);
}

__device__ __forceinline__ bool ge_nonneg(double a, double b) {  // a >= b for a, b >= 0, on the integer pipe
    return __double_as_longlong(a) >= __double_as_longlong(b);
}

// The threads that integrate one group in the workspace path, and the
// operations the path needs from them: a barrier, and reductions whose
// results do not depend on the order of combination (so both teams give the
// same values).  WarpTeam: one warp.
struct WarpTeam {
    static constexpr int T = 32;
    int t;  // lane
    __device__ void sync() const { __syncwarp(); }
    __device__ double min_nonneg(double v) const { return warp_min_nonneg(v); }
    __device__ void max_of(double *v, int cnt) const {  // fmax over the team of v[0..cnt), in place
        for (int k = 0; k < cnt; k++) v[k] = warp_max(v[k]);
    }
    __device__ int min_int(int v) const {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
        return v;
    }
    __device__ bool late(uint64_t t0) const {  // the launch's time limit, lane 0's clock
        int l = 0;
        if (t == 0) l = (global_timer_ns() - t0 > BS_TIME_LIMIT_NS) ? 1 : 0;
        return __shfl_sync(0xffffffffu, l, 0) != 0;
    }
};

// ClusterTeam: the BS_TEAM_CTAS CTAs of a thread-block cluster.  The barrier
// is the cluster barrier (release / acquire at cluster scope, which also
// orders the workspace in global memory); a reduction reduces each warp by
// shuffles, puts the warp results in its CTA's shared memory (two slots used
// alternately, so a slot is rewritten only after every thread has passed the
// next reduction's barrier) and every thread combines all warps' results
// through distributed shared memory.
struct ClusterTeam {
    static constexpr int T = BS_TEAM_CTAS * 32 * BS_WARPS;
    static constexpr int NW = BS_TEAM_CTAS * BS_WARPS;
    int t;
    double *red;  // this CTA's shared [2][BS_WARPS][BS_KMAX]
    int *redi;    // this CTA's shared [2][BS_WARPS]
    mutable unsigned k;  // reductions so far (selects the shared slot)
    __device__ void sync() const { cooperative_groups::this_cluster().sync(); }
    __device__ void max_of(double *v, int cnt) const {
        const int slot = k++ & 1, w = (threadIdx.x >> 5), lane = threadIdx.x & 31;
        for (int q = 0; q < cnt; q++) {
            const double m = warp_max(v[q]);
            if (lane == 0) red[(slot * BS_WARPS + w) * BS_KMAX + q] = m;
        }
        sync();
        auto cl = cooperative_groups::this_cluster();
        for (int r = 0; r < BS_TEAM_CTAS; r++) {
            const double *rr = cl.map_shared_rank(red, r);
            for (int ww = 0; ww < BS_WARPS; ww++)
                for (int q = 0; q < cnt; q++) {
                    const double x = rr[(slot * BS_WARPS + ww) * BS_KMAX + q];
                    v[q] = (r == 0 && ww == 0) ? x : fmax(v[q], x);  // fmax of every warp's value, as a warp does
                }
        }
    }
    __device__ double min_nonneg(double v) const {
        double b = -warp_min_nonneg(v);  // max of the negatives, via max_of on one value
        max_of(&b, 1);
        return -b;
    }
    __device__ int min_int(int v) const {
        const int slot = k++ & 1, w = (threadIdx.x >> 5), lane = threadIdx.x & 31;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) redi[slot * BS_WARPS + w] = v;
        sync();
        auto cl = cooperative_groups::this_cluster();
        int r0 = v;
        for (int r = 0; r < BS_TEAM_CTAS; r++) {
            const int *rr = cl.map_shared_rank(redi, r);
            for (int ww = 0; ww < BS_WARPS; ww++) r0 = min(r0, rr[slot * BS_WARPS + ww]);
        }
        return r0;
    }
    __device__ bool late(uint64_t t0) const {  // any warp past the time limit (its lane 0's clock)
        int l = 0;
        if ((threadIdx.x & 31) == 0) l = (global_timer_ns() - t0 > BS_TIME_LIMIT_NS) ? 1 : 0;
        l = __shfl_sync(0xffffffffu, l, 0);
        return min_int(-l) < 0;
    }
};

// Groups of up to 4 members, everything in registers: lane 8 q + k holds
// member q (q < n) for extrapolation column k; partners' positions come from
// lanes 8 p + k by shuffles.  The same arithmetic as bs_general, in the same
// order (central term, then partners in ascending body order).
__device__ void bs_small(const BSArgs &a, int s0, int n, int lane, uint64_t t0, bool &forced) {
    const int k = lane & 7, q = lane >> 3;
    const bool act = q < n;
    const int nk = 2 * (k + 1);
    double y[6] = {1.0, 0.0, 0.0, 0.0, 1.0, 0.0};  // inactive lanes: a harmless circular state
    double mq = 0.0, aq = 1.0, rcq = 1.0, Rq = 0.0;
    int tpq = 0, ghq = 0, v = -1;
    if (act) {
        v = a.gbody[s0 + q];
        const int kp = (int)a.iperm[v];
        y[0] = a.x[v]; y[1] = a.y[v]; y[2] = a.z[v];
        y[3] = a.vx[v]; y[4] = a.vy[v]; y[5] = a.vz[v];
        mq = a.m[v];
        aq = a.a_osc[kp];
        rcq = a.rc_eq1[kp];
        tpq = a.lo[kp].w != 0.f ? 1 : 0;
        ghq = signbit(mq) ? 1 : 0;  // a ghost (m = -0.0)
        if (a.radius) Rq = a.radius[v];
    }
    // partner constants (fixed over the drift, recomputed after a merger)
    double gm[4], rc2[4], lo2[4], inv9[4];
    bool use[4];
    auto partners = [&]() {
#pragma unroll
        for (int p = 0; p < 4; p++) {
            const double mp = shfl_d(mq, 8 * p), ap = shfl_d(aq, 8 * p), rcp = shfl_d(rcq, 8 * p);
            const int tpp = __shfl_sync(0xffffffffu, tpq, 8 * p), ghp = __shfl_sync(0xffffffffu, ghq, 8 * p);
            use[p] = act && p < n && p != q && !(tpq && tpp) && !ghq && !ghp;
            double rc = 1.0;
            if (use[p]) rc = pair_radius(a, mq, mp, aq, ap, rcq, rcp);
            const double rcl = rc / a.snl;  // the innermost radius: no force beyond it, all of it inside 0.1 of it
            gm[p] = a.G * mp;
            rc2[p] = rcl * rcl;
            lo2[p] = (0.1 * rcl) * (0.1 * rcl);
            inv9[p] = 1.0 / (0.9 * rc);
        }
    };
    partners();
    const double mgm = -a.G * a.Mstar;
    // level-1 acceleration of this lane's member at (x, y, z) of its column
    auto accel = [&](double x, double yy, double z, double &ax, double &ay, double &az) {
        double px[4], py[4], pz[4];
#pragma unroll
        for (int p = 0; p < 4; p++) {
            px[p] = shfl_d(x, 8 * p + k);
            py[p] = shfl_d(yy, 8 * p + k);
            pz[p] = shfl_d(z, 8 * p + k);
        }
        const double ir = rsqrt_fp64(x * x + yy * yy + z * z);
        const double c = mgm * (ir * ir * ir);
        ax = c * x;
        ay = c * yy;
        az = c * z;
        // member q's partners in ascending order: the jn-th is p = jn + (jn >= q).
        // One pass of the pair term per partner slot (n - 1 passes) instead of one
        // per member with the lanes of that member masked off (n passes: on this
        // GPU an FP64 warp instruction costs the same whatever lanes are active)
#pragma unroll
        for (int jn = 0; jn < 3; jn++) {
            if (jn >= n - 1) break;  // warp-uniform
            const int p = jn + (jn >= q ? 1 : 0);
            double sx = px[0], sy = py[0], sz = pz[0], gp = gm[0], r2p = rc2[0], l2p = lo2[0], i9p = inv9[0];
            bool up = use[0];
#pragma unroll
            for (int pp = 1; pp < 4; pp++)
                if (p == pp) {
                    sx = px[pp]; sy = py[pp]; sz = pz[pp];
                    gp = gm[pp]; r2p = rc2[pp]; l2p = lo2[pp]; i9p = inv9[pp];
                    up = use[pp];
                }
            if (!up) continue;
            const double dx = sx - x, dy = sy - yy, dz = sz - z;
            const double q2 = dx * dx + dy * dy + dz * dz;
            if (__double_as_longlong(q2) == 0 || ge_nonneg(q2, r2p)) continue;  // coincident / K = 1
            const double iq = rsqrt_fp64(q2);
            const double w = ge_nonneg(l2p, q2) ? 1.0 : bs_weight(a, q2 * iq, i9p);
            const double f = gp * w * (iq * iq * iq);
            ax = fma(f, dx, ax);
            ay = fma(f, dy, ay);
            az = fma(f, dz, az);
        }
    };
    double done = 0.0, frac;
    {  // first sub-step from the fastest interacting pair (lanes 8 q, partners p > q)
        double f = 1.0;
        double ox[6][4];
        int otp[4];
#pragma unroll
        for (int p = 0; p < 4; p++) {  // every lane takes part in the shuffles
#pragma unroll
            for (int c = 0; c < 6; c++) ox[c][p] = shfl_d(y[c], 8 * p);
            otp[p] = __shfl_sync(0xffffffffu, tpq, 8 * p);
        }
        if (act && k == 0) {
#pragma unroll
            for (int p = 1; p < 4; p++) {
                if (p <= q || p >= n || (tpq && otp[p])) continue;
                f = fmin(f, first_frac(ox[0][p] - y[0], ox[1][p] - y[1], ox[2][p] - y[2], ox[3][p] - y[3],
                                       ox[4][p] - y[4], ox[5][p] - y[5], fabs(a.dt)));
            }
        }
        frac = warp_min_nonneg(f);
    }
    for (int att = 0; att < BS_MAX_ATTEMPTS && done < 1.0; att++) {
        int late = 0;
        if (lane == 0) late = (global_timer_ns() - t0 > BS_TIME_LIMIT_NS) ? 1 : 0;
        late = __shfl_sync(0xffffffffu, late, 0);
        if (late) break;  // the rest of the drift on Kepler orbits, below
        const double h = frac * a.dt;
        const double H = h / nk;
        const double px2 = y[0] * y[0] + y[1] * y[1] + y[2] * y[2], pv2 = y[3] * y[3] + y[4] * y[4] + y[5] * y[5];
        const double isx = px2 > 0.0 ? rsqrt_fp64(px2) : 1.0, isv = pv2 > 0.0 ? rsqrt_fp64(pv2) : 1.0;
        double f0x, f0y, f0z;
        accel(y[0], y[1], y[2], f0x, f0y, f0z);
        const double f0[6] = {y[3], y[4], y[5], f0x, f0y, f0z};
        double zp[6], zc[6], T[6];
#pragma unroll
        for (int c = 0; c < 6; c++) {
            zp[c] = y[c];
            zc[c] = fma(H, f0[c], y[c]);
            T[c] = 0.0;
        }
        // The columns advance together and column kc is complete after stage
        // n_kc = 2 (kc + 1): its Neville row is built then, and the first
        // column kc >= 1 that meets the tolerance ends the stages (the later
        // columns could not change that choice).  Lane 8 q + c (c < 6) holds
        // component c of member q: the source lane of column kc sends each
        // of its six components in turn.
        const int c = k;
        const bool item = act && c < 6;
        const double isc = c < 3 ? isx : isv;
        double row[BS_KMAX];
        double pick = 0.0;  // T[kc][kc] of the last column built
        int acc_col = -1;
        for (int m = 1; m <= 2 * BS_KMAX; m++) {  // every lane evaluates (the shuffles need all lanes)
            double ax, ay, az;
            accel(zc[0], zc[1], zc[2], ax, ay, az);
            const double fv[6] = {zc[3], zc[4], zc[5], ax, ay, az};
            if (m < nk) {
#pragma unroll
                for (int c6 = 0; c6 < 6; c6++) {
                    const double zn = fma(2.0 * H, fv[c6], zp[c6]);
                    zp[c6] = zc[c6];
                    zc[c6] = zn;
                }
            } else if (m == nk) {
#pragma unroll
                for (int c6 = 0; c6 < 6; c6++) T[c6] = 0.5 * (zc[c6] + zp[c6] + H * fv[c6]);
            }
            if (m & 1) continue;
            const int kc = (m >> 1) - 1;  // warp-uniform
            double cur = 0.0;
#pragma unroll
            for (int cc = 0; cc < 6; cc++) {
                const double t = shfl_d(T[cc], 8 * q + kc);
                if (cc == c) cur = t;
            }
            double dprev = 0.0;
#pragma unroll
            for (int jn = 1; jn < BS_KMAX; jn++) {
                if (jn > kc) break;
                const double prev = row[jn - 1];  // T[kc-1][jn-1]
                row[jn - 1] = cur;                // T[kc][jn-1]
                dprev = cur;
                cur = fma(cur - prev, c_neville.c[kc * BS_KMAX + jn], cur);
            }
#pragma unroll
            for (int jj = 0; jj < BS_KMAX; jj++)
                if (jj == kc) row[jj] = cur;
            pick = cur;
            if (kc == 0) continue;
            const double e = warp_max_nonneg(item ? fabs(cur - dprev) * isc : 0.0);
            if (e <= a.tol) {
                acc_col = kc;
                break;
            }
        }
        if (acc_col < 0 && frac <= BS_MIN_FRAC) {  // pick holds the last column's T[7][7]
            acc_col = BS_KMAX - 1;
            forced = true;
        }
        if (acc_col < 0) {
            frac *= 0.5;
            continue;
        }
#pragma unroll
        for (int cc = 0; cc < 6; cc++) {
            const double nv = shfl_d(pick, 8 * q + cc);
            if (act) y[cc] = nv;
        }
        if (a.radius) {  // perfect mergers: the first overlapping pair (i < j), again until none
            for (int it = 0; it < 3; it++) {
                double ox[4], oy[4], oz[4], oR[4];
                int og[4];
#pragma unroll
                for (int p = 0; p < 4; p++) {
                    ox[p] = shfl_d(y[0], 8 * p);
                    oy[p] = shfl_d(y[1], 8 * p);
                    oz[p] = shfl_d(y[2], 8 * p);
                    oR[p] = shfl_d(Rq, 8 * p);
                    og[p] = __shfl_sync(0xffffffffu, ghq, 8 * p);
                }
                int code = 16;  // 4 i + j of the first overlapping pair, 16: none
                if (act && k == 0 && !ghq) {
#pragma unroll
                    for (int p = 3; p > 0; p--) {  // smallest j last
                        if (p <= q || p >= n || og[p]) continue;
                        const double dx = ox[p] - y[0], dy = oy[p] - y[1], dz = oz[p] - y[2];
                        const double rr = Rq + oR[p];
                        if (dx * dx + dy * dy + dz * dz < rr * rr) code = 4 * q + p;
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) code = min(code, __shfl_xor_sync(0xffffffffu, code, o));
                if (code == 16) break;
                const int fi = code >> 2, fj = code & 3;
                const double mi = shfl_d(mq, 8 * fi), mj = shfl_d(mq, 8 * fj), mt = mi + mj;
                double nyv[6];
#pragma unroll
                for (int cc = 0; cc < 6; cc++) {
                    const double u = shfl_d(y[cc], 8 * fi), w = shfl_d(y[cc], 8 * fj);
                    nyv[cc] = (mt > 0.0) ? (mi * u + mj * w) / mt : 0.5 * (u + w);
                }
                const double Ri = shfl_d(Rq, 8 * fi), Rj = shfl_d(Rq, 8 * fj);
                const double Rn = cbrt(Ri * Ri * Ri + Rj * Rj * Rj);
                if (q == fi) {
#pragma unroll
                    for (int cc = 0; cc < 6; cc++) y[cc] = nyv[cc];
                    mq = mt;
                    Rq = Rn;
                }
                if (q == fj) {
                    mq = 0.0;
                    Rq = 0.0;
                    ghq = 1;
                }
                partners();
            }
        }
        done += frac;
        if (acc_col <= BS_GROW_COL) frac *= 2.0;
        if (frac > 1.0 - done) frac = 1.0 - done;
    }
    if (done < 1.0) {  // out of attempts or time: the rest of the drift on Kepler orbits (level 0)
        forced = true;
        kepler_drift(a.G * a.Mstar, (1.0 - done) * a.dt, 50, y[0], y[1], y[2], y[3], y[4], y[5]);
    }
    if (act && k == 0) {
        a.x[v] = y[0]; a.y[v] = y[1]; a.z[v] = y[2];
        a.vx[v] = y[3]; a.vy[v] = y[4]; a.vz[v] = y[5];
        if (a.radius) {
            a.m[v] = ghq ? -0.0 : mq;
            a.radius[v] = Rq;
        }
        a.grp[v] = -1;
        a.gmark[v] = 0;
    }
}

template <class Team>
__device__ void bs_general(const BSArgs &a, int s0, int n, const Team &tm, uint64_t t0, bool &forced) {
    constexpr int T = Team::T;
    const int lane = tm.t;  // this thread's rank in the team
    const int kcol = lane & 7, qs = lane >> 3;
    const int nk = 2 * (kcol + 1);
    const Work W{a.bs, (size_t)a.slots};
    const int fz = F_Z + 18 * kcol;  // this lane's column: buffers fz + 6 b + c
    {
        const bool tab = n <= BS_PAIR_TAB;
        for (int q = lane; q < n; q += T) {
            const int s = s0 + q, v = a.gbody[s];
            const int k = (int)a.iperm[v];
            W(F_Y + 0, s) = a.x[v];
            W(F_Y + 1, s) = a.y[v];
            W(F_Y + 2, s) = a.z[v];
            W(F_Y + 3, s) = a.vx[v];
            W(F_Y + 4, s) = a.vy[v];
            W(F_Y + 5, s) = a.vz[v];
            W(F_M, s) = a.m[v];
            W(F_A, s) = a.a_osc[k];
            W(F_RC, s) = a.rc_eq1[k];
            W(F_RAD, s) = a.radius ? a.radius[v] : 0.0;
            a.tpf[s] = (a.lo[k].w != 0.f ? 1 : 0) | (signbit(a.m[v]) ? 2 : 0);
        }
        tm.sync();
        auto pair_table = [&]() {  // pair radii, fixed over the drift (masses change only in mergers)
            for (int idx = lane; idx < n * n; idx += T) {
                const int si = s0 + idx / n, ti = idx % n;
                const double rc = pair_radius(a, W(F_M, si), W(F_M, s0 + ti), W(F_A, si), W(F_A, s0 + ti),
                                              W(F_RC, si), W(F_RC, s0 + ti));
                const double rcl = rc / a.snl;
                W(F_PR2 + ti, si) = rcl * rcl;
                W(F_PIN + ti, si) = 1.0 / (0.9 * rc);
            }
            tm.sync();
        };
        if (tab) pair_table();
        double done = 0.0, frac;
        {  // first sub-step from the fastest interacting pair
            double f = 1.0;
            for (int idx = lane; idx < n * n; idx += T) {
                const int i = idx / n, j = idx % n;
                if (j <= i) continue;
                const int si = s0 + i, sj = s0 + j;
                if (a.tpf[si] & a.tpf[sj] & 1) continue;  // two test particles
                f = fmin(f, first_frac(W(F_Y, sj) - W(F_Y, si), W(F_Y + 1, sj) - W(F_Y + 1, si),
                                       W(F_Y + 2, sj) - W(F_Y + 2, si), W(F_Y + 3, sj) - W(F_Y + 3, si),
                                       W(F_Y + 4, sj) - W(F_Y + 4, si), W(F_Y + 5, sj) - W(F_Y + 5, si),
                                       fabs(a.dt)));
            }
            frac = tm.min_nonneg(f);
        }
        for (int att = 0; att < BS_MAX_ATTEMPTS && done < 1.0; att++) {
            if (tm.late(t0)) break;  // the rest of the drift on Kepler orbits, below
            const double h = frac * a.dt;
            for (int q = lane; q < n; q += T) {  // error scales and f(y)
                const int s = s0 + q;
                const double x = W(F_Y, s), y = W(F_Y + 1, s), z = W(F_Y + 2, s);
                const double u = W(F_Y + 3, s), v = W(F_Y + 4, s), w = W(F_Y + 5, s);
                const double px2 = x * x + y * y + z * z, pv2 = u * u + v * v + w * w;
                W(F_ISC, s) = px2 > 0.0 ? rsqrt_fp64(px2) : 1.0;
                W(F_ISC + 1, s) = pv2 > 0.0 ? rsqrt_fp64(pv2) : 1.0;
                double ax, ay, az;
                level1_acc(a, W, s, s0, n, F_Y, tab, ax, ay, az);
                W(F_F0, s) = ax;
                W(F_F0 + 1, s) = ay;
                W(F_F0 + 2, s) = az;
            }
            tm.sync();
            const double H = h / nk;
            for (int q = qs; q < n; q += T / 8) {  // z_0 = y, z_1 = y + H f(y), every column
                const int s = s0 + q;
                for (int c = 0; c < 6; c++) {
                    const double yc = W(F_Y + c, s);
                    const double fc = c < 3 ? W(F_Y + 3 + c, s) : W(F_F0 + c - 3, s);
                    W(fz + c, s) = yc;
                    W(fz + 6 + c, s) = fma(H, fc, yc);
                }
            }
            tm.sync();
            // stage m: z_{m+1} from z_m (m < n_k) or the smoothing step (m = n_k);
            // after m - 1 stages z_m is buffer m mod 3 and z_{m-1} buffer (m - 1) mod 3
            for (int m = 1; m <= 2 * BS_KMAX; m++) {
                if (m <= nk) {
                    const int bc = m % 3, bp = (m + 2) % 3, bn = (m + 1) % 3;
                    for (int q = qs; q < n; q += T / 8) {
                        const int s = s0 + q;
                        double ax, ay, az;
                        level1_acc(a, W, s, s0, n, fz + 6 * bc, tab, ax, ay, az);
                        const double fv[6] = {W(fz + 6 * bc + 3, s), W(fz + 6 * bc + 4, s), W(fz + 6 * bc + 5, s),
                                              ax, ay, az};
                        if (m < nk) {
                            for (int c = 0; c < 6; c++)
                                W(fz + 6 * bn + c, s) = fma(2.0 * H, fv[c], W(fz + 6 * bp + c, s));
                        } else {
                            for (int c = 0; c < 6; c++)
                                W(F_T + 6 * kcol + c, s) =
                                    0.5 * (W(fz + 6 * bc + c, s) + W(fz + 6 * bp + c, s) + H * fv[c]);
                        }
                    }
                }
                tm.sync();
            }
            // extrapolation and error per (member, component); a thread takes items lane, lane + T, ...
            double ek[BS_KMAX];
            for (int k = 0; k < BS_KMAX; k++) ek[k] = 0.0;
            for (int item = lane; item < 6 * n; item += T) {
                const int q = item / 6, c = item % 6, s = s0 + q;
                const double isc = W(F_ISC + (c < 3 ? 0 : 1), s);
                double row[BS_KMAX];   // row k of the table, in place
                double diag[BS_KMAX];  // T[k][k]
                for (int k = 0; k < BS_KMAX; k++) {
                    double cur = W(F_T + 6 * k + c, s);
                    double diag_prev = 0.0;
                    for (int j = 1; j <= k; j++) {
                        const double prev = row[j - 1];  // T[k-1][j-1]
                        row[j - 1] = cur;                // T[k][j-1]
                        diag_prev = cur;
                        cur = fma(cur - prev, c_neville.c[k * BS_KMAX + j], cur);
                    }
                    row[k] = cur;
                    diag[k] = cur;
                    if (k >= 1) ek[k] = fmax(ek[k], fabs(cur - diag_prev) * isc);
                }
                // the candidates T[k][k] stay in W(F_T) for the accepted column
                for (int k = 0; k < BS_KMAX; k++) W(F_T + 6 * k + c, s) = diag[k];
            }
            int acc_col = -1;
            tm.max_of(ek, BS_KMAX);  // every column's error over the team
            for (int k = 1; k < BS_KMAX; k++)
                if (acc_col < 0 && ek[k] <= a.tol) acc_col = k;
            tm.sync();
            if (acc_col < 0 && frac <= BS_MIN_FRAC) {
                acc_col = BS_KMAX - 1;
                forced = true;
            }
            if (acc_col < 0) {
                frac *= 0.5;
                continue;
            }
            for (int q = lane; q < n; q += T) {
                const int s = s0 + q;
                for (int c = 0; c < 6; c++) W(F_Y + c, s) = W(F_T + 6 * acc_col + c, s);
            }
            tm.sync();
            if (a.radius) {  // perfect mergers: the first overlapping pair (i < j), again until none
                for (int it = 0; it < n - 1; it++) {
                    int code = n * n;  // i n + j of the first overlapping pair
                    for (int idx = lane; idx < n * n; idx += T) {
                        const int i = idx / n, j = idx % n;
                        if (j <= i) continue;
                        const int si = s0 + i, sj = s0 + j;
                        if ((a.tpf[si] | a.tpf[sj]) & 2) continue;
                        const double dx = W(F_Y, sj) - W(F_Y, si), dy = W(F_Y + 1, sj) - W(F_Y + 1, si);
                        const double dz = W(F_Y + 2, sj) - W(F_Y + 2, si);
                        const double rr = W(F_RAD, si) + W(F_RAD, sj);
                        if (dx * dx + dy * dy + dz * dz < rr * rr) code = min(code, idx);
                    }
                    code = tm.min_int(code);
                    if (code == n * n) break;
                    const int si = s0 + code / n, sj = s0 + code % n;
                    if (lane == 0) {  // the team's first thread
                        const double mi = W(F_M, si), mj = W(F_M, sj), mt = mi + mj;
                        for (int c = 0; c < 6; c++) {
                            const double u = W(F_Y + c, si), w = W(F_Y + c, sj);
                            W(F_Y + c, si) = (mt > 0.0) ? (mi * u + mj * w) / mt : 0.5 * (u + w);
                        }
                        const double Ri = W(F_RAD, si), Rj = W(F_RAD, sj);
                        W(F_RAD, si) = cbrt(Ri * Ri * Ri + Rj * Rj * Rj);
                        W(F_M, si) = mt;
                        W(F_M, sj) = 0.0;
                        W(F_RAD, sj) = 0.0;
                        a.tpf[sj] |= 2;
                    }
                    tm.sync();
                    if (tab) pair_table();
                }
            }
            done += frac;
            if (acc_col <= BS_GROW_COL) frac *= 2.0;
            if (frac > 1.0 - done) frac = 1.0 - done;
        }
        if (done < 1.0) {  // out of attempts or time: the rest of the drift on Kepler orbits (level 0)
            forced = true;
            for (int q = lane; q < n; q += T) {
                const int s = s0 + q;
                double px = W(F_Y, s), py = W(F_Y + 1, s), pz = W(F_Y + 2, s);
                double u = W(F_Y + 3, s), vv = W(F_Y + 4, s), w = W(F_Y + 5, s);
                kepler_drift(a.G * a.Mstar, (1.0 - done) * a.dt, 50, px, py, pz, u, vv, w);
                W(F_Y, s) = px; W(F_Y + 1, s) = py; W(F_Y + 2, s) = pz;
                W(F_Y + 3, s) = u; W(F_Y + 4, s) = vv; W(F_Y + 5, s) = w;
            }
            tm.sync();
        }
        for (int q = lane; q < n; q += T) {
            const int s = s0 + q, v = a.gbody[s];
            a.x[v] = W(F_Y, s);
            a.y[v] = W(F_Y + 1, s);
            a.z[v] = W(F_Y + 2, s);
            a.vx[v] = W(F_Y + 3, s);
            a.vy[v] = W(F_Y + 4, s);
            a.vz[v] = W(F_Y + 5, s);
            if (a.radius) {
                a.m[v] = (a.tpf[s] & 2) ? -0.0 : W(F_M, s);
                a.radius[v] = W(F_RAD, s);
            }
            a.grp[v] = -1;
            a.gmark[v] = 0;
        }
    }
}

// Members of group (s0, n) in ascending body order (the order of every sum),
// by the threads t = 0, T, 2T, ... of a team.
__device__ __forceinline__ void sort_members(const BSArgs &a, int s0, int n, int t, int T) {
    for (int q = t; q < n; q += T) {
        const int v = a.gmem[s0 + q];
        int rank = 0;
        for (int r = 0; r < n; r++) rank += (a.gmem[s0 + r] < v) ? 1 : 0;
        a.gbody[s0 + rank] = v;
    }
}

// Launched as clusters of BS_TEAM_CTAS CTAs.  First every group of more than
// BS_TEAM_MIN members, one cluster per group (the k-th such group goes to
// cluster k mod clusters), on the workspace path with the cluster as its
// team; then every other group on one warp: the register path (n <= 4) or
// the workspace path.
__global__ void __cluster_dims__(BS_TEAM_CTAS, 1, 1) __launch_bounds__(32 * BS_WARPS, 2)
    bs_kernel(const __grid_constant__ BSArgs a) {
    static_assert(BS_KMAX == 8, "lane = 8 * member slice + column");
    __shared__ double s_red[2 * BS_WARPS * BS_KMAX];
    __shared__ int s_redi[2 * BS_WARPS];
    const int lane = threadIdx.x & 31;
    const int ng = *a.gcount;
    uint64_t t0 = 0;  // the time limit holds for the whole launch, however many groups a warp takes
    if (lane == 0) t0 = global_timer_ns();
    {
        auto cl = cooperative_groups::this_cluster();
        ClusterTeam tm{(int)cl.block_rank() * 32 * BS_WARPS + (int)threadIdx.x, s_red, s_redi, 0u};
        const int ncl = (int)(gridDim.x / BS_TEAM_CTAS), cid = (int)(blockIdx.x / BS_TEAM_CTAS);
        int big = 0;
        for (int g0 = 0; g0 < ng; g0 += 32) {  // every warp finds the same large groups
            const bool large = g0 + lane < ng && a.gsize[g0 + lane] > BS_TEAM_MIN;
            unsigned m = __ballot_sync(0xffffffffu, large);
            while (m) {
                const int g = g0 + __ffs((int)m) - 1;
                m &= m - 1u;
                if (big++ % ncl != cid) continue;
                const int s0 = a.gstart[g], n = a.gsize[g];
                sort_members(a, s0, n, tm.t, ClusterTeam::T);
                tm.sync();
                bool forced = false;
                bs_general(a, s0, n, tm, t0, forced);
                if (forced && tm.t == 0) atomicOr(a.status, GENGA_BIT(GENGA_ERR_BS));
                tm.sync();
            }
        }
    }
    const int gw = blockIdx.x * BS_WARPS + (threadIdx.x >> 5), nw = gridDim.x * BS_WARPS;
    const WarpTeam wt{lane};
    for (int g = gw; g < ng; g += nw) {
        const int s0 = a.gstart[g], n = a.gsize[g];
        if (n > BS_TEAM_MIN) continue;
        sort_members(a, s0, n, lane, 32);
        __syncwarp();
        bool forced = false;
        if (n <= 4) bs_small(a, s0, n, lane, t0, forced);
        else bs_general(a, s0, n, wt, t0, forced);
        if (forced && lane == 0) atomicOr(a.status, GENGA_BIT(GENGA_ERR_BS));
        __syncwarp();
    }
}

}  // namespace

cudaError_t launch_groups(const GroupArgs &g, cudaStream_t s) {
    group_kernel<<<1, GROUP_THREADS, 0, s>>>(g);
    return cudaGetLastError();
}

// Clusters of the level-1 kernel resident at once (queried when a context is
// created, outside any capture; one GPU model per process).
int g_bs_clusters = 0;

cudaError_t init_bs_kernel(int sm_count) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((2 * sm_count) / BS_TEAM_CTAS * BS_TEAM_CTAS));
    cfg.blockDim = dim3(32 * BS_WARPS);
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, (void *)bs_kernel, &cfg) != cudaSuccess) {
        cudaGetLastError();  // not fatal: one cluster at a time still runs every group
        ncl = 1;
    }
    g_bs_clusters = ncl > 0 ? ncl : 1;
    return cudaSuccess;
}

cudaError_t launch_bs(const BSArgs &b, int sm_count, cudaStream_t s) {
    // as many clusters as are resident at once (the kernel hands out its
    // groups statically, so a second wave of CTAs would run after the first),
    // at most two CTAs per SM
    const int resident = g_bs_clusters > 0 ? g_bs_clusters : 1;
    const int grid = std::min(resident, (2 * sm_count) / BS_TEAM_CTAS) * BS_TEAM_CTAS;
    bs_kernel<<<grid > 0 ? grid : BS_TEAM_CTAS, 32 * BS_WARPS, 0, s>>>(b);
    return cudaGetLastError();
}

}  // namespace genga
