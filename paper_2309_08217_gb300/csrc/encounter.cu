// encounter.cu -- the close-encounter level of the hybrid step (Sect. 1:
// level 1, the Bulirsch-Stoer integrator that takes over from the Kepler
// drift for bodies in close encounters; the changeover function splits each
// pair force between the kick and this level).
//
//   groups     the connected components of the encounter pairs of the step's
//              first kick (one CTA: hook-and-compress union-find over the
//              pairs, then the members of each group stored contiguously)
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
//
// The drift kernel skips the members (grp[i] >= 0): they get the central-
// body momentum drift only, and this level moves them over dt in between
// the two momentum drifts.  Everything here is FP64 (Sect. 1, last paragraph:
// close-encounter forces are always double precision).
#include "internal.cuh"

namespace genga {

namespace {

constexpr int GROUP_THREADS = 1024;
constexpr int GROUP_MAX_ROUNDS = 256;  // hook-and-compress rounds (a chain of n bodies needs about log2 n)

constexpr int BS_KMAX = 8;             // extrapolation columns: midpoint step counts 2, 4, ..., 16
constexpr int BS_GROW_COL = 2;         // a sub-step accepted by column <= 2 doubles the next one
constexpr double BS_MIN_FRAC = 0x1p-30;  // smallest sub-step, as a fraction of the drift
constexpr int BS_MAX_ATTEMPTS = 4096;  // sub-step attempts per group and drift
constexpr int BS_WARPS = 4;            // groups in flight per CTA (one warp each)
// Wall-clock bound of one group's integration; past it the rest of the drift
// is taken as one forced sub-step (GENGA_ERR_BS).
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

// One CTA.  In: the encounter pairs (body indices < N).  Out: gcount groups;
// group g has gsize[g] members gmem[gstart[g] ..] (in no particular order),
// grp[v] = the smallest body of v's group for every member (-1 elsewhere),
// gmark[v] = 1 for every member.  More members than `slots`: no groups, the
// marks are cleared again and GENGA_ERR_BS is raised (the bodies then get the
// plain Kepler drift).
__global__ void __launch_bounds__(GROUP_THREADS) group_kernel(const __grid_constant__ GroupArgs a) {
    __shared__ int s_flag, s_nmem, s_ngroups;
    __shared__ int warp_sums[32];
    const int tid = threadIdx.x;
    const int np = min(*a.enc_count, a.enc_cap);
    if (tid == 0) {
        s_nmem = 0;
        s_ngroups = 0;
    }
    // 1. every body of a pair starts as its own group
    for (int p = tid; p < np; p += GROUP_THREADS) {
        const int2 e = a.enc[p];
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
            const int2 e = a.enc[p];
            if (e.x < 0 || e.y < 0 || e.x >= a.N || e.y >= a.N) continue;
            const int li = ld_cg(a.grp + e.x), lj = ld_cg(a.grp + e.y);
            if (li != lj) {
                atomicMin(a.grp + max(li, lj), min(li, lj));
                s_flag = 1;
            }
        }
        __syncthreads();
        for (int p = tid; p < np; p += GROUP_THREADS) {
            const int2 e = a.enc[p];
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
        const int2 e = a.enc[p];
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
            const int2 e = a.enc[p];
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

// Changeover weight K(y) of the kick (Sect. 1): 0 for y <= 0, 1 for y >= 1.
__device__ __forceinline__ double changeover_weight(double y, int form) {
    if (y <= 0.0) return 0.0;
    if (y >= 1.0) return 1.0;
    if (form == GENGA_K_CHAMBERS) {
        const double y2 = y * y;
        return y2 / (2.0 * y2 - 2.0 * y + 1.0);
    }
    return y * y * y * (10.0 + y * (6.0 * y - 15.0));
}

// Scratch fields of the level-1 workspace, each `slots` doubles (slot = the
// member's position in gmem/gbody):
enum : int {
    F_Y = 0,                       // accepted state x, y, z, vx, vy, vz
    F_Z = 6,                       // three rotating midpoint states (6 fields each)
    F_F0 = F_Z + 18,               // acceleration at the accepted state
    F_T = F_F0 + 3,                // extrapolation row, BS_KMAX x 6 fields
    F_SC = F_T + 6 * BS_KMAX,      // error scales |x|, |v| of the sub-step
    F_M = F_SC + 2,                // mass
    F_A = F_M + 1,                 // osculating a of the first kick
    F_RC = F_A + 1,                // Eq. 1 radius of the first kick
    F_COUNT = F_RC + 1
};
static_assert(F_COUNT == GENGA_BS_FIELDS, "level-1 workspace fields");

struct Work {  // field f of slot s: base[f * stride + s]
    double *base;
    size_t stride;
    __device__ __forceinline__ double *f(int field) const { return base + (size_t)field * stride; }
    __device__ __forceinline__ double &operator()(int field, int s) const { return base[(size_t)field * stride + s]; }
};

// Level-1 acceleration of the member in slot s with the positions of buffer
// field p (fields p, p+1, p+2); members in slots [s0, s0 + n).
__device__ void level1_acc(const BSArgs &a, const Work &W, int s, int s0, int n, int p, double &ax, double &ay,
                           double &az) {
    const double *__restrict__ px = W.f(p);
    const double *__restrict__ py = W.f(p + 1);
    const double *__restrict__ pz = W.f(p + 2);
    const double *__restrict__ M = W.f(F_M);
    const double *__restrict__ A = W.f(F_A);
    const double *__restrict__ RC = W.f(F_RC);
    const double xi = px[s], yi = py[s], zi = pz[s];
    const double r2 = xi * xi + yi * yi + zi * zi;
    const double r = sqrt(r2);
    const double c = -a.G * a.Mstar / (r2 * r);
    ax = c * xi;
    ay = c * yi;
    az = c * zi;
    const bool tpi = a.tpf[s] != 0;
    const double mi = M[s], ai = A[s], rci = RC[s];
    for (int t = s0; t < s0 + n; t++) {
        if (t == s || (tpi && a.tpf[t] != 0)) continue;
        const double dx = px[t] - xi, dy = py[t] - yi, dz = pz[t] - zi;
        const double q2 = dx * dx + dy * dy + dz * dz;
        if (q2 == 0.0) continue;
        const double q = sqrt(q2);
        const double rc = (a.rcrit_mode == GENGA_RCRIT_EQ1)
                              ? fmax(rci, RC[t])
                              : a.n1 * cbrt((mi + M[t]) / (3.0 * a.Mstar)) * 0.5 * (ai + A[t]);
        if (q >= rc) continue;  // K = 1: the kick has all of it
        const double w = 1.0 - changeover_weight((q / rc - 0.1) / 0.9, a.changeover);
        const double f = a.G * M[t] * w / (q2 * q);
        ax += f * dx;
        ay += f * dy;
        az += f * dz;
    }
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// One warp per group.  Sub-steps are fractions of dt (exact binary values):
// each runs the modified midpoint rule with n_k = 2 (k + 1) steps,
//   z_0 = y, z_1 = z_0 + H f(z_0), z_{m+1} = z_{m-1} + 2H f(z_m),
//   T[k][0] = (z_n + z_{n-1} + H f(z_n)) / 2,
// and the Aitken-Neville table
//   T[k][j] = T[k][j-1] + (T[k][j-1] - T[k-1][j-1]) n_{k-j}^2 / (n_k^2 - n_{k-j}^2);
// column k >= 1 is accepted when max |T[k][k] - T[k][k-1]| <= tol |x| (position
// components) and tol |v| (velocity components) for every member.  No
// accepted column: the sub-step is halved; accepted by column <= BS_GROW_COL:
// the next one is doubled.  At BS_MIN_FRAC, at the last of BS_MAX_ATTEMPTS
// attempts (which takes the rest of dt) or past BS_TIME_LIMIT_NS the last
// column is accepted anyway and GENGA_ERR_BS is raised.  Only row k of the
// table is kept: T[k][j-1] overwrites T[k-1][j-1] once T[k][j] is formed.
__global__ void __launch_bounds__(32 * BS_WARPS) bs_kernel(const __grid_constant__ BSArgs a) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * BS_WARPS + (threadIdx.x >> 5), nw = gridDim.x * BS_WARPS;
    const int ng = *a.gcount;
    const Work W{a.bs, (size_t)a.slots};
    for (int g = gw; g < ng; g += nw) {
        const int s0 = a.gstart[g], n = a.gsize[g];
        // members in ascending body order (the order of every sum below)
        for (int q = lane; q < n; q += 32) {
            const int v = a.gmem[s0 + q];
            int rank = 0;
            for (int r = 0; r < n; r++) rank += (a.gmem[s0 + r] < v) ? 1 : 0;
            a.gbody[s0 + rank] = v;
        }
        __syncwarp();
        for (int q = lane; q < n; q += 32) {
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
            a.tpf[s] = a.lo[k].w != 0.f ? 1 : 0;
        }
        __syncwarp();
        uint64_t t0 = 0;
        if (lane == 0) t0 = global_timer_ns();
        double done = 0.0, frac = 1.0;
        bool forced = false;
        for (int att = 0; att < BS_MAX_ATTEMPTS && done < 1.0; att++) {
            int late = 0;
            if (lane == 0) late = (global_timer_ns() - t0 > BS_TIME_LIMIT_NS) ? 1 : 0;
            late = __shfl_sync(0xffffffffu, late, 0);
            const bool last = (att == BS_MAX_ATTEMPTS - 1) || late;
            if (last) frac = 1.0 - done;
            const double h = frac * a.dt;
            for (int q = lane; q < n; q += 32) {  // error scales and f(y)
                const int s = s0 + q;
                const double x = W(F_Y, s), y = W(F_Y + 1, s), z = W(F_Y + 2, s);
                const double u = W(F_Y + 3, s), v = W(F_Y + 4, s), w = W(F_Y + 5, s);
                const double px = sqrt(x * x + y * y + z * z), pv = sqrt(u * u + v * v + w * w);
                W(F_SC, s) = px > 0.0 ? px : 1.0;
                W(F_SC + 1, s) = pv > 0.0 ? pv : 1.0;
                double ax, ay, az;
                level1_acc(a, W, s, s0, n, F_Y, ax, ay, az);
                W(F_F0, s) = ax;
                W(F_F0 + 1, s) = ay;
                W(F_F0 + 2, s) = az;
            }
            __syncwarp();
            int acc_col = -1;
            for (int k = 0; k < BS_KMAX; k++) {
                const int nsub = 2 * (k + 1);
                const double H = h / nsub;
                for (int q = lane; q < n; q += 32) {  // z_0 = y, z_1 = y + H f(y)
                    const int s = s0 + q;
                    for (int c = 0; c < 6; c++) {
                        const double yc = W(F_Y + c, s);
                        const double fc = c < 3 ? W(F_Y + 3 + c, s) : W(F_F0 + c - 3, s);
                        W(F_Z + c, s) = yc;
                        W(F_Z + 6 + c, s) = yc + H * fc;
                    }
                }
                __syncwarp();
                int bp = 0, bc = 1, bn = 2;
                for (int mstep = 1; mstep < nsub; mstep++) {
                    for (int q = lane; q < n; q += 32) {
                        const int s = s0 + q;
                        double ax, ay, az;
                        level1_acc(a, W, s, s0, n, F_Z + 6 * bc, ax, ay, az);
                        for (int c = 0; c < 6; c++) {
                            const double fc = c < 3 ? W(F_Z + 6 * bc + 3 + c, s) : (c == 3 ? ax : (c == 4 ? ay : az));
                            W(F_Z + 6 * bn + c, s) = W(F_Z + 6 * bp + c, s) + 2.0 * H * fc;
                        }
                    }
                    __syncwarp();
                    const int t = bp;
                    bp = bc;
                    bc = bn;
                    bn = t;
                }
                double err = 0.0;
                for (int q = lane; q < n; q += 32) {  // smoothing step, extrapolation, error
                    const int s = s0 + q;
                    double ax, ay, az;
                    level1_acc(a, W, s, s0, n, F_Z + 6 * bc, ax, ay, az);
                    const double sx = W(F_SC, s), sv = W(F_SC + 1, s);
                    for (int c = 0; c < 6; c++) {
                        const double fc = c < 3 ? W(F_Z + 6 * bc + 3 + c, s) : (c == 3 ? ax : (c == 4 ? ay : az));
                        double cur = 0.5 * (W(F_Z + 6 * bc + c, s) + W(F_Z + 6 * bp + c, s) + H * fc);
                        for (int j = 1; j <= k; j++) {
                            const double nk = nsub, nkj = 2 * (k - j + 1);
                            const double cf = (nkj * nkj) / (nk * nk - nkj * nkj);
                            double &slot = W(F_T + 6 * (j - 1) + c, s);
                            const double prev = slot;  // T[k-1][j-1]
                            slot = cur;                // T[k][j-1]
                            cur = cur + (cur - prev) * cf;
                        }
                        W(F_T + 6 * k + c, s) = cur;
                        if (k >= 1) err = fmax(err, fabs(cur - W(F_T + 6 * (k - 1) + c, s)) / (c < 3 ? sx : sv));
                    }
                }
                err = warp_max(err);
                __syncwarp();
                if (k >= 1 && err <= a.tol) {
                    acc_col = k;
                    break;
                }
            }
            if (acc_col < 0 && (frac <= BS_MIN_FRAC || last)) {
                acc_col = BS_KMAX - 1;
                forced = true;
            }
            if (acc_col < 0) {
                frac *= 0.5;
                continue;
            }
            for (int q = lane; q < n; q += 32) {
                const int s = s0 + q;
                for (int c = 0; c < 6; c++) W(F_Y + c, s) = W(F_T + 6 * acc_col + c, s);
            }
            __syncwarp();
            done += frac;
            if (acc_col <= BS_GROW_COL) frac *= 2.0;
            if (frac > 1.0 - done) frac = 1.0 - done;
        }
        for (int q = lane; q < n; q += 32) {
            const int s = s0 + q, v = a.gbody[s];
            a.x[v] = W(F_Y, s);
            a.y[v] = W(F_Y + 1, s);
            a.z[v] = W(F_Y + 2, s);
            a.vx[v] = W(F_Y + 3, s);
            a.vy[v] = W(F_Y + 4, s);
            a.vz[v] = W(F_Y + 5, s);
            a.grp[v] = -1;
            a.gmark[v] = 0;
        }
        if (forced && lane == 0) atomicOr(a.status, GENGA_BIT(GENGA_ERR_BS));
        __syncwarp();
    }
}

}  // namespace

cudaError_t launch_groups(const GroupArgs &g, cudaStream_t s) {
    group_kernel<<<1, GROUP_THREADS, 0, s>>>(g);
    return cudaGetLastError();
}

cudaError_t launch_bs(const BSArgs &b, int sm_count, cudaStream_t s) {
    bs_kernel<<<2 * sm_count, 32 * BS_WARPS, 0, s>>>(b);
    return cudaGetLastError();
}

}  // namespace genga
