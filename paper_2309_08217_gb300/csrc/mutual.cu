// mutual.cu -- the mutual (symmetric) long-range passes of the kick, FP32
// and FP64 (Sect. 1, the single-precision long-range forces and the FP64
// kick they are measured against):
//
//   a_i = sum_{j != i} G m_j K(y_ij) (x_j - x_i) / r_ij^3
//
// evaluated once per unordered pair {i, j}: the pair's inverse cube serves
// both bodies, a_i += G m_j r^-3 (x_j - x_i) and a_j += G m_i r^-3 (x_i - x_j)
// (Newton's third law), so a pair costs 16 FP32 operations for two
// interactions instead of 12 for one.  The sums and their tolerances are
// those of the one-sided passes in kick.cu; only the order of the
// evaluation changes.  One plan and kernel serve a single disc and a batch
// of independent discs (a table of systems).
//
// Layout.  Bodies in the spatial (Morton) order, 64-body groups.  A CTA has
// CW consumer warps, one producer warp and three reducer warps.  A CTA's
// i-block is CW NP groups; consumer warp w holds NP of them in registers,
// interleaved over the block (groups w, w + CW, w + 2 CW, ...: a j-group
// next to one part of the block is then near one i-group of several warps,
// not of one warp only); packed register q holds bodies l and l + 32 of its
// group q (lane l).  The producer stages one
// 64-body j-group per ring slot (bulk copies completed on an mbarrier).  In a
// slot, lane l takes j-body (l + t) mod 32 at step t of a 32-step rotation:
// it adds the pair's i-side terms to its own i-sums and the j-side terms to a
// running j-sum that then moves one lane down (shuffle), so after 32 steps
// every j-sum is back in the lane of its j-body, complete over the warp's
// i-tile.  The reducer warps add the CW warps' j-sums of a slot in warp
// order (double-float) into the j-side partial row of the item's i-block,
// each a third of the (half, component) sums (so no scheduler of the SM
// carries the whole reduction), then free the slot; so every sum has a
// fixed order and results are bitwise reproducible.
//
// Work.  Items come from a table built on the host (plan_systems): the
// diagonal items of each i-block (its own groups, one-sided: every warp takes
// its i-groups against a range of the block's groups, each ordered pair from
// its i-side, the self pair screened out), then chunks of each block's strip
// (the groups of its system after the block, both sides), longest first, a
// tail of single-group items last.  A persistent grid takes items from a
// global counter; a CTA's producer claims its next item only when the
// leading consumer warp is close to the end of its queued slots.
//
// Precision.  Offsets come from positions relative to the centre c of the
// j-group: X_j = fl32(x_j - c) (the FP64 difference rounded, computed by the
// prep kernel) and X_i = fl32(fl32(x_i,hi - c) + x_i,lo).  A group is FAR for
// an i-tile when every pair is beyond both the r_crit bound and the group's
// precision distance (a tenth of its half-diagonal h), so the offset
// X_j - X_i is within 3 u (1 + 10) relative of x_j - x_i (u = 2^-24): there
// the pair terms need no screening.  Otherwise (NEAR) the offsets carry the
// exact residuals, every pair is compared with an FP32 upper bound of
// r_crit,ij^2, and the pairs under it are evaluated exactly in FP64
// afterwards (K-weighted, both sides, encounter list) -- close-encounter
// forces are always FP64 (Sect. 1).
// i-sums: FP32 per slot, folded every 2 slots into double-float per-body
// sums in shared memory, written as the item's i-row at its end.
#include <algorithm>
#include <cmath>
#include <functional>
#include <new>
#include <queue>
#include <vector>

#include "internal.cuh"
#include "pass_common.cuh"

namespace genga {

constexpr int MC_WAYS = 16;        // single-system plans kept per variant (one per padded length)
constexpr int MC_BATCH_WAYS = 4;   // batch plans kept per variant (one per batch layout)

struct MutualCache {            // host-built plans per variant slot
    struct Entry {
        unsigned long long key = ~0ull;  // the padded length (single systems) or the batch layout hash
        unsigned long long used = 0;     // last use (the least recently used entry is replaced)
        bool ok = false;  // false: no plan fits: one-sided passes instead
        int nb = 0, gpb = 0, items = 0, nsys = 0;
        int4 *d_item = nullptr;
        int2 *d_blk = nullptr;
        int32_t *d_bsys = nullptr;
        MSys *d_sys = nullptr;
    };
    Entry e[GENGA_MAX_VARIANTS][MC_WAYS];         // single systems: FP32 variants, then FP64 ones
    Entry eb[GENGA_MAX_VARIANTS][MC_BATCH_WAYS];  // batches: FP32 variants
    unsigned long long tick = 0;
};

namespace {

constexpr int MG = 64;           // bodies per staged j-group
constexpr int MUTUAL_MAX_ROWS = 192;  // partial rows a mutual plan may use (its workspace grows to them)
constexpr int M_FOLD = 2;        // slots between folds of the FP32 i-sums into double-float (2: max error 8e-6 at 200k bodies, 1.3e-5 with 4)
constexpr int NEAR_SPEC_NP = 2;  // NEAR loops specialised per set of NEAR i-groups up to this NP (NP = 3 measured slower overall)
constexpr int M_CLAIM = 3;       // a producer claims an item when the leading warp has at most M_CLAIM - 1 slots left

struct MHdr {
    int item, group, flags, pad;  // flags: 1 first slot of the item, 2 last, 4 no more work
};

// J += S.lo D.lo + S.hi D.hi: a j-body's terms from the two i-bodies of a
// packed register, in one scalar running sum (one shuffle per component and
// step instead of two; the same FMA-pipe cycles as one packed FMA)
__device__ __forceinline__ void jsum(float &J, f32x2 S, f32x2 D) {
    float s0, s1, d0, d1;
    up2(S, s0, s1);
    up2(D, d0, d1);
    J = fmaf(s1, d1, fmaf(s0, d0, J));
}

// Wait until the leading consumer warp has finished `target` slots, bounded
// like the mbarrier waits (a progress hint: no data passes through it).
__device__ __forceinline__ bool wait_lead(const unsigned *lead, unsigned target, uint32_t *status,
                                          uint64_t limit_ns) {
    if (*(volatile const unsigned *)lead >= target) return true;
    const uint64_t t0 = global_timer_ns();
    while (*(volatile const unsigned *)lead < target) {
        if (global_timer_ns() - t0 > limit_ns) {
            atomicOr(status, GENGA_BIT(GENGA_ERR_TIMEOUT));
            return false;
        }
        __nanosleep(32);
    }
    return true;
}

// f(integral_constant<unsigned, m>) for the run-time value m in [M, MAXM].
template <unsigned M, unsigned MAXM, class F>
__device__ __forceinline__ void dispatch_mask(unsigned m, F &f) {
    if constexpr (M <= MAXM) {
        if (m == M) {
            f(std::integral_constant<unsigned, M>{});
            return;
        }
        dispatch_mask<M + 1, MAXM>(m, f);
    }
}

__device__ __forceinline__ f32x2 rsq2(f32x2 r2) {
    float a, b;
    up2(r2, a, b);
    return pk2(rsqrt_sfu(a), rsqrt_sfu(b));
}

// True when every pair between box u (an i-tile) and box v (a j-group) is
// beyond the r_crit bound and beyond the group's precision distance.
__device__ __forceinline__ bool far_mutual(const Box &u, const Box &v, float prec) {
    if (u.lo.x > u.hi.x || v.lo.x > v.hi.x) return true;  // an empty box: no real body on that side
    const float gx = fmaxf(0.f, fmaxf(v.lo.x - u.hi.x, u.lo.x - v.hi.x));
    const float gy = fmaxf(0.f, fmaxf(v.lo.y - u.hi.y, u.lo.y - v.hi.y));
    const float gz = fmaxf(0.f, fmaxf(v.lo.z - u.hi.z, u.lo.z - v.hi.z));
    const float gap2 = gx * gx + gy * gy + gz * gz;
    const float need = fmaxf(fmaxf(u.lo.w, v.lo.w) * fmaxf(u.hi.w, v.hi.w) * (1.0f + 0x1p-10f), prec);
    return gap2 > need * need;
}

// x - c = X + residual to ~u^2, where X = fl(fl(xh - c) + xl) is the value
// the packed loop uses: the rounding error of xh - c (two-sum) plus that of
// the second addition.
__device__ __forceinline__ float centred_residual(float xh, float xl, float c, float X) {
    const float t = xh - c;
    const float bp = t - xh;
    const float e = (xh - (t - bp)) + (-c - bp);
    return e + ((t - X) + xl);
}

// The exact FP64 treatment of a screened pair (packed positions i, j of one
// system whose packed range starts at poff, Nd bodies from caller index off):
// the K-weighted terms on i (fi) and on j (fj).  The encounter pair and the
// predicted entry are recorded as (smaller, larger) body index -- for every
// visit when `both` (the pass visits the pair once), else only from the side
// with the smaller index (the one-sided own tile visits it twice).  Ghosts
// (mass -0.0) are never pairs.
__device__ __noinline__ void screened_pair_mutual(const PassArgs &a, int i, int j, int poff, int Nd, int off,
                                                  bool both, double3 *fi, double3 *fj) {
    *fi = *fj = make_double3(0.0, 0.0, 0.0);
    if (i - poff >= Nd || j - poff >= Nd || i == j) return;
    const double4_32a pi = a.p64[i], pj = a.p64[j];
    const double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
    const double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 == 0.0) return;  // coincident bodies: no direction, no force
    const double r = sqrt(r2);
    const int oi = (int)a.perm[off + i - poff], oj = (int)a.perm[off + j - poff];
    double rc;
    if (a.rcrit_mode == GENGA_RCRIT_EQ1) {
        rc = fmax(a.rc_eq1[i], a.rc_eq1[j]);
    } else {
        rc = a.n1 * cbrt((a.m[oi] + a.m[oj]) / (3.0 * a.Mstar)) * 0.5 * (a.a_osc[i] + a.a_osc[j]);
    }
    const bool record = both || oi < oj;
    const bool ghost = signbit(a.m[oi]) || signbit(a.m[oj]);
    const int lo = oi < oj ? oi : oj, hi = oi < oj ? oj : oi;
    double K = 1.0;
    if (r < rc) {
        if (record && !ghost) {
            const int pos = atomicAdd(a.enc_count, 1);
            if (pos < a.enc_cap) a.enc[pos] = make_int2(lo, hi);
        }
        K = changeover_K((r / rc - 0.1) / 0.9, a.changeover);
    } else if (a.predict && record && r < GENGA_PREDICT_RANGE * rc && !ghost) {
        // straight-line relative motion over the coming drift (rounded
        // products as written, no contraction; the test is the same from
        // either side)
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
            if (pos < a.enc_cap) a.pred[pos] = make_int2(lo, hi);
        }
    }
    if (K == 0.0) return;
    const double s = K / (r2 * r);
    const double si = pj.w * s, sj = -pi.w * s;
    *fi = make_double3(si * dx, si * dy, si * dz);
    *fj = make_double3(sj * dx, sj * dy, sj * dz);
}

template <int NP, int CW, int STAGES>
struct MLayout {
    static constexpr int BPT = 2 * NP, NC = CW * 32;
    static constexpr size_t r_off = 0;                                         // float4 [STAGES][MG]
    static constexpr size_t l_off = r_off + (size_t)STAGES * MG * 16;          // float4 [STAGES][MG]
    static constexpr size_t g_off = l_off + (size_t)STAGES * MG * 16;          // float4 [STAGES][4]
    static constexpr size_t p_off = g_off + (size_t)STAGES * 4 * 16;           // float [STAGES][CW][3][MG]
    static constexpr size_t a_off = p_off + (size_t)STAGES * CW * 3 * MG * 4;  // DF [3][BPT][NC]
    static constexpr size_t i_off = a_off + (size_t)3 * BPT * NC * 8;          // float4 [2][BPT][NC]
    static constexpr size_t q_off = i_off + (size_t)2 * BPT * NC * 16;         // float4 [CW][NP][2]
    static constexpr size_t m_off = q_off + (size_t)CW * NP * 2 * 16;          // uint32 [BPT][NC]
    static constexpr size_t e_off = m_off + (size_t)BPT * NC * 4;              // f32x2 [NP][3][NC]
    static constexpr size_t b_off = e_off + (size_t)NP * 3 * NC * 8;           // uint64 [3][STAGES]
    static constexpr size_t h_off = b_off + (size_t)3 * STAGES * 8;            // MHdr [STAGES]
    static constexpr size_t bytes = h_off + (size_t)STAGES * sizeof(MHdr);
    static_assert(bytes <= 227 * 1024, "one CTA per SM: at most 227 KB of shared memory");
};

// Registers per thread: as many as one CTA of `warps` warps per SM allows; a
// block's warps take registers in units of 4 warps (measured: 14 warps of 144
// registers do not launch), so the count is that of the next multiple of 4.
constexpr int mutual_maxreg(int warps) {
    return ((65536 / (((warps + 3) / 4) * 4 * 32)) / 8 * 8) > 255 ? 255
                                                                  : ((65536 / (((warps + 3) / 4) * 4 * 32)) / 8 * 8);
}

// NR reducer warps (warps CW + 1 ...): reducer r sums the (half, component)
// j-sums r, r + NR, ... of a slot, so with NR = 3 the reduction is spread
// over three of the SM's four schedulers instead of loading one.
template <int NP, int CW, int STAGES, int UNR, int NR>
__global__ void __maxnreg__(mutual_maxreg(CW + 1 + NR)) pass_mutual_kernel(const __grid_constant__ PassArgs a) {
    using L = MLayout<NP, CW, STAGES>;
    constexpr int BPT = L::BPT, NC = L::NC;
    constexpr int NEAR_UNR = NP <= 2 ? 2 : 1;  // NEAR-loop unroll (register budget)
    constexpr uint32_t STAGE_BYTES = 4 * MG * 4 + MG * 16 + 3 * 16;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float4 *s_r = reinterpret_cast<float4 *>(smem_raw + L::r_off);
    float4 *s_l = reinterpret_cast<float4 *>(smem_raw + L::l_off);
    float4 *s_g = reinterpret_cast<float4 *>(smem_raw + L::g_off);
    float *s_part = reinterpret_cast<float *>(smem_raw + L::p_off);
    DF *s_acc = reinterpret_cast<DF *>(smem_raw + L::a_off);
    float4 *s_ip = reinterpret_cast<float4 *>(smem_raw + L::i_off);
    float4 *s_qb = reinterpret_cast<float4 *>(smem_raw + L::q_off);
    uint32_t *mk = reinterpret_cast<uint32_t *>(smem_raw + L::m_off) + threadIdx.x;  // mk[k * NC]: screened pairs of i-body k
    f32x2 *res = reinterpret_cast<f32x2 *>(smem_raw + L::e_off) + threadIdx.x;     // res[(q * 3 + c) * NC]: residuals
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + L::b_off);
    uint64_t *pdone = full + STAGES, *empty = pdone + STAGES;
    MHdr *hdr = reinterpret_cast<MHdr *>(smem_raw + L::h_off);

    const MutualPlan &P = a.mp;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t wlim = pass_wait_limit(a.wait_ns_log2);
    float2 *rows = reinterpret_cast<float2 *>(a.partial);

    __shared__ unsigned s_lead;  // slots the leading consumer warp has finished
    __shared__ MSys s_wsys[CW];  // the system of each consumer warp's current item
    if (tid == 0) {
        for (int q = 0; q < STAGES; q++) {
            mbar_init(&full[q], 1);
            mbar_init(&pdone[q], CW);
            mbar_init(&empty[q], NR);
        }
        fence_barrier_init();
        s_lead = 0u;
    }
    __syncthreads();

    if (warp == CW) {  // -------------------------------------------- producer
        if (lane != 0) return;
        unsigned n = 0;
        for (;;) {
            // claim the next item only when the leading consumer warp is
            // within M_CLAIM - 1 filled slots of the end of this CTA's work
            // (inside an item the ring still runs up to STAGES slots ahead of
            // the slowest warp): a CTA then holds no queued slots that an
            // idle CTA could have taken, which evens out the CTAs' end times
            if (n >= (unsigned)M_CLAIM && !wait_lead(&s_lead, n - M_CLAIM + 1, a.status, wlim)) return;
            const int q = atomicAdd(a.work, 1);
            const bool done = q >= P.items;
            int4 it = done ? make_int4(0, 0, 0, 0) : P.item[q];
            if (!done && P.nreal > 0) {  // a plan for the padded length: only the groups that hold bodies
                const int greal = (P.nreal + MG - 1) / MG;
                if (it.x * P.gpb >= greal) continue;  // a block of padding only: its rows are never read
                it.z = min(it.z, greal);
                if (it.y >= it.z) {  // no j-group with bodies: one empty slot writes the item's (zero) i-row
                    it.y = -1;
                    it.z = 0;
                }
            }
            for (int g = it.y; done || g < it.z; g++, n++) {
                const int slot = n % STAGES;
                const unsigned u = n / STAGES;
                if (u > 0 && !mbar_wait_bounded(&empty[slot], (u - 1) & 1, a.status, wlim)) return;
                if (done) {
                    hdr[slot] = MHdr{q, 0, 4, 0};
                    mbar_arrive(&full[slot]);
                    return;
                }
                if (a.hold) return;  // test hook: no stage is ever filled (and no copy issued)
                hdr[slot] = MHdr{q, g, (g == it.y ? 1 : 0) | (g == it.z - 1 ? 2 : 0), 0};
                if (g < 0) {  // the empty slot: no copy
                    mbar_arrive(&full[slot]);
                    continue;
                }
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&full[slot], STAGE_BYTES);
                bulk_g2s(s_r + slot * MG, a.rel + (size_t)g * MG, MG * 16, &full[slot]);
                bulk_g2s(s_l + slot * MG, a.rell + (size_t)g * MG, MG * 16, &full[slot]);
                bulk_g2s(s_g + slot * 4, a.gbox_lo + g, 16, &full[slot]);
                bulk_g2s(s_g + slot * 4 + 1, a.gbox_hi + g, 16, &full[slot]);
                bulk_g2s(s_g + slot * 4 + 2, a.gctr + g, 16, &full[slot]);
            }
        }
    }

    if (warp > CW) {  // --------------------------------------------- reducers
        const int rw = NR == 1 ? 0 : warp - CW - 1;  // this reducer's share: (half, component) pairs rw, rw + NR, ...
        float2 *jrow = nullptr;    // NULL: a diagonal item (one-sided, no j-side sums)
        int jnp = 0, jpoff = 0;    // the j-row's length and first packed position
        for (unsigned n = 0;; n++) {
            const int slot = n % STAGES;
            const uint32_t par = (n / STAGES) & 1;
            if (!mbar_wait_bounded(&full[slot], par, a.status, wlim)) return;
            const MHdr h = hdr[slot];
            if (h.flags & 4) return;
            if (!mbar_wait_bounded(&pdone[slot], par, a.status, wlim)) return;
            if (h.flags & 1) {
                const int4 it = P.item[h.item];
                const MSys sy = P.sys[P.bsys[it.x]];
                jrow = it.w < sy.S ? nullptr : rows + sy.pbase + (size_t)(sy.irows + it.x - sy.blk0) * 3 * sy.np;
                jnp = sy.np;
                jpoff = sy.poff;
            }
            if (jrow && h.group >= 0) {
                const float *sp = s_part + (size_t)slot * CW * 3 * MG;
#pragma unroll
                for (int hc = rw; hc < 6; hc += NR) {
                    const int jj = lane + 32 * (hc / 3), c = hc % 3;
                    DF t{0.f, 0.f};
#pragma unroll
                    for (int w = 0; w < CW; w++) t = df_add(t, sp[(w * 3 + c) * MG + jj], 0.f);
                    jrow[(size_t)c * jnp + (h.group * MG + jj - jpoff)] = make_float2(t.hi, t.lo);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[slot]);
        }
    }

    // ---------------------------------------------------------------- consumers
    const int src = (lane + 1) & 31;  // the rotation: lane l receives lane l+1's j-sums
    f32x2 MN[NP], TX[NP], TY[NP], TZ[NP];
#pragma unroll
    for (int q = 0; q < NP; q++) MN[q] = TX[q] = TY[q] = TZ[q] = 0ull;
    Box wbox = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
    bool in = false, diag = false;
    int row = 0, gw = 0, nf = 0;
    unsigned qin = 0u;            // bit q: packed register q holds i-group gw + q CW of the block
    DF *acc = s_acc + tid;        // acc[(c * BPT + k) * NC]: double-float sums of i-body k, component c
    float4 *ip = s_ip + tid;      // ip[k * NC]: {x_hi, y_hi, z_hi, H}, ip[(BPT + k) * NC]: {x_lo, y_lo, z_lo, A}
    float4 *qb = s_qb + warp * NP * 2;  // the boxes of the warp's i-groups

    for (unsigned n = 0;; n++) {
        const int slot = n % STAGES;
        if (!mbar_wait_bounded(&full[slot], (n / STAGES) & 1, a.status, wlim)) return;
        const MHdr h = hdr[slot];
        if (h.flags & 4) return;
        if (h.flags & 1) {  // first slot of an item: this warp's i-tile
            const int4 it = P.item[h.item];
            row = it.w;
            if (lane == 0) {
                s_wsys[warp] = P.sys[P.bsys[it.x]];
                if (P.nreal > 0) s_wsys[warp].N = P.nreal;
            }
            __syncwarp();
            const MSys &sy = s_wsys[warp];
            diag = row < sy.S;
            // the warp's i-groups are interleaved over the block (gw, gw + CW,
            // ...), so a j-group next to one part of the block is near one
            // i-group of several warps rather than all of one warp's
            const int gb0 = sy.poff / MG + (it.x - sy.blk0) * P.gpb;
            const int gb1 = min(gb0 + P.gpb, (sy.poff + sy.N + MG - 1) / MG);  // groups holding bodies
            gw = gb0 + warp;
            qin = 0u;
#pragma unroll
            for (int q = 0; q < NP; q++)
                if (gw + q * CW < gb1) qin |= 1u << q;
            in = qin != 0u;
            if (in) {
                const float INF = __int_as_float(0x7f800000);
#pragma unroll
                for (int k = 0; k < BPT; k++) {
                    const bool ok = (qin >> (k >> 1)) & 1u;
                    const int i = (gw + (k >> 1) * CW) * MG + 32 * (k & 1) + lane;
                    // an i-group past a partial last block: massless, far away
                    const float4 hi = ok ? a.hi[i] : make_float4(GENGA_PAD_POS, GENGA_PAD_POS, GENGA_PAD_POS, 0.f);
                    const float4 lo = ok ? a.lo[i] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float2 sc = ok ? a.scr[i] : make_float2(0.f, 0.f);
                    ip[k * NC] = make_float4(hi.x, hi.y, hi.z, sc.x);
                    ip[(BPT + k) * NC] = make_float4(lo.x, lo.y, lo.z, sc.y);
                    if (k & 1) {
                        float m0, m1;
                        up2(MN[k >> 1], m0, m1);
                        MN[k >> 1] = pk2(m0, -hi.w);
                    } else {
                        MN[k >> 1] = pk2(-hi.w, 0.f);
                    }
                }
                if (lane < 2 * NP) {
                    const int q = lane >> 1;
                    const bool ok = (qin >> q) & 1u;
                    const float4 empty_lo = make_float4(INF, INF, INF, 0.f), empty_hi = make_float4(-INF, -INF, -INF, 0.f);
                    qb[lane] = (lane & 1) ? (ok ? a.gbox_hi[gw + q * CW] : empty_hi) : (ok ? a.gbox_lo[gw + q * CW] : empty_lo);
                }
#pragma unroll
                for (int k = 0; k < 3 * BPT; k++) acc[k * NC] = DF{0.f, 0.f};
            }
            __syncwarp();
            if (in) {  // the box of all the warp's i-groups
                wbox = Box{qb[0], qb[1]};
#pragma unroll
                for (int q = 1; q < NP; q++) {
                    const float4 l = qb[2 * q], u = qb[2 * q + 1];
                    wbox.lo = make_float4(fminf(wbox.lo.x, l.x), fminf(wbox.lo.y, l.y), fminf(wbox.lo.z, l.z),
                                          fmaxf(wbox.lo.w, l.w));
                    wbox.hi = make_float4(fmaxf(wbox.hi.x, u.x), fmaxf(wbox.hi.y, u.y), fmaxf(wbox.hi.z, u.z),
                                          fmaxf(wbox.hi.w, u.w));
                }
            }
            __syncwarp();
#pragma unroll
            for (int q = 0; q < NP; q++) TX[q] = TY[q] = TZ[q] = 0ull;
            nf = 0;
        }
        const int g = h.group;
        float *part = s_part + ((size_t)slot * CW + warp) * 3 * MG;
        if (in && g >= 0) {  // (g < 0: an item without j-groups, its i-row only)
            // strip items: both sides of every pair; diagonal items: the
            // i-side only (every ordered pair inside the block is visited)
            const bool both = !diag;
            const Box gb = {s_g[slot * 4], s_g[slot * 4 + 1]};
            const float4 ctr = s_g[slot * 4 + 2];
            const float4 *tr = s_r + slot * MG;  // {X, Y, Z, G m} of the j-group's bodies
            // the warp's i-bodies relative to the group centre
            f32x2 XI[NP], YI[NP], ZI[NP];
#pragma unroll
            for (int q = 0; q < NP; q++) {
                const float4 h0 = ip[(2 * q) * NC], h1 = ip[(2 * q + 1) * NC];
                const float4 l0 = ip[(BPT + 2 * q) * NC], l1 = ip[(BPT + 2 * q + 1) * NC];
                XI[q] = pk2((h0.x - ctr.x) + l0.x, (h1.x - ctr.x) + l1.x);
                YI[q] = pk2((h0.y - ctr.y) + l0.y, (h1.y - ctr.y) + l1.y);
                ZI[q] = pk2((h0.z - ctr.z) + l0.z, (h1.z - ctr.z) + l1.z);
            }
            // which i-groups are NEAR the j-group (all of them for a diagonal
            // item's own tile): a tile FAR as a whole needs no per-group test
            unsigned qnear = 0u;
            if (!far_mutual(wbox, gb, ctr.w)) {
#pragma unroll
                for (int q = 0; q < NP; q++)
                    if (!far_mutual(Box{qb[2 * q], qb[2 * q + 1]}, gb, ctr.w)) qnear |= 1u << q;
            }
            // ------------------------------------------------ FAR i-groups
            // plain terms; both sides (strip items) or the i-side only
            auto far_loop = [&](auto both_tag) {
                constexpr bool BOTH = decltype(both_tag)::value;
#pragma unroll 1
                for (int sb = 0; sb < 2; sb++) {
                    float JX = 0.f, JY = 0.f, JZ = 0.f;
#pragma unroll(UNR)
                    for (int t = 0; t < 32; t++) {
                        // consecutive j across the lanes: one conflict-free 16-byte load
                        const int j = sb * 32 + ((lane + t) & 31);
                        const float4 B = tr[j];
                        const f32x2 AX = pk2(B.x, B.x), AY = pk2(B.y, B.y), AZ = pk2(B.z, B.z), AM = pk2(B.w, B.w);
#pragma unroll
                        for (int q = 0; q < NP; q++) {
                            const f32x2 DX = sub2(AX, XI[q]), DY = sub2(AY, YI[q]), DZ = sub2(AZ, ZI[q]);
                            const f32x2 R2 = fma2(DZ, DZ, fma2(DY, DY, mul2(DX, DX)));
                            const f32x2 RI = rsq2(R2);
                            const f32x2 R3 = mul2(mul2(RI, RI), RI);
                            const f32x2 SI = mul2(AM, R3);
                            TX[q] = fma2(SI, DX, TX[q]);
                            TY[q] = fma2(SI, DY, TY[q]);
                            TZ[q] = fma2(SI, DZ, TZ[q]);
                            if constexpr (BOTH) {
                                const f32x2 SJ = mul2(MN[q], R3);
                                jsum(JX, SJ, DX);
                                jsum(JY, SJ, DY);
                                jsum(JZ, SJ, DZ);
                            }
                        }
                        if constexpr (BOTH) {
                            JX = __shfl_sync(0xffffffffu, JX, src);
                            JY = __shfl_sync(0xffffffffu, JY, src);
                            JZ = __shfl_sync(0xffffffffu, JZ, src);
                        }
                    }
                    if constexpr (BOTH) {
                        part[0 * MG + sb * 32 + lane] = JX;
                        part[1 * MG + sb * 32 + lane] = JY;
                        part[2 * MG + sb * 32 + lane] = JZ;
                    }
                }
            };
            if (qnear == 0u) {
                if (both) far_loop(std::true_type{});
                else far_loop(std::false_type{});
            } else {
                // ---------------------------------------------- NEAR i-groups
                // rotations over QP i-groups at a time: a FAR i-group takes
                // the plain terms, a NEAR one exact offsets (residuals) with
                // every pair screened
                const float4 *tl = s_l + slot * MG;
                // the group of the warp's own tile (diagonal items): i-body k
                // meets itself at step 0 of packed register q = the group's
                // place in the warp's set, half sb; that pair is always
                // screened out (its FP32 offset is zero only up to rounding)
                // and the FP64 pass skips i = j
                const int dg = g - gw;
                const int gself = (both || dg < 0 || dg % CW != 0 || dg / CW >= NP) ? -1 : dg / CW;
                // residuals of the NEAR i-groups (shared memory: they are read
                // only for those) and their screening bounds (the i-group's
                // largest H and A against the j-group's)
                float thr[NP];
                const unsigned qres = NP <= NEAR_SPEC_NP ? qnear : (1u << NP) - 1u;  // i-groups taking the NEAR treatment
#pragma unroll
                for (int q = 0; q < NP; q++) {
                    thr[q] = 0.f;
                    if (qres & (1u << q)) {
                        const float4 h0 = ip[(2 * q) * NC], h1 = ip[(2 * q + 1) * NC];
                        const float4 l0 = ip[(BPT + 2 * q) * NC], l1 = ip[(BPT + 2 * q + 1) * NC];
                        float x0, x1, y0, y1, z0, z1;
                        up2(XI[q], x0, x1);
                        up2(YI[q], y0, y1);
                        up2(ZI[q], z0, z1);
                        res[(q * 3 + 0) * NC] = pk2(centred_residual(h0.x, l0.x, ctr.x, x0), centred_residual(h1.x, l1.x, ctr.x, x1));
                        res[(q * 3 + 1) * NC] = pk2(centred_residual(h0.y, l0.y, ctr.y, y0), centred_residual(h1.y, l1.y, ctr.y, y1));
                        res[(q * 3 + 2) * NC] = pk2(centred_residual(h0.z, l0.z, ctr.z, z0), centred_residual(h1.z, l1.z, ctr.z, z1));
                        thr[q] = screen_threshold(qb[2 * q].w, qb[2 * q + 1].w, gb.lo.w, gb.hi.w);
                    }
                }
                // the NEAR loop, specialised on the set QN of NEAR i-groups
                // (known at compile time: no branches between the packed
                // chains); a screened pair's flag goes to a per-lane bit mask
                auto near_loop = [&](auto both_tag, auto mask_tag) {
                    constexpr bool BOTH = decltype(both_tag)::value;
                    constexpr unsigned QN = decltype(mask_tag)::value;
#pragma unroll 1
                    for (int sb = 0; sb < 2; sb++) {
                        float JX = 0.f, JY = 0.f, JZ = 0.f;
                        // bit jj of M0[q] / M1[q]: pair (i_{2q} / i_{2q+1}, j = sb * 32 + jj) is screened
                        unsigned M0[NP], M1[NP];
#pragma unroll
                        for (int q = 0; q < NP; q++) M0[q] = M1[q] = 0u;
#pragma unroll(NEAR_UNR)
                        for (int t = 0; t < 32; t++) {
                            const int jj = (lane + t) & 31, j = sb * 32 + jj;
                            const float4 B = tr[j];
                            const f32x2 AX = pk2(B.x, B.x), AY = pk2(B.y, B.y), AZ = pk2(B.z, B.z), AM = pk2(B.w, B.w);
                            const float4 R = tl[j];
                            const f32x2 RX = pk2(R.x, R.x), RY = pk2(R.y, R.y), RZ = pk2(R.z, R.z);
#pragma unroll
                            for (int q = 0; q < NP; q++) {
                                f32x2 DX = sub2(AX, XI[q]), DY = sub2(AY, YI[q]), DZ = sub2(AZ, ZI[q]);
                                if (((QN >> q) & 1u) != 0u) {  // folded at compile time (q unrolled)
                                    DX = add2(DX, sub2(RX, res[(q * 3 + 0) * NC]));
                                    DY = add2(DY, sub2(RY, res[(q * 3 + 1) * NC]));
                                    DZ = add2(DZ, sub2(RZ, res[(q * 3 + 2) * NC]));
                                }
                                const f32x2 R2 = fma2(DZ, DZ, fma2(DY, DY, mul2(DX, DX)));
                                const f32x2 RI = rsq2(R2);
                                const f32x2 R3 = mul2(mul2(RI, RI), RI);
                                f32x2 SI = mul2(AM, R3), SJ = mul2(MN[q], R3);
                                if (((QN >> q) & 1u) != 0u) {  // folded at compile time (q unrolled)
                                    float ra, rb, sa, sb_, ja, jb;
                                    up2(R2, ra, rb);
                                    const bool self = t == 0 && q == gself;
                                    const bool na = ra < thr[q] || (self && sb == 0);
                                    const bool nb = rb < thr[q] || (self && sb == 1);
                                    // screened pairs leave the FP32 sums (exact FP64 afterwards)
                                    up2(SI, sa, sb_);
                                    SI = pk2(na ? 0.f : sa, nb ? 0.f : sb_);
                                    up2(SJ, ja, jb);
                                    SJ = pk2(na ? 0.f : ja, nb ? 0.f : jb);
                                    M0[q] |= (unsigned)na << jj;
                                    M1[q] |= (unsigned)nb << jj;
                                }
                                TX[q] = fma2(SI, DX, TX[q]);
                                TY[q] = fma2(SI, DY, TY[q]);
                                TZ[q] = fma2(SI, DZ, TZ[q]);
                                if constexpr (BOTH) {
                                    jsum(JX, SJ, DX);
                                    jsum(JY, SJ, DY);
                                    jsum(JZ, SJ, DZ);
                                }
                            }
                            if constexpr (BOTH) {
                                JX = __shfl_sync(0xffffffffu, JX, src);
                                JY = __shfl_sync(0xffffffffu, JY, src);
                                JZ = __shfl_sync(0xffffffffu, JZ, src);
                            }
                        }
                        if constexpr (BOTH) {
                            part[0 * MG + sb * 32 + lane] = JX;
                            part[1 * MG + sb * 32 + lane] = JY;
                            part[2 * MG + sb * 32 + lane] = JZ;
                        }
#pragma unroll
                        for (int q = 0; q < NP; q++) {
                            mk[(2 * q) * NC] = M0[q];
                            mk[(2 * q + 1) * NC] = M1[q];
                        }
                        // the screened pairs of this half of the group, exactly in
                        // FP64: all lanes evaluate one pair each per round; the
                        // j-side terms are added in lane order (a fixed order)
                        __syncwarp();
                        for (;;) {
                            int kk = -1, jj = 0;
                            for (int k = 0; k < BPT && kk < 0; k++) {
                                const unsigned m = mk[k * NC];
                                if (m) {
                                    kk = k;
                                    jj = __ffs((int)m) - 1;
                                    mk[k * NC] = m & (m - 1u);
                                }
                            }
                            if (!__any_sync(0xffffffffu, kk >= 0)) break;
                            double3 fi = make_double3(0.0, 0.0, 0.0), fj = fi;
                            if (kk >= 0) {
                                const int i = (gw + (kk >> 1) * CW) * MG + 32 * (kk & 1) + lane, j = g * MG + sb * 32 + jj;
                                const MSys &sy = s_wsys[warp];
                                screened_pair_mutual(a, i, j, sy.poff, sy.N, sy.off, BOTH, &fi, &fj);
                                const double f3[3] = {fi.x, fi.y, fi.z};
#pragma unroll
                                for (int c = 0; c < 3; c++) {
                                    DF &t = acc[(c * BPT + kk) * NC];
                                    const DF d = df_of_double(f3[c]);
                                    t = df_add(t, d.hi, d.lo);
                                }
                            }
                            if constexpr (BOTH) {
                                const int js = kk >= 0 ? sb * 32 + jj : -1;
                                const float fx = (float)fj.x, fy = (float)fj.y, fz = (float)fj.z;
                                for (int s = 0; s < 32; s++) {
                                    const int j2 = __shfl_sync(0xffffffffu, js, s);
                                    const float gx = __shfl_sync(0xffffffffu, fx, s);
                                    const float gy = __shfl_sync(0xffffffffu, fy, s);
                                    const float gz = __shfl_sync(0xffffffffu, fz, s);
                                    if (lane == 0 && j2 >= 0) {
                                        part[0 * MG + j2] += gx;
                                        part[1 * MG + j2] += gy;
                                        part[2 * MG + j2] += gz;
                                    }
                                }
                                __syncwarp();
                            }
                        }
                    }
                };
                if constexpr (NP <= NEAR_SPEC_NP) {  // one instantiation per non-empty set of NEAR i-groups
                    auto run = [&](auto mask_tag) {
                        if (both) near_loop(std::true_type{}, mask_tag);
                        else near_loop(std::false_type{}, mask_tag);
                    };
                    dispatch_mask<1u, (1u << NP) - 1u>(qnear, run);
                } else {  // every i-group takes the NEAR treatment (residuals and thresholds of all)
                    constexpr unsigned ALL = (1u << NP) - 1u;
                    if (both) near_loop(std::true_type{}, std::integral_constant<unsigned, ALL>{});
                    else near_loop(std::false_type{}, std::integral_constant<unsigned, ALL>{});
                }
            }
        } else if (!diag && g >= 0) {
#pragma unroll
            for (int c = 0; c < 3; c++) part[c * MG + lane] = part[c * MG + 32 + lane] = 0.f;
        }
        __syncwarp();
        if (lane == 0) {
            mbar_arrive(&pdone[slot]);  // this warp's j-sums are in; the slot may be reduced
            atomicMax(&s_lead, n + 1);
        }
        if (in) {
            if (++nf == M_FOLD || (h.flags & 2)) {  // fold the FP32 i-sums into the double-float sums
#pragma unroll
                for (int q = 0; q < NP; q++) {
                    float e, o;
                    up2(TX[q], e, o);
                    acc[(0 * BPT + 2 * q) * NC] = df_add(acc[(0 * BPT + 2 * q) * NC], e, 0.f);
                    acc[(0 * BPT + 2 * q + 1) * NC] = df_add(acc[(0 * BPT + 2 * q + 1) * NC], o, 0.f);
                    up2(TY[q], e, o);
                    acc[(1 * BPT + 2 * q) * NC] = df_add(acc[(1 * BPT + 2 * q) * NC], e, 0.f);
                    acc[(1 * BPT + 2 * q + 1) * NC] = df_add(acc[(1 * BPT + 2 * q + 1) * NC], o, 0.f);
                    up2(TZ[q], e, o);
                    acc[(2 * BPT + 2 * q) * NC] = df_add(acc[(2 * BPT + 2 * q) * NC], e, 0.f);
                    acc[(2 * BPT + 2 * q + 1) * NC] = df_add(acc[(2 * BPT + 2 * q + 1) * NC], o, 0.f);
                    TX[q] = TY[q] = TZ[q] = 0ull;
                }
                nf = 0;
            }
            if (h.flags & 2) {  // last slot of the item: its i-row
                const MSys &sy = s_wsys[warp];
                float2 *out = rows + sy.pbase + (size_t)row * 3 * sy.np;
#pragma unroll
                for (int k = 0; k < BPT; k++) {
                    if (!((qin >> (k >> 1)) & 1u)) continue;
                    const size_t i = (size_t)((gw + (k >> 1) * CW) * MG + 32 * (k & 1) + lane - sy.poff);
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        const DF t = acc[(c * BPT + k) * NC];
                        out[(size_t)c * sy.np + i] = make_float2(t.hi, t.lo);
                    }
                }
            }
        }
    }
}

// The system of packed position p (the largest whose first position is <= p).
__device__ __forceinline__ int plan_system(const MutualPlan &P, int p) {
    int lo = 0, hi = P.nsys - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.sys[mid].poff <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// COMBINE_LANES lanes per (two consecutive bodies, component): lane r of
// the group adds rows r, r + COMBINE_LANES, ... of the bodies' rows (their
// i-rows, then the j-rows of the earlier blocks) in double-float; the
// partial sums are then joined in a fixed tree (lane r with r ^ 1, then
// with r ^ 2) and lane 0 writes the optional acc output and v += acc tau
// (acc[c * Ntot + body], body = perm[off + k]).  Every sum has a fixed order
// (bitwise reproducible); splitting a body's rows over lanes puts four
// times the loads in flight and gives a grid of several blocks per SM.  Two
// bodies per group make every row load 16 bytes per lane (128 contiguous
// bytes per 8 groups); both bodies are in the same i-block (blocks are
// whole 64-body groups of one system), so they share the rows.
constexpr int COMBINE_LANES = 4;

__global__ void combine_mutual_kernel(const double *__restrict__ partial, const __grid_constant__ MutualPlan P,
                                      int Ntot, int npad, const uint32_t *__restrict__ perm, double tau,
                                      double *__restrict__ acc, double *__restrict__ vx, double *__restrict__ vy,
                                      double *__restrict__ vz, uint32_t *__restrict__ status) {
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = 2 * (gt / COMBINE_LANES), r = gt % COMBINE_LANES;
    const int c = blockIdx.y;
    const unsigned gmask = 0xfu << (threadIdx.x & 28u);  // the group's lanes (every lane reaches the shuffles)
    MSys sy{};
    int k = 0;
    bool live = p < npad;
    if (live) {
        sy = P.sys[plan_system(P, p)];
        if (P.nreal > 0) sy.N = P.nreal;
        k = p - sy.poff;
        live = k < sy.N;
    }
    DF t0{0.f, 0.f}, t1{0.f, 0.f};
    if (live) {
        const int bl = (k / MG) / P.gpb;  // block within the system
        const size_t stride = 3 * (size_t)sy.np / 2;  // float4 units (two float2 entries)
        const float4 *pr = reinterpret_cast<const float4 *>(partial + sy.pbase) + ((size_t)c * sy.np + k) / 2;
        const int2 bk = P.blk[sy.blk0 + bl];
        // the rows in order: diagonal i-rows, strip i-rows, j-rows of the system's blocks before bl
        const int n0 = bk.x, n1 = n0 + bk.y, n2 = n1 + bl;
        constexpr int BATCH = 8;
        for (int r0 = r; r0 < n2; r0 += BATCH * COMBINE_LANES) {
            float4 v[BATCH];
#pragma unroll
            for (int u = 0; u < BATCH; u++) {
                const int rw = r0 + u * COMBINE_LANES;
                const int rr = rw < n0 ? rw : rw < n1 ? sy.S + (rw - n0) : sy.irows + (rw - n1);
                v[u] = rw < n2 ? pr[(size_t)rr * stride] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < BATCH; u++)
                if (r0 + u * COMBINE_LANES < n2) {
                    t0 = df_add(t0, v[u].x, v[u].y);
                    t1 = df_add(t1, v[u].z, v[u].w);
                }
        }
    }
#pragma unroll
    for (int o = 1; o < COMBINE_LANES; o <<= 1) {
        const float h0 = __shfl_xor_sync(gmask, t0.hi, o), l0 = __shfl_xor_sync(gmask, t0.lo, o);
        const float h1 = __shfl_xor_sync(gmask, t1.hi, o), l1 = __shfl_xor_sync(gmask, t1.lo, o);
        t0 = df_add(t0, h0, l0);
        t1 = df_add(t1, h1, l1);
    }
    if (!live || r != 0) return;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        if (k + h >= sy.N) break;
        const DF &t = h ? t1 : t0;
        const double s = (double)t.hi + (double)t.lo;
        if (!isfinite(s)) atomicOr(status, GENGA_BIT(GENGA_ERR_NONFINITE));
        const int i = (int)perm[sy.off + k + h];
        if (acc) acc[c * (size_t)Ntot + i] = s;
        if (tau != 0.0) {
            double *v = c == 0 ? vx : (c == 1 ? vy : vz);
            v[i] += s * tau;
        }
    }
}

// ------------------------------------------------------- FP64 mutual pass
// The same plan, staging and reduction with FP64 arithmetic (the FP64 kick
// of Sect. 1): i-bodies as FP64 registers, j-groups as the FP64 records
// {x, y, z, G m}, 1/r from an FP32 SFU seed with a third-order correction,
// FP64 sums per slot folded into Neumaier-compensated per-body sums.  NEAR
// means inside the r_crit bound only (FP64 offsets need no precision
// distance).  On this GPU every FP64 warp instruction holds the FP64 pipe for
// tens of cycles, so the pair's 20 FP64 operations for two interactions (17
// for one in the one-sided pass) set the time; everything else overlaps.
struct CompS {  // Neumaier-compensated FP64 sum
    double s, c;
};

__device__ __forceinline__ void comp_add(CompS &a, double v) {
    const double t = a.s + v;
    // |a.s| >= |v| compared on the bit patterns (integer pipe, not FP64)
    const bool big = (__double_as_longlong(a.s) & 0x7fffffffffffffffll) >= (__double_as_longlong(v) & 0x7fffffffffffffffll);
    a.c += big ? ((a.s - t) + v) : ((v - t) + a.s);
    a.s = t;
}

template <int BPT, int CW, int STAGES>
struct M64Layout {
    static constexpr int NC = CW * 32, NPG = BPT / 2;
    static constexpr size_t p_off = 0;                                          // double4 [STAGES][MG]
    static constexpr size_t g_off = p_off + (size_t)STAGES * MG * 32;           // float4 [STAGES][2]
    static constexpr size_t j_off = g_off + (size_t)STAGES * 2 * 16;            // double [STAGES][CW][3][MG]
    static constexpr size_t c_off = j_off + (size_t)STAGES * CW * 3 * MG * 8;   // CompS [3][BPT][NC]
    static constexpr size_t q_off = c_off + (size_t)3 * BPT * NC * 16;          // float4 [CW][NPG][2]
    static constexpr size_t m_off = q_off + (size_t)CW * NPG * 2 * 16;          // uint32 [BPT][NC]
    static constexpr size_t b_off = m_off + (size_t)BPT * NC * 4;               // uint64 [3][STAGES]
    static constexpr size_t h_off = b_off + (size_t)3 * STAGES * 8;             // MHdr [STAGES]
    static constexpr size_t bytes = h_off + (size_t)STAGES * sizeof(MHdr);
    static_assert(bytes <= 227 * 1024, "one CTA per SM: at most 227 KB of shared memory");
};

template <int BPT, int CW, int STAGES, int NR>
__global__ void __maxnreg__(mutual_maxreg(CW + 1 + NR)) pass_mutual64_kernel(const __grid_constant__ PassArgs a) {
    using L = M64Layout<BPT, CW, STAGES>;
    constexpr int NC = L::NC, NPG = L::NPG;
    constexpr uint32_t STAGE_BYTES = MG * 32 + 2 * 16;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    double4_32a *s_p = reinterpret_cast<double4_32a *>(smem_raw + L::p_off);
    float4 *s_g = reinterpret_cast<float4 *>(smem_raw + L::g_off);
    double *s_part = reinterpret_cast<double *>(smem_raw + L::j_off);
    CompS *s_acc = reinterpret_cast<CompS *>(smem_raw + L::c_off);
    float4 *s_qb = reinterpret_cast<float4 *>(smem_raw + L::q_off);
    uint32_t *mk = reinterpret_cast<uint32_t *>(smem_raw + L::m_off) + threadIdx.x;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + L::b_off);
    uint64_t *pdone = full + STAGES, *empty = pdone + STAGES;
    MHdr *hdr = reinterpret_cast<MHdr *>(smem_raw + L::h_off);

    const MutualPlan &P = a.mp;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t wlim = pass_wait_limit(a.wait_ns_log2);
    double *rows = a.partial;

    __shared__ unsigned s_lead;  // slots the leading consumer warp has finished
    __shared__ MSys s_wsys[CW];  // the system of each consumer warp's current item
    if (tid == 0) {
        for (int q = 0; q < STAGES; q++) {
            mbar_init(&full[q], 1);
            mbar_init(&pdone[q], CW);
            mbar_init(&empty[q], NR);
        }
        fence_barrier_init();
        s_lead = 0u;
    }
    __syncthreads();

    if (warp == CW) {  // -------------------------------------------- producer
        if (lane != 0) return;
        unsigned n = 0;
        for (;;) {
            // claim the next item only when the leading consumer warp is
            // within M_CLAIM - 1 filled slots of the end of this CTA's work
            // (inside an item the ring still runs up to STAGES slots ahead of
            // the slowest warp): a CTA then holds no queued slots that an
            // idle CTA could have taken, which evens out the CTAs' end times
            if (n >= (unsigned)M_CLAIM && !wait_lead(&s_lead, n - M_CLAIM + 1, a.status, wlim)) return;
            const int q = atomicAdd(a.work, 1);
            const bool done = q >= P.items;
            int4 it = done ? make_int4(0, 0, 0, 0) : P.item[q];
            if (!done && P.nreal > 0) {  // a plan for the padded length: only the groups that hold bodies
                const int greal = (P.nreal + MG - 1) / MG;
                if (it.x * P.gpb >= greal) continue;  // a block of padding only: its rows are never read
                it.z = min(it.z, greal);
                if (it.y >= it.z) {  // no j-group with bodies: one empty slot writes the item's (zero) i-row
                    it.y = -1;
                    it.z = 0;
                }
            }
            for (int g = it.y; done || g < it.z; g++, n++) {
                const int slot = n % STAGES;
                const unsigned u = n / STAGES;
                if (u > 0 && !mbar_wait_bounded(&empty[slot], (u - 1) & 1, a.status, wlim)) return;
                if (done) {
                    hdr[slot] = MHdr{q, 0, 4, 0};
                    mbar_arrive(&full[slot]);
                    return;
                }
                if (a.hold) return;  // test hook: no stage is ever filled (and no copy issued)
                hdr[slot] = MHdr{q, g, (g == it.y ? 1 : 0) | (g == it.z - 1 ? 2 : 0), 0};
                if (g < 0) {  // the empty slot: no copy
                    mbar_arrive(&full[slot]);
                    continue;
                }
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&full[slot], STAGE_BYTES);
                bulk_g2s(s_p + slot * MG, a.p64 + (size_t)g * MG, MG * 32, &full[slot]);
                bulk_g2s(s_g + slot * 2, a.gbox_lo + g, 16, &full[slot]);
                bulk_g2s(s_g + slot * 2 + 1, a.gbox_hi + g, 16, &full[slot]);
            }
        }
    }

    if (warp > CW) {  // --------------------------------------------- reducers
        const int rw = NR == 1 ? 0 : warp - CW - 1;  // (half, component) pairs rw, rw + NR, ... as in the FP32 pass
        double *jrow = nullptr;
        int jnp = 0, jpoff = 0;
        for (unsigned n = 0;; n++) {
            const int slot = n % STAGES;
            const uint32_t par = (n / STAGES) & 1;
            if (!mbar_wait_bounded(&full[slot], par, a.status, wlim)) return;
            const MHdr h = hdr[slot];
            if (h.flags & 4) return;
            if (!mbar_wait_bounded(&pdone[slot], par, a.status, wlim)) return;
            if (h.flags & 1) {
                const int4 it = P.item[h.item];
                const MSys sy = P.sys[P.bsys[it.x]];
                jrow = it.w < sy.S ? nullptr : rows + sy.pbase + (size_t)(sy.irows + it.x - sy.blk0) * 3 * sy.np;
                jnp = sy.np;
                jpoff = sy.poff;
            }
            if (jrow && h.group >= 0) {
                const double *sp = s_part + (size_t)slot * CW * 3 * MG;
#pragma unroll
                for (int hc = rw; hc < 6; hc += NR) {
                    const int jj = lane + 32 * (hc / 3), c = hc % 3;
                    CompS t{0.0, 0.0};
#pragma unroll
                    for (int w = 0; w < CW; w++) comp_add(t, sp[(w * 3 + c) * MG + jj]);
                    jrow[(size_t)c * jnp + (h.group * MG + jj - jpoff)] = t.s + t.c;
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[slot]);
        }
    }

    // ---------------------------------------------------------------- consumers
    const int src = (lane + 1) & 31;
    double XI[BPT], YI[BPT], ZI[BPT], MN[BPT];
#pragma unroll
    for (int k = 0; k < BPT; k++) XI[k] = YI[k] = ZI[k] = MN[k] = 0.0;
    Box wbox = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
    bool in = false, diag = false;
    int row = 0, gw = 0;
    unsigned qin = 0u;
    CompS *acc = s_acc + tid;           // acc[(c * BPT + k) * NC]
    float4 *qb = s_qb + warp * NPG * 2;

    for (unsigned n = 0;; n++) {
        const int slot = n % STAGES;
        if (!mbar_wait_bounded(&full[slot], (n / STAGES) & 1, a.status, wlim)) return;
        const MHdr h = hdr[slot];
        if (h.flags & 4) return;
        if (h.flags & 1) {  // first slot of an item: this warp's i-bodies (groups gw + q CW)
            const int4 it = P.item[h.item];
            row = it.w;
            if (lane == 0) {
                s_wsys[warp] = P.sys[P.bsys[it.x]];
                if (P.nreal > 0) s_wsys[warp].N = P.nreal;
            }
            __syncwarp();
            const MSys &sy = s_wsys[warp];
            diag = row < sy.S;
            const int gb0 = sy.poff / MG + (it.x - sy.blk0) * P.gpb;
            const int gb1 = min(gb0 + P.gpb, (sy.poff + sy.N + MG - 1) / MG);  // groups holding bodies
            gw = gb0 + warp;
            qin = 0u;
#pragma unroll
            for (int q = 0; q < NPG; q++)
                if (gw + q * CW < gb1) qin |= 1u << q;
            in = qin != 0u;
            if (in) {
                const float INF = __int_as_float(0x7f800000);
#pragma unroll
                for (int k = 0; k < BPT; k++) {
                    const bool ok = (qin >> (k >> 1)) & 1u;
                    const int i = (gw + (k >> 1) * CW) * MG + 32 * (k & 1) + lane;
                    const double4_32a p = ok ? a.p64[i] : make_double4_32a(GENGA_PAD_POS, GENGA_PAD_POS, GENGA_PAD_POS, 0.0);
                    XI[k] = p.x;
                    YI[k] = p.y;
                    ZI[k] = p.z;
                    MN[k] = -p.w;
                }
                if (lane < 2 * NPG) {
                    const int q = lane >> 1;
                    const bool ok = (qin >> q) & 1u;
                    qb[lane] = (lane & 1) ? (ok ? a.gbox_hi[gw + q * CW] : make_float4(-INF, -INF, -INF, 0.f))
                                          : (ok ? a.gbox_lo[gw + q * CW] : make_float4(INF, INF, INF, 0.f));
                }
#pragma unroll
                for (int k = 0; k < 3 * BPT; k++) acc[k * NC] = CompS{0.0, 0.0};
            }
            __syncwarp();
            if (in) {
                wbox = Box{qb[0], qb[1]};
#pragma unroll
                for (int q = 1; q < NPG; q++) {
                    const float4 l = qb[2 * q], u = qb[2 * q + 1];
                    wbox.lo = make_float4(fminf(wbox.lo.x, l.x), fminf(wbox.lo.y, l.y), fminf(wbox.lo.z, l.z),
                                          fmaxf(wbox.lo.w, l.w));
                    wbox.hi = make_float4(fmaxf(wbox.hi.x, u.x), fmaxf(wbox.hi.y, u.y), fmaxf(wbox.hi.z, u.z),
                                          fmaxf(wbox.hi.w, u.w));
                }
            }
        }
        const int g = h.group;
        double *part = s_part + ((size_t)slot * CW + warp) * 3 * MG;
        if (in && g >= 0) {  // (g < 0: an item without j-groups, its i-row only)
            const bool both = !diag;
            const Box gb = {s_g[slot * 2], s_g[slot * 2 + 1]};
            const double4_32a *tp = s_p + slot * MG;
            // NEAR i-groups (inside the r_crit bound of the j-group): their
            // pairs are compared with the screening bound (integer compare of
            // the FP64 bit patterns of r^2 and of the bound: both positive)
            unsigned qnear = 0u;
            long long thr[NPG];
#pragma unroll
            for (int q = 0; q < NPG; q++) {
                thr[q] = 0;
                if (!far_pair_of_boxes(wbox, gb, false) && !far_pair_of_boxes(Box{qb[2 * q], qb[2 * q + 1]}, gb, false)) {
                    qnear |= 1u << q;
                    thr[q] = __double_as_longlong((double)screen_threshold(qb[2 * q].w, qb[2 * q + 1].w, gb.lo.w, gb.hi.w));
                }
            }
            const int dg = g - gw;
            const int gself = (both || dg < 0 || dg % CW != 0 || dg / CW >= NPG) ? -1 : dg / CW;
            double PX[BPT], PY[BPT], PZ[BPT];
#pragma unroll
            for (int k = 0; k < BPT; k++) PX[k] = PY[k] = PZ[k] = 0.0;
#pragma unroll 1
            for (int sb = 0; sb < 2; sb++) {
                double JX = 0.0, JY = 0.0, JZ = 0.0;
                if (qnear) {
#pragma unroll
                    for (int k = 0; k < BPT; k++) mk[k * NC] = 0u;
                }
#pragma unroll 2
                for (int t = 0; t < 32; t++) {
                    const int jj = (lane + t) & 31;
                    const double4_32a pj = tp[sb * 32 + jj];
#pragma unroll
                    for (int k = 0; k < BPT; k++) {
                        const double dx = pj.x - XI[k], dy = pj.y - YI[k], dz = pj.z - ZI[k];
                        const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
                        const double r3 = rsqrt3_fp64(r2);
                        double si = pj.w * r3, sj = MN[k] * r3;
                        if ((qnear >> (k >> 1)) & 1u) {
                            const bool self = t == 0 && (k >> 1) == gself && (k & 1) == sb;
                            if (__double_as_longlong(r2) < thr[k >> 1] || self) {  // rare: exact FP64 afterwards
                                si = 0.0;
                                sj = 0.0;
                                mk[k * NC] |= 1u << jj;
                            }
                        }
                        PX[k] = fma(si, dx, PX[k]);
                        PY[k] = fma(si, dy, PY[k]);
                        PZ[k] = fma(si, dz, PZ[k]);
                        if (both) {
                            JX = fma(sj, dx, JX);
                            JY = fma(sj, dy, JY);
                            JZ = fma(sj, dz, JZ);
                        }
                    }
                    if (both) {
                        JX = __shfl_sync(0xffffffffu, JX, src);
                        JY = __shfl_sync(0xffffffffu, JY, src);
                        JZ = __shfl_sync(0xffffffffu, JZ, src);
                    }
                }
                if (both) {
                    part[0 * MG + sb * 32 + lane] = JX;
                    part[1 * MG + sb * 32 + lane] = JY;
                    part[2 * MG + sb * 32 + lane] = JZ;
                }
                if (qnear) {  // screened pairs exactly (K-weighted), both sides
                    __syncwarp();
                    for (;;) {
                        int kk = -1, jj = 0;
                        for (int k = 0; k < BPT && kk < 0; k++) {
                            const unsigned m = mk[k * NC];
                            if (m) {
                                kk = k;
                                jj = __ffs((int)m) - 1;
                                mk[k * NC] = m & (m - 1u);
                            }
                        }
                        if (!__any_sync(0xffffffffu, kk >= 0)) break;
                        double3 fi = make_double3(0.0, 0.0, 0.0), fj = fi;
                        if (kk >= 0) {
                            const int i = (gw + (kk >> 1) * CW) * MG + 32 * (kk & 1) + lane, j = g * MG + sb * 32 + jj;
                            const MSys &sy = s_wsys[warp];
                            screened_pair_mutual(a, i, j, sy.poff, sy.N, sy.off, both, &fi, &fj);
                            comp_add(acc[(0 * BPT + kk) * NC], fi.x);
                            comp_add(acc[(1 * BPT + kk) * NC], fi.y);
                            comp_add(acc[(2 * BPT + kk) * NC], fi.z);
                        }
                        if (both) {
                            const int js = kk >= 0 ? sb * 32 + jj : -1;
                            for (int s2 = 0; s2 < 32; s2++) {
                                const int j2 = __shfl_sync(0xffffffffu, js, s2);
                                const double gx = __shfl_sync(0xffffffffu, fj.x, s2);
                                const double gy = __shfl_sync(0xffffffffu, fj.y, s2);
                                const double gz = __shfl_sync(0xffffffffu, fj.z, s2);
                                if (lane == 0 && j2 >= 0) {
                                    part[0 * MG + j2] += gx;
                                    part[1 * MG + j2] += gy;
                                    part[2 * MG + j2] += gz;
                                }
                            }
                            __syncwarp();
                        }
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < BPT; k++) {  // this slot's sums into the compensated per-body sums
                comp_add(acc[(0 * BPT + k) * NC], PX[k]);
                comp_add(acc[(1 * BPT + k) * NC], PY[k]);
                comp_add(acc[(2 * BPT + k) * NC], PZ[k]);
            }
        } else if (!diag && g >= 0) {
#pragma unroll
            for (int c = 0; c < 3; c++) part[c * MG + lane] = part[c * MG + 32 + lane] = 0.0;
        }
        __syncwarp();
        if (lane == 0) {
            mbar_arrive(&pdone[slot]);
            atomicMax(&s_lead, n + 1);
        }
        if (in && (h.flags & 2)) {  // last slot of the item: its i-row
            const MSys &sy = s_wsys[warp];
            double *out = rows + sy.pbase + (size_t)row * 3 * sy.np;
#pragma unroll
            for (int k = 0; k < BPT; k++) {
                if (!((qin >> (k >> 1)) & 1u)) continue;
                const size_t i = (size_t)((gw + (k >> 1) * CW) * MG + 32 * (k & 1) + lane - sy.poff);
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const CompS t = acc[(c * BPT + k) * NC];
                    out[(size_t)c * sy.np + i] = t.s + t.c;
                }
            }
        }
    }
}

// The FP64 rows of a mutual FP64 pass, combined as in combine_mutual_kernel
// (COMBINE_LANES lanes per two bodies and component, 16-byte loads, a fixed
// tree), Neumaier-compensated.
__global__ void combine_mutual64_kernel(const double *__restrict__ partial, const __grid_constant__ MutualPlan P,
                                        int Ntot, int npad, const uint32_t *__restrict__ perm, double tau,
                                        double *__restrict__ acc, double *__restrict__ vx, double *__restrict__ vy,
                                        double *__restrict__ vz, uint32_t *__restrict__ status) {
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = 2 * (gt / COMBINE_LANES), r = gt % COMBINE_LANES;
    const int c = blockIdx.y;
    const unsigned gmask = 0xfu << (threadIdx.x & 28u);
    MSys sy{};
    int k = 0;
    bool live = p < npad;
    if (live) {
        sy = P.sys[plan_system(P, p)];
        if (P.nreal > 0) sy.N = P.nreal;
        k = p - sy.poff;
        live = k < sy.N;
    }
    CompS t0{0.0, 0.0}, t1{0.0, 0.0};
    if (live) {
        const int bl = (k / MG) / P.gpb;
        const size_t stride = 3 * (size_t)sy.np / 2;  // double2 units
        const double2 *pr = reinterpret_cast<const double2 *>(partial + sy.pbase) + ((size_t)c * sy.np + k) / 2;
        const int2 bk = P.blk[sy.blk0 + bl];
        const int n0 = bk.x, n1 = n0 + bk.y, n2 = n1 + bl;
        constexpr int BATCH = 8;
        for (int r0 = r; r0 < n2; r0 += BATCH * COMBINE_LANES) {
            double2 v[BATCH];
#pragma unroll
            for (int u = 0; u < BATCH; u++) {
                const int rw = r0 + u * COMBINE_LANES;
                const int rr = rw < n0 ? rw : rw < n1 ? sy.S + (rw - n0) : sy.irows + (rw - n1);
                v[u] = rw < n2 ? pr[(size_t)rr * stride] : make_double2(0.0, 0.0);
            }
#pragma unroll
            for (int u = 0; u < BATCH; u++)
                if (r0 + u * COMBINE_LANES < n2) {
                    comp_add(t0, v[u].x);
                    comp_add(t1, v[u].y);
                }
        }
    }
#pragma unroll
    for (int o = 1; o < COMBINE_LANES; o <<= 1) {
        const double s0 = __shfl_xor_sync(gmask, t0.s, o), c0 = __shfl_xor_sync(gmask, t0.c, o);
        const double s1 = __shfl_xor_sync(gmask, t1.s, o), c1 = __shfl_xor_sync(gmask, t1.c, o);
        comp_add(t0, s0);
        t0.c += c0;
        comp_add(t1, s1);
        t1.c += c1;
    }
    if (!live || r != 0) return;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        if (k + h >= sy.N) break;
        const CompS &t = h ? t1 : t0;
        const double s = t.s + t.c;
        if (!isfinite(s)) atomicOr(status, GENGA_BIT(GENGA_ERR_NONFINITE));
        const int i = (int)perm[sy.off + k + h];
        if (acc) acc[c * (size_t)Ntot + i] = s;
        if (tau != 0.0) {
            double *v = c == 0 ? vx : (c == 1 ? vy : vz);
            v[i] += s * tau;
        }
    }
}

// --------------------------------------------------------------- variants
struct MVariant {
    int np, cw, nr;
    void (*fn)(const PassArgs);
    size_t smem;
};
#define GENGA_MV(NP, CW, ST, UNR, NR) \
    {NP, CW, NR, pass_mutual_kernel<NP, CW, ST, UNR, NR>, MLayout<NP, CW, ST>::bytes}
// three reducer warps in every shape (one reducer: 0.562 against 0.552 ms
// for the (2, 12, 4, 8) pass at 40k)
const MVariant kMVariants[] = {GENGA_MV(2, 12, 4, 8, 3), GENGA_MV(2, 12, 8, 4, 3), GENGA_MV(2, 12, 8, 8, 3),
                               GENGA_MV(4, 8, 6, 4, 3)};
#undef GENGA_MV
constexpr int kNumMVariants = sizeof(kMVariants) / sizeof(kMVariants[0]);

struct M64Variant {
    int bpt, cw, nr;
    void (*fn)(const PassArgs);
    size_t smem;
};
#define GENGA_M64(BPT, CW, ST, NR) \
    {BPT, CW, NR, pass_mutual64_kernel<BPT, CW, ST, NR>, M64Layout<BPT, CW, ST>::bytes}
const M64Variant kM64Variants[] = {GENGA_M64(4, 8, 4, 3), GENGA_M64(8, 4, 4, 3), GENGA_M64(2, 12, 4, 3)};
#undef GENGA_M64
constexpr int kNumM64Variants = sizeof(kM64Variants) / sizeof(kM64Variants[0]);
static_assert(kNumMVariants + kNumM64Variants <= GENGA_MAX_VARIANTS, "plan cache slots");

// ---------------------------------------------------------------- planner
// Cost model, in units of one slot of far pairs for both sides (every warp
// on one group): groups next to an i-block (its own, in the diagonal items,
// evaluated one-sided; the first near_span groups of its strip) are mostly
// NEAR and cost about DIAG_COST and NEAR_COST.
constexpr double DIAG_COST = 1.5, NEAR_COST = 2.0, ITEM_COST = 0.1;

struct Chunk {
    double cost;
    int4 item;
    int tail;     // 1: a tail item (handed out last)
    double near;  // share of the item's cost in NEAR groups (its cost is the least certain)
};

// Items of one plan: diagonal items (the block's groups in D ranges); each
// strip's first near_span groups (next to the block, mostly NEAR) in chunks
// of at most Ln groups, the rest in chunks of Lm groups (Lm = 0: about R
// chunks per strip, their length following the strip's, so that handing the
// items out longest first ends on the short chunks of the short strips), its
// last T groups in single-group tail items.  Strip i-rows follow the diagonal
// items' rows in strip order; handout order: largest first, the tail last.
void build_items(int ngroups, int gpb, int D, int R, int Lm, int Ln, int near_span, int T, std::vector<Chunk> *out,
                 std::vector<int2> *blk, int *S) {
    const int nb = (ngroups + gpb - 1) / gpb;
    out->clear();
    blk->assign(nb, make_int2(0, 0));
    *S = 0;
    for (int b = 0; b < nb; b++) {
        const int g0 = b * gpb, g1 = std::min(g0 + gpb, ngroups), n = g1 - g0;
        const int d = std::min(D, n);
        for (int k = 0; k < d; k++) {
            const int a0 = g0 + (int)((long long)n * k / d), a1 = g0 + (int)((long long)n * (k + 1) / d);
            out->push_back(Chunk{(a1 - a0) * DIAG_COST + ITEM_COST, make_int4(b, a0, a1, k), 0, 1.0});
        }
        (*blk)[b].x = d;
        *S = std::max(*S, d);
    }
    for (int b = 0; b < nb; b++) {
        const int s0 = (b + 1) * gpb, Sb = std::max(0, ngroups - s0);
        const int tail0 = std::max(0, Sb - T);
        const int nspan = std::min(near_span, tail0);
        const int Lb = Lm > 0 ? Lm : std::max(1, (Sb + R - 1) / R);
        int pos = 0, nch = 0;
        auto emit = [&](int L, int tl) {
            const int nnear = std::max(0, std::min(pos + L, near_span) - pos);
            const double c = nnear * NEAR_COST + (L - nnear) + ITEM_COST;
            out->push_back(Chunk{c, make_int4(b, s0 + pos, s0 + pos + L, -1), tl, nnear * NEAR_COST / c});
            pos += L;
            nch++;
        };
        while (pos < nspan) emit(std::min(std::min(Ln, Lb), nspan - pos), 0);
        while (pos < tail0) emit(std::min(Lb, tail0 - pos), 0);
        while (pos < Sb) emit(1, 1);
        (*blk)[b].y = nch;
    }
    std::vector<int> next(nb, 0);
    for (Chunk &c : *out)
        if (c.item.w < 0) c.item.w = *S + next[c.item.x]++;
    std::stable_sort(out->begin(), out->end(), [](const Chunk &x, const Chunk &y) {
        return x.tail != y.tail ? y.tail : x.cost > y.cost;
    });
}

// Makespan of handing the items in order to the first free of C CTAs, the
// worst of a few draws in which each item's cost is off by a fixed
// pseudo-random factor (up to +-60 % of its NEAR share, +-10 % otherwise):
// the cost model is rough, so plans whose balance rests on it are avoided.
double makespan(const std::vector<Chunk> &items, int C) {
    double worst = 0.0;
    for (uint32_t seed = 1; seed <= 3; seed++) {
        std::priority_queue<double, std::vector<double>, std::greater<double>> q;
        for (int k = 0; k < C; k++) q.push(0.0);
        double m = 0.0;
        uint32_t h = seed * 2654435761u;
        for (const Chunk &c : items) {
            h ^= h << 13;
            h ^= h >> 17;
            h ^= h << 5;
            const double r = (double)(h & 0xffff) / 65535.0 * 2.0 - 1.0;  // in [-1, 1]
            const double t = q.top() + c.cost * (1.0 + r * (0.1 + 0.5 * c.near));
            q.pop();
            q.push(t);
            m = std::max(m, t);
        }
        worst = std::max(worst, m);
    }
    return worst;
}

// A system as the planner sees it: packed range [poff, poff + np), N bodies,
// caller indices from off.
struct HSys {
    int poff, np, N, off;
};

struct PlanOut {
    std::vector<int4> item;
    std::vector<int2> blk;
    std::vector<int32_t> bsys;
    std::vector<MSys> sys;
    size_t row_entries = 0;  // 8-byte entries of all partial rows
};

// The plan with the best estimated makespan over all systems' items (plus a
// small cost per partial row a body reads in the combine) over the diagonal
// split, the chunks per strip and the tail (single groups, a few per CTA in
// all); each system's rows at most max_rows.  out->item is empty when no
// plan fits.
void plan_systems(const std::vector<HSys> &hs, int cw, int NPg, int ctas, int max_rows, PlanOut *out) {
    const int gpb = cw * NPg;
    const int ns = (int)hs.size();
    std::vector<int> G(ns), nbs(ns);
    int nstrips = 0;
    long long npos = 0;
    for (int d = 0; d < ns; d++) {
        G[d] = (hs[d].N + MG - 1) / MG;
        nbs[d] = (G[d] + gpb - 1) / gpb;
        nstrips += std::max(0, nbs[d] - 1);
        npos += hs[d].np;
    }
    nstrips = std::max(1, nstrips);
    std::vector<Chunk> items, all;
    std::vector<int2> blk;
    int S = 0;
    double total = 0.0;
    for (int d = 0; d < ns; d++) {
        build_items(G[d], gpb, 1, 1, 1, NPg, 2 * gpb, 0, &items, &blk, &S);
        for (const Chunk &c : items) total += c.cost;
    }
    const double per = total / ctas;
    // two families: fixed chunk lengths (fractions of a CTA's share) and a
    // fixed number of chunks per strip
    struct Shape {
        int R, Lm;
    };
    std::vector<Shape> shapes;
    for (int R : {16, 24, 32, 48, 64}) shapes.push_back(Shape{R, 0});
    for (double f : {0.06, 0.09, 0.12, 0.18, 0.25}) shapes.push_back(Shape{0, std::max(1, (int)std::lround(per * f))});
    double best = 1e300;
    out->item.clear();
    PlanOut cand;
    for (int D : {2, 4, 8, 12}) {
        for (const Shape &sh : shapes) {
            for (int tau : {2, 4, 6}) {
                const int T = (tau * ctas + nstrips - 1) / nstrips;
                all.clear();
                cand.blk.clear();
                cand.bsys.clear();
                cand.sys.clear();
                bool fits = true;
                int blk0 = 0;
                double rows_read = 0.0;  // partial rows per packed position, on average
                for (int d = 0; d < ns && fits; d++) {
                    if (G[d] == 0) continue;
                    build_items(G[d], gpb, D, sh.R, sh.Lm, NPg, 2 * gpb, T, &items, &blk, &S);
                    int irows = 0;
                    for (const int2 &b : blk) irows = std::max(irows, S + b.y);
                    const int rows = irows + (int)blk.size();
                    if (rows > max_rows) fits = false;
                    const int g0 = hs[d].poff / MG, sd = (int)cand.sys.size();
                    for (Chunk c : items) {
                        c.item.x += blk0;
                        c.item.y += g0;
                        c.item.z += g0;
                        all.push_back(c);
                    }
                    for (const int2 &b : blk) {
                        cand.blk.push_back(b);
                        cand.bsys.push_back(sd);
                    }
                    cand.sys.push_back(MSys{hs[d].poff, hs[d].np, hs[d].N, hs[d].off, irows, S, g0 + G[d], blk0, 0});
                    blk0 += (int)blk.size();
                    rows_read += (double)rows * hs[d].np / (double)npos;
                }
                if (!fits || (int)all.size() > GENGA_MUTUAL_MAX_ITEMS) continue;
                std::stable_sort(all.begin(), all.end(), [](const Chunk &x, const Chunk &y) {
                    return x.tail != y.tail ? y.tail : x.cost > y.cost;
                });
                const double score = makespan(all, ctas) + 0.01 * rows_read;
                if (score < best) {
                    best = score;
                    out->item.clear();
                    for (const Chunk &c : all) out->item.push_back(c.item);
                    out->blk = cand.blk;
                    out->bsys = cand.bsys;
                    out->sys = cand.sys;
                }
            }
        }
    }
    size_t pb = 0;  // each system's rows (irows + its blocks) after the previous systems'
    for (size_t q = 0; q < out->sys.size(); q++) {
        MSys &y = out->sys[q];
        const int nb = (q + 1 < out->sys.size() ? out->sys[q + 1].blk0 : (int)out->blk.size()) - y.blk0;
        y.pbase = (long long)pb;
        pb += (size_t)(y.irows + nb) * 3 * (size_t)y.np;
    }
    out->row_entries = pb;
}

}  // namespace

int num_mutual_variants() { return kNumMVariants; }
int num_mutual64_variants() { return kNumM64Variants; }
void mutual64_variant_shape(int v, int *cw, int *bpt) {
    *cw = kM64Variants[v].cw;
    *bpt = kM64Variants[v].bpt;
}
void mutual_variant_shape(int v, int *cw, int *bpt) {
    *cw = kMVariants[v].cw;
    *bpt = 2 * kMVariants[v].np;
}

void free_mutual_cache(genga_ctx *c) {
    if (!c->mcache) return;
    auto drop = [](MutualCache::Entry &e) {
        if (e.d_item) cudaFree(e.d_item);
        if (e.d_blk) cudaFree(e.d_blk);
        if (e.d_bsys) cudaFree(e.d_bsys);
        if (e.d_sys) cudaFree(e.d_sys);
    };
    for (int q = 0; q < GENGA_MAX_VARIANTS; q++) {
        for (MutualCache::Entry &e : c->mcache->e[q]) drop(e);
        for (MutualCache::Entry &e : c->mcache->eb[q]) drop(e);
    }
    delete c->mcache;
    c->mcache = nullptr;
}

// The plan of cache entry e for `key` (the systems hs, cw consumer warps of
// npg groups each), built and uploaded on first use.  Returns false when it
// must be built while `s` is being captured, or when no plan fits: the caller
// then uses a one-sided variant.
static bool plan_cached(genga_ctx *c, MutualCache::Entry *ways, int nways, unsigned long long key,
                        const std::vector<HSys> &hs, int cw, int npg, cudaStream_t s, MutualPlan *P) {
    MutualCache::Entry *pe = nullptr;
    for (int w = 0; w < nways && !pe; w++)
        if (ways[w].key == key) pe = &ways[w];
    if (!pe) {  // the least recently used entry makes room
        pe = &ways[0];
        for (int w = 1; w < nways; w++)
            if (ways[w].used < pe->used) pe = &ways[w];
    }
    MutualCache::Entry &e = *pe;
    e.used = ++c->mcache->tick;
    if (e.key != key) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return false;
        PlanOut po;
        plan_systems(hs, cw, npg, c->sm_count, MUTUAL_MAX_ROWS, &po);
        if (cudaStreamSynchronize(s) != cudaSuccess) return false;  // the old tables may be in use
        if (e.d_item) cudaFree(e.d_item);
        if (e.d_blk) cudaFree(e.d_blk);
        if (e.d_bsys) cudaFree(e.d_bsys);
        if (e.d_sys) cudaFree(e.d_sys);
        e = MutualCache::Entry{};
        e.key = key;  // remembered also when no plan fits, so that it is not searched again
        e.used = c->mcache->tick;
        if (po.item.empty() || po.sys.empty()) return false;
        const size_t need = po.row_entries;
        if (need > c->partial_cap) {  // a larger workspace for the rows; captured step graphs used the old one
            double *bigger = nullptr;
            if (cudaMalloc(&bigger, need * sizeof(double)) != cudaSuccess) {
                cudaGetLastError();
                return false;
            }
            cudaFree(c->partial);
            c->partial = bigger;
            c->partial_cap = need;
            if (c->step_exec) {
                cudaGraphExecDestroy(c->step_exec);
                c->step_exec = nullptr;
            }
        }
        if (cudaMalloc(&e.d_item, po.item.size() * sizeof(int4)) != cudaSuccess ||
            cudaMalloc(&e.d_blk, po.blk.size() * sizeof(int2)) != cudaSuccess ||
            cudaMalloc(&e.d_bsys, po.bsys.size() * sizeof(int32_t)) != cudaSuccess ||
            cudaMalloc(&e.d_sys, po.sys.size() * sizeof(MSys)) != cudaSuccess)
            return false;
        if (cudaMemcpy(e.d_item, po.item.data(), po.item.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(e.d_blk, po.blk.data(), po.blk.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(e.d_bsys, po.bsys.data(), po.bsys.size() * sizeof(int32_t), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemcpy(e.d_sys, po.sys.data(), po.sys.size() * sizeof(MSys), cudaMemcpyHostToDevice) != cudaSuccess)
            return false;
        e.nb = (int)po.blk.size();
        e.gpb = cw * npg;
        e.items = (int)po.item.size();
        e.nsys = (int)po.sys.size();
        e.ok = true;
    }
    if (!e.ok) return false;
    *P = MutualPlan{e.nb, e.gpb, e.items, e.nsys, 0, e.d_item, e.d_blk, e.d_bsys, e.d_sys};
    return true;
}

static MutualCache *cache_of(genga_ctx *c) {
    if (!c->mcache) c->mcache = new (std::nothrow) MutualCache();
    return c->mcache;
}

// Single systems: the plan is built for the padded length (every group of
// it, the padding bodies massless) and serves every N of that length; the
// bodies' count goes with the returned plan.
bool mutual_plan(genga_ctx *c, int N, int v, cudaStream_t s, MutualPlan *P) {
    if (N <= 0 || v < 0 || v >= kNumMVariants || !cache_of(c)) return false;
    const int npad = (N + GENGA_PAD - 1) / GENGA_PAD * GENGA_PAD;
    if (!plan_cached(c, c->mcache->e[v], MC_WAYS, (unsigned long long)npad, {HSys{0, npad, npad, 0}},
                     kMVariants[v].cw, kMVariants[v].np, s, P))
        return false;
    P->nreal = N;
    return true;
}

bool mutual64_plan(genga_ctx *c, int N, int v, cudaStream_t s, MutualPlan *P) {
    if (N <= 0 || v < 0 || v >= kNumM64Variants || !cache_of(c)) return false;
    const int npad = (N + GENGA_PAD - 1) / GENGA_PAD * GENGA_PAD;
    if (!plan_cached(c, c->mcache->e[kNumMVariants + v], MC_WAYS, (unsigned long long)npad,
                     {HSys{0, npad, npad, 0}}, kM64Variants[v].cw, kM64Variants[v].bpt / 2, s, P))
        return false;
    P->nreal = N;
    return true;
}

bool mutual_plan_batched(genga_ctx *c, const BatchBodies &bb, unsigned long long key, int v, cudaStream_t s,
                         MutualPlan *P) {
    if (v < 0 || v >= kNumMVariants || !cache_of(c)) return false;
    std::vector<HSys> hs;
    for (int d = 0; d < bb.D; d++) {
        const int n = bb.off[d + 1] - bb.off[d];
        if (n > 0) hs.push_back(HSys{bb.poff[d], bb.poff[d + 1] - bb.poff[d], n, bb.off[d]});
    }
    if (hs.empty()) return false;
    return plan_cached(c, c->mcache->eb[v], MC_BATCH_WAYS, key, hs, kMVariants[v].cw, kMVariants[v].np, s, P);
}

cudaError_t init_mutual_kernels() {
    for (int q = 0; q < kNumMVariants; q++) {
        cudaError_t e = cudaFuncSetAttribute(kMVariants[q].fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kMVariants[q].smem);
        if (e != cudaSuccess) return e;
    }
    for (int q = 0; q < kNumM64Variants; q++) {
        cudaError_t e = cudaFuncSetAttribute(kM64Variants[q].fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kM64Variants[q].smem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_pass_mutual64(const PassArgs &a0, int v, int sm_count, cudaStream_t s) {
    PassArgs a = a0;
    const M64Variant &mv = kM64Variants[v];
    cudaError_t e = cudaMemsetAsync(a.work, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const int grid = std::min(sm_count, a.mp.items);
    mv.fn<<<grid, (mv.cw + 1 + mv.nr) * 32, mv.smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_combine_mutual64(const double *partial, const MutualPlan &P, int N, int npad, const uint32_t *perm,
                                    double tau, double *acc, double *vx, double *vy, double *vz, uint32_t *status,
                                    cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    combine_mutual64_kernel<<<dim3((npad / 2 * COMBINE_LANES + 255) / 256, 3), 256, 0, s>>>(partial, P, N, npad, perm, tau, acc, vx,
                                                                             vy, vz, status);
    return cudaGetLastError();
}

cudaError_t launch_pass_mutual(const PassArgs &a0, int v, int sm_count, cudaStream_t s) {
    PassArgs a = a0;
    const MVariant &mv = kMVariants[v];
    cudaError_t e = cudaMemsetAsync(a.work, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const int grid = std::min(sm_count, a.mp.items);
    mv.fn<<<grid, (mv.cw + 1 + mv.nr) * 32, mv.smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_combine_mutual(const double *partial, const MutualPlan &P, int N, int npad, const uint32_t *perm,
                                  double tau, double *acc, double *vx, double *vy, double *vz, uint32_t *status,
                                  cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    combine_mutual_kernel<<<dim3((npad / 2 * COMBINE_LANES + 255) / 256, 3), 256, 0, s>>>(partial, P, N, npad, perm, tau, acc, vx,
                                                                           vy, vz, status);
    return cudaGetLastError();
}

}  // namespace genga

// ------------------------------------------------- host check of a plan
// Builds the mutual plan of a batch of systems of n[d] bodies (padded to
// GENGA_PAD, a single system for nsys = 1) for cw consumer warps of npg
// groups, and verifies by enumeration what the pass relies on: inside a
// block every ordered pair of groups is visited once by its diagonal items;
// every pair of groups in different blocks of a system once, by a strip item
// of the earlier block; no item crosses a system or reaches a group without
// bodies; each block's rows are the rows its combine reads, each written by
// one item; the rows fit the plan's row space.
extern "C" genga_status genga_mutual_plan_check(int32_t nsys, const int32_t *n, int32_t cw, int32_t npg,
                                                int32_t ctas, int64_t *stats) {
    using namespace genga;
    if (nsys < 1 || nsys > GENGA_MAX_DISCS || !n || cw < 1 || npg < 1 || ctas < 1 || !stats)
        return GENGA_ERR_INVALID_ARG;
    std::vector<HSys> hs;
    int poff = 0, off = 0;
    for (int d = 0; d < nsys; d++) {
        if (n[d] < 0) return GENGA_ERR_INVALID_ARG;
        const int np = (n[d] + GENGA_PAD - 1) / GENGA_PAD * GENGA_PAD;
        if (n[d] > 0) hs.push_back(HSys{poff, np, n[d], off});
        poff += np;
        off += n[d];
    }
    for (int q = 0; q < 4; q++) stats[q] = 0;
    if (hs.empty()) return GENGA_OK;
    PlanOut po;
    plan_systems(hs, cw, npg, ctas, MUTUAL_MAX_ROWS, &po);
    if (po.item.empty()) return GENGA_ERR_CAPACITY;  // no plan fits
    const int gpb = cw * npg;
    const int ngr = poff / MG;
    std::vector<int> gsys(ngr, -1);  // system of each group holding bodies
    for (size_t d = 0; d < po.sys.size(); d++)
        for (int g = po.sys[d].poff / MG; g < po.sys[d].g1; g++) gsys[g] = (int)d;
    auto block_of = [&](int g) {
        const MSys &y = po.sys[gsys[g]];
        return y.blk0 + (g - y.poff / MG) / gpb;
    };
    auto block_groups = [&](int B, int *g0, int *g1) {
        const MSys &y = po.sys[po.bsys[B]];
        *g0 = y.poff / MG + (B - y.blk0) * gpb;
        *g1 = std::min(*g0 + gpb, y.g1);
    };
    // visits of each (i-group, j-group): ordered for diagonal items, unordered
    // (counted on (earlier, later)) for strip items
    std::vector<std::vector<int>> rows_seen(po.blk.size());
    std::vector<std::vector<uint8_t>> hit(ngr);
    for (size_t d = 0; d < po.sys.size(); d++)  // row gi: the groups of its system
        for (int g = po.sys[d].poff / MG; g < po.sys[d].g1; g++) hit[g].assign(po.sys[d].g1 - po.sys[d].poff / MG, 0);
    long long visits = 0;
    for (const int4 &it : po.item) {
        if (it.x < 0 || it.x >= (int)po.blk.size()) return GENGA_ERR_INVALID_ARG;
        int b0, b1;
        block_groups(it.x, &b0, &b1);
        const MSys &y = po.sys[po.bsys[it.x]];
        if (it.y < y.poff / MG || it.z > y.g1 || it.y >= it.z) return GENGA_ERR_INVALID_ARG;
        rows_seen[it.x].push_back(it.w);
        const bool diag = it.w < y.S;
        if (diag && (it.y < b0 || it.z > b1)) return GENGA_ERR_INVALID_ARG;
        if (!diag && it.y < b1) return GENGA_ERR_INVALID_ARG;  // strips start after the block
        for (int gi = b0; gi < b1; gi++)
            for (int gj = it.y; gj < it.z; gj++) {
                if (++hit[gi][gj - y.poff / MG] > 1) return GENGA_ERR_INVALID_ARG;
                visits++;
            }
    }
    for (size_t d = 0; d < po.sys.size(); d++) {
        const int a0 = po.sys[d].poff / MG, a1 = po.sys[d].g1;
        for (int gi = a0; gi < a1; gi++)
            for (int gj = a0; gj < a1; gj++) {
                const int bi = block_of(gi), bj = block_of(gj);
                const int want = bi == bj ? 1 : (bi < bj ? 1 : 0);
                if (hit[gi][gj - a0] != want) return GENGA_ERR_INVALID_ARG;
            }
    }
    int max_rows = 0;
    for (size_t B = 0; B < po.blk.size(); B++) {
        const MSys &y = po.sys[po.bsys[B]];
        const int nb = (po.bsys[B] + 1 < (int)po.sys.size() ? po.sys[po.bsys[B] + 1].blk0 : (int)po.blk.size()) - y.blk0;
        std::vector<int> want;
        for (int r = 0; r < po.blk[B].x; r++) want.push_back(r);
        for (int r = 0; r < po.blk[B].y; r++) want.push_back(y.S + r);
        std::vector<int> got = rows_seen[B];
        std::sort(got.begin(), got.end());
        if (got != want) return GENGA_ERR_INVALID_ARG;  // each row written once, every row read is written
        for (int r : got)
            if (r >= y.irows) return GENGA_ERR_INVALID_ARG;
        max_rows = std::max(max_rows, y.irows + nb);
    }
    stats[0] = (int64_t)po.item.size();
    stats[1] = max_rows;
    stats[2] = visits;
    stats[3] = (int64_t)po.row_entries;
    return GENGA_OK;
}
