// kick.cu -- the long-range pass of the GENGA kick (Sect. 1):
//
//   a_i = sum_{j != i} G m_j K(y_ij) (x_j - x_i) / r_ij^3,
//   y_ij = (r_ij / r_crit,ij - 0.1) / 0.9,  K = 1 for r_ij >= r_crit,ij.
//
// Layout.  Bodies sit in the spatial (Morton) order of order.cu.  A CTA owns
// KB * BPT consecutive i-bodies; warp w holds the 32 * BPT consecutive bodies
// ibase + w*32*BPT + k*32 + lane (k < BPT) in registers, so each warp covers a
// compact region.  j-bodies stream through shared memory in tiles of TILE
// (one-dimensional bulk copies completed on an mbarrier, STAGES-deep ring)
// and are read back as broadcasts.  Slices of the j range run in separate
// CTAs (grid.y) so the grid fills the GPU; their FP64 partial sums are
// combined afterwards in a fixed order, so results are bitwise reproducible.
//
// Tile classes.  For every (warp, tile) the bounding boxes of the two body
// sets give a lower bound D on every pair distance.  A tile is FAR for a warp
// when D exceeds an upper bound of r_crit,ij over the two sets (so K = 1 for
// every pair) and, in FP32, also 0.025 * (largest |coordinate|), which keeps
// the offset of two rounded FP32 positions within ~5e-6 of the true offset.
// FAR tiles run the plain loop (packed FP32 pairs); NEAR tiles run the
// screened loop below.
//
// Precision.  FP32 pass (the single-precision kick of Sect. 1): FAR pairs use
// the FP32-rounded positions; NEAR pairs use the hi/lo split of the FP64
// positions, dx = (x_j,hi - x_i,hi) + (x_j,lo - x_i,lo); r^2 in FP32, rsqrt on
// the SFU, each tile's terms summed in FP32 registers and added once per tile
// into double-float (hi + lo, ~48-bit) per-body accumulators, which are also
// the partial rows the combine adds up; FP64 appears only in screened pairs
// and in the final hi + lo.  FP64 pass: the same in FP64, with its
// own inverse square root (FP32 SFU seed + one third-order correction) and
// Neumaier-compensated accumulation every 32 terms.
//
// Screened pairs.  In NEAR tiles every pair is compared with an FP32 upper
// bound of r_crit,ij^2; a pair under it leaves the FP32/FP64 fast arithmetic
// and is evaluated exactly in FP64: r_crit,ij, K and the weighted force
// (close-encounter forces are always FP64, Sect. 1), and, if r_ij < r_crit,ij,
// it is appended to the encounter list (once, from the side with the smaller
// body index).
#include <algorithm>
#include <type_traits>
#include <cmath>

#include "internal.cuh"
#include "pass_common.cuh"

namespace genga {

namespace {

constexpr int KB = 256;  // threads per CTA of the pass kernels


// ----------------------------------------------------------- FP32 pass ----
// Persistent and warp-specialised.  Work items are (i-block, chunk of
// j-tiles), handed out by a global counter, so busy regions of the disc do
// not hold up the rest of the GPU.  One producer warp fetches
// items and fills a STAGES-deep ring of j-tiles with bulk copies (mbarrier
// "full" per slot, with a small header naming the item and tile); eight
// consumer warps compute and release each slot on its "empty" mbarrier, so
// warps with more NEAR work fall behind by up to STAGES tiles without
// stalling the others.  Each item's result goes to its own partial row
// (chunk, body), so the combined sum does not depend on which CTA ran it.
// FAR/NEAR is decided per (warp, 64-body group of the tile).  Registers hold
// only the FP32-rounded i positions and FP32 tile sums; the double-float
// per-body sums live in shared memory, touched once per tile.

struct StageHdr {
    int item, tile, flags, pad;  // flags: 1 first tile of item, 2 last tile, 4 no more work
};

// Work item q -> (i-block b, chunk k), k-major: q = k * iblocks + b.  Chunk k
// of an i-block covers the j-tiles of ranks u in the i-block's own order of
// tiles by distance from its diagonal tile (ranks 0, 1, 2, 3, 4, ... are the
// offsets 0, +1, -1, +2, -2, ...).  Chunk lengths come in tiers of
// decreasing length: the near tiles, with the NEAR groups and screened
// pairs, go out first in long items; the pass ends with single far tiles, so
// the CTAs run out of work at nearly the same time while the partial rows
// (one per chunk) stay few.
__device__ __forceinline__ void item_of(int q, int iblocks, int *b, int *k) {
    *k = q / iblocks;
    *b = q - *k * iblocks;
}

// Ranks [u0, u1) of chunk k: tiers of cnt[t] chunks of len[t] ranks, the
// first chunk shorter by `excess`.
__device__ __forceinline__ void chunk_ranks(int k, int ntier, int excess, const int *len, const int *cnt, int *u0,
                                            int *u1) {
    int u = -excess;
    for (int t = 0; t < ntier; t++) {
        if (k < cnt[t]) {
            const int a = u + k * len[t];
            *u0 = a > 0 ? a : 0;
            *u1 = a + len[t];
            return;
        }
        k -= cnt[t];
        u += cnt[t] * len[t];
    }
    *u0 = *u1 = 0;  // not reached for k < the number of chunks
}

__device__ __forceinline__ int tile_of_rank(int tdiag, int u, int ntiles) {
    const int off = (u & 1) ? (u + 1) / 2 : -(u / 2);
    return ((tdiag + off) % ntiles + ntiles) % ntiles;
}

// Geometry of the system a work item belongs to, with its chunk tiers.
struct ItemGeo {
    int poff, npad, Nd, off, nchunks, iblocks, ntier, excess;
    const int *tlen, *tcnt;
    long long pbase;
    int dt0;  // >= 0: the item covers tiles dt0.. of its system directly (test-particle i-blocks)
};

// Work items of a single system (the whole packed range).
struct SingleItems {
    __device__ int total(const PassArgs &a, int IB) const {
        return ((a.npad + IB - 1) / IB - a.tp_b0) * a.split + a.tp_b0;
    }
    __device__ void decode(const PassArgs &a, int IB, int, int q, int *ib, int *chunk, ItemGeo *g) const {
        const int nA = (a.npad + IB - 1) / IB - a.tp_b0;  // i-blocks with every tile (all of them without mode 2)
        *g = ItemGeo{0, a.npad, a.N, 0, a.split, nA, a.ntier, a.excess, a.tier_len, a.tier_n, 0, -1};
        if (q < nA * a.split) {
            item_of(q, nA, ib, chunk);
            *ib += a.tp_b0;
        } else {  // a test-particle i-block: the tiles with big bodies, row 0
            *ib = q - nA * a.split;
            *chunk = 0;
            g->dt0 = a.tp_t0;
        }
    }
};

// Work items of a batch: ranks of systems in handout order (largest items
// first), each system's items in the order of item_of, one tier of chunks
// per system (the small systems handed out last make the tail).
struct BatchPolicy {
    BatchBodies bb;
    BatchItems bi;
    __device__ int total(const PassArgs &, int) const { return bi.items_total; }
    __device__ void decode(const PassArgs &, int, int, int q, int *ib, int *chunk, ItemGeo *g) const {
        const int r = find_segment(bi.item0, bb.D, q);
        const int d = bi.order[r];
        const int np = bb.poff[d + 1] - bb.poff[d];
        *g = ItemGeo{bb.poff[d],        np, bb.off[d + 1] - bb.off[d], bb.off[d], bi.nchunks[d], bi.iblocks[d], 1,
                     bi.nchunks[d] * bi.blen[d] - np / GENGA_TILE_T, &bi.blen[d], &bi.nchunks[d],
                     (long long)bi.pbase[d], -1};
        item_of(q - bi.item0[r], g->iblocks, ib, chunk);
    }
};


// Scalar value of i-body k from its packed register: the j-packed loop keeps
// {x_k, x_k}, the i-packed loop {x_2q, x_2q+1} in register q.
template <bool IPACK>
__device__ __forceinline__ float ival(const f32x2 *V, int k) {
    float e, o;
    up2(V[IPACK ? k >> 1 : k], e, o);
    return (IPACK && (k & 1)) ? o : e;
}

// Two packed-loop flavours (the autotuner picks per size):
//   j-packed (IPACK = false): a lane pair holds two consecutive j-bodies
//     against one i-body held twice; j-tiles staged tile-blocked
//     x[TILE] y[TILE] z[TILE] w[TILE] (one 128-bit load covers four j);
//   i-packed (IPACK = true): a lane pair holds two i-bodies of the thread
//     against one j-body held twice; j-tiles staged as the duplicated-pair
//     copy {x, x, y, y}, {z, z, w, w} (two 128-bit loads per j).  Half the
//     registers for i positions and sums, so more bodies per thread fit.
template <int BPT, int CW, int TILE, int STAGES, int MINB, int UNR, bool IPACK, class Pol, bool TP>
__global__ void __launch_bounds__((CW + 1) * 32, MINB)
    pass_fp32_kernel(const __grid_constant__ PassArgs a, const __grid_constant__ Pol pol) {
    static_assert(TILE == GENGA_TILE_T, "the staged tile is one block of the tile-blocked copy");
    static_assert(!IPACK || BPT % 2 == 0, "the i-packed loop pairs the bodies of a thread");
    constexpr int NC = CW * 32;              // consumer threads (CW consumer warps + 1 producer warp)
    constexpr int IB = NC * BPT;             // i-bodies per item (the last i-block may be partial)
    constexpr int NG = TILE / 64;            // 64-body groups per tile
    constexpr int HF4 = IPACK ? 2 * TILE : TILE;  // float4 per staged hi slot
    constexpr int NP = IPACK ? BPT / 2 : BPT;     // packed registers per i coordinate
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float4 *s_hi = reinterpret_cast<float4 *>(smem_raw);
    float4 *s_lo = s_hi + STAGES * HF4;
    float4 *s_glo = s_lo + STAGES * TILE;  // [STAGES][NG] group boxes of each staged tile
    float4 *s_ghi = s_glo + STAGES * NG;
    float4 *s_tb = s_ghi + STAGES * NG;  // [STAGES][2] box of each staged tile (union of its groups)
    int32_t *s_gf = reinterpret_cast<int32_t *>(s_tb + 2 * STAGES);  // [STAGES][NG + 1] group flags, tile flags
    uint64_t *full = reinterpret_cast<uint64_t *>(s_gf + STAGES * (NG + 4));
    uint64_t *empty = full + STAGES;
    StageHdr *hdr = reinterpret_cast<StageHdr *>(empty + STAGES);
    __shared__ DF s_acc[3 * BPT * NC];      // [c][k][thread] double-float per-body sums
    __shared__ float4 s_ilo[BPT * NC];      // lo parts of this thread's i-bodies (current item)
    __shared__ float2 s_iscr[BPT * NC];     // and their screening factors
    __shared__ unsigned long long s_mask[BPT * NC];  // screened j of the current NEAR group, per i-body

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nitems = pol.total(a, IB);

    if (tid == 0) {
        for (int q = 0; q < STAGES; q++) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], CW);
        }
        fence_barrier_init();
    }
    __syncthreads();

    const uint64_t wlim = pass_wait_limit(a.wait_ns_log2);
    if (warp == CW) {  // ------------------------------------------ producer
        if (lane != 0) return;
        if (a.hold) return;  // test hook: no slot is ever filled (and no copy issued)
        constexpr uint32_t TBH = HF4 * sizeof(float4), TBL = TILE * sizeof(float4);
        unsigned n = 0;
        for (;;) {
            const int q = atomicAdd(a.work, 1);
            if (q >= nitems) {
                const int slot = n % STAGES;
                const unsigned u = n / STAGES;
                if (u > 0 && !mbar_wait_bounded(&empty[slot], (u - 1) & 1, a.status, wlim)) return;
                hdr[slot] = StageHdr{q, 0, 4, 0};
                mbar_arrive(&full[slot]);
                return;
            }
            int ib, chunk;
            ItemGeo geo;
            pol.decode(a, IB, TILE, q, &ib, &chunk, &geo);
            const int t0 = geo.poff / TILE, nt = geo.npad / TILE;  // first tile and tiles of the system
            const int tdiag = (ib * IB) / TILE;                      // the i-block's diagonal tile
            int u0, u1;
            if (geo.dt0 >= 0) {
                u0 = geo.dt0;
                u1 = nt;
            } else {
                chunk_ranks(chunk, geo.ntier, geo.excess, geo.tlen, geo.tcnt, &u0, &u1);
            }
            for (int ur = u0; ur < u1; ur++, n++) {
                const int t = t0 + (geo.dt0 >= 0 ? ur : tile_of_rank(tdiag, ur, nt));
                const int slot = n % STAGES;
                const unsigned u = n / STAGES;
                if (u > 0 && !mbar_wait_bounded(&empty[slot], (u - 1) & 1, a.status, wlim)) return;
                hdr[slot] = StageHdr{q, t, (ur == u0 ? 1 : 0) | (ur == u1 - 1 ? 2 : 0), 0};
                const Box tbx = group_box<NG>(a.gbox_lo, a.gbox_hi, t * NG);
                s_tb[2 * slot] = tbx.lo;
                s_tb[2 * slot + 1] = tbx.hi;
                if constexpr (TP) {  // test-particle mode 2: which kinds of bodies the groups hold
                    int32_t tf = 0;
#pragma unroll
                    for (int q = 0; q < NG; q++) {
                        const int32_t f = a.gflag[(size_t)t * NG + q];
                        s_gf[slot * (NG + 4) + q] = f;
                        tf |= f;
                    }
                    s_gf[slot * (NG + 4) + NG] = tf;
                }
                fence_proxy_async_smem();
                constexpr uint32_t GB = NG * sizeof(float4);
                mbar_arrive_expect_tx(&full[slot], TBH + TBL + 2 * GB);
                const void *src_hi = IPACK ? static_cast<const void *>(a.hid + (size_t)t * 2 * TILE)
                                           : static_cast<const void *>(a.hit + (size_t)t * 4 * TILE);
                bulk_g2s(s_hi + slot * HF4, src_hi, TBH, &full[slot]);
                bulk_g2s(s_lo + slot * TILE, a.lo + (size_t)t * TILE, TBL, &full[slot]);
                bulk_g2s(s_glo + slot * NG, a.gbox_lo + (size_t)t * NG, GB, &full[slot]);
                bulk_g2s(s_ghi + slot * NG, a.gbox_hi + (size_t)t * NG, GB, &full[slot]);
            }
        }
    }

    // ---------------------------------------------------------- consumers
    f32x2 XI[NP], YI[NP], ZI[NP];
#pragma unroll
    for (int q = 0; q < NP; q++) XI[q] = YI[q] = ZI[q] = 0ull;
    Box wbox = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
    int wbase = 0;
    bool in = false;  // this warp holds real i-bodies of the current item
    int32_t wflag = GENGA_GROUP_BIG;  // kinds of bodies the warp holds (test-particle mode 2)
    for (unsigned n = 0;; n++) {
        const int slot = n % STAGES;
        if (!mbar_wait_bounded(&full[slot], (n / STAGES) & 1, a.status, wlim)) return;
        const StageHdr h = hdr[slot];
        if (h.flags & 4) return;
        if (h.flags & 1) {  // first tile of an item: load this warp's i-bodies
            int ib, chunk;
            ItemGeo geo;
            pol.decode(a, IB, TILE, h.item, &ib, &chunk, &geo);
            wbase = geo.poff + ib * IB + warp * 32 * BPT;
            in = wbase - geo.poff < geo.npad;  // warps past the padded end hold dummy bodies
            float4 p[BPT];
#pragma unroll
            for (int k = 0; k < BPT; k++) {
                const int i = wbase + k * 32 + lane;
                p[k] = in ? a.hi[i] : make_float4(GENGA_PAD_POS, 0.f, 0.f, 0.f);
                s_ilo[k * NC + tid] = in ? a.lo[i] : make_float4(0.f, 0.f, 0.f, 0.f);
                s_iscr[k * NC + tid] = in ? a.scr[i] : make_float2(0.f, 0.f);
#pragma unroll
                for (int c = 0; c < 3; c++) s_acc[(c * BPT + k) * NC + tid] = DF{0.f, 0.f};
                s_mask[k * NC + tid] = 0ull;
            }
#pragma unroll
            for (int q = 0; q < NP; q++) {
                const float4 &u = p[IPACK ? 2 * q : q], &v = p[IPACK ? 2 * q + 1 : q];
                XI[q] = pk2(u.x, v.x);
                YI[q] = pk2(u.y, v.y);
                ZI[q] = pk2(u.z, v.z);
            }
            wflag = GENGA_GROUP_BIG;
            if (TP && in) {
                wflag = 0;
#pragma unroll
                for (int q = 0; q < BPT / 2; q++) wflag |= a.gflag[wbase / 64 + q];
            }
            if (in) {
                wbox = group_box<BPT / 2>(a.gbox_lo, a.gbox_hi, wbase / 64);
            } else {  // empty box: every tile is FAR, nothing is written
                const float INF = __int_as_float(0x7f800000);
                wbox = {make_float4(INF, INF, INF, 0.f), make_float4(-INF, -INF, -INF, 0.f)};
            }
        }
        // FP32 sums of this tile: i-packed, packed pairs TX; j-packed, scalar
        // ax (FAR groups accumulate packed even/odd-j sums and fold them in at
        // the end of the group)
        f32x2 TX[IPACK ? NP : 1], TY[IPACK ? NP : 1], TZ[IPACK ? NP : 1];
        float ax[BPT], ay[BPT], az[BPT];
#pragma unroll
        for (int q = 0; q < (IPACK ? NP : 1); q++) TX[q] = TY[q] = TZ[q] = 0ull;
#pragma unroll
        for (int k = 0; k < BPT; k++) ax[k] = ay[k] = az[k] = 0.f;
        const float4 *th = s_hi + slot * HF4;
        // test-particle mode 2: a warp of test particles skips the groups of
        // test particles; a warp holding test particles runs the groups that
        // hold test particles through the NEAR loop, which masks their pairs
        constexpr bool tp2 = TP;  // the kernel instantiated for test-particle mode 2 (n_big >= 0)
        const int32_t tflag = tp2 ? s_gf[slot * (NG + 4) + NG] : GENGA_GROUP_BIG;
        const bool tile_skip = tp2 && !(wflag & GENGA_GROUP_BIG) && !(tflag & GENGA_GROUP_BIG);
        // a warp of both kinds against a tile of test particles: every pair of
        // its test-particle lanes is excluded, so the tile is run as usual and
        // those lanes' tile sums are dropped
        const bool drop_tp = tp2 && (wflag & GENGA_GROUP_TP) && (wflag & GENGA_GROUP_BIG) && !(tflag & GENGA_GROUP_BIG);
        const bool tile_mixed = tp2 && !drop_tp && (wflag & GENGA_GROUP_TP) && (tflag & GENGA_GROUP_TP);
        // a tile FAR as a whole needs no per-group test (the tile box holds
        // every group box, so its gap is smaller and its bound larger)
        const bool tile_far =
            !tile_mixed && far_pair_of_boxes(wbox, Box{s_tb[2 * slot], s_tb[2 * slot + 1]}, true);
        for (int g = 0; g < NG; g++) {
            if (tile_skip) break;
            const int32_t gflag = tp2 ? s_gf[slot * (NG + 4) + g] : GENGA_GROUP_BIG;
            if (tp2 && !(wflag & GENGA_GROUP_BIG) && !(gflag & GENGA_GROUP_BIG)) continue;  // no pair interacts
            const bool masked = tile_mixed && (wflag & GENGA_GROUP_TP) && (gflag & GENGA_GROUP_TP);
            const Box gb = {s_glo[slot * NG + g], s_ghi[slot * NG + g]};
            const float *tx = reinterpret_cast<const float *>(th) + g * 64, *ty = tx + TILE, *tz = tx + 2 * TILE,
                        *tw = tx + 3 * TILE;     // j-packed layout
            const float4 *td = th + g * 128;  // i-packed layout: two float4 per j
            if (!masked && (tile_far || far_pair_of_boxes(wbox, gb, true))) {
                // every pair: K = 1, FP32-rounded positions accurate enough
                if constexpr (IPACK) {
#pragma unroll(UNR)
                    for (int jj = 0; jj < 64; jj++) {
                        const ulonglong2 A = *reinterpret_cast<const ulonglong2 *>(td + 2 * jj);      // {xx}, {yy}
                        const ulonglong2 B = *reinterpret_cast<const ulonglong2 *>(td + 2 * jj + 1);  // {zz}, {ww}
#pragma unroll
                        for (int q = 0; q < NP; q++) {
                            const f32x2 DX = sub2(A.x, XI[q]), DY = sub2(A.y, YI[q]), DZ = sub2(B.x, ZI[q]);
                            const f32x2 R2 = fma2(DZ, DZ, fma2(DY, DY, mul2(DX, DX)));
                            float ra, rb;
                            up2(R2, ra, rb);
                            const f32x2 RI = pk2(rsqrt_sfu(ra), rsqrt_sfu(rb));
                            const f32x2 S = mul2(mul2(B.y, RI), mul2(RI, RI));
                            TX[q] = fma2(S, DX, TX[q]);
                            TY[q] = fma2(S, DY, TY[q]);
                            TZ[q] = fma2(S, DZ, TZ[q]);
                        }
                    }
                } else {
                    // two consecutive j per packed register, four j per step
                    f32x2 AX[BPT], AY[BPT], AZ[BPT];  // (even j, odd j) sums
#pragma unroll
                    for (int k = 0; k < BPT; k++) AX[k] = AY[k] = AZ[k] = 0ull;
#pragma unroll(UNR)
                    for (int jj = 0; jj < 64; jj += 4) {
                        const ulonglong2 X4 = *reinterpret_cast<const ulonglong2 *>(tx + jj);
                        const ulonglong2 Y4 = *reinterpret_cast<const ulonglong2 *>(ty + jj);
                        const ulonglong2 Z4 = *reinterpret_cast<const ulonglong2 *>(tz + jj);
                        const ulonglong2 W4 = *reinterpret_cast<const ulonglong2 *>(tw + jj);
#pragma unroll
                        for (int half = 0; half < 2; half++) {
                            const f32x2 JX = half ? X4.y : X4.x, JY = half ? Y4.y : Y4.x;
                            const f32x2 JZ = half ? Z4.y : Z4.x, JW = half ? W4.y : W4.x;
#pragma unroll
                            for (int k = 0; k < BPT; k++) {
                                const f32x2 DX = sub2(JX, XI[k]), DY = sub2(JY, YI[k]), DZ = sub2(JZ, ZI[k]);
                                const f32x2 R2 = fma2(DZ, DZ, fma2(DY, DY, mul2(DX, DX)));
                                float ra, rb;
                                up2(R2, ra, rb);
                                const f32x2 RI = pk2(rsqrt_sfu(ra), rsqrt_sfu(rb));
                                const f32x2 S = mul2(mul2(JW, RI), mul2(RI, RI));
                                AX[k] = fma2(S, DX, AX[k]);
                                AY[k] = fma2(S, DY, AY[k]);
                                AZ[k] = fma2(S, DZ, AZ[k]);
                            }
                        }
                    }
#pragma unroll
                    for (int k = 0; k < BPT; k++) {
                        float e0, e1;
                        up2(AX[k], e0, e1);
                        ax[k] += e0 + e1;
                        up2(AY[k], e0, e1);
                        ay[k] += e0 + e1;
                        up2(AZ[k], e0, e1);
                        az[k] += e0 + e1;
                    }
                }
            } else {
                // NEAR group: hi/lo offsets, every pair screened; sums into sx, sy, sz
                // MASK: the group and the warp both hold test particles (mode 2):
                // pairs of two test particles are skipped pair by pair
                auto near_group = [&](auto mask_tag, float(&sx)[BPT], float(&sy)[BPT], float(&sz)[BPT]) {
                    constexpr bool MASK = decltype(mask_tag)::value;
                    const float4 *tl = s_lo + slot * TILE + g * 64;
                    float xl[BPT], yl[BPT], zl[BPT], thr[BPT];
                    unsigned itp = 0u;  // bit k: i_k is a test particle (masked groups only)
#pragma unroll
                    for (int k = 0; k < BPT; k++) {
                        const float4 l = s_ilo[k * NC + tid];
                        const float2 sc = s_iscr[k * NC + tid];
                        xl[k] = l.x; yl[k] = l.y; zl[k] = l.z;
                        thr[k] = screen_threshold(sc.x, sc.y, gb.lo.w, gb.hi.w);
                        if constexpr (MASK) itp |= (unsigned)(l.w != 0.f) << k;
                    }
#pragma unroll 2
                    for (int jj = 0; jj < 64; jj++) {
                        float jx, jy, jz, jw;
                        if constexpr (IPACK) {
                            const float4 A = td[2 * jj], B = td[2 * jj + 1];
                            jx = A.x; jy = A.z; jz = B.x; jw = B.z;
                        } else {
                            jx = tx[jj]; jy = ty[jj]; jz = tz[jj]; jw = tw[jj];
                        }
                        const float4 pl = tl[jj];
                        unsigned screened = 0u;  // bit k: pair (i_k, j) is under the screening bound
#pragma unroll
                        for (int k = 0; k < BPT; k++) {
                            const float dx = (jx - ival<IPACK>(XI, k)) + (pl.x - xl[k]);
                            const float dy = (jy - ival<IPACK>(YI, k)) + (pl.y - yl[k]);
                            const float dz = (jz - ival<IPACK>(ZI, k)) + (pl.z - zl[k]);
                            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                            const float ri = rsqrt_sfu(r2);
                            bool skip = false;
                            if constexpr (MASK) skip = (itp >> k & 1u) && pl.w != 0.f;  // two test particles
                            const bool near = r2 < thr[k] && !skip;
                            screened |= (unsigned)near << k;
                            const float sf = (near || skip) ? 0.f : (jw * ri) * (ri * ri);
                            sx[k] = fmaf(sf, dx, sx[k]);
                            sy[k] = fmaf(sf, dy, sy[k]);
                            sz[k] = fmaf(sf, dz, sz[k]);
                        }
                        if (screened) {  // rare: noted here, evaluated after the loop
#pragma unroll
                            for (int k = 0; k < BPT; k++)
                                if (screened & (1u << k)) s_mask[k * NC + tid] |= 1ull << jj;
                        }
                    }
                    // the screened pairs of this group, exactly in FP64 (the
                    // pair of a body with itself contributes nothing)
#pragma unroll 1
                    for (int k = 0; k < BPT; k++) {
                        unsigned long long msk = s_mask[k * NC + tid];
                        if (!msk) continue;
                        s_mask[k * NC + tid] = 0ull;
                        const int i = wbase + k * 32 + lane;
                        int ib_, ch_;
                        ItemGeo geo;
                        pol.decode(a, IB, TILE, h.item, &ib_, &ch_, &geo);
                        double fx = 0.0, fy = 0.0, fz = 0.0;
                        do {
                            const int jj = __ffsll((long long)msk) - 1;
                            msk &= msk - 1;
                            const int j = h.tile * TILE + g * 64 + jj;
                            if (j != i) {
                                const double3 f = screened_pair(a, i, j, geo.poff, geo.Nd, geo.off);
                                fx += f.x;
                                fy += f.y;
                                fz += f.z;
                            }
                        } while (msk);
                        const double f3[3] = {fx, fy, fz};
#pragma unroll
                        for (int c = 0; c < 3; c++) {
                            DF &t = s_acc[(c * BPT + k) * NC + tid];
                            const DF d = df_of_double(f3[c]);
                            t = df_add(t, d.hi, d.lo);
                        }
                    }
                };
                if constexpr (IPACK) {
                    float nx[BPT], ny[BPT], nz[BPT];
#pragma unroll
                    for (int k = 0; k < BPT; k++) nx[k] = ny[k] = nz[k] = 0.f;
                    if (masked)
                        near_group(std::true_type{}, nx, ny, nz);
                    else
                        near_group(std::false_type{}, nx, ny, nz);
#pragma unroll
                    for (int q = 0; q < NP; q++) {
                        TX[q] = add2(TX[q], pk2(nx[2 * q], nx[2 * q + 1]));
                        TY[q] = add2(TY[q], pk2(ny[2 * q], ny[2 * q + 1]));
                        TZ[q] = add2(TZ[q], pk2(nz[2 * q], nz[2 * q + 1]));
                    }
                } else {
                    if (masked)
                        near_group(std::true_type{}, ax, ay, az);
                    else
                        near_group(std::false_type{}, ax, ay, az);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);  // this warp is done reading the slot
        if constexpr (IPACK) {
#pragma unroll
            for (int k = 0; k < BPT; k++) {
                ax[k] = ival<true>(TX, k);
                ay[k] = ival<true>(TY, k);
                az[k] = ival<true>(TZ, k);
            }
        }
        if (drop_tp) {
#pragma unroll
            for (int k = 0; k < BPT; k++)
                if (s_ilo[k * NC + tid].w != 0.f) ax[k] = ay[k] = az[k] = 0.f;
        }
#pragma unroll
        for (int k = 0; k < BPT; k++) {  // fold the tile's FP32 sums into the double-float sums
            DF &tx_ = s_acc[(0 * BPT + k) * NC + tid];
            DF &ty_ = s_acc[(1 * BPT + k) * NC + tid];
            DF &tz_ = s_acc[(2 * BPT + k) * NC + tid];
            tx_ = df_add(tx_, ax[k], 0.f);
            ty_ = df_add(ty_, ay[k], 0.f);
            tz_ = df_add(tz_, az[k], 0.f);
        }
        if ((h.flags & 2) && in) {  // last tile of the item: write its partial row
            int ib, chunk;
            ItemGeo geo;
            pol.decode(a, IB, TILE, h.item, &ib, &chunk, &geo);
            const size_t np = (size_t)geo.npad;
            // partial rows of the FP32 pass: double-float pairs (8 bytes, like a double)
            float2 *out = reinterpret_cast<float2 *>(a.partial + geo.pbase) + (size_t)chunk * 3 * np;
#pragma unroll
            for (int k = 0; k < BPT; k++) {
                const int i = wbase - geo.poff + k * 32 + lane;
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const DF t = s_acc[(c * BPT + k) * NC + tid];
                    out[c * np + i] = make_float2(t.hi, t.lo);
                }
            }
        }
    }
}

// ----------------------------------------------------------- FP64 pass ----
struct Comp {  // Neumaier-compensated FP64 accumulator
    double s, c;
    __device__ __forceinline__ void add(double v) {
        const double t = s + v;
        c += (fabs(s) >= fabs(v)) ? ((s - t) + v) : ((v - t) + s);
        s = t;
    }
};

template <int BPT, int TILE, int STAGES>
__global__ void __launch_bounds__(KB, 2) pass_fp64_kernel(const __grid_constant__ PassArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    double4_32a *s_p = reinterpret_cast<double4_32a *>(smem_raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(s_p + STAGES * TILE);
    __shared__ int s_abort;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ibase = blockIdx.x * (KB * BPT);
    const int wbase = ibase + warp * 32 * BPT;
    const int slice = blockIdx.y;
    // test-particle mode 2 plan: an i-block of test particles only needs the
    // tiles from the first big body on, in its first slice (partial row 0)
    const bool tp_block = (int)blockIdx.x < a.tp_b0;
    if (tp_block && slice != 0) return;
    const int t0 = tp_block ? a.tp_t0 : (int)((long long)a.ntiles * slice / a.split);
    const int t1 = tp_block ? a.ntiles : (int)((long long)a.ntiles * (slice + 1) / a.split);

    double xi[BPT], yi[BPT], zi[BPT];
    float H[BPT], A[BPT];
    Comp CX[BPT], CY[BPT], CZ[BPT];
#pragma unroll
    for (int k = 0; k < BPT; k++) {
        const int i = wbase + k * 32 + lane;
        const double4_32a p = a.p64[i];
        const float2 s = a.scr[i];
        xi[k] = p.x; yi[k] = p.y; zi[k] = p.z;
        H[k] = s.x; A[k] = s.y;
        CX[k] = CY[k] = CZ[k] = Comp{0.0, 0.0};
    }
    const Box wbox = group_box<(BPT + 1) / 2>(a.gbox_lo, a.gbox_hi, wbase / 64);
    // test-particle mode 2: kinds of bodies the warp holds; its test particles
    const bool tp2 = a.n_big >= 0;
    int32_t wflag = GENGA_GROUP_BIG;
    unsigned itp = 0u;
    if (tp2) {
        wflag = 0;
#pragma unroll
        for (int q = 0; q < (BPT + 1) / 2; q++) wflag |= a.gflag[wbase / 64 + q];
#pragma unroll
        for (int k = 0; k < BPT; k++) itp |= (unsigned)(a.lo[wbase + k * 32 + lane].w != 0.f) << k;
    }

    constexpr uint32_t TB = TILE * sizeof(double4_32a);
    if (tid == 0) {
        for (int s = 0; s < STAGES; s++) mbar_init(&bars[s], 1);
        fence_barrier_init();
        s_abort = 0;
    }
    __syncthreads();
    if (tid == 0) {
        for (int s = 0; s < STAGES - 1 && t0 + s < t1; s++) {
            mbar_arrive_expect_tx(&bars[s], TB);
            bulk_g2s(s_p + s * TILE, a.p64 + (size_t)(t0 + s) * TILE, TB, &bars[s]);
        }
    }

    for (int t = t0; t < t1; t++) {
        const int it = t - t0;
        const int stage = it % STAGES;
        if (tid == 0) {
            const int tn = t + STAGES - 1;
            if (tn < t1) {
                const int sn = (it + STAGES - 1) % STAGES;
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&bars[sn], TB);
                bulk_g2s(s_p + sn * TILE, a.p64 + (size_t)tn * TILE, TB, &bars[sn]);
            }
        }
        const Box tbox = group_box<TILE / 64>(a.gbox_lo, a.gbox_hi, t * (TILE / 64));
        int32_t tflag = GENGA_GROUP_BIG;
        if (tp2) {
            tflag = 0;
#pragma unroll
            for (int q = 0; q < TILE / 64; q++) tflag |= a.gflag[t * (TILE / 64) + q];
        }
        const bool skip_tile = tp2 && !(wflag & GENGA_GROUP_BIG) && !(tflag & GENGA_GROUP_BIG);
        // both kinds in the warp, test particles only in the tile: run it as
        // usual and drop the test-particle lanes' sums
        const bool drop_tp = tp2 && (wflag & GENGA_GROUP_TP) && (wflag & GENGA_GROUP_BIG) && !(tflag & GENGA_GROUP_BIG);
        const bool masked = tp2 && !drop_tp && (wflag & GENGA_GROUP_TP) && (tflag & GENGA_GROUP_TP);
        const bool far = !masked && far_pair_of_boxes(wbox, tbox, false);
        double thr[BPT];
#pragma unroll
        for (int k = 0; k < BPT; k++) thr[k] = (double)screen_threshold(H[k], A[k], tbox.lo.w, tbox.hi.w);

        if (!mbar_wait_bounded(&bars[stage], (uint32_t)((it / STAGES) & 1), a.status)) s_abort = 1;

        const double4_32a *tp = s_p + stage * TILE;
        for (int j0 = 0; j0 < (skip_tile ? 0 : TILE); j0 += 32) {
            double px[BPT], py[BPT], pz[BPT];
#pragma unroll
            for (int k = 0; k < BPT; k++) px[k] = py[k] = pz[k] = 0.0;
            if (far) {
#pragma unroll 2
                for (int jj = j0; jj < j0 + 32; jj++) {
                    const double4_32a pj = tp[jj];
#pragma unroll
                    for (int k = 0; k < BPT; k++) {
                        const double dx = pj.x - xi[k], dy = pj.y - yi[k], dz = pj.z - zi[k];
                        const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
                        const double s = pj.w * rsqrt3_fp64(r2);
                        px[k] = fma(s, dx, px[k]);
                        py[k] = fma(s, dy, py[k]);
                        pz[k] = fma(s, dz, pz[k]);
                    }
                }
            } else {
#pragma unroll 2
                for (int jj = j0; jj < j0 + 32; jj++) {
                    const double4_32a pj = tp[jj];
                    const bool jtp = masked && a.lo[t * TILE + jj].w != 0.f;  // j is a test particle
                    unsigned screened = 0u;
#pragma unroll
                    for (int k = 0; k < BPT; k++) {
                        const double dx = pj.x - xi[k], dy = pj.y - yi[k], dz = pj.z - zi[k];
                        const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
                        const bool skip = jtp && (itp >> k & 1u);  // two test particles: no force
                        const bool near = r2 < thr[k] && !skip;
                        screened |= (unsigned)near << k;
                        const double s = (near || skip) ? 0.0 : pj.w * rsqrt3_fp64(r2);
                        px[k] = fma(s, dx, px[k]);
                        py[k] = fma(s, dy, py[k]);
                        pz[k] = fma(s, dz, pz[k]);
                    }
                    if (screened) {
#pragma unroll
                        for (int k = 0; k < BPT; k++) {
                            if (screened & (1u << k)) {
                                const double3 f = screened_pair(a, wbase + k * 32 + lane, t * TILE + jj, 0, a.N, 0);
                                CX[k].add(f.x);
                                CY[k].add(f.y);
                                CZ[k].add(f.z);
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < BPT; k++) {
                if (drop_tp && (itp >> k & 1u)) px[k] = py[k] = pz[k] = 0.0;
                CX[k].add(px[k]);
                CY[k].add(py[k]);
                CZ[k].add(pz[k]);
            }
        }
        __syncthreads();
        if (s_abort) break;
    }

    const size_t np = (size_t)a.npad;
    double *out = a.partial + (size_t)slice * 3 * np;
#pragma unroll
    for (int k = 0; k < BPT; k++) {
        const int i = wbase + k * 32 + lane;
        out[i] = CX[k].s + CX[k].c;
        out[np + i] = CY[k].s + CY[k].c;
        out[2 * np + i] = CZ[k].s + CZ[k].c;
    }
}

// ------------------------------------------------------------ combine ----
// One thread per (body, component): the body's partial rows summed in row
// order -- double-float pairs of the FP32 pass in double-float arithmetic,
// FP64 rows of the FP64 pass Neumaier-compensated.  The rows are fetched
// COMBINE_BATCH at a time before any of them is added, so a thread waits for
// a few memory round trips, not one per row.  Then the optional acc output
// and v_c += acc_c * tau for the body's caller index; non-finite
// accelerations raise NONFINITE.
constexpr int COMBINE_BATCH = 16;

__device__ __forceinline__ double df_row_sum(const float2 *__restrict__ p, size_t stride, int nrows) {
    DF t{0.f, 0.f};
    for (int q0 = 0; q0 < nrows; q0 += COMBINE_BATCH) {
        float2 v[COMBINE_BATCH];
#pragma unroll
        for (int u = 0; u < COMBINE_BATCH; u++)
            v[u] = (q0 + u < nrows) ? p[(size_t)(q0 + u) * stride] : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < COMBINE_BATCH; u++)
            if (q0 + u < nrows) t = df_add(t, v[u].x, v[u].y);
    }
    return (double)t.hi + (double)t.lo;
}

__device__ __forceinline__ double comp_row_sum(const double *__restrict__ p, size_t stride, int nrows) {
    Comp s{0.0, 0.0};
    for (int q0 = 0; q0 < nrows; q0 += COMBINE_BATCH) {
        double v[COMBINE_BATCH];
#pragma unroll
        for (int u = 0; u < COMBINE_BATCH; u++) v[u] = (q0 + u < nrows) ? p[(size_t)(q0 + u) * stride] : 0.0;
#pragma unroll
        for (int u = 0; u < COMBINE_BATCH; u++)
            if (q0 + u < nrows) s.add(v[u]);
    }
    return s.s + s.c;
}

__device__ __forceinline__ void apply_component(double t, int c, int i, size_t NT, double tau, double *acc,
                                                double *vx, double *vy, double *vz, uint32_t *status) {
    if (!isfinite(t)) atomicOr(status, GENGA_BIT(GENGA_ERR_NONFINITE));
    if (acc) acc[c * NT + i] = t;
    if (tau != 0.0) {
        double *v = c == 0 ? vx : (c == 1 ? vy : vz);
        v[i] += t * tau;
    }
}

// grid (ceil(N / 256), 3): blockIdx.y is the component
__global__ void combine_kernel(const double *__restrict__ partial, int split, int one_row_end, int N, int npad,
                               int fp64_rows,
                               const uint32_t *__restrict__ perm, double tau, double *__restrict__ acc,
                               double *__restrict__ vx, double *__restrict__ vy, double *__restrict__ vz,
                               uint32_t *__restrict__ status) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (k >= N) return;
    const size_t off = (size_t)c * npad + k, stride = 3 * (size_t)npad;
    const int rows = k < one_row_end ? 1 : split;  // test-particle i-blocks of a mode-2 plan: row 0 only
    const double t = fp64_rows ? comp_row_sum(partial + off, stride, rows)
                               : df_row_sum(reinterpret_cast<const float2 *>(partial) + off, stride, rows);
    apply_component(t, c, (int)perm[k], (size_t)N, tau, acc, vx, vy, vz, status);
}

// Batched: packed position p of system d; rows of d start at pbase[d], one
// per j-chunk, each npad_d long (double-float pairs of the FP32 pass).  grid
// (ceil(npad_total / 256), 3).
__global__ void combine_batched_kernel(const double *__restrict__ partial, const uint32_t *__restrict__ perm,
                                       double tau, double *__restrict__ acc, double *__restrict__ vx,
                                       double *__restrict__ vy, double *__restrict__ vz, uint32_t *__restrict__ status,
                                       const __grid_constant__ BatchBodies bb, const __grid_constant__ BatchItems bi) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (p >= bb.npad_total) return;
    const int d = find_segment(bb.poff, bb.D, p);
    const int k = p - bb.poff[d];
    if (k >= bb.off[d + 1] - bb.off[d]) return;
    const size_t np = (size_t)(bb.poff[d + 1] - bb.poff[d]);
    const double t =
        df_row_sum(reinterpret_cast<const float2 *>(partial + bi.pbase[d]) + (size_t)c * np + k, 3 * np, bi.nchunks[d]);
    apply_component(t, c, (int)perm[bb.off[d] + k], (size_t)bb.N_total, tau, acc, vx, vy, vz, status);
}

// ------------------------------------------------------ encounter list ----
// One CTA sorts the list (keys i * 2^32 + j, ascending) with a bitonic
// network: in shared memory up to 8192 entries, in place in global memory
// above that (enc_cap is a power of two, so the padded length fits).
constexpr int SORT_THREADS = 1024;
constexpr int SORT_SMEM = 8192;

__device__ __forceinline__ unsigned long long pair_key(int2 p) {
    return ((unsigned long long)(unsigned)p.x << 32) | (unsigned)p.y;
}

__global__ void __launch_bounds__(SORT_THREADS) sort_pairs_kernel(int2 *__restrict__ enc, int32_t cap,
                                                                  const int32_t *__restrict__ count) {
    __shared__ unsigned long long sk[SORT_SMEM];
    const int n = min(*count, cap);
    if (n <= 1) return;
    int L = 1;
    while (L < n) L <<= 1;
    const unsigned long long SENT = ~0ull;
    if (L <= SORT_SMEM) {
        for (int q = threadIdx.x; q < L; q += SORT_THREADS) sk[q] = (q < n) ? pair_key(enc[q]) : SENT;
        __syncthreads();
        for (int k = 2; k <= L; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int q = threadIdx.x; q < L; q += SORT_THREADS) {
                    const int p = q ^ j;
                    if (p > q) {
                        const bool up = (q & k) == 0;
                        const unsigned long long u = sk[q], v = sk[p];
                        if ((u > v) == up) { sk[q] = v; sk[p] = u; }
                    }
                }
                __syncthreads();
            }
        }
        for (int q = threadIdx.x; q < n; q += SORT_THREADS)
            enc[q] = make_int2((int)(sk[q] >> 32), (int)(sk[q] & 0xffffffffu));
        return;
    }
    // large list: pad with sentinels, then the same network on global memory
    for (int q = n + threadIdx.x; q < L; q += SORT_THREADS) enc[q] = make_int2(-1, -1);
    __syncthreads();
    for (int k = 2; k <= L; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int q = threadIdx.x; q < L; q += SORT_THREADS) {
                const int p = q ^ j;
                if (p > q) {
                    const bool up = (q & k) == 0;
                    const int2 u2 = enc[q], v2 = enc[p];
                    const unsigned long long u = pair_key(u2), v = pair_key(v2);
                    if ((u > v) == up) { enc[q] = v2; enc[p] = u2; }
                }
            }
            __syncthreads();
        }
    }
}

__global__ void copy_pairs_kernel(const int2 *__restrict__ enc, const int32_t *__restrict__ count,
                                  int32_t enc_cap, int32_t *__restrict__ pairs, int32_t capacity,
                                  int32_t *__restrict__ count_out, uint32_t *__restrict__ status) {
    const int total = *count;
    const int avail = min(total, enc_cap);
    const int n = min(avail, capacity);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const int2 p = enc[q];
        pairs[2 * q] = p.x;
        pairs[2 * q + 1] = p.y;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (count_out) *count_out = total;
        if (total > capacity || total > enc_cap) atomicOr(status, GENGA_BIT(GENGA_ERR_CAPACITY));
    }
}

// ------------------------------------------------------------ variants ----
constexpr int F32_TILE = 256;
constexpr int F32_TAIL_ITEMS = 5;  // single-tile work items per resident CTA at the end of a pass

// FP32 pass variants (packing, bodies per thread, consumer warps, CTAs per
// SM, FAR-loop unroll, ring stages); the autotuner in api.cu times them per N
// bucket and keeps the fastest.  The first entry is the default where no
// tuning is possible (stream capture, batched passes).
struct F32Variant {
    bool ipack;
    int bpt, cw, minb, stages;  // bodies per thread, consumer warps, resident CTAs per SM, ring depth
    void (*fn)(const PassArgs, const SingleItems);
    void (*fnb)(const PassArgs, const BatchPolicy);
    void (*fn_tp)(const PassArgs, const SingleItems);  // test-particle mode 2 instantiations
    void (*fnb_tp)(const PassArgs, const BatchPolicy);
};
#define GENGA_F32V(IP, BPT, CW, MINB, UNR, ST)                                                           \
    {IP,                                                                                                 \
     BPT,                                                                                                \
     CW,                                                                                                 \
     MINB,                                                                                               \
     ST,                                                                                                 \
     pass_fp32_kernel<BPT, CW, F32_TILE, ST, MINB, UNR, IP, SingleItems, false>,                        \
     pass_fp32_kernel<BPT, CW, F32_TILE, ST, MINB, UNR, IP, BatchPolicy, false>,                        \
     pass_fp32_kernel<BPT, CW, F32_TILE, ST, MINB, UNR, IP, SingleItems, true>,                         \
     pass_fp32_kernel<BPT, CW, F32_TILE, ST, MINB, UNR, IP, BatchPolicy, true>}
const F32Variant kF32Variants[] = {
    GENGA_F32V(true, 2, 8, 2, 4, 4), GENGA_F32V(true, 2, 4, 4, 8, 3),  GENGA_F32V(true, 2, 4, 4, 4, 3),
    GENGA_F32V(true, 2, 8, 2, 4, 3), GENGA_F32V(true, 2, 8, 2, 8, 4),  GENGA_F32V(false, 2, 8, 2, 8, 4),
    GENGA_F32V(true, 2, 16, 1, 8, 4), GENGA_F32V(true, 4, 8, 2, 2, 4),
};
#undef GENGA_F32V
constexpr int kNumF32Variants = sizeof(kF32Variants) / sizeof(kF32Variants[0]);
static_assert(kNumF32Variants <= GENGA_MAX_VARIANTS, "the context records tuning times of GENGA_MAX_VARIANTS variants");
constexpr int F64_BPT = 2, F64_TILE = 128, F64_STAGES = 3;
constexpr int F64_WAVES = 16;  // FP64 pass: j-slices so that the CTAs fill about this many waves

size_t smem_fp32(bool ipack, int stages) {
    const size_t hf4 = ipack ? 2 * F32_TILE : F32_TILE;
    return (size_t)stages * (hf4 + F32_TILE) * sizeof(float4) + (size_t)stages * (F32_TILE / 64 + 1) * 2 * sizeof(float4) +
           (size_t)stages * (F32_TILE / 64 + 4) * sizeof(int32_t) +
           2 * stages * sizeof(uint64_t) + stages * sizeof(StageHdr);
}
size_t smem_fp64() { return (size_t)F64_STAGES * F64_TILE * sizeof(double4_32a) + F64_STAGES * sizeof(uint64_t); }

}  // namespace

// Work decomposition of one pass.
// FP32 (persistent): split j-chunks per i-block in tiers of chunk lengths,
// built from the end of the pass: F32_TAIL_ITEMS single tiles per resident
// CTA come last; each earlier tier has chunks as long as the work of all the
// tiers after it per CTA (so an item of that tier started late still ends
// while the later, shorter items keep the other CTAs busy) and about as much
// work as they have together; lengths stop growing at a quarter of a CTA's share of
// the pass, and the first tier takes what is left (its first chunk made
// shorter to fit).  split = partial rows per body; grid = resident CTAs.
// FP64: `split` contiguous j-slices per i-block, one CTA each, sized to
// F64_WAVES waves of two CTAs per SM (one wave left the SMs holding a second
// CTA to finish alone).  In both cases split * 3 * npad partial sums
// (8 bytes each) fit in partial_cap.
int num_fp32_variants() { return kNumF32Variants; }

// Test-particle mode 2 (n_big >= 0): the big bodies are ordered after the
// test particles, so i-blocks that end before position N - n_big hold test
// particles only: their one item covers the tiles from the first big body on
// (TP-only tiles have no pair with them); the i-blocks from there on get the
// whole plan.  Sets tp_b0, tp_t0, tp_rows_end; returns the i-blocks with the
// whole plan.
int plan_tp2(int N, int iblocks, int ib, int tile, PassArgs *a) {
    a->tp_b0 = a->tp_t0 = a->tp_rows_end = 0;
    if (a->n_big < 0 || a->n_big == 0 || a->n_big >= N) return iblocks;
    const int first_big = N - a->n_big;
    const int b0 = first_big / ib;
    if (b0 <= 0) return iblocks;
    a->tp_b0 = b0;
    a->tp_t0 = first_big / tile;
    a->tp_rows_end = b0 * ib;
    return iblocks - b0;
}

void plan_pass(int N, int precision, int variant, int sm_count, size_t partial_cap, PassArgs *a, int *grid) {
    const int npad = (N + GENGA_PAD - 1) / GENGA_PAD * GENGA_PAD;
    const int cap = (int)(partial_cap / (3 * (size_t)npad));
    if (precision != GENGA_FP32) {
        const int ntiles = npad / F64_TILE, iblocks = (npad + KB * F64_BPT - 1) / (KB * F64_BPT);
        const int nA = plan_tp2(N, iblocks, KB * F64_BPT, F64_TILE, a);
        int sp = (F64_WAVES * 2 * sm_count + nA - 1) / nA;  // several waves of 2 CTAs per SM: even end
        sp = sp > ntiles ? ntiles : sp;
        sp = sp > cap ? cap : sp;
        a->split = sp < 1 ? 1 : sp;
        a->ntier = 1;
        a->excess = 0;
        a->tier_len[0] = 1;
        a->tier_n[0] = a->split;
        *grid = iblocks;
        return;
    }
    const F32Variant &v = kF32Variants[variant];
    const int ntiles = npad / F32_TILE, ib = v.cw * 32 * v.bpt, iblocks = (npad + ib - 1) / ib;
    const int ctas = v.minb * sm_count;
    const int nA = plan_tp2(N, iblocks, ib, F32_TILE, a);
    const double r = (double)nA / ctas;  // single-tile items per CTA of one chunk per i-block
    const int lmax = std::max(1, (int)(0.25 * ntiles * r));
    int len[GENGA_MAX_TIERS], cnt[GENGA_MAX_TIERS], nt = 0, rows = 0;
    int R = ntiles;
    double drain = 0.0;  // work per CTA of the tiers already placed (after this one in time)
    while (R > 0) {
        int L = nt == 0 ? 1 : std::min(lmax, std::max(1, (int)drain));
        int n = nt == 0 ? (int)std::ceil(F32_TAIL_ITEMS / r) : (int)std::ceil(drain / (L * r));
        n = std::max(1, n);
        if (nt == GENGA_MAX_TIERS - 1 || L == lmax || (long long)n * L >= R) n = (R + L - 1) / L;  // last tier
        len[nt] = L;
        cnt[nt] = n;
        nt++;
        rows += n;
        R -= n * L;
        drain += n * L * r;
    }
    if (rows > cap) {  // too many partial rows: one tier of equal chunks
        const int L = (ntiles + cap - 1) / cap;
        nt = 1;
        len[0] = L;
        cnt[0] = (ntiles + L - 1) / L;
        R = ntiles - cnt[0] * L;
        rows = cnt[0];
    }
    a->ntier = nt;
    a->excess = -R;  // the first-processed chunk is this much shorter
    for (int t = 0; t < nt; t++) {  // first-processed tier first
        a->tier_len[t] = len[nt - 1 - t];
        a->tier_n[t] = cnt[nt - 1 - t];
    }
    a->split = rows;
    const int nitems = nA * rows + a->tp_b0;
    *grid = nitems < ctas ? nitems : ctas;
}

// Dynamic shared memory above the 48 KB default needs an opt-in per kernel
// (the FP32 pass also holds its FP64 accumulators in static shared memory).
cudaError_t init_pass_kernels() {
    for (int q = 0; q < kNumF32Variants; q++) {
        const int sm = (int)smem_fp32(kF32Variants[q].ipack, kF32Variants[q].stages);
        cudaError_t e = cudaFuncSetAttribute(kF32Variants[q].fn, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kF32Variants[q].fnb, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kF32Variants[q].fn_tp, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kF32Variants[q].fnb_tp, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e != cudaSuccess) return e;
    }
    return cudaFuncSetAttribute(pass_fp64_kernel<F64_BPT, F64_TILE, F64_STAGES>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_fp64());
}

cudaError_t launch_pass(const PassArgs &a0, int precision, int variant, int grid, cudaStream_t s) {
    PassArgs a = a0;
    if (precision == GENGA_FP32) {
        a.ntiles = a.npad / F32_TILE;
        cudaError_t e = cudaMemsetAsync(a.work, 0, sizeof(int32_t), s);
        if (e != cudaSuccess) return e;
        const F32Variant &v = kF32Variants[variant];
        (a.n_big >= 0 ? v.fn_tp : v.fn)<<<grid, (v.cw + 1) * 32, smem_fp32(v.ipack, v.stages), s>>>(a, SingleItems{});
    } else {
        a.ntiles = a.npad / F64_TILE;
        auto k = pass_fp64_kernel<F64_BPT, F64_TILE, F64_STAGES>;
        dim3 g(grid, a.split);
        k<<<g, KB, smem_fp64(), s>>>(a);
    }
    return cudaGetLastError();
}

int fp32_variant_ib(int variant) { return kF32Variants[variant].cw * 32 * kF32Variants[variant].bpt; }
void fp32_variant_shape(int variant, int *cw, int *bpt, int *ctas_per_sm) {
    *cw = kF32Variants[variant].cw;
    *bpt = kF32Variants[variant].bpt;
    *ctas_per_sm = kF32Variants[variant].minb;
}
int fp32_variant_minb(int variant) { return kF32Variants[variant].minb; }

cudaError_t launch_pass_batched(const PassArgs &a0, const BatchBodies &bb, const BatchItems &bi, int variant, int grid,
                                cudaStream_t s) {
    PassArgs a = a0;
    a.ntiles = bb.npad_total / F32_TILE;
    cudaError_t e = cudaMemsetAsync(a.work, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const F32Variant &v = kF32Variants[variant];
    BatchPolicy pol;
    pol.bb = bb;
    pol.bi = bi;
    (a.n_big >= 0 ? v.fnb_tp : v.fnb)<<<grid, (v.cw + 1) * 32, smem_fp32(v.ipack, v.stages), s>>>(a, pol);
    return cudaGetLastError();
}

cudaError_t launch_combine_batched(const BatchBodies &bb, const BatchItems &bi, const double *partial,
                                   const uint32_t *perm, double tau, double *acc, double *vx, double *vy, double *vz,
                                   uint32_t *status, cudaStream_t s) {
    if (bb.N_total <= 0) return cudaSuccess;
    combine_batched_kernel<<<dim3((bb.npad_total + 255) / 256, 3), 256, 0, s>>>(partial, perm, tau, acc, vx, vy, vz, status,
                                                                       bb, bi);
    return cudaGetLastError();
}

cudaError_t launch_combine(const double *partial, int split, int one_row_end, int N, int npad, int fp64_rows,
                           const uint32_t *perm,
                           double tau, double *acc, double *vx, double *vy, double *vz, uint32_t *status,
                           cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    combine_kernel<<<dim3((N + 255) / 256, 3), 256, 0, s>>>(partial, split, one_row_end, N, npad, fp64_rows, perm, tau, acc, vx, vy, vz,
                                                   status);
    return cudaGetLastError();
}

cudaError_t launch_sort_pairs(int2 *enc, int32_t cap, const int32_t *count, cudaStream_t s) {
    sort_pairs_kernel<<<1, SORT_THREADS, 0, s>>>(enc, cap, count);
    return cudaGetLastError();
}

cudaError_t launch_copy_pairs(const int2 *enc, const int32_t *count, int32_t enc_cap, int32_t *pairs,
                              int32_t capacity, int32_t *count_out, uint32_t *status, cudaStream_t s) {
    copy_pairs_kernel<<<64, 256, 0, s>>>(enc, count, enc_cap, pairs, capacity, count_out, status);
    return cudaGetLastError();
}

void fp64_pass_shape(int *warps, int *bpt) {
    *warps = KB / 32;
    *bpt = F64_BPT;
}

}  // namespace genga
