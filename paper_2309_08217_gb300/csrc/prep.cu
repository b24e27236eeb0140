// prep.cu -- per-body work done before each long-range pass (O(N), FP64):
//
//   * P = sum_j m_j v_j, a deterministic reduction over 64 CTAs;
//   * the Eq. (1) inputs and radius of every body (Sect. 1): osculating
//     semi-major axis a_i (1/a = 2/r - v_hel^2 / mu_i, mu_i = G (M* + m_i),
//     a_i = r_i for unbound orbits), heliocentric speed v_hel = |v + P/M*|,
//     r_crit,i = max(n1 a_i (m_i / 3M*)^(1/3), n2 dt v_hel);
//   * the packed copies the pass kernels read, in the spatial (Morton) order
//     of order.cu: FP32 hi/lo split of each position plus G m in FP32 (the
//     single-precision kick of Sect. 1 takes its pair offsets from these),
//     an FP64 {x, y, z, G m} record, and the FP32 screening factors
//     {H_i, A_i} with r_crit,ij <= max(H_i, H_j) * max(A_i, A_j) for every
//     pair (rounded up; with the close-encounter level on, of GENGA_PREDICT_RANGE
//     r_crit,ij, so that the pass also sees the pairs that may enter r_crit
//     within the drift); per 64-body group, the bounding box of the FP32
//     positions and the maxima of the screening factors;
//   * iperm: the packed position of every body (the close-encounter level
//     reads a_i, r_crit,i and the test-particle flag of its members there).
#include "internal.cuh"
#include "pass_common.cuh"

namespace genga {

namespace {


constexpr int MOM_BLOCKS = 64, MOM_THREADS = 256;

// P = sum_j m_j v_j over MOM_BLOCKS CTAs (FP64 throughput is low on this
// part, so the few adds per body are spread over many SMs).  Block b sums a
// contiguous chunk (strided per thread, then a fixed-shape tree); the last
// block to finish adds the 64 block sums with a fixed warp-shuffle tree.
// Every add happens in the same order on every run, so the result is
// bitwise reproducible.
__global__ void __launch_bounds__(MOM_THREADS) momentum_kernel(const double *__restrict__ vx,
                                                               const double *__restrict__ vy,
                                                               const double *__restrict__ vz,
                                                               const double *__restrict__ m, int N,
                                                               double *__restrict__ P, double *__restrict__ part,
                                                               unsigned *__restrict__ ticket,
                                                               int32_t *__restrict__ zero_me) {
    __shared__ double sh[3][MOM_THREADS];
    __shared__ bool last;
    const int chunk = (N + MOM_BLOCKS - 1) / MOM_BLOCKS;
    const int lo = blockIdx.x * chunk, hi = min(N, lo + chunk);
    double px = 0.0, py = 0.0, pz = 0.0;
    for (int i = lo + threadIdx.x; i < hi; i += MOM_THREADS) {
        const double mi = m[i];
        px += mi * vx[i];
        py += mi * vy[i];
        pz += mi * vz[i];
    }
    sh[0][threadIdx.x] = px;
    sh[1][threadIdx.x] = py;
    sh[2][threadIdx.x] = pz;
    __syncthreads();
    for (int w = MOM_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            for (int c = 0; c < 3; c++) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int c = 0; c < 3; c++) part[3 * blockIdx.x + c] = sh[c][0];
        __threadfence();
        last = (atomicAdd(ticket, 1u) == MOM_BLOCKS - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (w < 3) {  // warp c sums component c of the 64 block sums
        const volatile double *vp = part;
        double t = vp[3 * lane + w] + vp[3 * (lane + 32) + w];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) P[w] = t;
    }
    if (threadIdx.x == 0) {
        *ticket = 0u;
        if (zero_me) zero_me[0] = zero_me[1] = 0;  // encounter pairs, predicted entries
    }
}

constexpr int PREP_THREADS = 64;  // one block = one 64-body group

// Tile-blocked copy of {x_hi, y_hi, z_hi, G m}: the 256-body tile t holds
// x[256], y[256], z[256], w[256], so a 64-bit shared load gives the values of
// two consecutive bodies (the packed-pair loop of the FP32 pass).
__device__ __forceinline__ void store_tiled(float *hit, int k, float x, float y, float z, float w) {
    float *t = hit + (size_t)(k / GENGA_TILE_T) * 4 * GENGA_TILE_T + (k % GENGA_TILE_T);
    t[0] = x;
    t[GENGA_TILE_T] = y;
    t[2 * GENGA_TILE_T] = z;
    t[3 * GENGA_TILE_T] = w;
}

// Duplicated-pair copy: body k as {x, x, y, y}, {z, z, w, w}, so a 64-bit
// lane pair broadcasts one j-body to two i-bodies (the i-packed FP32 loop).
__device__ __forceinline__ void store_dup(float4 *hid, int k, float x, float y, float z, float w) {
    hid[2 * (size_t)k] = make_float4(x, x, y, y);
    hid[2 * (size_t)k + 1] = make_float4(z, z, w, w);
}

// Fills packed position k with body i (i >= 0) or with padding body number
// `pad` (i < 0); returns the screening factors and the FP32 position.
__device__ __forceinline__ float2 prep_body(int k, int i, int pad, const double *__restrict__ x,
                                           const double *__restrict__ y, const double *__restrict__ z,
                                           const double *__restrict__ vx, const double *__restrict__ vy,
                                           const double *__restrict__ vz, const double *__restrict__ m,
                                           const double *__restrict__ P, double G, double Mstar, double dt, double n1,
                                           double n2, int rcrit_mode, float4 *__restrict__ hi, float *__restrict__ hit, float4 *__restrict__ hid,
                                           float4 *__restrict__ lo, double4_32a *__restrict__ p64,
                                           float2 *__restrict__ scr, double *__restrict__ a_osc,
                                           double *__restrict__ rc_eq1, bool tp, double sscale, float3 *pos,
                                           bool *real, double4 *pos64) {
    float2 s = make_float2(0.f, 0.f);
    if (i >= 0) {
        // osculating a from the heliocentric velocity u = v + P / M*:
        // 1/a = 2/r - u^2 / (G (M* + m)); FP64 reciprocals by series-corrected
        // SFU seeds (the FP64 pipe is the slow one on this GPU)
        const double xi = x[i], yi = y[i], zi = z[i], mi = m[i];
        const double iM = rcp_fp64(Mstar);
        const double ux = fma(P[0], iM, vx[i]);
        const double uy = fma(P[1], iM, vy[i]);
        const double uz = fma(P[2], iM, vz[i]);
        const double v2 = ux * ux + uy * uy + uz * uz;
        const double r2 = xi * xi + yi * yi + zi * zi;
        const double ri = rsqrt_fp64(r2);
        const double mu = G * (Mstar + mi);
        const double inva = 2.0 * ri - v2 * rcp_fp64(mu);
        const double a = (inva > 0.0) ? rcp_fp64(inva) : r2 * ri;
        a_osc[k] = a;
        if (rcrit_mode == GENGA_RCRIT_EQ1) {
            // r_crit,ij = max(rc_i, rc_j) = max(1, 1) * max(rc_i, rc_j)
            const double rc = fmax(n1 * a * cbrt(mi / (3.0 * Mstar)), n2 * dt * sqrt(v2));
            rc_eq1[k] = rc;
            s = make_float2(1.0f, __double2float_ru(rc * sscale));
        } else {
            // n1 ((m_i+m_j)/3M)^(1/3) (a_i+a_j)/2 <= n1 (2 max(m)/3M)^(1/3) * max(a); the FP32
            // cube root (error ~1 ulp) is inflated by 2^-16 to stay an upper bound
            rc_eq1[k] = 0.0;
            const float h = n1 * cbrtf(__double2float_ru(2.0 * mi / (3.0 * Mstar))) * (1.0f + 0x1p-16f);
            s = make_float2(h, __double2float_ru(a * (1.0 + 1e-12) * sscale));
        }
        const float hx = __double2float_rn(xi), hy = __double2float_rn(yi), hz = __double2float_rn(zi);
        const double gm = G * mi;
        hi[k] = make_float4(hx, hy, hz, __double2float_rn(gm));
        store_tiled(hit, k, hx, hy, hz, __double2float_rn(gm));
        store_dup(hid, k, hx, hy, hz, __double2float_rn(gm));
        lo[k] = make_float4(__double2float_rn(xi - (double)hx), __double2float_rn(yi - (double)hy),
                            __double2float_rn(zi - (double)hz), tp ? 1.f : 0.f);  // w: test particle (mode 2)
        p64[k] = make_double4_32a(xi, yi, zi, gm);
        *pos = make_float3(hx, hy, hz);
        *pos64 = make_double4(xi, yi, zi, gm);
        *real = true;
    } else {
        const float px = GENGA_PAD_POS + 64.0f * (float)pad;
        hi[k] = make_float4(px, GENGA_PAD_POS, GENGA_PAD_POS, 0.f);
        store_tiled(hit, k, px, GENGA_PAD_POS, GENGA_PAD_POS, 0.f);
        store_dup(hid, k, px, GENGA_PAD_POS, GENGA_PAD_POS, 0.f);
        lo[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        p64[k] = make_double4_32a((double)px, GENGA_PAD_POS, GENGA_PAD_POS, 0.0);
        a_osc[k] = 0.0;
        rc_eq1[k] = 0.0;
        *pos64 = make_double4((double)px, GENGA_PAD_POS, GENGA_PAD_POS, 0.0);
        *real = false;
    }
    scr[k] = s;
    return s;
}

// Bounding box of the group's real bodies (FP32 hi positions), the maxima of
// its screening factors and its flags (GENGA_GROUP_BIG: holds a body that is
// not a test particle, GENGA_GROUP_TP: holds a test particle); one block =
// one 64-body group.
__device__ __forceinline__ Box group_reduce_store(float2 s, float3 pos, bool real, bool tp,
                                                  float4 *__restrict__ gbox_lo, float4 *__restrict__ gbox_hi,
                                                  int32_t *__restrict__ gflag) {
    const unsigned big_w = __ballot_sync(0xffffffffu, real && !tp), tp_w = __ballot_sync(0xffffffffu, real && tp);
    const float INF = __int_as_float(0x7f800000);
    float3 bl = real ? pos : make_float3(INF, INF, INF);
    float3 bh = real ? pos : make_float3(-INF, -INF, -INF);
    float hmax = s.x, amax = s.y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        hmax = fmaxf(hmax, __shfl_xor_sync(0xffffffffu, hmax, o));
        amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        bl.x = fminf(bl.x, __shfl_xor_sync(0xffffffffu, bl.x, o));
        bl.y = fminf(bl.y, __shfl_xor_sync(0xffffffffu, bl.y, o));
        bl.z = fminf(bl.z, __shfl_xor_sync(0xffffffffu, bl.z, o));
        bh.x = fmaxf(bh.x, __shfl_xor_sync(0xffffffffu, bh.x, o));
        bh.y = fmaxf(bh.y, __shfl_xor_sync(0xffffffffu, bh.y, o));
        bh.z = fmaxf(bh.z, __shfl_xor_sync(0xffffffffu, bh.z, o));
    }
    __shared__ float4 wl[PREP_THREADS / 32], wh[PREP_THREADS / 32];
    __shared__ int32_t wf[PREP_THREADS / 32];
    __shared__ Box box;
    if ((threadIdx.x & 31) == 0) {
        wl[threadIdx.x >> 5] = make_float4(bl.x, bl.y, bl.z, hmax);
        wh[threadIdx.x >> 5] = make_float4(bh.x, bh.y, bh.z, amax);
        wf[threadIdx.x >> 5] = (big_w ? GENGA_GROUP_BIG : 0) | (tp_w ? GENGA_GROUP_TP : 0);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float4 l = wl[0], h = wh[0];
        int32_t f = wf[0];
        for (int w = 1; w < PREP_THREADS / 32; w++) {
            f |= wf[w];
            l = make_float4(fminf(l.x, wl[w].x), fminf(l.y, wl[w].y), fminf(l.z, wl[w].z), fmaxf(l.w, wl[w].w));
            h = make_float4(fmaxf(h.x, wh[w].x), fmaxf(h.y, wh[w].y), fmaxf(h.z, wh[w].z), fmaxf(h.w, wh[w].w));
        }
        gbox_lo[blockIdx.x] = l;
        gbox_hi[blockIdx.x] = h;
        gflag[blockIdx.x] = f;
        box = Box{l, h};
    }
    __syncthreads();
    return box;
}

// Group-centred copies for the mutual FP32 pass: c = the centre of the
// group's box (an FP32 value), each body's offset from it as the FP64
// difference rounded to FP32 (X = fl32(x - c)), stored as the record
// {X, Y, Z, G m} (the pass reads a j-body with one 16-byte load), and its
// rounding residual
// {x - c - X, y - c - Y, z - c - Z, test-particle flag}; per group
// {c, PRECISION_KAPPA * h}, h an upper bound of |x - c| over the group.  The
// pass treats a group as far from a set of bodies only beyond that distance:
// with |x_j - c| <= h, |x_i - c| <= r + h and three roundings (X_j, the
// two-step X_i, the difference) the offset X_j - X_i is within
// 3 u (r + h) of x_j - x_i, a relative error of at most
// 3 u (1 + 1/PRECISION_KAPPA) = 33 u ~ 2e-6 (u = 2^-24), about 6e-6 on the
// pair's force.  An empty group (padding only) has c = 0 and distance 0.
constexpr float PRECISION_KAPPA = 0.1f;

__device__ __forceinline__ void store_centred(int k, const Box &b, double4 p, bool tp, float4 *__restrict__ rel,
                                              float4 *__restrict__ rell, float4 *__restrict__ gctr) {
    const bool empty = !(b.lo.x <= b.hi.x);
    const float cx = empty ? 0.f : 0.5f * (b.lo.x + b.hi.x), cy = empty ? 0.f : 0.5f * (b.lo.y + b.hi.y);
    const float cz = empty ? 0.f : 0.5f * (b.lo.z + b.hi.z);
    const double dx = p.x - (double)cx, dy = p.y - (double)cy, dz = p.z - (double)cz;
    const float X = __double2float_rn(dx), Y = __double2float_rn(dy), Z = __double2float_rn(dz);
    const float w = __double2float_rn(p.w);
    rel[k] = make_float4(X, Y, Z, w);
    rell[k] = make_float4(__double2float_rn(dx - (double)X), __double2float_rn(dy - (double)Y),
                          __double2float_rn(dz - (double)Z), tp ? 1.f : 0.f);
    if (threadIdx.x == 0) {
        float h = 0.f;
        if (!empty) {  // half-diagonal of the box about c, rounded up
            const float ex = fmaxf(b.hi.x - cx, cx - b.lo.x), ey = fmaxf(b.hi.y - cy, cy - b.lo.y);
            const float ez = fmaxf(b.hi.z - cz, cz - b.lo.z);
            h = __fsqrt_ru(__fmaf_ru(ex, ex, __fmaf_ru(ey, ey, __fmul_ru(ez, ez)))) * (1.0f + 0x1p-20f);
        }
        gctr[blockIdx.x] = make_float4(cx, cy, cz, PRECISION_KAPPA * h);
    }
}

// Position k of the packed arrays holds body perm[k] (the Morton order);
// k >= N are padding bodies: zero mass, 64 au apart, far from everything.
__global__ void __launch_bounds__(PREP_THREADS) prep_kernel(
    const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
    const double *__restrict__ vx, const double *__restrict__ vy, const double *__restrict__ vz,
    const double *__restrict__ m, int N, const uint32_t *__restrict__ perm, const double *__restrict__ P, double G,
    double Mstar, double dt, double n1, double n2, int rcrit_mode, float4 *__restrict__ hi, float *__restrict__ hit, float4 *__restrict__ hid,
    float4 *__restrict__ lo, double4_32a *__restrict__ p64, float2 *__restrict__ scr, float4 *__restrict__ gbox_lo,
    float4 *__restrict__ gbox_hi, int32_t *__restrict__ gflag, double *__restrict__ a_osc,
    double *__restrict__ rc_eq1, int n_big, uint32_t *__restrict__ iperm, double sscale, float4 *__restrict__ rel,
    float4 *__restrict__ rell, float4 *__restrict__ gctr) {
    const int k = blockIdx.x * PREP_THREADS + threadIdx.x;
    float3 pos = make_float3(0.f, 0.f, 0.f);
    double4 p4;
    bool real = false;
    const int i = k < N ? (int)perm[k] : -1;
    if (i >= 0) iperm[i] = (uint32_t)k;
    const bool tp = i >= 0 && n_big >= 0 && i >= n_big;
    const float2 s = prep_body(k, i, k - N, x, y, z, vx, vy, vz, m, P, G, Mstar, dt, n1, n2,
                               rcrit_mode, hi, hit, hid, lo, p64, scr, a_osc, rc_eq1, tp, sscale, &pos, &real, &p4);
    const Box b = group_reduce_store(s, pos, real, tp, gbox_lo, gbox_hi, gflag);
    store_centred(k, b, p4, tp, rel, rell, gctr);
}

// Batched: packed position p belongs to system d = segment of p in poff; its
// k-th body (k = p - poff[d]) is body perm[off[d] + k] of the caller's arrays
// (the batched Morton sort keeps each system's bodies together).
__global__ void __launch_bounds__(PREP_THREADS) prep_batched_kernel(
    const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
    const double *__restrict__ vx, const double *__restrict__ vy, const double *__restrict__ vz,
    const double *__restrict__ m, const uint32_t *__restrict__ perm, const double *__restrict__ Pd, double G,
    double Mstar, double dt, double n1, double n2, int rcrit_mode, float4 *__restrict__ hi, float *__restrict__ hit, float4 *__restrict__ hid,
    float4 *__restrict__ lo, double4_32a *__restrict__ p64, float2 *__restrict__ scr, float4 *__restrict__ gbox_lo,
    float4 *__restrict__ gbox_hi, int32_t *__restrict__ gflag, double *__restrict__ a_osc,
    double *__restrict__ rc_eq1, int n_big, uint32_t *__restrict__ iperm, double sscale, float4 *__restrict__ rel,
    float4 *__restrict__ rell, float4 *__restrict__ gctr, const __grid_constant__ BatchBodies bb) {
    const int p = blockIdx.x * PREP_THREADS + threadIdx.x;
    const int d = find_segment(bb.poff, bb.D, p);
    const int k = p - bb.poff[d], Nd = bb.off[d + 1] - bb.off[d];
    float3 pos = make_float3(0.f, 0.f, 0.f);
    double4 p4;
    bool real = false;
    const int i = k < Nd ? (int)perm[bb.off[d] + k] : -1;
    if (i >= 0) iperm[i] = (uint32_t)p;
    const bool tp = i >= 0 && n_big >= 0 && i - bb.off[d] >= n_big;
    const float2 s = prep_body(p, i, k - Nd, x, y, z, vx, vy, vz, m, Pd + 3 * d, G, Mstar, dt, n1, n2, rcrit_mode, hi,
                               hit, hid, lo, p64, scr, a_osc, rc_eq1, tp, sscale, &pos, &real, &p4);
    const Box b = group_reduce_store(s, pos, real, tp, gbox_lo, gbox_hi, gflag);
    store_centred(p, b, p4, tp, rel, rell, gctr);
}

// Batched momentum: block d sums system d (strided per thread, fixed tree).
__global__ void __launch_bounds__(MOM_THREADS) momentum_batched_kernel(
    const double *__restrict__ vx, const double *__restrict__ vy, const double *__restrict__ vz,
    const double *__restrict__ m, double *__restrict__ Pd, int32_t *__restrict__ zero_me,
    const __grid_constant__ BatchBodies bb) {
    __shared__ double sh[3][MOM_THREADS];
    const int d = blockIdx.x;
    double px = 0.0, py = 0.0, pz = 0.0;
    for (int i = bb.off[d] + threadIdx.x; i < bb.off[d + 1]; i += MOM_THREADS) {
        const double mi = m[i];
        px += mi * vx[i];
        py += mi * vy[i];
        pz += mi * vz[i];
    }
    sh[0][threadIdx.x] = px;
    sh[1][threadIdx.x] = py;
    sh[2][threadIdx.x] = pz;
    __syncthreads();
    for (int w = MOM_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 3; c++) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) Pd[3 * d + threadIdx.x] = sh[threadIdx.x][0];
    if (d == 0 && threadIdx.x == 0 && zero_me) zero_me[0] = zero_me[1] = 0;
}

}  // namespace

cudaError_t launch_momentum(const double *vx, const double *vy, const double *vz, const double *m, int N,
                            double *P, int32_t *zero_me, cudaStream_t s) {
    // P[0..2] result, P[8..8+3*MOM_BLOCKS) block partials, ticket after them
    momentum_kernel<<<MOM_BLOCKS, MOM_THREADS, 0, s>>>(vx, vy, vz, m, N, P, P + 8,
                                                       reinterpret_cast<unsigned *>(P + 8 + 3 * MOM_BLOCKS),
                                                       zero_me);
    return cudaGetLastError();
}

cudaError_t launch_prep(const genga_system &sys, const genga_params &p, genga_ctx *c, cudaStream_t s) {
    const int npad = (sys.N + GENGA_PAD - 1) / GENGA_PAD * GENGA_PAD;
    prep_kernel<<<npad / PREP_THREADS, PREP_THREADS, 0, s>>>(
        sys.x, sys.y, sys.z, sys.vx, sys.vy, sys.vz, sys.m, sys.N, c->perm, c->mom, p.G, p.Mstar, p.dt, p.n1,
        p.n2, p.rcrit_mode, c->pk_hi, c->pk_t, c->pk_d, c->pk_lo, c->pk64, c->scr, c->gbox_lo, c->gbox_hi, c->gflag,
        c->a_osc, c->rc_eq1, p.n_big, c->iperm, p.bs_tol > 0.0 ? GENGA_PREDICT_RANGE : 1.0, c->pk_r, c->pk_rl,
        c->gctr);
    return cudaGetLastError();
}

}  // namespace genga

namespace genga {

cudaError_t launch_momentum_batched(const genga_system &all, const BatchBodies &bb, double *Pd, int32_t *zero_me,
                                    cudaStream_t s) {
    momentum_batched_kernel<<<bb.D, MOM_THREADS, 0, s>>>(all.vx, all.vy, all.vz, all.m, Pd, zero_me, bb);
    return cudaGetLastError();
}

cudaError_t launch_prep_batched(const genga_system &all, const BatchBodies &bb, const genga_params &p, genga_ctx *c,
                                cudaStream_t s) {
    prep_batched_kernel<<<bb.npad_total / PREP_THREADS, PREP_THREADS, 0, s>>>(
        all.x, all.y, all.z, all.vx, all.vy, all.vz, all.m, c->perm, c->Pd, p.G, p.Mstar, p.dt, p.n1, p.n2,
        p.rcrit_mode, c->pk_hi, c->pk_t, c->pk_d, c->pk_lo, c->pk64, c->scr, c->gbox_lo, c->gbox_hi, c->gflag, c->a_osc,
        c->rc_eq1, p.n_big, c->iperm, p.bs_tol > 0.0 ? GENGA_PREDICT_RANGE : 1.0, c->pk_r, c->pk_rl, c->gctr, bb);
    return cudaGetLastError();
}

}  // namespace genga
