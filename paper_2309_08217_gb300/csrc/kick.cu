// kick.cu -- the long-range pass of the GENGA kick (Sect. 1):
//
//   a_i = sum_{j != i} G m_j K(y_ij) (x_j - x_i) / r_ij^3,
//   y_ij = (r_ij / r_crit,ij - 0.1) / 0.9,  K = 1 for r_ij >= r_crit,ij.
//
// Layout of one pass.  A CTA owns KB * BPT i-bodies (BPT per thread, held in
// registers) and a contiguous slice of j-tiles; TILE j-bodies at a time are
// staged into shared memory by one-dimensional bulk copies completed on an
// mbarrier (STAGES-deep ring), and every warp reads them back as broadcasts.
// Slices of the j range run in separate CTAs (grid.y) so that N = 40k still
// fills all SMs; their FP64 partial sums are combined afterwards in a fixed
// order, so results are bitwise reproducible.
//
// Precision.  The FP32 pass (the single-precision kick of Sect. 1) forms
// each pair offset from the FP32 hi/lo split of the FP64 positions,
//   dx = (x_j,hi - x_i,hi) + (x_j,lo - x_i,lo),
// squares it in FP32, takes rsqrt on the SFU, and accumulates each tile's
// terms in FP32 registers that are added into FP64 per-body accumulators
// once per tile.  The FP64 pass does the same arithmetic in FP64, with its
// own inverse square root (FP32 SFU seed + one third-order correction) and
// Neumaier-compensated accumulation every 32 terms.
//
// Changeover pairs.  Both passes screen every pair against an FP32 upper
// bound of r_crit,ij (per i-body and j-tile); a pair under the bound leaves
// the fast loop and is evaluated exactly in FP64: r_crit,ij, K and the
// weighted force (close-encounter forces are always FP64, Sect. 1), and, if
// r_ij < r_crit,ij and i < j, it is appended to the encounter list.
#include "internal.cuh"

namespace genga {

namespace {

constexpr int KB = 256;  // threads per CTA of the pass kernels

__device__ __forceinline__ float rsqrt_sfu(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/sqrt(x) in FP64: FP32 SFU seed y0 (relative error ~1e-7), then the
// third-order correction y = y0 (1 + e/2 + 3e^2/8), e = 1 - x y0^2, from the
// binomial series of (1 - e)^(-1/2); the truncation error is O(e^3) ~ 1e-21.
// Valid for x in the FP32 normal range.
__device__ __forceinline__ double rsqrt_fp64(double x) {
    const double y0 = (double)rsqrt_sfu(__double2float_rn(x));
    const double t = x * y0;
    const double e = fma(-t, y0, 1.0);
    const double p = fma(e, 0.375, 0.5);
    return fma(y0 * e, p, y0);
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

// Exact FP64 treatment of one screened pair: returns the K-weighted
// acceleration of i due to j and records (i, j) when it is an encounter.
__device__ __noinline__ double3 screened_pair(const PassArgs &a, int i, int j) {
    double3 f = make_double3(0.0, 0.0, 0.0);
    if (i >= a.N || j >= a.N || i == j) return f;
    const double4_32a pi = a.p64[i], pj = a.p64[j];
    const double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
    const double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 == 0.0) return f;  // coincident bodies: no direction, no force
    const double r = sqrt(r2);
    double rc;
    if (a.rcrit_mode == GENGA_RCRIT_EQ1) {
        rc = fmax(a.rc_eq1[i], a.rc_eq1[j]);
    } else {
        rc = a.n1 * cbrt((a.m[i] + a.m[j]) / (3.0 * a.Mstar)) * 0.5 * (a.a_osc[i] + a.a_osc[j]);
    }
    double K = 1.0;
    if (r < rc) {
        if (i < j) {
            const int pos = atomicAdd(a.enc_count, 1);
            if (pos < a.enc_cap) a.enc[pos] = make_int2(i, j);
        }
        K = changeover_K((r / rc - 0.1) / 0.9, a.changeover);
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

template <int TILE>
__device__ __forceinline__ float2 tile_maxima(const float2 *__restrict__ tm, int t) {
    float Hm = 0.f, Am = 0.f;
#pragma unroll
    for (int q = 0; q < TILE / 64; q++) {
        const float2 v = tm[t * (TILE / 64) + q];
        Hm = fmaxf(Hm, v.x);
        Am = fmaxf(Am, v.y);
    }
    return make_float2(Hm, Am);
}

// ----------------------------------------------------------- FP32 pass ----
template <int BPT, int TILE, int STAGES>
__global__ void __launch_bounds__(KB, 2) pass_fp32_kernel(const __grid_constant__ PassArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float4 *s_hi = reinterpret_cast<float4 *>(smem_raw);
    float4 *s_lo = s_hi + STAGES * TILE;
    uint64_t *bars = reinterpret_cast<uint64_t *>(s_lo + STAGES * TILE);
    __shared__ int s_abort;

    const int tid = threadIdx.x;
    const int ibase = blockIdx.x * (KB * BPT);
    const int slice = blockIdx.y;
    const int t0 = (int)((long long)a.ntiles * slice / a.split);
    const int t1 = (int)((long long)a.ntiles * (slice + 1) / a.split);

    float xh[BPT], yh[BPT], zh[BPT], xl[BPT], yl[BPT], zl[BPT], H[BPT], A[BPT];
    double AX[BPT], AY[BPT], AZ[BPT];
#pragma unroll
    for (int k = 0; k < BPT; k++) {
        const int i = ibase + k * KB + tid;
        const float4 h = a.hi[i], l = a.lo[i];
        const float2 s = a.scr[i];
        xh[k] = h.x; yh[k] = h.y; zh[k] = h.z;
        xl[k] = l.x; yl[k] = l.y; zl[k] = l.z;
        H[k] = s.x; A[k] = s.y;
        AX[k] = AY[k] = AZ[k] = 0.0;
    }

    constexpr uint32_t TB = TILE * sizeof(float4);
    if (tid == 0) {
        for (int s = 0; s < STAGES; s++) mbar_init(&bars[s], 1);
        fence_barrier_init();
        s_abort = 0;
    }
    __syncthreads();
    if (tid == 0) {
        for (int s = 0; s < STAGES - 1 && t0 + s < t1; s++) {
            mbar_arrive_expect_tx(&bars[s], 2 * TB);
            bulk_g2s(s_hi + s * TILE, a.hi + (size_t)(t0 + s) * TILE, TB, &bars[s]);
            bulk_g2s(s_lo + s * TILE, a.lo + (size_t)(t0 + s) * TILE, TB, &bars[s]);
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
                mbar_arrive_expect_tx(&bars[sn], 2 * TB);
                bulk_g2s(s_hi + sn * TILE, a.hi + (size_t)tn * TILE, TB, &bars[sn]);
                bulk_g2s(s_lo + sn * TILE, a.lo + (size_t)tn * TILE, TB, &bars[sn]);
            }
        }
        const float2 tm = tile_maxima<TILE>(a.tile_max, t);
        float thr[BPT];
#pragma unroll
        for (int k = 0; k < BPT; k++) thr[k] = screen_threshold(H[k], A[k], tm.x, tm.y);

        if (!mbar_wait_bounded(&bars[stage], (uint32_t)((it / STAGES) & 1), a.status)) s_abort = 1;

        float ax[BPT], ay[BPT], az[BPT];
#pragma unroll
        for (int k = 0; k < BPT; k++) ax[k] = ay[k] = az[k] = 0.f;
        const float4 *th = s_hi + stage * TILE;
        const float4 *tl = s_lo + stage * TILE;
#pragma unroll 2
        for (int jj = 0; jj < TILE; jj++) {
            const float4 ph = th[jj];
            const float4 pl = tl[jj];
#pragma unroll
            for (int k = 0; k < BPT; k++) {
                const float dx = (ph.x - xh[k]) + (pl.x - xl[k]);
                const float dy = (ph.y - yh[k]) + (pl.y - yl[k]);
                const float dz = (ph.z - zh[k]) + (pl.z - zl[k]);
                const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                const float ri = rsqrt_sfu(r2);
                float s = (ph.w * ri) * (ri * ri);
                if (r2 < thr[k]) {
                    const double3 f = screened_pair(a, ibase + k * KB + tid, t * TILE + jj);
                    AX[k] += f.x;
                    AY[k] += f.y;
                    AZ[k] += f.z;
                    s = 0.f;
                }
                ax[k] = fmaf(s, dx, ax[k]);
                ay[k] = fmaf(s, dy, ay[k]);
                az[k] = fmaf(s, dz, az[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < BPT; k++) {
            AX[k] += (double)ax[k];
            AY[k] += (double)ay[k];
            AZ[k] += (double)az[k];
        }
        __syncthreads();
        if (s_abort) break;
    }

    const size_t np = (size_t)a.npad;
    double *out = a.partial + (size_t)slice * 3 * np;
#pragma unroll
    for (int k = 0; k < BPT; k++) {
        const int i = ibase + k * KB + tid;
        out[i] = AX[k];
        out[np + i] = AY[k];
        out[2 * np + i] = AZ[k];
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

    const int tid = threadIdx.x;
    const int ibase = blockIdx.x * (KB * BPT);
    const int slice = blockIdx.y;
    const int t0 = (int)((long long)a.ntiles * slice / a.split);
    const int t1 = (int)((long long)a.ntiles * (slice + 1) / a.split);

    double xi[BPT], yi[BPT], zi[BPT];
    float H[BPT], A[BPT];
    Comp CX[BPT], CY[BPT], CZ[BPT];
#pragma unroll
    for (int k = 0; k < BPT; k++) {
        const int i = ibase + k * KB + tid;
        const double4_32a p = a.p64[i];
        const float2 s = a.scr[i];
        xi[k] = p.x; yi[k] = p.y; zi[k] = p.z;
        H[k] = s.x; A[k] = s.y;
        CX[k] = CY[k] = CZ[k] = Comp{0.0, 0.0};
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
        const float2 tm = tile_maxima<TILE>(a.tile_max, t);
        double thr[BPT];
#pragma unroll
        for (int k = 0; k < BPT; k++) thr[k] = (double)screen_threshold(H[k], A[k], tm.x, tm.y);

        if (!mbar_wait_bounded(&bars[stage], (uint32_t)((it / STAGES) & 1), a.status)) s_abort = 1;

        const double4_32a *tp = s_p + stage * TILE;
        for (int j0 = 0; j0 < TILE; j0 += 32) {
            double px[BPT], py[BPT], pz[BPT];
#pragma unroll
            for (int k = 0; k < BPT; k++) px[k] = py[k] = pz[k] = 0.0;
#pragma unroll 2
            for (int jj = j0; jj < j0 + 32; jj++) {
                const double4_32a pj = tp[jj];
#pragma unroll
                for (int k = 0; k < BPT; k++) {
                    const double dx = pj.x - xi[k], dy = pj.y - yi[k], dz = pj.z - zi[k];
                    const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
                    const double ri = rsqrt_fp64(r2);
                    double s = (pj.w * ri) * (ri * ri);
                    if (r2 < thr[k]) {
                        const double3 f = screened_pair(a, ibase + k * KB + tid, t * TILE + jj);
                        CX[k].add(f.x);
                        CY[k].add(f.y);
                        CZ[k].add(f.z);
                        s = 0.0;
                    }
                    px[k] = fma(s, dx, px[k]);
                    py[k] = fma(s, dy, py[k]);
                    pz[k] = fma(s, dz, pz[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < BPT; k++) {
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
        const int i = ibase + k * KB + tid;
        out[i] = CX[k].s + CX[k].c;
        out[np + i] = CY[k].s + CY[k].c;
        out[2 * np + i] = CZ[k].s + CZ[k].c;
    }
}

// ------------------------------------------------------------ combine ----
// acc_i = sum over slices (Neumaier, slice order); optional acc output and
// v_i += acc_i * tau; non-finite accelerations raise GENGA_ERR_NONFINITE.
__global__ void combine_kernel(const double *__restrict__ partial, int split, int N, int npad, double tau,
                               double *__restrict__ acc, double *__restrict__ vx, double *__restrict__ vy,
                               double *__restrict__ vz, uint32_t *__restrict__ status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double a3[3];
    bool finite = true;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        Comp s{0.0, 0.0};
        for (int q = 0; q < split; q++) s.add(partial[((size_t)q * 3 + c) * npad + i]);
        a3[c] = s.s + s.c;
        finite = finite && isfinite(a3[c]);
    }
    if (!finite) atomicOr(status, GENGA_BIT(GENGA_ERR_NONFINITE));
    if (acc) {
        acc[i] = a3[0];
        acc[(size_t)N + i] = a3[1];
        acc[2 * (size_t)N + i] = a3[2];
    }
    if (tau != 0.0) {
        vx[i] += a3[0] * tau;
        vy[i] += a3[1] * tau;
        vz[i] += a3[2] * tau;
    }
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
                    const int2 a = enc[q], b = enc[p];
                    const unsigned long long u = pair_key(a), v = pair_key(b);
                    if ((u > v) == up) { enc[q] = b; enc[p] = a; }
                }
            }
            __threadfence_block();
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
template <int BPT, int TILE, int STAGES>
size_t smem_fp32() { return (size_t)STAGES * TILE * 2 * sizeof(float4) + STAGES * sizeof(uint64_t); }
template <int BPT, int TILE, int STAGES>
size_t smem_fp64() { return (size_t)STAGES * TILE * sizeof(double4_32a) + STAGES * sizeof(uint64_t); }

constexpr int F32_BPT = 4, F32_TILE = 256, F32_STAGES = 3;
constexpr int F64_BPT = 2, F64_TILE = 128, F64_STAGES = 3;

}  // namespace

int choose_split(int N, int precision, int sm_count, int max_split) {
    const int npad = (N + GENGA_PAD - 1) / GENGA_PAD * GENGA_PAD;
    const int bpt = (precision == GENGA_FP32) ? F32_BPT : F64_BPT;
    const int tile = (precision == GENGA_FP32) ? F32_TILE : F64_TILE;
    const int iblocks = npad / (KB * bpt);
    const int ntiles = npad / tile;
    const int want = 2 * sm_count;                  // two resident CTAs per SM
    int split = (want + iblocks - 1) / iblocks;
    split = split < 1 ? 1 : split;
    split = split > ntiles ? ntiles : split;
    split = split > max_split ? max_split : split;
    return split;
}

cudaError_t launch_pass(const PassArgs &a0, int precision, int sm_count, cudaStream_t s) {
    (void)sm_count;
    PassArgs a = a0;
    if (precision == GENGA_FP32) {
        a.ntiles = a.npad / F32_TILE;
        auto k = pass_fp32_kernel<F32_BPT, F32_TILE, F32_STAGES>;
        const size_t sm = smem_fp32<F32_BPT, F32_TILE, F32_STAGES>();
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        dim3 grid(a.npad / (KB * F32_BPT), a.split);
        k<<<grid, KB, sm, s>>>(a);
    } else {
        a.ntiles = a.npad / F64_TILE;
        auto k = pass_fp64_kernel<F64_BPT, F64_TILE, F64_STAGES>;
        const size_t sm = smem_fp64<F64_BPT, F64_TILE, F64_STAGES>();
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        dim3 grid(a.npad / (KB * F64_BPT), a.split);
        k<<<grid, KB, sm, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_combine(const double *partial, int split, int N, int npad, double tau, double *acc,
                           double *vx, double *vy, double *vz, uint32_t *status, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    combine_kernel<<<(N + 255) / 256, 256, 0, s>>>(partial, split, N, npad, tau, acc, vx, vy, vz, status);
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

}  // namespace genga
