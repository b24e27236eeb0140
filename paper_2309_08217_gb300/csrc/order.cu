// order.cu -- spatial order of the bodies for the long-range pass.
//
// Bodies are sorted along a 3-D Morton curve (7 bits per axis over the cube
// [-R, R]^3, R = the largest |coordinate|), so that a warp's i-bodies and a
// 256-body j-tile each cover a compact region; the pass kernels then test
// (warp, tile) bounding boxes and run most tiles without per-pair screening.
// Massive bodies (m > GENGA_HEAVY_MASS * M*: embryos, giant planets) come
// after all others: their r_crit bound is large, and inside a group of
// planetesimals one of them would make every group NEAR for its warp.  The
// order only changes which pairs share a tile, never which pairs are summed,
// so it affects speed, not the definition of the result.
//
// The sort is a stable least-significant-digit radix sort of the 22-bit keys
// (heavy flag above the 21 Morton bits) with 8-bit digits (three passes of
// histogram / scan / scatter; four in batched mode, where the system index
// fills the top byte).  Stable
// ranks inside a CTA come from warp match masks and per-warp digit counts, so
// the permutation is the same on every run.
#include "internal.cuh"

namespace genga {

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 4;
constexpr int RS_CHUNK = RS_THREADS * RS_ITEMS;  // keys per CTA
constexpr int RS_BITS = 8;
constexpr int RS_BINS = 1 << RS_BITS;
constexpr int RS_WARPS = RS_THREADS / 32;

// R = max |coordinate| (as float bits: non-negative floats order like uints).
__global__ void extent_kernel(const double *__restrict__ x, const double *__restrict__ y,
                              const double *__restrict__ z, int N, unsigned *__restrict__ rbits) {
    float r = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        r = fmaxf(r, fmaxf(fabsf((float)x[i]), fmaxf(fabsf((float)y[i]), fabsf((float)z[i]))));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    if ((threadIdx.x & 31) == 0) atomicMax(rbits, __float_as_uint(r));
}

__device__ __forceinline__ uint32_t spread3(uint32_t v) {  // 8 bits -> every third bit
    v &= 0xffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ uint32_t quant7(double c, float inv) {
    float f = ((float)c * inv + 1.0f) * 64.0f;
    f = fminf(fmaxf(f, 0.0f), 127.0f);
    return (uint32_t)f;
}

// Heavy flag and 21-bit Morton code of one body (k = its index in its system;
// in test-particle mode 2 the flag marks the bodies that are not test
// particles, so groups hold one kind only).
__device__ __forceinline__ uint32_t body_key(double x, double y, double z, double m, double heavy_mass, int k,
                                             int n_big, float inv) {
    const uint32_t heavy = (n_big >= 0 ? k < n_big : m > heavy_mass) ? 1u : 0u;
    return (heavy << 21) | spread3(quant7(x, inv)) | (spread3(quant7(y, inv)) << 1) | (spread3(quant7(z, inv)) << 2);
}

__global__ void keys_kernel(const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
                            const double *__restrict__ m, int N, double heavy_mass, int n_big,
                            const unsigned *__restrict__ rbits,
                            uint32_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float R = fmaxf(__uint_as_float(*rbits), 1e-30f) * 1.0001f;
    const float inv = 1.0f / R;
    keys[i] = body_key(x[i], y[i], z[i], m[i], heavy_mass, i, n_big, inv);
    vals[i] = (uint32_t)i;
}

// Batched: the system index d takes the top 8 bits, so one sort orders the
// bodies by system first and along the Morton curve inside each system.
__global__ void keys_batched_kernel(const double *__restrict__ x, const double *__restrict__ y,
                                    const double *__restrict__ z, const double *__restrict__ m, double heavy_mass,
                                    int n_big,
                                    const unsigned *__restrict__ rbits, uint32_t *__restrict__ keys,
                                    uint32_t *__restrict__ vals, const __grid_constant__ BatchBodies bb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= bb.N_total) return;
    const int d = find_segment(bb.off, bb.D, i);
    const float R = fmaxf(__uint_as_float(*rbits), 1e-30f) * 1.0001f;
    const float inv = 1.0f / R;
    keys[i] = ((uint32_t)d << 24) | body_key(x[i], y[i], z[i], m[i], heavy_mass, i - bb.off[d], n_big, inv);
    vals[i] = (uint32_t)i;
}

__global__ void __launch_bounds__(RS_THREADS) hist_kernel(const uint32_t *__restrict__ keys, int n, int shift,
                                                          uint32_t *__restrict__ hist, int nblk) {
    __shared__ uint32_t h[RS_BINS];
    for (int b = threadIdx.x; b < RS_BINS; b += RS_THREADS) h[b] = 0;
    __syncthreads();
    const int base = blockIdx.x * RS_CHUNK;
#pragma unroll
    for (int q = 0; q < RS_ITEMS; q++) {
        const int i = base + q * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & (RS_BINS - 1)], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < RS_BINS; b += RS_THREADS) hist[b * nblk + blockIdx.x] = h[b];
}

// Exclusive scan of hist[0 .. total) in place, one CTA of 1024 threads:
// segments of 8192 entries are loaded coalesced into shared memory, each
// thread scans 8 consecutive entries, a warp-shuffle scan combines the
// thread sums, and a running carry links the segments.
constexpr int SCAN_THREADS = 1024, SCAN_PER = 8, SCAN_SEG = SCAN_THREADS * SCAN_PER;

__global__ void __launch_bounds__(SCAN_THREADS) scan_kernel(uint32_t *__restrict__ hist, int total) {
    __shared__ uint32_t seg[SCAN_SEG];
    __shared__ uint32_t wsum[SCAN_THREADS / 32];
    __shared__ uint32_t carry_s;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry_s = 0;
    for (int base = 0; base < total; base += SCAN_SEG) {
        for (int q = threadIdx.x; q < SCAN_SEG; q += SCAN_THREADS)
            seg[q] = (base + q < total) ? hist[base + q] : 0u;
        __syncthreads();
        uint32_t v[SCAN_PER], t = 0;
#pragma unroll
        for (int q = 0; q < SCAN_PER; q++) {
            v[q] = t;
            t += seg[threadIdx.x * SCAN_PER + q];
        }
        uint32_t incl = t;  // inclusive scan of thread sums within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        if (w == 0) {
            uint32_t ws = wsum[lane], wi = ws;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            wsum[lane] = wi - ws;  // exclusive prefix of warp sums
        }
        __syncthreads();
        const uint32_t off = carry_s + wsum[w] + incl - t;
#pragma unroll
        for (int q = 0; q < SCAN_PER; q++) seg[threadIdx.x * SCAN_PER + q] = off + v[q];
        __syncthreads();
        for (int q = threadIdx.x; q < SCAN_SEG; q += SCAN_THREADS)
            if (base + q < total) hist[base + q] = seg[q];
        if (threadIdx.x == SCAN_THREADS - 1) carry_s = off + t;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(RS_THREADS) scatter_kernel(const uint32_t *__restrict__ kin,
                                                             const uint32_t *__restrict__ vin,
                                                             uint32_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                             int n, int shift, const uint32_t *__restrict__ offs,
                                                             int nblk) {
    __shared__ uint32_t run[RS_BINS];
    __shared__ uint32_t wcnt[RS_WARPS][RS_BINS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int b = threadIdx.x; b < RS_BINS; b += RS_THREADS) run[b] = offs[b * nblk + blockIdx.x];
    const int base = blockIdx.x * RS_CHUNK;
    for (int q = 0; q < RS_ITEMS; q++) {
        for (int e = threadIdx.x; e < RS_WARPS * RS_BINS; e += RS_THREADS) (&wcnt[0][0])[e] = 0u;
        __syncthreads();
        const int i = base + q * RS_THREADS + threadIdx.x;
        const bool valid = i < n;
        const uint32_t key = valid ? kin[i] : 0u;
        const uint32_t d = valid ? ((key >> shift) & (RS_BINS - 1)) : (uint32_t)RS_BINS;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const unsigned lt = (1u << lane) - 1u;
        const uint32_t rank = __popc(peers & lt);
        if (valid && lane == __ffs(peers) - 1) wcnt[w][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pre = 0;
            for (int v = 0; v < w; v++) pre += wcnt[v][d];
            const uint32_t pos = run[d] + pre + rank;
            kout[pos] = key;
            vout[pos] = vin[i];
        }
        __syncthreads();
        for (int b = threadIdx.x; b < RS_BINS; b += RS_THREADS) {
            uint32_t t = 0;
            for (int v = 0; v < RS_WARPS; v++) t += wcnt[v][b];
            run[b] += t;
        }
        __syncthreads();
    }
}

}  // namespace

size_t order_hist_entries(int nmax) { return (size_t)RS_BINS * ((nmax + RS_CHUNK - 1) / RS_CHUNK); }

// LSD radix sort of ord_keys[0] / ord_vals[0] (N entries) over `passes`
// 8-bit digits; the sorted values (body indices) end in c->perm.
void radix_to_perm(genga_ctx *c, int N, int passes, cudaStream_t s) {
    const int nblk = (N + RS_CHUNK - 1) / RS_CHUNK;
    int cur = 0;
    for (int pass = 0; pass < passes; pass++) {
        const int shift = pass * RS_BITS;
        hist_kernel<<<nblk, RS_THREADS, 0, s>>>(c->ord_keys[cur], N, shift, c->ord_hist, nblk);
        scan_kernel<<<1, SCAN_THREADS, 0, s>>>(c->ord_hist, RS_BINS * nblk);
        uint32_t *vout = (pass == passes - 1) ? c->perm : c->ord_vals[1 - cur];
        scatter_kernel<<<nblk, RS_THREADS, 0, s>>>(c->ord_keys[cur], c->ord_vals[cur], c->ord_keys[1 - cur], vout,
                                                   N, shift, c->ord_hist, nblk);
        cur = 1 - cur;
    }
}

// perm[k] = index of the body at position k of the Morton order (k < N).
cudaError_t launch_order(const genga_system &sys, double Mstar, int n_big, genga_ctx *c, cudaStream_t s) {
    const int N = sys.N;
    if (N <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(c->ord_rbits, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    extent_kernel<<<64, 256, 0, s>>>(sys.x, sys.y, sys.z, N, c->ord_rbits);
    keys_kernel<<<(N + 255) / 256, 256, 0, s>>>(sys.x, sys.y, sys.z, sys.m, N, GENGA_HEAVY_MASS * Mstar, n_big,
                                                c->ord_rbits, c->ord_keys[0], c->ord_vals[0]);
    radix_to_perm(c, N, 3, s);
    return cudaGetLastError();
}

// Batched: the 22-bit keys below the 8-bit system index, four passes.
cudaError_t launch_order_batched(const genga_system &all, const BatchBodies &bb, double Mstar, int n_big,
                                 genga_ctx *c, cudaStream_t s) {
    const int N = bb.N_total;
    if (N <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(c->ord_rbits, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    extent_kernel<<<64, 256, 0, s>>>(all.x, all.y, all.z, N, c->ord_rbits);
    keys_batched_kernel<<<(N + 255) / 256, 256, 0, s>>>(all.x, all.y, all.z, all.m, GENGA_HEAVY_MASS * Mstar,
                                                        n_big, c->ord_rbits, c->ord_keys[0], c->ord_vals[0], bb);
    radix_to_perm(c, N, 4, s);
    return cudaGetLastError();
}

}  // namespace genga
