// compact.cu -- removal of ghosts from the caller's arrays (genga_compact):
// bodies that merged into others or crossed a removal radius (Sect. 2) carry
// the mass -0.0 (set by the close-encounter level and the drift); a stable
// device-side compaction moves the others to the front, in order.
//
//   count    block b counts the live bodies of [1024 b, 1024 b + 1024)
//   scan     one CTA: exclusive scan of the block counts, the new N
//   scatter  block b ranks its live bodies (block scan) and copies them to the
//            scratch arrays at offset[b] + rank
//   copy     scratch -> caller's arrays (the first new-N entries)
#include "internal.cuh"

namespace genga {

namespace {

constexpr int CT = 1024;  // bodies per block

__device__ int block_excl_scan(int v, int *warp_sums, int *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[w] = incl;
    __syncthreads();
    if (w == 0) {
        int s = warp_sums[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    const int r = incl - v + (w > 0 ? warp_sums[w - 1] : 0);
    *total = warp_sums[31];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(CT) count_kernel(const double *__restrict__ m, int N, int32_t *__restrict__ cnt) {
    __shared__ int warp_sums[32];
    const int i = blockIdx.x * CT + threadIdx.x;
    const int live = (i < N && !signbit(m[i])) ? 1 : 0;
    int total;
    block_excl_scan(live, warp_sums, &total);
    if (threadIdx.x == 0) cnt[blockIdx.x] = total;
}

__global__ void __launch_bounds__(CT) scan_kernel(const int32_t *__restrict__ cnt, int nb, int32_t *__restrict__ off,
                                                  int32_t *__restrict__ newN) {
    __shared__ int warp_sums[32];
    int carry = 0;
    for (int base = 0; base < nb; base += CT) {
        const int b = base + threadIdx.x;
        const int v = b < nb ? cnt[b] : 0;
        int total;
        const int r = block_excl_scan(v, warp_sums, &total);
        if (b < nb) off[b] = carry + r;
        carry += total;
    }
    if (threadIdx.x == 0) *newN = carry;
}

struct CompactArrays {
    double *f[8];     // x, y, z, vx, vy, vz, m, radius (radius may be NULL)
    int32_t *id;      // optional
    double *tmp;      // 9 fields of `stride` doubles
    size_t stride;
};

__global__ void __launch_bounds__(CT) scatter_kernel(const __grid_constant__ CompactArrays c, int N,
                                                     const int32_t *__restrict__ off) {
    __shared__ int warp_sums[32];
    const int i = blockIdx.x * CT + threadIdx.x;
    const int live = (i < N && !signbit(c.f[6][i])) ? 1 : 0;
    int total;
    const int r = block_excl_scan(live, warp_sums, &total);
    if (!live) return;
    const size_t d = (size_t)off[blockIdx.x] + r;
    for (int k = 0; k < 8; k++)
        if (c.f[k]) c.tmp[(size_t)k * c.stride + d] = c.f[k][i];
    if (c.id) c.tmp[8 * c.stride + d] = (double)c.id[i];
}

__global__ void copy_back_kernel(const __grid_constant__ CompactArrays c, int N, const int32_t *__restrict__ newN) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N || i >= *newN) return;
    for (int k = 0; k < 8; k++)
        if (c.f[k]) c.f[k][i] = c.tmp[(size_t)k * c.stride + i];
    if (c.id) c.id[i] = (int32_t)c.tmp[8 * c.stride + i];
}

}  // namespace

// Compacts the N bodies of sys (and id), dropping those of mass -0.0; the new count goes to
// *count (device).  Scratch: ctx->partial (9 N doubles), ctx->gsize / gstart
// (block counts and offsets, N / 1024 entries).
cudaError_t launch_compact(genga_ctx *c, genga_system &sys, int32_t *id, int32_t *count, cudaStream_t s) {
    const int N = sys.N, nb = (N + CT - 1) / CT;
    CompactArrays a;
    a.f[0] = sys.x; a.f[1] = sys.y; a.f[2] = sys.z;
    a.f[3] = sys.vx; a.f[4] = sys.vy; a.f[5] = sys.vz;
    a.f[6] = sys.m; a.f[7] = sys.radius;
    a.id = id;
    a.tmp = c->partial;
    a.stride = (size_t)N;
    count_kernel<<<nb, CT, 0, s>>>(sys.m, N, c->gsize);
    scan_kernel<<<1, CT, 0, s>>>(c->gsize, nb, c->gstart, count);
    scatter_kernel<<<nb, CT, 0, s>>>(a, N, c->gstart);
    copy_back_kernel<<<(N + 255) / 256, 256, 0, s>>>(a, N, count);
    return cudaGetLastError();
}

}  // namespace genga
