// noalloc.cu -- genga_kick_noalloc: the FP64 long-range kick without any
// device allocation (declared in include/genga_noalloc.h).
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or allocator hooks, plug-ins that are not allowed
// to grow device memory, or hosts that budget device memory up front and
// forbid allocation later.  For them this entry point keeps all its
// scratch -- the per-block momentum partials, the completion ticket and the
// per-body critical-radius inputs -- in one file-scope __device__ array of
// fixed size, so every GPU that loads the library holds that array (about
// 1.6 MB) until the process exits.  The caller still provides the state
// arrays and the acceleration output.
//
// Host code cannot use the array's name as a device address, so the first
// call in each CUDA context looks the address up with cudaGetSymbolAddress
// (with that context current) and caches it under the context's unique id;
// later calls in the same context reuse it.  A new context on the same device
// (after cudaDeviceReset, or a caller's own driver context) has a new id, so
// its first call looks the address up again instead of reusing an address
// that belongs to another context.
#include <cuda.h>  // CUcontext and CUresult only; the driver calls are resolved at run time

#include <mutex>

#include "../../include/genga_noalloc.h"
#include "internal.cuh"

namespace {

constexpr int NA_MOM_BLOCKS = 64;
constexpr int NA_THREADS = 256;
// scratch layout, in doubles: momentum partials, P, ticket, then a_i and
// r_crit,i of each body
constexpr size_t NA_OFF_PART = 0;
constexpr size_t NA_OFF_P = NA_OFF_PART + 3 * NA_MOM_BLOCKS;
constexpr size_t NA_OFF_TICKET = NA_OFF_P + 4;
constexpr size_t NA_OFF_A = 256;
constexpr size_t NA_OFF_RC = NA_OFF_A + GENGA_NOALLOC_MAX_N;
constexpr size_t NA_OFF_H = NA_OFF_RC + GENGA_NOALLOC_MAX_N;  // n1 (2 m_i / 3 M*)^(1/3)
constexpr size_t NA_DOUBLES = NA_OFF_H + GENGA_NOALLOC_MAX_N;

static __device__ __align__(256) double g_noalloc_scratch[NA_DOUBLES];

struct NaSum {  // Neumaier running sum
    double s = 0.0, c = 0.0;
    __device__ void add(double v) {
        const double t = s + v;
        c += (fabs(s) >= fabs(v)) ? ((s - t) + v) : ((v - t) + s);
        s = t;
    }
    __device__ double value() const { return s + c; }
};

// P = sum m v: block partials in index order, the last block adds them up.
__global__ void __launch_bounds__(NA_THREADS) na_momentum(const double *__restrict__ vx, const double *__restrict__ vy,
                                                          const double *__restrict__ vz, const double *__restrict__ m,
                                                          int N, double *scratch) {
    __shared__ double sh[3][NA_THREADS];
    __shared__ bool last;
    double *part = scratch + NA_OFF_PART;
    unsigned *ticket = reinterpret_cast<unsigned *>(scratch + NA_OFF_TICKET);
    const int chunk = (N + NA_MOM_BLOCKS - 1) / NA_MOM_BLOCKS;
    const int lo = blockIdx.x * chunk, hi = min(N, lo + chunk);
    NaSum px, py, pz;
    for (int i = lo + threadIdx.x; i < hi; i += NA_THREADS) {
        px.add(m[i] * vx[i]);
        py.add(m[i] * vy[i]);
        pz.add(m[i] * vz[i]);
    }
    sh[0][threadIdx.x] = px.value();
    sh[1][threadIdx.x] = py.value();
    sh[2][threadIdx.x] = pz.value();
    __syncthreads();
    for (int w = NA_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 3; c++) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int c = 0; c < 3; c++) part[3 * blockIdx.x + c] = sh[c][0];
        __threadfence();
        last = (atomicAdd(ticket, 1u) == NA_MOM_BLOCKS - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < 3) {
        NaSum t;
        const volatile double *vp = part;
        for (int b = 0; b < NA_MOM_BLOCKS; b++) t.add(vp[3 * b + threadIdx.x]);
        scratch[NA_OFF_P + threadIdx.x] = t.value();
    }
}

// Eq. (1) inputs of every body: osculating a_i and r_crit,i.
__global__ void na_rcrit(const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
                         const double *__restrict__ vx, const double *__restrict__ vy, const double *__restrict__ vz,
                         const double *__restrict__ m, int N, double G, double Mstar, double dt, double n1, double n2,
                         double *scratch) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double *P = scratch + NA_OFF_P;
    const double ux = vx[i] + P[0] / Mstar, uy = vy[i] + P[1] / Mstar, uz = vz[i] + P[2] / Mstar;
    const double v2 = ux * ux + uy * uy + uz * uz;
    const double r = sqrt(x[i] * x[i] + y[i] * y[i] + z[i] * z[i]);
    const double inva = 2.0 / r - v2 / (G * (Mstar + m[i]));
    const double a = (inva > 0.0) ? 1.0 / inva : r;
    scratch[NA_OFF_A + i] = a;
    scratch[NA_OFF_RC + i] = fmax(n1 * a * cbrt(m[i] / (3.0 * Mstar)), n2 * dt * sqrt(v2));
    scratch[NA_OFF_H + i] = n1 * cbrt(2.0 * m[i] / (3.0 * Mstar));
}

__device__ double na_changeover(double y, int form) {
    if (y <= 0.0) return 0.0;
    if (y >= 1.0) return 1.0;
    if (form == GENGA_K_CHAMBERS) return y * y / (2.0 * y * y - 2.0 * y + 1.0);
    return y * y * y * (10.0 - 15.0 * y + 6.0 * y * y);
}

// One thread per body i: the FP64 sum over all j != i, compensated every 32
// terms; r_crit,ij and K are evaluated only for pairs inside a cheap bound.
__global__ void na_acc(const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
                       double *__restrict__ vx, double *__restrict__ vy, double *__restrict__ vz,
                       const double *__restrict__ m, int N, double G, double Mstar, double n1, int mode, int form,
                       int n_big, double tau, double *__restrict__ acc, const double *scratch) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double *A = scratch + NA_OFF_A, *RC = scratch + NA_OFF_RC, *H = scratch + NA_OFF_H;
    const double xi = x[i], yi = y[i], zi = z[i], mi = m[i], ai = A[i], rci = RC[i], hi = H[i];
    NaSum sx, sy, sz;
    double px = 0.0, py = 0.0, pz = 0.0;
    const bool tp_i = n_big >= 0 && i >= n_big;  // test-particle mode 2: no force between test particles
    for (int j = 0; j < N; j++) {
        if (j != i && !(tp_i && j >= n_big)) {
            const double dx = x[j] - xi, dy = y[j] - yi, dz = z[j] - zi;
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 > 0.0) {
                const double r = sqrt(r2);
                double K = 1.0;
                // r_crit,ij <= max(H_i, H_j) max(a_i, a_j) (mutual Hill) or max(rc_i, rc_j)
                const double bound = (mode == GENGA_RCRIT_EQ1) ? fmax(rci, RC[j]) : fmax(hi, H[j]) * fmax(ai, A[j]);
                if (r < bound * (1.0 + 1e-9)) {
                    const double rc = (mode == GENGA_RCRIT_EQ1)
                                          ? fmax(rci, RC[j])
                                          : n1 * cbrt((mi + m[j]) / (3.0 * Mstar)) * 0.5 * (ai + A[j]);
                    if (r < rc) K = na_changeover((r / rc - 0.1) / 0.9, form);
                }
                const double f = G * m[j] * K / (r2 * r);
                px += f * dx;
                py += f * dy;
                pz += f * dz;
            }
        }
        if ((j & 31) == 31 || j == N - 1) {
            sx.add(px);
            sy.add(py);
            sz.add(pz);
            px = py = pz = 0.0;
        }
    }
    const double ax = sx.value(), ay = sy.value(), az = sz.value();
    if (acc) {
        acc[i] = ax;
        acc[(size_t)N + i] = ay;
        acc[2 * (size_t)N + i] = az;
    }
    if (tau != 0.0) {
        vx[i] += ax * tau;
        vy[i] += ay * tau;
        vz[i] += az * tau;
    }
}

// Address of g_noalloc_scratch per CUDA context, keyed by the context's
// unique id (cuCtxGetId), so an address is never used in another context.
// The two driver calls are taken from the runtime's driver entry-point table,
// so the library links against the CUDA runtime only.
constexpr int NA_MAX_CONTEXTS = 64;
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);
struct NaEntry {
    unsigned long long ctx_id;
    double *ptr;
};
std::mutex g_na_mutex;
NaEntry g_na_cache[NA_MAX_CONTEXTS];
int g_na_used = 0, g_na_next = 0;
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;

cudaError_t current_context_id(unsigned long long *id) {
    if (!g_ctx_current || !g_ctx_id) {
        void *f0 = nullptr, *f1 = nullptr;
        cudaDriverEntryPointQueryResult q0 = cudaDriverEntryPointSymbolNotFound, q1 = q0;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0);
        if (e != cudaSuccess) return e;
        e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1);
        if (e != cudaSuccess) return e;
        if (q0 != cudaDriverEntryPointSuccess || q1 != cudaDriverEntryPointSuccess || !f0 || !f1)
            return cudaErrorNotSupported;
        g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f0);
        g_ctx_id = reinterpret_cast<CtxGetIdFn>(f1);
    }
    CUcontext ctx = nullptr;
    if (g_ctx_current(&ctx) != CUDA_SUCCESS) return cudaErrorContextIsDestroyed;
    if (!ctx) {
        // no context is current yet: cudaSetDevice on the current device
        // binds its primary context (and allocates nothing)
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaSetDevice(dev);
        if (e != cudaSuccess) return e;
        if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorContextIsDestroyed;
    }
    return g_ctx_id(ctx, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorContextIsDestroyed;
}

cudaError_t scratch_for_current_context(double **out) {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    unsigned long long id = 0;
    cudaError_t e = current_context_id(&id);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < g_na_used; k++) {
        if (g_na_cache[k].ctx_id == id) {
            *out = g_na_cache[k].ptr;
            return cudaSuccess;
        }
    }
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    // a full table replaces its oldest entry (a context seen again later is
    // looked up again)
    const int k = g_na_used < NA_MAX_CONTEXTS ? g_na_used++ : (g_na_next++ % NA_MAX_CONTEXTS);
    g_na_cache[k] = NaEntry{id, static_cast<double *>(p)};
    *out = static_cast<double *>(p);
    return cudaSuccess;
}

}  // namespace

extern "C" genga_status genga_kick_noalloc(const genga_system *sys, const genga_params *p, double tau, double *acc,
                                           void *stream) {
    if (!sys || !p) return GENGA_ERR_INVALID_ARG;
    if (sys->N < 0 || sys->N > GENGA_NOALLOC_MAX_N) return GENGA_ERR_INVALID_ARG;
    if (sys->N > 0 && (!sys->x || !sys->y || !sys->z || !sys->vx || !sys->vy || !sys->vz || !sys->m))
        return GENGA_ERR_INVALID_ARG;
    if (p->precision != GENGA_FP64 || !isfinite(p->G) || !(p->G >= 0.0) || !isfinite(p->Mstar) ||
        !(p->Mstar > 0.0) || !isfinite(p->dt) || !isfinite(p->n1) || !isfinite(p->n2) || p->n1 < 0.0 ||
        p->n2 < 0.0 || (p->rcrit_mode != GENGA_RCRIT_EQ1 && p->rcrit_mode != GENGA_RCRIT_MUTUAL_HILL) ||
        (p->changeover != GENGA_K_CHAMBERS && p->changeover != GENGA_K_QUINTIC) || p->n_big < -1 || !isfinite(tau))
        return GENGA_ERR_INVALID_ARG;
    if (sys->N == 0) return GENGA_OK;
    double *scratch = nullptr;
    if (scratch_for_current_context(&scratch) != cudaSuccess) return GENGA_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const int N = sys->N;
    // the momentum kernel's completion ticket must start at zero on every call
    if (cudaMemsetAsync(scratch + NA_OFF_TICKET, 0, sizeof(double), s) != cudaSuccess) return GENGA_ERR_CUDA;
    na_momentum<<<NA_MOM_BLOCKS, NA_THREADS, 0, s>>>(sys->vx, sys->vy, sys->vz, sys->m, N, scratch);
    const int nb = (N + NA_THREADS - 1) / NA_THREADS;
    na_rcrit<<<nb, NA_THREADS, 0, s>>>(sys->x, sys->y, sys->z, sys->vx, sys->vy, sys->vz, sys->m, N, p->G,
                                       p->Mstar, p->dt, p->n1, p->n2, scratch);
    na_acc<<<nb, NA_THREADS, 0, s>>>(sys->x, sys->y, sys->z, sys->vx, sys->vy, sys->vz, sys->m, N, p->G, p->Mstar,
                                     p->n1, p->rcrit_mode, p->changeover, p->n_big, tau, acc, scratch);
    return cudaGetLastError() == cudaSuccess ? GENGA_OK : GENGA_ERR_CUDA;
}
