// measure.cu -- measurement hooks (include/genga_measure.h): CUDA events
// around the long-range pass launches, and an FFMA / DFMA throughput
// microbenchmark used as the arithmetic roofline of the pass kernels.
#include <stdlib.h>

#include <new>

#include "../../include/genga_measure.h"
#include "internal.cuh"

namespace genga {

void profile_before_pass(genga_ctx *c, cudaStream_t s) {
    Profile *p = c->prof;
    if (!p || !p->enabled || p->n >= Profile::CAP) return;
    cudaEventRecord(p->ev[2 * p->n], s);
}

void profile_after_pass(genga_ctx *c, cudaStream_t s) {
    Profile *p = c->prof;
    if (!p || !p->enabled || p->n >= Profile::CAP) return;
    cudaEventRecord(p->ev[2 * p->n + 1], s);
    p->n++;
}

void profile_free(genga_ctx *c) {
    Profile *p = c->prof;
    if (!p) return;
    for (int k = 0; k < p->created; k++) cudaEventDestroy(p->ev[k]);
    free(p->ev);
    delete p;
    c->prof = nullptr;
}

namespace {

constexpr int PEAK_ITERS = 4096;

// Eight independent FMA chains per thread; the result is stored only if it
// equals an impossible value, so the compiler keeps the work.
template <class T>
__global__ void fma_peak_kernel(T a, T b, T *out) {
    T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
      x7 = x0 + 7;
#pragma unroll 16
    for (int it = 0; it < PEAK_ITERS; it++) {
        x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
        x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
    const T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == (T)-1.2345) out[0] = s;
}

// The same with packed two-lane FP32 FMAs (fma.rn.f32x2): eight chains of
// two lanes each.
__global__ void fma2_peak_kernel(float a, float b, float *out) {
    unsigned long long A, B, x[8];
    asm("mov.b64 %0, {%1, %1};" : "=l"(A) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(B) : "f"(b));
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const float v = (float)(threadIdx.x + c);
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[c]) : "f"(v), "f"(v + 0.5f));
    }
#pragma unroll 16
    for (int it = 0; it < PEAK_ITERS; it++) {
#pragma unroll
        for (int c = 0; c < 8; c++) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(A), "l"(B));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        float u, w;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(u), "=f"(w) : "l"(x[c]));
        s += u + w;
    }
    if (s == -1.2345f) out[0] = s;
}

double run_peak_fma2(int sms, float *out) {
    const int threads = 256, blocks = sms * 8;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fma2_peak_kernel<<<blocks, threads>>>(0.999999f, 1e-7f, out);
    float best = 1e30f;
    for (int rep = 0; rep < 5; rep++) {
        cudaEventRecord(e0);
        fma2_peak_kernel<<<blocks, threads>>>(0.999999f, 1e-7f, out);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double flops = 2.0 * 2.0 * 8.0 * PEAK_ITERS * (double)threads * blocks;
    return flops / (best * 1e-3) / 1e12;
}

template <class T>
double run_peak(int sms, T *out) {
    const int threads = 256, blocks = sms * 8;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fma_peak_kernel<T><<<blocks, threads>>>((T)0.999999, (T)1e-7, out);  // warm-up
    float best = 1e30f;
    for (int rep = 0; rep < 5; rep++) {
        cudaEventRecord(e0);
        fma_peak_kernel<T><<<blocks, threads>>>((T)0.999999, (T)1e-7, out);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double flops = 2.0 * 8.0 * PEAK_ITERS * (double)threads * blocks;
    return flops / (best * 1e-3) / 1e12;
}

}  // namespace
}  // namespace genga

using namespace genga;

extern "C" {

genga_status genga_profile_enable(genga_ctx *c, int32_t enable) {
    if (!c) return GENGA_ERR_INVALID_ARG;
    if (!c->prof) {
        Profile *p = new (std::nothrow) Profile();
        if (!p) return GENGA_ERR_CUDA;
        p->ev = (cudaEvent_t *)calloc(2 * Profile::CAP, sizeof(cudaEvent_t));
        if (!p->ev) {
            delete p;
            return GENGA_ERR_CUDA;
        }
        c->prof = p;
    }
    Profile *p = c->prof;
    int dev_prev = -1;
    cudaGetDevice(&dev_prev);
    if (dev_prev != c->device) cudaSetDevice(c->device);
    // events are created lazily up to what a run needs; create a first batch
    const int want = enable ? 2 * 4096 : 0;
    while (p->created < want && p->created < 2 * Profile::CAP) {
        if (cudaEventCreate(&p->ev[p->created]) != cudaSuccess) break;
        p->created++;
    }
    if (dev_prev >= 0 && dev_prev != c->device) cudaSetDevice(dev_prev);
    p->enabled = enable != 0;
    p->n = 0;
    return GENGA_OK;
}

genga_status genga_profile_read(genga_ctx *c, double *pass_ms, int32_t *launches, int32_t reset) {
    if (!c || !pass_ms || !launches) return GENGA_ERR_INVALID_ARG;
    *pass_ms = 0.0;
    *launches = 0;
    Profile *p = c->prof;
    if (!p) return GENGA_OK;
    double tot = 0.0;
    for (int k = 0; k < p->n; k++) {
        if (cudaEventSynchronize(p->ev[2 * k + 1]) != cudaSuccess) return GENGA_ERR_CUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p->ev[2 * k], p->ev[2 * k + 1]) != cudaSuccess) return GENGA_ERR_CUDA;
        tot += ms;
    }
    *pass_ms = tot;
    *launches = p->n;
    if (reset) p->n = 0;
    return GENGA_OK;
}

genga_status genga_launch_count(genga_ctx *c, int64_t *count) {
    if (!c || !count) return GENGA_ERR_INVALID_ARG;
    *count = c->launches;
    return GENGA_OK;
}

genga_status genga_tuning_times(genga_ctx *c, int32_t N, float *ms, int32_t n) {
    if (!c || !ms || n < 0 || N < 0) return GENGA_ERR_INVALID_ARG;
    int b = 0;
    for (int v = (N + GENGA_PAD - 1) / GENGA_PAD * GENGA_PAD; v > 1; v >>= 1) b++;
    b = b < 32 ? b : 31;
    const int nv = num_fp32_variants() + num_mutual_variants();
    for (int q = 0; q < n; q++) ms[q] = (q < GENGA_MAX_VARIANTS && q < nv) ? c->tune_ms[b][q] : 0.f;
    return GENGA_OK;
}

genga_status genga_set_kernel_variant(genga_ctx *c, int32_t variant) {
    if (!c || variant < -1 || variant >= num_fp32_variants() + num_mutual_variants()) return GENGA_ERR_INVALID_ARG;
    c->forced_variant = variant;
    return GENGA_OK;
}

genga_status genga_kernel_variant_info(int32_t variant, int32_t *kind, int32_t *warps, int32_t *bodies_per_thread,
                                       int32_t *ctas_per_sm) {
    const int n1 = num_fp32_variants();
    if (!kind || !warps || !bodies_per_thread || !ctas_per_sm || variant < 0 || variant >= n1 + num_mutual_variants())
        return GENGA_ERR_INVALID_ARG;
    int cw = 0, bpt = 0, minb = 1;
    if (variant < n1) {
        fp32_variant_shape(variant, &cw, &bpt, &minb);
        *kind = 0;
    } else {
        mutual_variant_shape(variant - n1, &cw, &bpt);
        *kind = 1;
    }
    *warps = cw;
    *bodies_per_thread = bpt;
    *ctas_per_sm = minb;
    return GENGA_OK;
}

genga_status genga_set_fp64_variant(genga_ctx *c, int32_t variant) {
    if (!c || variant < -1 || variant >= 1 + num_mutual64_variants()) return GENGA_ERR_INVALID_ARG;
    c->forced_f64 = variant;
    return GENGA_OK;
}

genga_status genga_get_fp64_variant(genga_ctx *c, int32_t N, int32_t *variant, int32_t *num_variants) {
    if (!c || !variant || !num_variants || N < 0) return GENGA_ERR_INVALID_ARG;
    int b = 0;
    for (int v = (N + GENGA_PAD - 1) / GENGA_PAD * GENGA_PAD; v > 1; v >>= 1) b++;
    b = b < 32 ? b : 31;
    *variant = (c->forced_f64 >= 0) ? c->forced_f64 : c->f64_variant[b];
    *num_variants = 1 + num_mutual64_variants();
    return GENGA_OK;
}

genga_status genga_fp64_variant_info(int32_t variant, int32_t *kind, int32_t *warps, int32_t *bodies_per_thread) {
    if (!kind || !warps || !bodies_per_thread || variant < 0 || variant >= 1 + num_mutual64_variants())
        return GENGA_ERR_INVALID_ARG;
    int cw = 0, bpt = 0;
    if (variant == 0) {
        fp64_pass_shape(&cw, &bpt);
        *kind = 0;
    } else {
        mutual64_variant_shape(variant - 1, &cw, &bpt);
        *kind = 1;
    }
    *warps = cw;
    *bodies_per_thread = bpt;
    return GENGA_OK;
}

genga_status genga_fp64_tuning_times(genga_ctx *c, int32_t N, float *ms, int32_t n) {
    if (!c || !ms || n < 0 || N < 0) return GENGA_ERR_INVALID_ARG;
    int b = 0;
    for (int v = (N + GENGA_PAD - 1) / GENGA_PAD * GENGA_PAD; v > 1; v >>= 1) b++;
    b = b < 32 ? b : 31;
    const int nv = 1 + num_mutual64_variants();
    for (int q = 0; q < n; q++) ms[q] = (q < GENGA_MAX_VARIANTS && q < nv) ? c->tune64_ms[b][q] : 0.f;
    return GENGA_OK;
}

genga_status genga_set_test_waits(genga_ctx *c, int32_t wait_ns_log2, int32_t hold) {
    if (!c || wait_ns_log2 < 0 || wait_ns_log2 > 40) return GENGA_ERR_INVALID_ARG;
    c->test_wait_log2 = wait_ns_log2;
    c->test_hold = hold ? 1 : 0;
    return GENGA_OK;
}

genga_status genga_set_step_graphs(genga_ctx *c, int32_t enable) {
    if (!c) return GENGA_ERR_INVALID_ARG;
    c->step_graphs = enable ? 1 : 0;
    return GENGA_OK;
}

genga_status genga_get_kernel_variant(genga_ctx *c, int32_t N, int32_t *variant, int32_t *num_variants) {
    if (!c || !variant || !num_variants || N < 0) return GENGA_ERR_INVALID_ARG;
    int b = 0;
    for (int v = (N + GENGA_PAD - 1) / GENGA_PAD * GENGA_PAD; v > 1; v >>= 1) b++;
    b = b < 32 ? b : 31;
    *variant = (c->forced_variant >= 0) ? c->forced_variant : c->f32_variant[0][b];
    *num_variants = num_fp32_variants() + num_mutual_variants();
    return GENGA_OK;
}

genga_status genga_measure_fma2_peak(int32_t device, double *tflops) {
    if (!tflops) return GENGA_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) return GENGA_ERR_CUDA;
    if (device < 0 || device >= ndev) return GENGA_ERR_INVALID_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    void *buf = nullptr;
    genga_status st = GENGA_OK;
    if (cudaMalloc(&buf, 64) != cudaSuccess) {
        st = GENGA_ERR_CUDA;
    } else {
        *tflops = run_peak_fma2(sms, (float *)buf);
        if (cudaGetLastError() != cudaSuccess) st = GENGA_ERR_CUDA;
        cudaFree(buf);
    }
    if (prev >= 0) cudaSetDevice(prev);
    return st;
}

genga_status genga_measure_alu_peaks(int32_t device, double *fp32_tflops, double *fp64_tflops) {
    if (!fp32_tflops || !fp64_tflops) return GENGA_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) return GENGA_ERR_CUDA;
    if (device < 0 || device >= ndev) return GENGA_ERR_INVALID_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    void *buf = nullptr;
    genga_status st = GENGA_OK;
    if (cudaMalloc(&buf, 64) != cudaSuccess) {
        st = GENGA_ERR_CUDA;
    } else {
        *fp32_tflops = run_peak<float>(sms, (float *)buf);
        *fp64_tflops = run_peak<double>(sms, (double *)buf);
        if (cudaGetLastError() != cudaSuccess) st = GENGA_ERR_CUDA;
        cudaFree(buf);
    }
    if (prev >= 0) cudaSetDevice(prev);
    return st;
}

}  // extern "C"
