/*
 * genga_measure.h -- measurement hooks of libgenga.  The paper has no
 * counterpart for these; they exist so that a benchmark can time the
 * dominant kernel live and compare it with the chip's arithmetic peaks.
 */
#ifndef GENGA_MEASURE_H
#define GENGA_MEASURE_H

#include "genga.h"

#ifdef __cplusplus
extern "C" {
#endif

/* enable != 0: from now on, record a CUDA event pair around every launch of
 * the long-range pass kernel, on the stream it is launched on (at most 65536
 * pairs; later launches are not recorded).  enable == 0 stops recording.
 * Either call discards pairs recorded so far. */
genga_status genga_profile_enable(genga_ctx *ctx, int32_t enable);

/* Synchronise the recorded events and return the summed device time of the
 * recorded pass launches (*pass_ms) and their number (*launches); both
 * pointers are HOST memory.  reset != 0 discards the pairs afterwards. */
genga_status genga_profile_read(genga_ctx *ctx, double *pass_ms, int32_t *launches, int32_t reset);

/* Arithmetic throughput microbenchmark on `device`: independent FFMA and
 * DFMA chains over every SM; results in TFLOP/s (2 flops per FMA), HOST
 * memory.  Synchronous; allocates and frees a small result buffer. */
genga_status genga_measure_alu_peaks(int32_t device, double *fp32_tflops, double *fp64_tflops);

/* The same microbenchmark with packed two-lane FP32 FMAs (fma.rn.f32x2, the
 * form the FP32 pass uses); TFLOP/s counting 4 flops per packed FMA. */
genga_status genga_measure_fma2_peak(int32_t device, double *tflops);

/* The autotuner's measured pass time (ms) of each FP32 variant for systems of
 * N bodies (0 where not measured); ms is HOST memory [n]. */
genga_status genga_tuning_times(genga_ctx *ctx, int32_t N, float *ms, int32_t n);

/* Number of CUDA kernels the context has launched so far (HOST memory);
 * autotuning trial launches included. */
genga_status genga_launch_count(genga_ctx *ctx, int64_t *count);

/* Kernel variant of the FP32 long-range pass (bodies per thread, resident
 * CTAs per SM, loop unroll).  variant >= 0 forces that variant for every
 * size; variant = -1 (the default) lets the context time all variants the
 * first time it meets a size bucket (a power of two of the padded N) and keep
 * the fastest -- that first pass synchronises its stream.  Out-of-range
 * values return GENGA_ERR_INVALID_ARG. */
genga_status genga_set_kernel_variant(genga_ctx *ctx, int32_t variant);

/* The FP32 variant the context uses for systems of N bodies (-1 when that
 * size has not been tuned yet), and the number of variants; HOST memory. */
genga_status genga_get_kernel_variant(genga_ctx *ctx, int32_t N, int32_t *variant, int32_t *num_variants);

/* Shape of FP32 pass variant `variant` (HOST memory outputs): kind 0 = the
 * one-sided pass (every ordered pair from the side of its i-body), 1 = the
 * mutual pass (each unordered pair once, its terms added to both bodies);
 * consumer warps per CTA, i-bodies per thread, resident CTAs per SM.
 * Out-of-range variant: GENGA_ERR_INVALID_ARG. */
genga_status genga_kernel_variant_info(int32_t variant, int32_t *kind, int32_t *warps, int32_t *bodies_per_thread,
                                       int32_t *ctas_per_sm);

/* FP64 pass variants: 0 = the one-sided FP64 pass, 1 .. = the mutual FP64
 * pass (each unordered pair once, its terms added to both bodies) in several
 * shapes.  genga_set_fp64_variant forces `variant` (>= 0) or, with -1 (the
 * default), lets the context time every variant the first time it meets a
 * size bucket and keep the fastest, as for the FP32 pass; test-particle mode
 * 2 always takes variant 0.  Out-of-range values: GENGA_ERR_INVALID_ARG. */
genga_status genga_set_fp64_variant(genga_ctx *ctx, int32_t variant);

/* The FP64 variant used for systems of N bodies (-1 when not tuned yet) and
 * the number of FP64 variants; HOST memory. */
genga_status genga_get_fp64_variant(genga_ctx *ctx, int32_t N, int32_t *variant, int32_t *num_variants);

/* Shape of FP64 variant `variant` (HOST memory outputs): kind 0 one-sided,
 * 1 mutual; warps per CTA doing pair work; i-bodies per thread. */
genga_status genga_fp64_variant_info(int32_t variant, int32_t *kind, int32_t *warps, int32_t *bodies_per_thread);

/* The autotuner's measured pass time (ms) of each FP64 variant for systems of
 * N bodies (0 where not measured); ms is HOST memory [n]. */
genga_status genga_fp64_tuning_times(genga_ctx *ctx, int32_t N, float *ms, int32_t n);

/* Batched mode: the FP32 variant the context tuned for the batch layout
 * `offsets` (D + 1 ints, HOST memory, as for genga_kick_batched) in the
 * autotuned precision mode GENGA_FP32 -- -1 when this layout has not been
 * tuned (or was forgotten: a context remembers the last 8 layouts and modes)
 * -- and the batched pass + combine time (ms) of each variant measured then
 * (0 where not measured); variant and ms[n] are HOST memory.  A layout is
 * tuned by its first batched kick or step outside a stream capture (every
 * variant of the mode's family: one-sided and mutual for GENGA_FP32;
 * genga_set_kernel_variant skips that). */
genga_status genga_batched_tuning(genga_ctx *ctx, const int32_t *offsets, int32_t D, int32_t *variant, float *ms,
                                  int32_t n);

/* Host-only self-check of the mutual passes' work plan (no device, no
 * context): builds the plan for a batch of nsys systems of n[d] bodies (HOST
 * memory; nsys = 1: a single system) for cw consumer warps of npg 64-body
 * groups each and ctas persistent CTAs, and verifies by enumeration that
 * every pair of groups of a system is visited exactly once (both orders
 * inside an i-block, one visit across blocks), that no item leaves its
 * system or reaches a group without bodies, and that each block's partial
 * rows are exactly the rows its combine reads, each written by one item.
 * stats (HOST, 4 values): items, the largest rows of a system, group-pair
 * visits, 8-byte entries of all rows.  GENGA_ERR_CAPACITY: no plan fits;
 * GENGA_ERR_INVALID_ARG: bad arguments or a check failed. */
genga_status genga_mutual_plan_check(int32_t nsys, const int32_t *n, int32_t cw, int32_t npg, int32_t ctas,
                                     int64_t *stats);

/* Name of the most recent CUDA runtime error (cudaGetErrorName) that an
 * entry point called from this thread turned into GENGA_ERR_CUDA, or
 * "cudaSuccess" if none has; a static string. */
const char *genga_last_cuda_error(void);

/* Failure-detection test hook for the bounded waits of the pipelined passes
 * (the FP32 passes and the mutual FP64 pass; every mbarrier wait of a pass
 * gives up after a time limit, sets GENGA_ERR_TIMEOUT in the sticky status
 * and returns, so a stalled pipeline ends the kernel instead of hanging the
 * GPU).  wait_ns_log2 > 0 sets that
 * limit to 2^wait_ns_log2 ns (0: the default of 2 s); hold != 0 makes each
 * CTA's producer warp return before it fills its first ring slot, without
 * issuing any copy, so that the consumers' waits run out and the next
 * genga_get_status returns GENGA_ERR_TIMEOUT; the context stays usable.  Both
 * are off by default and stay set until changed.  wait_ns_log2 outside
 * [0, 40]: GENGA_ERR_INVALID_ARG. */
genga_status genga_set_test_waits(genga_ctx *ctx, int32_t wait_ns_log2, int32_t hold);

/* Step graphs: genga_step and genga_step_batched capture a CUDA graph of 4
 * steps (one rebuild of the spatial order per block) and replay it for the
 * whole 4-step blocks of a call, once the order has just been rebuilt and the
 * FP32 variant is tuned; the graph is captured again when the arrays, N, the
 * batch layout, the parameters or the variant change.  enable = 0 launches
 * every step's kernels one by one (same kernels, same order, bitwise the
 * same results).  Enabled by default; profiling also uses the step-by-step
 * path. */
genga_status genga_set_step_graphs(genga_ctx *ctx, int32_t enable);

#ifdef __cplusplus
}
#endif

#endif /* GENGA_MEASURE_H */
