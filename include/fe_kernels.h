/*
 * fe_kernels.h -- single hot-path steps of the expansion exposed through the C
 * ABI, so each kernel can be checked on its own against the CPU oracle.
 * They run on the context's stream and return when the result is ready.
 * All pointers are DEVICE pointers on the context's device; the caller owns
 * them.  Matrices are row-major with the given leading dimension.  Errors:
 * FE_EINVAL for bad sizes/pointers, FE_ENOMEM, FE_ECUDA, FE_ETIMEOUT.
 */
#ifndef FE_KERNELS_H
#define FE_KERNELS_H

#include <stdint.h>

#include "fe.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Gershgorin bounds of a symmetric H (Sec. II-C: spectral bounds eps_1,
 * eps_N of H are needed to scale it into [0, 1]).
 * out4 (HOST, 4 doubles): [0] = min_i (H_ii - sum_{j!=i} |H_ij|),
 * [1] = max_i (H_ii + sum_{j!=i} |H_ij|), [2] = tr H, [3] = 1.0 if H holds a
 * NaN/Inf else 0.0. */
FE_API int fe_k_gershgorin(fe_ctx *ctx, const double *H, int64_t n, int64_t ld, double *out4);

/* The Gershgorin bounds of fe_k_gershgorin without a context, through a path
 * that allocates nothing.  No counterpart in the paper: it serves callers that
 * cannot allocate device memory where they need the bounds (a framework whose
 * caching pool owns the GPU's memory, or a latency-critical loop that must not
 * hit the device-wide synchronisation of cudaMalloc / cudaFree).
 * H and out4 are DEVICE pointers on the current device; out4 receives the
 * same 4 doubles as fe_k_gershgorin.  The work is queued on cuda_stream (NULL:
 * the legacy default stream) and the call returns without waiting; out4 is
 * ready when that stream reaches this point.  Per-row scratch lives in one
 * fixed device array of 32768 rows (1 MiB) per device: n > 32768 returns
 * FE_EINVAL.  All calls on a device share that array, so calls that overlap
 * in time race; calls ordered on one stream do not.  The first call on a
 * device (with it current) looks up the array's address, which may load the
 * module; make that first call before any stream capture.
 * Errors: FE_EINVAL (NULL pointers, n < 1, ld < n, n too large), FE_ECUDA. */
FE_API int fe_k_gershgorin_noalloc(const double *H, int64_t n, int64_t ld, double *out4,
                                   void *cuda_stream);

/* C = Y * Y for a symmetric FP32 matrix Y, computed by the tensor-core kernel
 * of the SP2 step (Sec. II-B1 Eq. (1); the product is the dominant cost,
 * Sec. III-B): Y is scaled by a power of two s with s * bound <= 2^14 and
 * split into FP16 slices (nslices = 1: fp16(sY); nslices = 2: hi + lo), the
 * slice products are accumulated in FP32 in tensor memory, and only the upper
 * triangle of 128x128 blocks is computed and mirrored.  bound must satisfy
 * |Y_ij| <= bound.  C (FP32, ldc) is written whole and exactly symmetric. */
FE_API int fe_k_sym_square(fe_ctx *ctx, const float *Y, int64_t n, int64_t ldy, float *C, int64_t ldc,
                    int nslices, double bound);

/* P = X * X for a symmetric FP64 matrix X with ||X||_2 <= 2, computed by the
 * FP64-accurate tensor-core kernel of the polishing steps (Sec. III-A: the
 * last SP2 iterations run in FP64): X/4 is split into 7 balanced base-256
 * digit matrices held exactly in FP16, the 28 digit products of levels
 * a + c <= 6 are summed exactly in FP32 tensor memory per K block of 128 and
 * drained into int64 fixed point (unit 2^-60 of P).  Error of each entry
 * about n^(1/2) 2^-64 beyond FP64 rounding.  P (FP64, ldp) is written whole
 * and exactly symmetric. */
FE_API int fe_k_digit_square(fe_ctx *ctx, const double *X, int64_t n, int64_t ld, double *P, int64_t ldp);

/* Measurement hooks (no counterpart in the paper; they time the hot path).
 * fe_k_profile(ctx, 1) makes every following solve record CUDA events around
 * each tensor-core and FP64 step launch on the context's stream.
 * fe_k_profile_read fills out8 (HOST) from the last profiled solve:
 * [0] ms in tensor-core step launches that did work, [1] their count,
 * [2] ms in FP64 step launches that did work, [3] their count,
 * [4] ms of the whole solve, [5] kernels launched by the context so far,
 * [6] ms in all tensor-core step launches, [7] their count. */
FE_API int fe_k_profile(fe_ctx *ctx, int enable);
FE_API int fe_k_profile_read(fe_ctx *ctx, double *out8);
/* Per step of the last profiled solve: ms of its tensor-core step launch
 * (out, HOST, up to max_steps values; *count = values written).  Steps run in
 * phase order, so with fe_result's iters_by_phase the first iters_by_phase[0]
 * values are single-FP16 products and the next iters_by_phase[1] split ones. */
FE_API int fe_k_profile_steps(fe_ctx *ctx, double *out, int max_steps, int *count);

/* The last profiled solve's step launches summed by the kind of step
 * (measurement hook, no counterpart in the paper; first problem of the
 * batch), HOST out: ms8[k] milliseconds and n8[k] launches of kind k,
 * 1 single-FP16 tensor-core product, 2 split-FP16 product, 3 native FP64
 * product, 5 epilogue-only tensor-core step, 6 FP64-accurate digit product
 * (its digit split included), 7 second product of a polishing pair (split
 * FP16, added to the FP64 iterate); other entries 0. */
FE_API int fe_k_profile_kinds(fe_ctx *ctx, double *ms8, int *n8);

/* Test hook (no counterpart in the paper): every following solve on ctx,
 * blocking or submitted, shrinks its Lanczos estimate of the spectral bounds
 * about the interval's centre by `factor` (1 = off, the default) before the
 * estimate is certified.  A factor below 1 leaves eigenvalues of Hp outside
 * the estimate; the certificate (three logistic steps X <- 4 X (I - X) from X0
 * on the estimate, i.e. the Chebyshev polynomial T_8) must widen the bounds
 * until they contain the spectrum again (fe_result's eps_min / eps_max are the
 * bounds used).  Call it while no submitted solve is running.
 * Errors: FE_EINVAL (ctx NULL, factor outside (0, 1]). */
FE_API int fe_k_narrow_bounds(fe_ctx *ctx, double factor);

/* Failure-detection hook (no counterpart in the paper).  Every wait inside
 * the tensor-core kernels (TMA data, shared-memory stages, tensor-memory
 * hand-offs, the partner of a tile split between two CTAs) is bounded: when
 * one runs out the kernel records an error code, waits (bounded) for its own
 * copies and products in flight, frees its tensor memory and returns; the
 * control kernel then ends every problem of the run, and the call returns
 * FE_ETIMEOUT with the context still usable.  This sets the limit of those
 * waits for later solves on ctx (limit_ms, default 2000) and, with
 * fail_partner != 0, makes the second CTA of every split tile wait on a word
 * that nothing writes, so that its wait runs out: a way to exercise the
 * expiry path without any fault.  Call it while no submitted solve runs.
 * Errors: FE_EINVAL (ctx NULL, limit_ms outside (0, 60000]), FE_ECUDA. */
FE_API int fe_k_set_wait(fe_ctx *ctx, double limit_ms, int fail_partner);

/* Where the last blocking solve or batch on ctx spent its device time
 * (measurement hook, no counterpart in the paper; CUDA events, always on).
 * out4 (HOST): [0] ms of set-up (Hp staging, bounds, X0, first control step),
 * [1] ms of the step loop, [2] ms of the output kernels, [3] steps the loop
 * ran.  After fe_project / fe_rotate: [0] ms of the operand split (max and
 * FP16 slices), [1] ms of the tensor-core product (k_gemm_split), [2] ms of
 * the reduction of the K parts, [3] work units of the product.  Zeros before
 * the first call. */
FE_API int fe_k_phase_ms(fe_ctx *ctx, double *out4);

/* Tile-shape table hooks (tests; see fe_autotune in fe.h).  set: make problems
 * with n's number of 128-row panels under policy prec (an FE_PREC_* value,
 * FE_PREC_MIXED = 0 included) use tile width bn (128 or 256; 0 removes the
 * entry).  get: the width such a problem would use now (HOST out).
 * fe_k_sym_square looks its width up under FE_PREC_FP32 (two slices) or
 * FE_PREC_TRY_FP16 (one slice). */
FE_API int fe_k_set_tile_width(fe_ctx *ctx, int64_t n, uint32_t prec, int bn);
FE_API int fe_k_tile_width(fe_ctx *ctx, int64_t n, uint32_t prec, int *bn);

/* Serving counters (measurement hook, no counterpart in the paper), HOST out4:
 * [0] requests submitted, [1] requests that had to wait at least once for a
 * free part of the HBM budget (at submission or at a later admission pass),
 * [2] the largest number of requests waiting at once, [3] the largest
 * number of requests on the device at once; since fe_create or the last
 * call with reset != 0. */
FE_API int fe_k_serve_stats(fe_ctx *ctx, int64_t *out4, int reset);

/* Number of kernels this context has launched since fe_create (HOST out). */
FE_API int fe_k_launch_count(fe_ctx *ctx, int64_t *out);

/* Per-step record of problem `index` of the last solve or batch (measurement
 * hook, no counterpart in the paper).  out (HOST) receives up to max_rows rows
 * of 6 doubles: phase (0 single FP16, 1 split FP16, 2 FP64-accurate), kind of
 * the product that produced the iterate (0 none, 1 single, 2 split, 3 FP64,
 * 4 double-float), tr X - N_e, tr X - ||X||_F^2, ||X^2 - X||_F of that
 * product's input (-1 before the first product), RelTr (-1 at step 0).
 * *rows = rows written. */
FE_API int fe_k_history(fe_ctx *ctx, int index, double *out, int max_rows, int *rows);

#ifdef __cplusplus
}
#endif
#endif /* FE_KERNELS_H */
