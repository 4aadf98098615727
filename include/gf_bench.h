/*
 * gf_bench.h -- measurement helpers of libgf.so (no counterpart in the paper).
 *
 * The ray kernels are bound by the FP64 (or FP32) non-tensor pipes, whose
 * peaks a copy-bandwidth or tensor-GEMM measurement does not give; these
 * helpers measure them on the current device with independent FMA chains.
 */
#ifndef GF_BENCH_H
#define GF_BENCH_H

#include <stdint.h>

#include "gf.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * gf_bench_fma_peak -- time a kernel of independent fused multiply-add chains
 * (8 per thread, `iters` iterations, 2 flops each) over blocks_per_sm x SM
 * count blocks of 256 threads, in double (GF_F64) or float (GF_F32).
 * Synchronous.  out_tflops: achieved TFLOP/s; out_ms: kernel time (CUDA events).
 * Allocates and frees one small device buffer.  Errors: GF_ERR_INVALID_ARG
 * (iters <= 0, blocks_per_sm <= 0, NULL outputs), GF_ERR_CUDA, GF_ERR_OOM.
 */
gf_status gf_bench_fma_peak(gf_precision prec, int64_t iters, int32_t blocks_per_sm,
                            double *out_tflops, double *out_ms);

/*
 * gf_bench_set_counters -- from the next launch on, kernels add their work
 * to device unsigned 64-bit words owned by the caller; NULL turns counting
 * off.  gf_trace_rk4 (two words): counters[0]
 * right-hand-side evaluations, counters[1] blob terms actually evaluated
 * (not skipped as negligible).  gf_trace_adjoint and gf_trace_adjoint_static
 * (four words): counters[0] evaluations of the forward recomputation,
 * counters[1] their blob terms, counters[2] blob terms of the reverse sweep,
 * counters[3] recomputed segment-end states that differ in any bit from the
 * next checkpoint of the forward trace (0 when the recomputation reproduces
 * the forward trace).  The setting is process-wide and not thread-safe (a
 * measurement aid).
 * Errors: GF_ERR_INVALID_ARG (not device memory).
 */
gf_status gf_bench_set_counters(unsigned long long *counters);

/*
 * gf_bench_exp -- evaluate the library's table-driven base-2 exponential 2^a
 * (used for every Gaussian-blob term of the FP64 evaluator, whose rows carry
 * the exponent in base 2; defined for a <= 0, returning 0 for a <= -1021),
 * in the form that uses no FP64 operation, and CUDA's exp2 on n device
 * doubles `in`, writing out_lib and out_cuda (device, n each), so that tests
 * can bound its error.  Stream-ordered on `stream`.
 * Errors: GF_ERR_INVALID_ARG (n < 0, non-device pointers), GF_ERR_CUDA.
 */
gf_status gf_bench_exp(const double *in, double *out_lib, double *out_cuda, int64_t n, void *stream);

/*
 * gf_bench_exp_fp -- the same exponential in its other form (the table
 * product as one FP64 fused multiply-add, for kernels whose FP32 and integer
 * pipes are busy), on n device doubles `in`, writing `out` (device); it must
 * return gf_bench_exp's bits exactly.  Errors: GF_ERR_INVALID_ARG, GF_ERR_CUDA.
 */
gf_status gf_bench_exp_fp(const double *in, double *out, int64_t n, void *stream);

/*
 * gf_bench_blob_gauss -- evaluate the Gaussian of the FP64 evaluator's blob
 * terms, G = 2^(-(u0^2 + u1^2 + u2^2)), with |u|^2 summed exactly in integer
 * fixed point, for n points u (device, [3][n] structure of arrays), in both
 * forms of the table product: out_int (no FP64 operation) and out_fp (one
 * FP64 FMA), device, n each; the two must be the same bits.  A negligible
 * term (|u|^2 >= 58.5 or some |u_i| >= 8) gives +0, a non-finite u a NaN.
 * Stream-ordered on `stream`.
 * Errors: GF_ERR_INVALID_ARG (n < 0, non-device pointers), GF_ERR_CUDA.
 */
gf_status gf_bench_blob_gauss(const double *u, double *out_int, double *out_fp, int64_t n, void *stream);

/*
 * gf_bench_exp_df -- evaluate the double-float base-2 exponential 2^a of the
 * GF_F64X blob evaluator (defined for -63 < a <= 0) on n device doubles
 * (each first split into a float pair), writing hi + lo as doubles to `out`
 * (device).  Errors: GF_ERR_INVALID_ARG, GF_ERR_CUDA.
 */
gf_status gf_bench_exp_df(const double *in, double *out, int64_t n, void *stream);

/*
 * gf_bench_recip -- evaluate the FP64 evaluator's reciprocal of n^2 (an FP32
 * seed refined by one cubic Newton step; out_recip[i] = 1/in[i] for in[i] > 0,
 * 0 otherwise) and its double -> float truncation of positions (out_narrow)
 * on n device doubles `in`, so that tests can bound their errors.
 * Stream-ordered on `stream`.  Errors: GF_ERR_INVALID_ARG (n < 0, non-device
 * pointers), GF_ERR_CUDA.
 */
gf_status gf_bench_recip(const double *in, double *out_recip, float *out_narrow, int64_t n, void *stream);

/*
 * gf_fault_inject -- failure testing without a device fault (the paper has no
 * counterpart).  After gf_fault_inject(n) with n >= 1, the n-th CUDA call that
 * the library checks from then on (allocations, copies, launches, graph
 * capture and instantiation, pointer queries), counted across all entry
 * points and threads, reports GF_ERR_CUDA with a message containing
 * "injected fault", although the call itself ran and succeeded; its entry
 * point then takes its ordinary error path, which must release what it took
 * and leave every object and stream usable.  Fires once; n <= 0 disarms.
 * Host only: nothing is enqueued and the device is not touched.  Always GF_OK.
 */
gf_status gf_fault_inject(int64_t n);

/*
 * gf_bench_live_allocations -- the number of device allocations the library
 * holds now (media, batches and their caches, scratch of calls in progress);
 * their total size in bytes is written to *bytes when bytes is not NULL.
 * Host only.  Never fails.
 */
int64_t gf_bench_live_allocations(size_t *bytes);

#ifdef __cplusplus
}
#endif

#endif /* GF_BENCH_H */
