/*
 * gf_bench.h -- measurement helpers of libgf.so (no counterpart in the paper).
 *
 * The ray kernels are bound by the FP64 (or FP32) non-tensor pipes, whose
 * peaks are not in the measured peak table; these helpers measure
 * them on the current device with independent FMA chains.
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

#ifdef __cplusplus
}
#endif

#endif /* GF_BENCH_H */
