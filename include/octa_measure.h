/*
 * octa_measure.h -- measurement utilities of the OctaOctree library (no
 * counterpart in the paper): a microbenchmark that gives the FP32 CUDA-core
 * kernels (the FP32 decoder engine) a measured peak to report their
 * roofline against, in place of a figure derived from unit counts.
 */
#ifndef OCTA_MEASURE_H
#define OCTA_MEASURE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* octa_measure_ffma -- enqueue one launch of `blocks` x `threads` threads,
 * each running `iters` iterations of 16 independent binary32 fused
 * multiply-add chains: packed == 0 as scalar FMAs (fma.rn.f32), packed != 0
 * as 8 chains of the packed pair form (fma.rn.f32x2, two FMAs per
 * instruction).  Either way one launch performs
 * blocks * threads * iters * 16 FMAs = twice that many flops; time it with
 * CUDA events on `stream` (NULL: the legacy default stream).  out: device
 * float32 [blocks * threads], one result per thread, written so that the
 * compiler cannot drop the chains (its values have no meaning).
 * Errors: OCTA_EINVAL (NULL out, blocks / threads / iters < 1, threads >
 * 1024), OCTA_ECUDA (launch error).                                       */
int octa_measure_ffma(float* out, int32_t blocks, int32_t threads, int32_t iters, int32_t packed,
                      void* stream);

#ifdef __cplusplus
}
#endif
#endif /* OCTA_MEASURE_H */
