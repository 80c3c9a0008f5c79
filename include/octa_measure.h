/*
 * octa_measure.h -- measurement utilities of the OctaOctree library (no
 * counterpart in the paper): a microbenchmark that gives the FP32 CUDA-core
 * kernels (the FP32 decoder engine) a measured peak to report their
 * roofline against, in place of a figure derived from unit counts, and one
 * that measures the cost of a tensor-core MMA of the decoders' shapes (the
 * instruction rate that bounds the tensor-core training pass).
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

/* octa_measure_mma -- enqueue one single-CTA launch that times the 5th-
 * generation tensor-core MMA of the decoders (tcgen05.mma kind::f16: BF16
 * operands in canonical K-major shared-memory tiles without swizzle, FP32
 * accumulator in tensor memory, M = 128 rows, N = n columns, K = 16 per
 * instruction).  `issuers` threads (1 or 2, each with its own tiles,
 * accumulator columns and mbarrier) each issue k_steps MMAs along K
 * (descriptors advancing 16 elements per step) and commit, `reps` times;
 * the operands are pseudo-random BF16 values.  out: device int64[3],
 * written when the launch completes: [0] the first issuer's cycles
 * (clock64) spent issuing, [1] its cycles from the first issue to the
 * commit's completion, both summed over reps - 1 repetitions (the first is
 * a warm-up), [2] 1, or 0 if a completion wait ran out (100 ms bound).
 * Divide by (reps - 1) * k_steps for cycles per MMA.  n: multiple of 16 in
 * [16, 256]; k_steps in [1, 8]; reps in [2, 10000].  Uses 193 KB of shared
 * memory and 512 tensor-memory columns of one SM.
 * Errors: OCTA_EINVAL (argument out of range, NULL out), OCTA_ECUDA.     */
int octa_measure_mma(int64_t* out, int32_t n, int32_t k_steps, int32_t reps, int32_t issuers,
                     void* stream);

#ifdef __cplusplus
}
#endif
#endif /* OCTA_MEASURE_H */
