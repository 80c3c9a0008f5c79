// FP32 FMA throughput microbenchmark (include/octa_measure.h): the measured
// peak against which the FP32 decoder engine's roofline is reported.
#include <cuda_runtime.h>

#include "octa_internal.h"
#include "octa_measure.h"
#include "octaoctree.h"

namespace octa {
namespace {

constexpr int kChains = 16;

// Scalar form: 16 independent chains acc = acc * a + b per iteration.
__global__ void ffma_scalar_kernel(float* out, int iters, float a, float b) {
  float acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = static_cast<float>(threadIdx.x + c);
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = fmaf(acc[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Packed form: 8 chains of fma.rn.f32x2 (two FMAs each) per iteration.
__global__ void ffma_packed_kernel(float* out, int iters, float a, float b) {
  unsigned long long acc[kChains / 2];
  unsigned long long A, B;
  asm("mov.b64 %0, {%1, %1};" : "=l"(A) : "f"(a));
  asm("mov.b64 %0, {%1, %1};" : "=l"(B) : "f"(b));
#pragma unroll
  for (int c = 0; c < kChains / 2; ++c) {
    const float lo = static_cast<float>(threadIdx.x + 2 * c), hi = lo + 1.f;
    asm("mov.b64 %0, {%1, %2};" : "=l"(acc[c]) : "f"(lo), "f"(hi));
  }
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c)
      asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(acc[c]) : "l"(A), "l"(B));
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains / 2; ++c) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(acc[c]));
    s += lo + hi;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace octa

extern "C" int octa_measure_ffma(float* out, int32_t blocks, int32_t threads, int32_t iters,
                                 int32_t packed, void* stream) {
  using namespace octa;
  clear_error();
  if (!out) return fail(OCTA_EINVAL, "NULL out");
  if (blocks < 1 || threads < 1 || threads > 1024 || iters < 1)
    return fail(OCTA_EINVAL, "blocks, threads (<= 1024) and iters must be >= 1");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // a = 1 - 2^-12, b = 2^-10: the chains stay finite and normal for any count
  if (packed)
    ffma_packed_kernel<<<blocks, threads, 0, st>>>(out, iters, 0.999755859375f, 0.0009765625f);
  else
    ffma_scalar_kernel<<<blocks, threads, 0, st>>>(out, iters, 0.999755859375f, 0.0009765625f);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(OCTA_ECUDA, "ffma probe launch: %s", cudaGetErrorString(e));
  return OCTA_OK;
}
