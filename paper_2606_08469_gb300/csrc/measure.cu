// Measurement microbenchmarks (include/octa_measure.h): the FP32 FMA peak
// against which the FP32 decoder engine's roofline is reported, and the
// cost of one tcgen05.mma of the decoder's shapes.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "octa_internal.h"
#include "octa_measure.h"
#include "octaoctree.h"
#include "tc_ptx.cuh"

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

// One CTA: `issuers` threads (lane 0 of warps 0 and 4), each with its own
// operand tiles (canonical K-major, no swizzle, pseudo-random BF16 values),
// mbarrier and n tensor-memory columns, issue k_steps MMAs (M = 128, N = n,
// K = 16 each, the descriptors advancing along K) and commit, `reps` times;
// issuer 0's issue and issue-to-completion cycles are summed over reps 1..
// (rep 0 warms up).  Each wait is bounded (100 ms); the loops have fixed
// trip counts; whole warps take each branch.
constexpr int kMmaMaxK = 128, kMmaMaxN = 256;
constexpr int kMmaABytes = 128 * kMmaMaxK * 2, kMmaBBytes = kMmaMaxN * kMmaMaxK * 2;
constexpr int kMmaGroupBytes = kMmaABytes + kMmaBBytes;  // 96 KB
constexpr int kMmaSmem = 2 * kMmaGroupBytes + 64;

__global__ void __launch_bounds__(256, 1)
    mma_probe_kernel(long long* out, int n, int k_steps, int reps, int issuers) {
  using namespace tc;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * kMmaGroupBytes);
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + 2 * kMmaGroupBytes + 16);
  const int kdim = 16 * k_steps;
  const int elems = (128 + n) * kdim;  // per group: A then B
  for (int g = 0; g < issuers; ++g)
    for (int i = threadIdx.x; i < elems; i += blockDim.x) {
      uint32_t h = (static_cast<uint32_t>(i) + 1u + 7919u * g) * 2654435761u;
      h ^= h >> 13;
      reinterpret_cast<__nv_bfloat16*>(smem + g * kMmaGroupBytes)[i] =
          __float2bfloat16_rn(static_cast<float>(h & 0xFFFFu) / 65536.f - 0.5f);
    }
  if (threadIdx.x == 0) {
    mbar_init(smem_addr(bars), 1);
    mbar_init(smem_addr(bars + 1), 1);
  }
  if (threadIdx.x < 32) {
    tmem_alloc(smem_addr(slot), 512);
    tmem_relinquish();
  }
  fence_proxy_async();
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem = *slot;
  const int warp = threadIdx.x >> 5, g = warp / 4;
  const bool issuer_warp = (warp == 0) || (warp == 4 && issuers == 2);
  long long t_issue = 0, t_done = 0;
  bool ok_all = true;
  if (issuer_warp) {
    const bool issuer = (threadIdx.x & 31) == 0;
    const uint32_t mbar = smem_addr(bars + g);
    const uint32_t a_sa = smem_addr(smem + g * kMmaGroupBytes);
    const uint32_t b_sa = a_sa + static_cast<uint32_t>(128 * kdim * 2);
    const uint32_t d = tmem + static_cast<uint32_t>(g * kMmaMaxN);
    const uint32_t idesc = idesc_bf16(128, n);
    uint32_t phase = 0;
    for (int r = 0; r < reps; ++r) {
      long long t0 = clock64(), t1 = t0;
      if (issuer) {
        tc_fence_after_sync();
        for (int k = 0; k < k_steps; ++k)
          mma_bf16(d, kmajor_desc(a_sa, 16 * k, kdim), kmajor_desc(b_sa, 16 * k, kdim), idesc,
                   k > 0 ? 1u : 0u);
        mma_commit(mbar);
        t1 = clock64();
      }
      __syncwarp();
      bool ok = true;
      if (issuer) ok = mbar_wait_bounded(mbar, phase, 100000000ull);
      const long long t2 = clock64();
      phase ^= 1u;
      ok_all = ok_all && ok;
      if (issuer && g == 0 && r > 0) {
        t_issue += t1 - t0;
        t_done += t2 - t0;
      }
      tc_fence_before_sync();
      __syncwarp();
    }
  }
  const int all_ok = __syncthreads_and(ok_all ? 1 : 0);
  tc_fence_after_sync();
  if (threadIdx.x < 32) tmem_dealloc(tmem, 512);
  if (threadIdx.x == 0) {
    out[0] = t_issue;
    out[1] = t_done;
    out[2] = all_ok;
  }
}

}  // namespace
}  // namespace octa

extern "C" int octa_measure_mma(int64_t* out, int32_t n, int32_t k_steps, int32_t reps,
                                int32_t issuers, void* stream) {
  using namespace octa;
  clear_error();
  if (!out) return fail(OCTA_EINVAL, "NULL out");
  if (n < 16 || n > kMmaMaxN || n % 16 != 0)
    return fail(OCTA_EINVAL, "n must be a multiple of 16 in [16, %d]", kMmaMaxN);
  if (k_steps < 1 || 16 * k_steps > kMmaMaxK)
    return fail(OCTA_EINVAL, "k_steps must be in [1, %d]", kMmaMaxK / 16);
  if (reps < 2 || reps > 10000) return fail(OCTA_EINVAL, "reps must be in [2, 10000]");
  if (issuers < 1 || issuers > 2) return fail(OCTA_EINVAL, "issuers must be 1 or 2");
  cudaError_t e = cudaFuncSetAttribute(mma_probe_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kMmaSmem);
  if (e != cudaSuccess) return fail(OCTA_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  mma_probe_kernel<<<1, 256, kMmaSmem, st>>>(reinterpret_cast<long long*>(out), n, k_steps, reps,
                                             issuers);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(OCTA_ECUDA, "mma probe launch: %s", cudaGetErrorString(e));
  return OCTA_OK;
}

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
