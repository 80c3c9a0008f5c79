// The disparity predictor g_psi of Eq. 7 (Section 3.5): a multiresolution
// hash encoding of the position and a tiny MLP on [encoding, omega_r].
#include <cuda_runtime.h>

#include <algorithm>

#include "gather.cuh"
#include "octa_internal.h"
#include "tc_path.h"

namespace octa {
namespace {

constexpr int kPredThreads = 128;
constexpr int kH = OCTA_PRED_HIDDEN;
constexpr int kMaxIn = 2 * OCTA_PRED_MAX_LEVELS + 3;  // widest MLP input
constexpr int kW1Row = (kMaxIn + 3) / 4 * 4;           // W1 row in shared memory (float4s)

struct PredParams {
  const float* table;
  const float* weights;
  const float* x;
  const float* omega;
  const float* normal;
  float* disparity;
  int64_t n;
  int32_t levels;
  uint32_t tmask;                  // T - 1
  int32_t res[OCTA_PRED_MAX_LEVELS];
  int32_t dense[OCTA_PRED_MAX_LEVELS];  // (res + 1)^3 <= T
};

// One thread per query; the MLP's weights live in shared memory with W1's
// rows padded to kW1Row columns (zeros past the encoding's width), so every
// loop has a compile-time trip count, and are read as float4 (one shared
// load per four FMAs; all threads of a warp read the same address).
__global__ void __launch_bounds__(kPredThreads, 3) disparity_kernel(const __grid_constant__ PredParams p) {
  __shared__ __align__(16) float w1[kH * kW1Row];
  __shared__ __align__(16) float w2[kH * kH];
  __shared__ __align__(16) float w3[kH];
  const int in_w = 2 * p.levels + 3;
  for (int i = threadIdx.x; i < kH * kW1Row; i += blockDim.x) {
    const int o = i / kW1Row, c = i % kW1Row;
    w1[i] = c < in_w ? p.weights[o * in_w + c] : 0.f;
  }
  for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) w2[i] = p.weights[kH * in_w + i];
  for (int i = threadIdx.x; i < kH; i += blockDim.x) w3[i] = p.weights[kH * in_w + kH * kH + i];
  __syncthreads();
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < p.n; q += stride) {
    const float xs[3] = {clamp01(p.x[3 * q]), clamp01(p.x[3 * q + 1]), clamp01(p.x[3 * q + 2])};
    float in[kW1Row];
#pragma unroll
    for (int c = 0; c < kW1Row; ++c) in[c] = 0.f;
#pragma unroll
    for (int l = 0; l < OCTA_PRED_MAX_LEVELS; ++l) {
      if (l >= p.levels) break;
      const float2* tab = reinterpret_cast<const float2*>(p.table) + size_t(l) * (p.tmask + 1u);
      const float2 e = hash_level(tab, xs, p.res[l], p.dense[l] != 0, p.tmask);
      const float s0 = e.x, s1 = e.y;
      in[2 * l] = s0;
      in[2 * l + 1] = s1;
    }
    const float w0[3] = {p.omega[3 * q], p.omega[3 * q + 1], p.omega[3 * q + 2]};
    const float n0[3] = {p.normal[3 * q], p.normal[3 * q + 1], p.normal[3 * q + 2]};
    float wr[3];
    reflect_f32_rn(w0, n0, wr);
    // omega_r follows the encoding: columns 2 L .. 2 L + 2 of W1
#pragma unroll
    for (int l = 0; l <= OCTA_PRED_MAX_LEVELS; ++l)
      if (l == p.levels) {
        in[2 * l] = wr[0];
        in[2 * l + 1] = wr[1];
        in[2 * l + 2] = wr[2];
      }
    // four outputs at a time: four independent FMA chains per thread
    float h1[kH];
#pragma unroll
    for (int o = 0; o < kH; o += 4) {
      float s[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int c = 0; c < kW1Row / 4; ++c) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float4 w = reinterpret_cast<const float4*>(w1 + (o + r) * kW1Row)[c];
          s[r] = fmaf(w.x, in[4 * c], s[r]);
          s[r] = fmaf(w.y, in[4 * c + 1], s[r]);
          s[r] = fmaf(w.z, in[4 * c + 2], s[r]);
          s[r] = fmaf(w.w, in[4 * c + 3], s[r]);
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) h1[o + r] = fmaxf(s[r], 0.f);
    }
    float z = 0.f;
#pragma unroll 1
    for (int o = 0; o < kH; o += 4) {
      float s[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int c = 0; c < kH / 4; ++c) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float4 w = reinterpret_cast<const float4*>(w2 + (o + r) * kH)[c];
          s[r] = fmaf(w.x, h1[4 * c], s[r]);
          s[r] = fmaf(w.y, h1[4 * c + 1], s[r]);
          s[r] = fmaf(w.z, h1[4 * c + 2], s[r]);
          s[r] = fmaf(w.w, h1[4 * c + 3], s[r]);
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) z = fmaf(w3[o + r], fmaxf(s[r], 0.f), z);
    }
    p.disparity[q] = expf(z);
  }
}

int sm_count_here() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 148;
}

}  // namespace
}  // namespace octa

using namespace octa;

extern "C" int octa_disparity(const octa_predictor* pred, const octa_queries* q, float* disparity,
                              void* stream) {
  clear_error();
  if (!pred || !q) return fail(OCTA_EINVAL, "pred and q must be non-NULL");
  if (pred->levels < 1 || pred->levels > OCTA_PRED_MAX_LEVELS)
    return fail(OCTA_ERANGE, "predictor levels %d outside [1, %d]", pred->levels,
                OCTA_PRED_MAX_LEVELS);
  if (pred->log2_T < 4 || pred->log2_T > 24)
    return fail(OCTA_ERANGE, "predictor log2_T %d outside [4, 24]", pred->log2_T);
  if (pred->weights_bf16 && pred->levels > 14)
    return fail(OCTA_ERANGE, "the tensor-core predictor takes at most 14 levels");
  if (!pred->table || !pred->weights) return fail(OCTA_EINVAL, "NULL predictor table or weights");
  if (reinterpret_cast<uintptr_t>(pred->table) & 7u)
    return fail(OCTA_EINVAL, "predictor table not 8-byte aligned");
  if (q->n < 0) return fail(OCTA_EINVAL, "negative query count");
  if (q->n == 0) return OCTA_OK;
  if (!q->x || !q->omega || !q->normal || !disparity)
    return fail(OCTA_EINVAL, "x, omega, normal and disparity must be non-NULL");
  if (pred->weights_bf16) {  // the MLP on the tensor cores
    for (int l = 0; l < pred->levels; ++l)
      if (pred->res[l] < 1 || pred->res[l] > 65535)
        return fail(OCTA_ERANGE, "predictor res[%d] = %d outside [1, 65535]", l, pred->res[l]);
    return tc::predictor_fwd(pred, q, disparity, static_cast<cudaStream_t>(stream));
  }
  PredParams p{};
  p.table = pred->table;
  p.weights = pred->weights;
  p.x = q->x;
  p.omega = q->omega;
  p.normal = q->normal;
  p.disparity = disparity;
  p.n = q->n;
  p.levels = pred->levels;
  const int64_t T = int64_t(1) << pred->log2_T;
  p.tmask = static_cast<uint32_t>(T - 1);
  for (int l = 0; l < pred->levels; ++l) {
    const int N = pred->res[l];
    if (N < 1 || N > 65535) return fail(OCTA_ERANGE, "predictor res[%d] = %d outside [1, 65535]", l, N);
    p.res[l] = N;
    const int64_t side = N + 1;
    p.dense[l] = side * side * side <= T ? 1 : 0;
  }
  const int64_t want = (q->n + kPredThreads - 1) / kPredThreads;
  const int blocks = static_cast<int>(std::min<int64_t>(want, 8LL * sm_count_here()));
  disparity_kernel<<<blocks, kPredThreads, 0, static_cast<cudaStream_t>(stream)>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(OCTA_ECUDA, "octa_disparity: %s", cudaGetErrorString(e));
  return OCTA_OK;
}
