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

// ---------------------------------------------------------------------------
// g_psi's backward (FP32, CUDA cores): the gradients of sum_q c_q d_q
// ---------------------------------------------------------------------------
// A persistent CTA of 128 threads takes tiles of 128 queries.  Phase A, one
// thread per query: recompute the input row (hash features, omega_r), the
// hidden layers a1 = relu(W1 in), a2 = relu(W2 a1) and d = exp(W3 a2), then
// delta3 = c d (the derivative of exp is exp), delta2 = delta3 W3 * 1[a2 > 0],
// delta1 = (W2^T delta2) * 1[a1 > 0] and the input gradient W1^T delta1,
// whose hash columns are scattered into the cell's 8 vertices of each level
// with the trilinear weights (float2 atomics).  The rows in, a1, a2, delta1,
// delta2 and delta3 of the tile stay in shared memory, feature-major.  Phase
// B, all threads: dW3 += sum_q delta3 a2, dW2 += sum_q delta2 a1^T and
// dW1 += sum_q delta1 in^T over the tile, kept in registers across the CTA's
// tiles and added to the gradient once at the end.
constexpr int kBwdThreads = 128;
constexpr int kBQ = 128;             // queries per tile
constexpr int kLDQ = kBQ + 4;        // row stride of the tile rows (floats)
constexpr int kW1Half = kW1Row / 2;  // W1 columns per thread in phase B

struct PredBwdSmem {
  static constexpr size_t W1 = 0;
  static constexpr size_t W2 = W1 + sizeof(float) * kH * kW1Row;
  static constexpr size_t W3 = W2 + sizeof(float) * kH * kH;
  static constexpr size_t IN = W3 + sizeof(float) * kH;
  static constexpr size_t A1 = IN + sizeof(float) * kW1Row * kLDQ;
  static constexpr size_t A2 = A1 + sizeof(float) * kH * kLDQ;
  static constexpr size_t D2 = A2 + sizeof(float) * kH * kLDQ;
  static constexpr size_t D1 = D2 + sizeof(float) * kH * kLDQ;
  static constexpr size_t D3 = D1 + sizeof(float) * kH * kLDQ;
  static constexpr size_t BYTES = D3 + sizeof(float) * kLDQ;
};
static_assert(PredBwdSmem::BYTES <= 227 * 1024, "g_psi backward shared memory");

struct PredBwdParams {
  PredParams p;
  const float* d_disp;
  float* d_table;
  float* d_weights;
  int64_t n_tiles;
};

__global__ void __launch_bounds__(kBwdThreads, 1) disparity_bwd_kernel(
    const __grid_constant__ PredBwdParams bp) {
  const PredParams& p = bp.p;
  extern __shared__ __align__(16) uint8_t sm[];
  float* w1 = reinterpret_cast<float*>(sm + PredBwdSmem::W1);
  float* w2 = reinterpret_cast<float*>(sm + PredBwdSmem::W2);
  float* w3 = reinterpret_cast<float*>(sm + PredBwdSmem::W3);
  float* in_sm = reinterpret_cast<float*>(sm + PredBwdSmem::IN);
  float* a1_sm = reinterpret_cast<float*>(sm + PredBwdSmem::A1);
  float* a2_sm = reinterpret_cast<float*>(sm + PredBwdSmem::A2);
  float* d2_sm = reinterpret_cast<float*>(sm + PredBwdSmem::D2);
  float* d1_sm = reinterpret_cast<float*>(sm + PredBwdSmem::D1);
  float* d3_sm = reinterpret_cast<float*>(sm + PredBwdSmem::D3);
  const int in_w = 2 * p.levels + 3;
  const int t = threadIdx.x;
  for (int i = t; i < kH * kW1Row; i += kBwdThreads) {
    const int o = i / kW1Row, c = i % kW1Row;
    w1[i] = c < in_w ? p.weights[o * in_w + c] : 0.f;
  }
  for (int i = t; i < kH * kH; i += kBwdThreads) w2[i] = p.weights[kH * in_w + i];
  for (int i = t; i < kH; i += kBwdThreads) w3[i] = p.weights[kH * in_w + kH * kH + i];
  // phase B's weight-gradient accumulators: row ob of dW2 (columns
  // cb .. cb + 31) and of dW1 (columns c1 .. c1 + kW1Half - 1); t < 64: dW3[t]
  const int ob = t >> 1, cb = (t & 1) * 32, c1 = (t & 1) * kW1Half;
  float g2[32], g1[kW1Half], g3 = 0.f;
#pragma unroll
  for (int i = 0; i < 32; ++i) g2[i] = 0.f;
#pragma unroll
  for (int i = 0; i < kW1Half; ++i) g1[i] = 0.f;
  __syncthreads();

  for (int64_t tile = blockIdx.x; tile < bp.n_tiles; tile += gridDim.x) {
    const int64_t q = tile * kBQ + t;
    const bool valid = q < p.n;
    // ---- phase A: one thread per query
    float in[kW1Row];
#pragma unroll
    for (int c = 0; c < kW1Row; ++c) in[c] = 0.f;
    float xs[3] = {0.f, 0.f, 0.f};
    if (valid) {
      xs[0] = clamp01(p.x[3 * q]);
      xs[1] = clamp01(p.x[3 * q + 1]);
      xs[2] = clamp01(p.x[3 * q + 2]);
#pragma unroll
      for (int l = 0; l < OCTA_PRED_MAX_LEVELS; ++l) {
        if (l >= p.levels) break;
        const float2* tab = reinterpret_cast<const float2*>(p.table) + size_t(l) * (p.tmask + 1u);
        const float2 e = hash_level(tab, xs, p.res[l], p.dense[l] != 0, p.tmask);
        in[2 * l] = e.x;
        in[2 * l + 1] = e.y;
      }
      const float w0[3] = {p.omega[3 * q], p.omega[3 * q + 1], p.omega[3 * q + 2]};
      const float n0[3] = {p.normal[3 * q], p.normal[3 * q + 1], p.normal[3 * q + 2]};
      float wr[3];
      reflect_f32_rn(w0, n0, wr);
#pragma unroll
      for (int l = 0; l <= OCTA_PRED_MAX_LEVELS; ++l)
        if (l == p.levels) {
          in[2 * l] = wr[0];
          in[2 * l + 1] = wr[1];
          in[2 * l + 2] = wr[2];
        }
    }
    __syncthreads();  // the previous tile's phase B is done with the rows
#pragma unroll
    for (int c = 0; c < kW1Row; ++c) in_sm[c * kLDQ + t] = in[c];
    float a1[kH];
#pragma unroll
    for (int o = 0; o < kH; o += 4) {
      float s4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int c = 0; c < kW1Row / 4; ++c) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float4 w = reinterpret_cast<const float4*>(w1 + (o + r) * kW1Row)[c];
          s4[r] = fmaf(w.x, in[4 * c], s4[r]);
          s4[r] = fmaf(w.y, in[4 * c + 1], s4[r]);
          s4[r] = fmaf(w.z, in[4 * c + 2], s4[r]);
          s4[r] = fmaf(w.w, in[4 * c + 3], s4[r]);
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        a1[o + r] = fmaxf(s4[r], 0.f);
        a1_sm[(o + r) * kLDQ + t] = a1[o + r];
      }
    }
    float z3 = 0.f;
#pragma unroll 1
    for (int o = 0; o < kH; o += 4) {
      float s4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int c = 0; c < kH / 4; ++c) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float4 w = reinterpret_cast<const float4*>(w2 + (o + r) * kH)[c];
          s4[r] = fmaf(w.x, a1[4 * c], s4[r]);
          s4[r] = fmaf(w.y, a1[4 * c + 1], s4[r]);
          s4[r] = fmaf(w.z, a1[4 * c + 2], s4[r]);
          s4[r] = fmaf(w.w, a1[4 * c + 3], s4[r]);
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float a = fmaxf(s4[r], 0.f);
        a2_sm[(o + r) * kLDQ + t] = a;
        z3 = fmaf(w3[o + r], a, z3);
      }
    }
    const float delta3 = valid ? bp.d_disp[q] * expf(z3) : 0.f;
    d3_sm[t] = delta3;
    // delta2 (registers, reusing a1's storage pattern) and its row
    float d2[kH];
#pragma unroll
    for (int o = 0; o < kH; ++o) {
      d2[o] = a2_sm[o * kLDQ + t] > 0.f ? delta3 * w3[o] : 0.f;
      d2_sm[o * kLDQ + t] = d2[o];
    }
    // delta1 = (W2^T delta2) * 1[a1 > 0]
    float d1[kH];
#pragma unroll
    for (int c = 0; c < kH; c += 4) {
      float s4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int o = 0; o < kH; ++o) {
        const float4 w = reinterpret_cast<const float4*>(w2 + o * kH)[c / 4];
        s4[0] = fmaf(w.x, d2[o], s4[0]);
        s4[1] = fmaf(w.y, d2[o], s4[1]);
        s4[2] = fmaf(w.z, d2[o], s4[2]);
        s4[3] = fmaf(w.w, d2[o], s4[3]);
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        d1[c + r] = a1[c + r] > 0.f ? s4[r] : 0.f;
        d1_sm[(c + r) * kLDQ + t] = d1[c + r];
      }
    }
    // the input gradient's hash columns, scattered level by level
    if (valid) {
#pragma unroll 1
      for (int l = 0; l < p.levels; ++l) {
        float ga = 0.f, gb = 0.f;
#pragma unroll
        for (int o = 0; o < kH; ++o) {
          const float2 w = *reinterpret_cast<const float2*>(w1 + o * kW1Row + 2 * l);
          ga = fmaf(w.x, d1[o], ga);
          gb = fmaf(w.y, d1[o], gb);
        }
        float2* dtab = reinterpret_cast<float2*>(bp.d_table) + size_t(l) * (p.tmask + 1u);
        hash_level_scatter(dtab, xs, p.res[l], p.dense[l] != 0, p.tmask, ga, gb);
      }
    }
    __syncthreads();
    // ---- phase B: the tile's weight gradients
#pragma unroll 1
    for (int q4 = 0; q4 < kBQ; q4 += 4) {
      const float4 dv = *reinterpret_cast<const float4*>(d2_sm + ob * kLDQ + q4);
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const float4 a = *reinterpret_cast<const float4*>(a1_sm + (cb + c) * kLDQ + q4);
        g2[c] = fmaf(dv.x, a.x, fmaf(dv.y, a.y, fmaf(dv.z, a.z, fmaf(dv.w, a.w, g2[c]))));
      }
      const float4 ev = *reinterpret_cast<const float4*>(d1_sm + ob * kLDQ + q4);
#pragma unroll
      for (int c = 0; c < kW1Half; ++c) {
        const float4 a = *reinterpret_cast<const float4*>(in_sm + (c1 + c) * kLDQ + q4);
        g1[c] = fmaf(ev.x, a.x, fmaf(ev.y, a.y, fmaf(ev.z, a.z, fmaf(ev.w, a.w, g1[c]))));
      }
      if (t < kH) {
        const float4 dv3 = *reinterpret_cast<const float4*>(d3_sm + q4);
        const float4 a = *reinterpret_cast<const float4*>(a2_sm + t * kLDQ + q4);
        g3 = fmaf(dv3.x, a.x, fmaf(dv3.y, a.y, fmaf(dv3.z, a.z, fmaf(dv3.w, a.w, g3))));
      }
    }
  }
  // the CTA's sums into the weight gradient (layout of the weights)
  float* dW1 = bp.d_weights;
  float* dW2 = dW1 + kH * in_w;
  float* dW3 = dW2 + kH * kH;
#pragma unroll
  for (int c = 0; c < 32; ++c) atomicAdd(dW2 + ob * kH + cb + c, g2[c]);
#pragma unroll
  for (int c = 0; c < kW1Half; ++c)
    if (c1 + c < in_w) atomicAdd(dW1 + ob * in_w + c1 + c, g1[c]);
  if (t < kH) atomicAdd(dW3 + t, g3);
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

extern "C" int octa_disparity_bwd(const octa_predictor* pred, const octa_queries* q,
                                  const float* d_disp, float* d_table, float* d_weights,
                                  void* stream) {
  clear_error();
  if (!pred || !q) return fail(OCTA_EINVAL, "pred and q must be non-NULL");
  if (pred->levels < 1 || pred->levels > OCTA_PRED_MAX_LEVELS)
    return fail(OCTA_ERANGE, "predictor levels %d outside [1, %d]", pred->levels,
                OCTA_PRED_MAX_LEVELS);
  if (pred->log2_T < 4 || pred->log2_T > 24)
    return fail(OCTA_ERANGE, "predictor log2_T %d outside [4, 24]", pred->log2_T);
  if (!pred->table || !pred->weights) return fail(OCTA_EINVAL, "NULL predictor table or weights");
  if (q->n < 0) return fail(OCTA_EINVAL, "negative query count");
  if (q->n == 0) return OCTA_OK;
  if (!q->x || !q->omega || !q->normal || !d_disp || !d_table || !d_weights)
    return fail(OCTA_EINVAL, "x, omega, normal, d_disp, d_table and d_weights must be non-NULL");
  if ((reinterpret_cast<uintptr_t>(pred->table) | reinterpret_cast<uintptr_t>(d_table)) & 7u)
    return fail(OCTA_EINVAL, "predictor table and its gradient must be 8-byte aligned");
  if (pred->weights_bf16) {  // the MLP on the tensor cores
    if (pred->levels > 14)
      return fail(OCTA_ERANGE, "the tensor-core predictor takes at most 14 levels");
    for (int l = 0; l < pred->levels; ++l)
      if (pred->res[l] < 1 || pred->res[l] > 65535)
        return fail(OCTA_ERANGE, "predictor res[%d] = %d outside [1, 65535]", l, pred->res[l]);
    return tc::predictor_bwd(pred, q, d_disp, d_table, d_weights, static_cast<cudaStream_t>(stream));
  }
  PredBwdParams bp{};
  PredParams& p = bp.p;
  p.table = pred->table;
  p.weights = pred->weights;
  p.x = q->x;
  p.omega = q->omega;
  p.normal = q->normal;
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
  bp.d_disp = d_disp;
  bp.d_table = d_table;
  bp.d_weights = d_weights;
  bp.n_tiles = (q->n + kBQ - 1) / kBQ;
  const size_t smem = PredBwdSmem::BYTES;
  cudaError_t e = cudaFuncSetAttribute(disparity_bwd_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return fail(OCTA_ECUDA, "octa_disparity_bwd: %s", cudaGetErrorString(e));
  const int blocks = static_cast<int>(std::min<int64_t>(bp.n_tiles, sm_count_here()));
  disparity_bwd_kernel<<<blocks, kBwdThreads, smem, static_cast<cudaStream_t>(stream)>>>(bp);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(OCTA_ECUDA, "octa_disparity_bwd: %s", cudaGetErrorString(e));
  return OCTA_OK;
}
