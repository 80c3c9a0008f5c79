// Training-side entry points: the residual loss (Eq. 3, Eq. 14) and the Adam
// step with dynamic loss scaling.  Both reduce in FP64 (the loss value and
// the gradient norm) through per-block partials in the caller's workspace;
// the last block to finish sums the partials in a fixed order, so results are
// deterministic for a given launch shape.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "octa_device.cuh"
#include "octa_internal.h"

namespace octa {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 1024;
// workspace layout: [kMaxBlocks] doubles of partials, then the completion
// counter (uint32) and, 16 bytes after it, Adam's two bias corrections
constexpr size_t kPartialBytes = sizeof(double) * kMaxBlocks;
constexpr size_t kWorkspaceBytes = kPartialBytes + 256;

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 148;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
  return t;  // valid in thread 0
}

// Publishes this block's partial; the last block to finish sums all partials
// with every one of its threads (fixed strided order, then the fixed-order
// block reduction), so the total is deterministic for a given grid.  Returns
// true in thread 0 of the last block, which then holds the total in *total.
__device__ __forceinline__ bool last_block_total(double mine, double* partials,
                                                 unsigned* counter, double* total,
                                                 double* red) {
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = mine;
    __threadfence();
    const unsigned done = atomicAdd(counter, 1u);
    is_last = done == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double t = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += kThreads)
    t += reinterpret_cast<volatile double*>(partials)[b];
  __syncthreads();  // red[] reuse
  t = block_sum(t, red);
  if (threadIdx.x != 0) return false;
  *counter = 0;  // ready for the next call
  *total = t;
  return true;
}

// Eq. 14 per channel: T = E + w L_s, r = (L_p - T) / (L_p + T + eps), loss =
// mean r^2; gradients of S * loss with the normaliser detached.
__global__ void __launch_bounds__(kThreads) residual_loss_kernel(
    const float* __restrict__ Lp, const float* __restrict__ Ls, const float* __restrict__ E,
    const float* __restrict__ w, int64_t n3, float eps, int rhs_grad,
    const octa_scaler* __restrict__ scaler, double* loss_dev, float* __restrict__ dLp,
    float* __restrict__ dLs, double* partials, unsigned* counter) {
  __shared__ double red[kThreads / 32];
  const float S = scaler ? scaler->scale : 1.f;
  const float gscale = 2.f * S / static_cast<float>(n3);
  double acc = 0.0;
  const int64_t stride = int64_t(gridDim.x) * kThreads;
  for (int64_t i = int64_t(blockIdx.x) * kThreads + threadIdx.x; i < n3; i += stride) {
    const float lp = Lp[i], ls = Ls[i], ww = w[i];
    const float T = E[i] + ww * ls;
    const float den = lp + T + eps;
    const float r = (lp - T) / den;
    acc += double(r) * double(r);
    const float g = gscale * r / den;
    dLp[i] = g;
    if (dLs) dLs[i] = rhs_grad ? -g * ww : 0.f;
  }
  const double bsum = block_sum(acc, red);
  double total;
  if (last_block_total(bsum, partials, counter, &total, red)) *loss_dev = total / double(n3);
}

// Eq. 14 against Eq. 3's M-sample target, one warp per pair: the pair's 3M
// secondary radiances and weights are read coalesced (lane j takes elements
// j, j + 32, ... of the pair's [M][3] block), each lane sums w * L_s per
// channel in FP32 with two partial sums, and the warp reduces the three
// channel sums by shuffles; the gradients of the secondaries are written
// back by the lanes that read them.
__global__ void __launch_bounds__(kThreads) residual_loss_multi_kernel(
    const float* __restrict__ Lp, const float* __restrict__ Ls, const float* __restrict__ E,
    const float* __restrict__ w, int64_t n_pairs, int M, float eps, int rhs_grad,
    const octa_scaler* __restrict__ scaler, double* loss_dev, float* __restrict__ dLp,
    float* __restrict__ dLs, double* partials, unsigned* counter) {
  __shared__ double red[kThreads / 32];
  const float S = scaler ? scaler->scale : 1.f;
  const float gscale = 2.f * S / static_cast<float>(3 * n_pairs);
  const float invM = 1.f / static_cast<float>(M);
  const int lane = threadIdx.x & 31;
  const int64_t warps = int64_t(gridDim.x) * (kThreads / 32);
  const int per = 3 * M;  // elements of a pair
  double acc = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * (kThreads / 32) + (threadIdx.x >> 5); i < n_pairs;
       i += warps) {
    const float* ls = Ls + i * per;
    const float* ww = w + i * per;
    float s0[3] = {0.f, 0.f, 0.f}, s1[3] = {0.f, 0.f, 0.f};
    int e = lane, c = lane % 3;  // element and its channel
    bool odd = false;
    for (; e < per; e += 32, c = (c + 2) % 3) {  // 32 = 2 (mod 3)
      const float v = __ldg(ww + e) * __ldcs(ls + e);
#pragma unroll
      for (int k = 0; k < 3; ++k) {  // registers only: no indexing by c
        const float add = c == k ? v : 0.f;
        if (odd)
          s1[k] += add;
        else
          s0[k] += add;
      }
      odd = !odd;
    }
    float T[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float v = s0[k] + s1[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      T[k] = E[3 * i + k] + v * invM;
    }
    float g[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float lp = Lp[3 * i + k];
      const float den = lp + T[k] + eps;
      const float r = (lp - T[k]) / den;
      if (lane == 0) acc += double(r) * double(r);
      g[k] = gscale * r / den;
    }
    auto pick = [&](int k) { return k == 0 ? g[0] : (k == 1 ? g[1] : g[2]); };
    if (lane < 3) dLp[3 * i + lane] = pick(lane);
    if (dLs) {
      float* dls = dLs + i * per;
      c = lane % 3;
      for (e = lane; e < per; e += 32, c = (c + 2) % 3)
        dls[e] = rhs_grad ? -pick(c) * ww[e] * invM : 0.f;
    }
  }
  const double bsum = block_sum(acc, red);
  double total;
  if (last_block_total(bsum, partials, counter, &total, red))
    *loss_dev = total / double(3 * n_pairs);
}

struct AdamParams {
  octa_param_group g[OCTA_MAX_GROUPS];
  int32_t vec4[OCTA_MAX_GROUPS];  // group may use 16-byte vector accesses
  int32_t n_groups;
  float beta1, beta2, eps;
  octa_scaler* scaler;
  double* partials;
  unsigned* counter;
  float* bias_corr;  // [2]: 1 - beta1^t, 1 - beta2^t of the step being applied
};

// Pass 1: FP64 sum of squares of the unscaled gradient; the last block takes
// the skip / scale decision and advances the step count.
__global__ void __launch_bounds__(kThreads) adam_norm_kernel(const __grid_constant__ AdamParams p) {
  __shared__ double red[kThreads / 32];
  const float inv_s = 1.f / p.scaler->scale;
  double acc = 0.0;
  const int64_t stride = int64_t(gridDim.x) * kThreads;
  const int64_t first = int64_t(blockIdx.x) * kThreads + threadIdx.x;
  for (int gi = 0; gi < p.n_groups; ++gi) {
    const float* __restrict__ g = p.g[gi].grad;
    const int64_t n = p.g[gi].n;
    int64_t done = 0;
    if (p.vec4[gi]) {  // four elements per load, squared and summed in FP32
      const float4* __restrict__ g4 = reinterpret_cast<const float4*>(g);
      const int64_t n4 = n / 4;
      constexpr int UN = 4;  // loads in flight per thread
      for (int64_t i0 = first; i0 < n4; i0 += UN * stride) {
        float4 gv[UN];
#pragma unroll
        for (int u = 0; u < UN; ++u) {
          const int64_t i = i0 + u * stride;
          gv[u] = i < n4 ? g4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        acc += sum_sq4_batch(gv, inv_s);
      }
      done = n4 * 4;
    }
    for (int64_t i = done + first; i < n; i += stride) {
      const double v = double(g[i] * inv_s);
      acc += v * v;
    }
  }
  const double bsum = block_sum(acc, red);
  double total;
  if (last_block_total(bsum, p.partials, p.counter, &total, red)) {
    octa_scaler* s = p.scaler;
    s->inv_scale_used = inv_s;
    s->grad_norm = sqrt(total);
    if (!isfinite(total)) {  // inf or NaN anywhere makes the sum non-finite
      s->skipped = 1;
      s->n_skipped += 1;
      if (s->growth_interval > 0) {
        s->scale *= 0.5f;
        s->good_steps = 0;
      }
    } else {
      s->skipped = 0;
      s->step += 1;
      if (s->growth_interval > 0 && ++s->good_steps >= s->growth_interval) {
        s->scale *= 2.f;
        s->good_steps = 0;
      }
      p.bias_corr[0] = adam_bias_correction(p.beta1, s->step);
      p.bias_corr[1] = adam_bias_correction(p.beta2, s->step);
    }
  }
}

__device__ __forceinline__ float adam_one(float& pm, float& m, float& v, float g, float lr,
                                          float b1, float b2, float eps, float bc1, float bc2) {
  m = b1 * m + (1.f - b1) * g;
  v = b2 * v + (1.f - b2) * g * g;
  pm = pm - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
  return pm;
}

// Pass 2: Adam with bias correction (Kingma & Ba 2015) unless the step was
// skipped; working copies refreshed; gradients zeroed either way.
__global__ void __launch_bounds__(kThreads) adam_update_kernel(const __grid_constant__ AdamParams p) {
  const octa_scaler* s = p.scaler;
  const bool skip = s->skipped != 0;
  const float inv_s = s->inv_scale_used;
  const float bc1 = skip ? 1.f : p.bias_corr[0], bc2 = skip ? 1.f : p.bias_corr[1];
  const float b1 = p.beta1, b2 = p.beta2, eps = p.eps;
  const int64_t stride = int64_t(gridDim.x) * kThreads;
  const int64_t first = int64_t(blockIdx.x) * kThreads + threadIdx.x;
  for (int gi = 0; gi < p.n_groups; ++gi) {
    const octa_param_group& G = p.g[gi];
    const float lr = G.lr;
    int64_t done = 0;
    if (p.vec4[gi]) {  // 4 elements per thread and iteration
      const int64_t n4 = G.n / 4;
      float4* P = reinterpret_cast<float4*>(G.param);
      float4* Gr = reinterpret_cast<float4*>(G.grad);
      float4* M = reinterpret_cast<float4*>(G.m);
      float4* V = reinterpret_cast<float4*>(G.v);
      // UB elements per iteration, all their loads issued before any store
      constexpr int UB = 2;
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int64_t i0 = first; i0 < n4; i0 += UB * stride) {
        float4 g[UB], pm[UB], m[UB], v[UB];
#pragma unroll
        for (int u = 0; u < UB; ++u) {
          const int64_t i = i0 + u * stride;
          const bool in = i < n4;
          g[u] = in ? Gr[i] : z4;
          pm[u] = in && !skip ? P[i] : z4;
          m[u] = in && !skip ? M[i] : z4;
          v[u] = in && !skip ? V[i] : z4;
        }
#pragma unroll
        for (int u = 0; u < UB; ++u) {
          const int64_t i = i0 + u * stride;
          if (i >= n4) break;
          Gr[i] = z4;
          if (skip) continue;
          adam_one(pm[u].x, m[u].x, v[u].x, g[u].x * inv_s, lr, b1, b2, eps, bc1, bc2);
          adam_one(pm[u].y, m[u].y, v[u].y, g[u].y * inv_s, lr, b1, b2, eps, bc1, bc2);
          adam_one(pm[u].z, m[u].z, v[u].z, g[u].z * inv_s, lr, b1, b2, eps, bc1, bc2);
          adam_one(pm[u].w, m[u].w, v[u].w, g[u].w * inv_s, lr, b1, b2, eps, bc1, bc2);
          P[i] = pm[u];
          M[i] = m[u];
          V[i] = v[u];
          if (G.work) {
            if (G.work_dtype == OCTA_F16) {
              __half2* w = reinterpret_cast<__half2*>(G.work) + 2 * i;
              w[0] = __floats2half2_rn(pm[u].x, pm[u].y);
              w[1] = __floats2half2_rn(pm[u].z, pm[u].w);
            } else {
              __nv_bfloat162* w = reinterpret_cast<__nv_bfloat162*>(G.work) + 2 * i;
              w[0] = __floats2bfloat162_rn(pm[u].x, pm[u].y);
              w[1] = __floats2bfloat162_rn(pm[u].z, pm[u].w);
            }
          }
        }
      }
      done = n4 * 4;
    }
    for (int64_t i = done + first; i < G.n; i += stride) {
      const float g = G.grad[i] * inv_s;
      G.grad[i] = 0.f;
      if (skip) continue;
      float pm = G.param[i], m = G.m[i], v = G.v[i];
      adam_one(pm, m, v, g, lr, b1, b2, eps, bc1, bc2);
      G.param[i] = pm;
      G.m[i] = m;
      G.v[i] = v;
      if (G.work) {
        if (G.work_dtype == OCTA_F16)
          static_cast<__half*>(G.work)[i] = __float2half_rn(pm);
        else
          static_cast<__nv_bfloat16*>(G.work)[i] = __float2bfloat16_rn(pm);
      }
    }
  }
}

int check_workspace(void* ws, size_t bytes) {
  if (!ws) return fail(OCTA_EINVAL, "workspace must be non-NULL");
  if (reinterpret_cast<uintptr_t>(ws) & 255u)
    return fail(OCTA_EINVAL, "workspace must be 256-byte aligned");
  if (bytes < kWorkspaceBytes)
    return fail(OCTA_EINVAL, "workspace of %zu bytes < %zu", bytes, kWorkspaceBytes);
  return OCTA_OK;
}

int launched(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(OCTA_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  return OCTA_OK;
}

}  // namespace
}  // namespace octa

using namespace octa;

extern "C" size_t octa_workspace_bytes(int32_t op, int64_t n) {
  (void)n;
  if (op == OCTA_OP_LOSS || op == OCTA_OP_ADAM) return kWorkspaceBytes;
  if (op == OCTA_OP_STEP) return 256 + sizeof(double) * 1024;  // barrier words + CTA partials
  return 0;
}

extern "C" int residual_loss(const float* L_p, const float* L_s, const float* E, const float* w,
                             int64_t n_pairs, float eps, int32_t rhs_grad,
                             const octa_scaler* scaler, double* loss_dev, float* dL_p,
                             float* dL_s, void* workspace, size_t workspace_bytes,
                             void* stream) {
  clear_error();
  if (n_pairs < 1) return fail(OCTA_EINVAL, "n_pairs must be >= 1");
  if (!L_p || !L_s || !E || !w || !loss_dev || !dL_p)
    return fail(OCTA_EINVAL, "NULL array argument");
  if (rhs_grad && !dL_s) return fail(OCTA_EINVAL, "dL_s must be non-NULL when rhs_grad");
  if (!(eps > 0.f)) return fail(OCTA_EINVAL, "eps must be > 0");
  int rc = check_workspace(workspace, workspace_bytes);
  if (rc) return rc;
  const int64_t n3 = 3 * n_pairs;
  const int blocks = static_cast<int>(
      std::min<int64_t>({(n3 + kThreads - 1) / kThreads, int64_t(kMaxBlocks), 4LL * sm_count()}));
  double* partials = static_cast<double*>(workspace);
  unsigned* counter = reinterpret_cast<unsigned*>(static_cast<char*>(workspace) + kPartialBytes);
  residual_loss_kernel<<<blocks, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      L_p, L_s, E, w, n3, eps, rhs_grad, scaler, loss_dev, dL_p, dL_s, partials, counter);
  return launched("residual_loss");
}

extern "C" int residual_loss_multi(const float* L_p, const float* L_s, const float* E,
                                   const float* w, int64_t n_pairs, int32_t n_samples, float eps,
                                   int32_t rhs_grad, const octa_scaler* scaler, double* loss_dev,
                                   float* dL_p, float* dL_s, void* workspace,
                                   size_t workspace_bytes, void* stream) {
  clear_error();
  if (n_pairs < 1) return fail(OCTA_EINVAL, "n_pairs must be >= 1");
  if (n_samples < 1) return fail(OCTA_EINVAL, "n_samples must be >= 1");
  if (n_pairs > (int64_t(1) << 40) / n_samples) return fail(OCTA_ERANGE, "n_pairs * n_samples too large");
  if (!L_p || !L_s || !E || !w || !loss_dev || !dL_p)
    return fail(OCTA_EINVAL, "NULL array argument");
  if (rhs_grad && !dL_s) return fail(OCTA_EINVAL, "dL_s must be non-NULL when rhs_grad");
  if (!(eps > 0.f)) return fail(OCTA_EINVAL, "eps must be > 0");
  int rc = check_workspace(workspace, workspace_bytes);
  if (rc) return rc;
  constexpr int kWarps = kThreads / 32;
  const int blocks = static_cast<int>(std::min<int64_t>(
      {(n_pairs + kWarps - 1) / kWarps, int64_t(kMaxBlocks), 4LL * sm_count()}));
  double* partials = static_cast<double*>(workspace);
  unsigned* counter = reinterpret_cast<unsigned*>(static_cast<char*>(workspace) + kPartialBytes);
  residual_loss_multi_kernel<<<blocks, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      L_p, L_s, E, w, n_pairs, n_samples, eps, rhs_grad, scaler, loss_dev, dL_p, dL_s, partials,
      counter);
  return launched("residual_loss_multi");
}

extern "C" int adam_step(const octa_param_group* groups, int32_t n_groups,
                         const octa_adam_cfg* cfg, octa_scaler* scaler, void* workspace,
                         size_t workspace_bytes, void* stream) {
  clear_error();
  if (!groups || !cfg || !scaler) return fail(OCTA_EINVAL, "NULL argument");
  if (n_groups < 1 || n_groups > OCTA_MAX_GROUPS)
    return fail(OCTA_ERANGE, "n_groups %d outside [1, %d]", n_groups, OCTA_MAX_GROUPS);
  if (!(cfg->beta1 >= 0.f && cfg->beta1 < 1.f && cfg->beta2 >= 0.f && cfg->beta2 < 1.f &&
        cfg->eps >= 0.f))
    return fail(OCTA_EINVAL, "Adam hyper-parameters out of range");
  int rc = check_workspace(workspace, workspace_bytes);
  if (rc) return rc;
  AdamParams p{};
  int64_t total = 0;
  for (int i = 0; i < n_groups; ++i) {
    const octa_param_group& g = groups[i];
    if (g.n < 0) return fail(OCTA_EINVAL, "group %d: negative size", i);
    if (g.n > 0 && (!g.param || !g.grad || !g.m || !g.v))
      return fail(OCTA_EINVAL, "group %d: NULL array", i);
    if (g.work && g.work_dtype != OCTA_F16 && g.work_dtype != OCTA_BF16)
      return fail(OCTA_EINVAL, "group %d: working copy dtype must be F16 or BF16", i);
    p.g[i] = g;
    const uintptr_t mask = reinterpret_cast<uintptr_t>(g.param) | reinterpret_cast<uintptr_t>(g.grad) |
                           reinterpret_cast<uintptr_t>(g.m) | reinterpret_cast<uintptr_t>(g.v);
    p.vec4[i] = (mask & 15u) == 0 && (!g.work || (reinterpret_cast<uintptr_t>(g.work) & 7u) == 0);
    total += g.n;
  }
  p.n_groups = n_groups;
  p.beta1 = cfg->beta1;
  p.beta2 = cfg->beta2;
  p.eps = cfg->eps;
  p.scaler = scaler;
  p.partials = static_cast<double*>(workspace);
  p.counter = reinterpret_cast<unsigned*>(static_cast<char*>(workspace) + kPartialBytes);
  p.bias_corr = reinterpret_cast<float*>(static_cast<char*>(workspace) + kPartialBytes + 16);
  const int blocks = static_cast<int>(std::max<int64_t>(
      1, std::min<int64_t>({(total / 4 + kThreads - 1) / kThreads, int64_t(kMaxBlocks),
                            6LL * sm_count()})));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  adam_norm_kernel<<<blocks, kThreads, 0, st>>>(p);
  rc = launched("adam_step (norm)");
  if (rc) return rc;
  adam_update_kernel<<<blocks, kThreads, 0, st>>>(p);
  return launched("adam_step (update)");
}

// ---------------------------------------------------------------------------
// residual_loss_static: the residual loss without a caller workspace.
// ---------------------------------------------------------------------------
// Some callers cannot hand the library a device workspace: code that runs in
// a renderer's per-frame path, where a cudaMalloc may synchronise the device
// and stall the frame, or a plug-in whose host application owns every device
// allocation and exposes none to it.  For them the loss reduction takes its
// scratch (per-block FP64 partials and the completion counter) from the
// fixed array below, which every GPU that loads this library keeps until the
// process exits.
namespace octa {
namespace {

constexpr int kStaticSlots = 2048;                  // per-block partials
constexpr int64_t kStaticElemsPerBlock = 16 * kThreads;
// largest n_pairs whose 3 * n_pairs elements fit kStaticSlots blocks
constexpr int64_t kStaticMaxPairs = kStaticSlots * kStaticElemsPerBlock / 3;

// partials [kStaticSlots] doubles, then 256 bytes holding the counter
static __device__ __align__(256) double g_loss_scratch[kStaticSlots + 32] = {};

constexpr int kStaticMaxDevices = 64;
void* g_loss_scratch_addr[kStaticMaxDevices] = {};
std::mutex g_loss_scratch_mutex;

// Device address of g_loss_scratch on the current device, looked up once per
// device (the host-side symbol is only a stand-in for it).
int loss_scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(OCTA_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kStaticMaxDevices)
    return fail(OCTA_ERANGE, "device index %d beyond %d", dev, kStaticMaxDevices);
  std::lock_guard<std::mutex> lock(g_loss_scratch_mutex);
  if (!g_loss_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_loss_scratch);
    if (e != cudaSuccess || !p)
      return fail(OCTA_ECUDA, "cudaGetSymbolAddress(loss scratch): %s", cudaGetErrorString(e));
    g_loss_scratch_addr[dev] = p;
  }
  *out = g_loss_scratch_addr[dev];
  return OCTA_OK;
}

}  // namespace
}  // namespace octa

extern "C" int residual_loss_static(const float* L_p, const float* L_s, const float* E,
                                    const float* w, int64_t n_pairs, float eps, int32_t rhs_grad,
                                    const octa_scaler* scaler, double* loss_dev, float* dL_p,
                                    float* dL_s, void* stream) {
  clear_error();
  if (n_pairs < 1) return fail(OCTA_EINVAL, "n_pairs must be >= 1");
  if (n_pairs > kStaticMaxPairs)
    return fail(OCTA_ERANGE,
                "residual_loss_static: n_pairs %lld exceeds its fixed scratch limit of %lld pairs; "
                "use residual_loss with a workspace",
                static_cast<long long>(n_pairs), static_cast<long long>(kStaticMaxPairs));
  if (!L_p || !L_s || !E || !w || !loss_dev || !dL_p)
    return fail(OCTA_EINVAL, "NULL array argument");
  if (rhs_grad && !dL_s) return fail(OCTA_EINVAL, "dL_s must be non-NULL when rhs_grad");
  if (!(eps > 0.f)) return fail(OCTA_EINVAL, "eps must be > 0");
  void* scratch = nullptr;
  int rc = loss_scratch_address(&scratch);
  if (rc) return rc;
  double* partials = static_cast<double*>(scratch);
  unsigned* counter = reinterpret_cast<unsigned*>(partials + kStaticSlots);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the completion counter must start at zero in every call
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return fail(OCTA_ECUDA, "clearing the loss scratch: %s", cudaGetErrorString(e));
  const int64_t n3 = 3 * n_pairs;
  const int blocks = static_cast<int>((n3 + kStaticElemsPerBlock - 1) / kStaticElemsPerBlock);
  residual_loss_kernel<<<blocks, kThreads, 0, st>>>(L_p, L_s, E, w, n3, eps, rhs_grad, scaler,
                                                    loss_dev, dL_p, dL_s, partials, counter);
  return launched("residual_loss_static");
}
