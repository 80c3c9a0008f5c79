// BF16 tensor-core path of the query: the decoder (Eq. 13) runs on the
// tcgen05 tensor cores with FP32 accumulation in tensor memory.
//
// One CTA of 128 threads owns a tile of 128 queries (one query per thread
// and per tensor-memory lane).  Per tile:
//   locate   fold omega and walk the octree (one thread per query);
//   gather   one thread per (query, level): bilinear blend in FP32 of the 4
//            wrapped texels, rounded to BF16 and stored as one 16-byte row of
//            a core matrix of the canonical K-major operand tile (the level
//            concatenation of Eq. 11 is the K index);
//   decoder  per layer one elected thread issues K/16 MMAs of 128 x N x 16
//            (A = activations, B = the layer's weights, both in shared
//            memory), commits to an mbarrier; after the bounded wait every
//            thread pulls its row of the accumulator from tensor memory,
//            applies ReLU, rounds to BF16 and writes the next A tile.  The
//            last layer (N padded to 16) ends in exp().
// Several CTAs share an SM (64 tensor-memory columns each), so one CTA's
// gather overlaps another's MMAs.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "engine_f32.cuh"
#include "launch_util.h"
#include "octa_internal.h"
#include "tc_path.h"
#include "tc_ptx.cuh"

namespace octa {
namespace tc {

constexpr int NT = 128;   // threads per CTA = queries per tile
constexpr int NOUT = 16;  // padded output width of the last layer

template <int F_, int WP_, int H_, int NH_>
struct Shape {
  static constexpr int F = F_, WP = WP_, H = H_, NH = NH_, NL = NH_ + 1;
  static constexpr int KPAD = WP / F;
  static constexpr int AK = WP > H ? WP : H;
  static_assert(WP % 16 == 0 && H % 16 == 0 && H <= 128, "MMA shapes");
  static constexpr uint32_t W0_BYTES = H * WP * 2;
  static constexpr uint32_t WH_BYTES = H * H * 2;
  static constexpr uint32_t WL_BYTES = NOUT * H * 2;
  static constexpr uint32_t W_BYTES = W0_BYTES + (NH - 1) * WH_BYTES + WL_BYTES;
  static constexpr uint32_t ACT_BYTES = NT * AK * 2;
  static constexpr uint32_t NODE_BYTES = KPAD * NT * 4;
  static constexpr uint32_t U_BYTES = 2 * NT * 4;
  static constexpr uint32_t OFF_ACT = W_BYTES;
  static constexpr uint32_t OFF_NODE = OFF_ACT + ACT_BYTES;
  static constexpr uint32_t OFF_U = OFF_NODE + NODE_BYTES;
  static constexpr uint32_t OFF_BAR = (OFF_U + U_BYTES + 15) & ~15u;
  static constexpr size_t SMEM = OFF_BAR + 16;
  static constexpr uint32_t TMEM_COLS = H <= 32 ? 32 : (H <= 64 ? 64 : 128);
  __host__ __device__ static constexpr uint32_t w_off(int layer) {
    return layer == 0 ? 0u : W0_BYTES + static_cast<uint32_t>(layer - 1) * WH_BYTES;
  }
  __host__ __device__ static constexpr int kdim(int layer) { return layer == 0 ? WP : H; }
  __host__ __device__ static constexpr int ndim(int layer) { return layer == NL - 1 ? NOUT : H; }
};

// Weights of one scene into shared memory, canonical K-major, zero padded.
template <class S>
__device__ void load_weights_bf16(const DevScene& sc, uint8_t* smem) {
  const __nv_bfloat16* Wg = static_cast<const __nv_bfloat16*>(sc.weights);
#pragma unroll 1
  for (int l = 0; l < S::NL; ++l) {
    const int K = S::kdim(l), N = S::ndim(l);
    const int in = sc.widths[l], out = sc.widths[l + 1];
    __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(smem + S::w_off(l));
    for (int i = threadIdx.x; i < N * K; i += NT) {
      const int n = i / K, k = i % K;
      const __nv_bfloat16 v =
          (n < out && k < in) ? Wg[sc.w_offset[l] + n * in + k] : __float2bfloat16_rn(0.f);
      dst[kmajor_offset(n, k, K) / 2] = v;
    }
  }
}

// Locate and gather of one query per thread, fused: the thread folds omega,
// walks its query's path down the octree, loads the map base of every
// present level, then gathers two levels at a time (both levels' texel loads
// in flight together; one at a time for 32-byte texels) into its row of the
// layer-0 operand tile.  node_sm /
// u_sm (nullable) keep the path and the folded direction for a later scatter.
template <class S, typename TT>
__device__ __forceinline__ void locate_gather_bf16(const QueryParams& p, const DevScene& sc,
                                                   int64_t q0, int nq, uint8_t* act,
                                                   int* node_sm, float* u_sm) {
  constexpr int F = S::F, KP = S::KPAD;
  // levels gathered together: two for texels of up to 16 bytes, else one
  constexpr int WIN = TexelRaw<TT, F>::BYTES <= 16 ? 2 : 1;
  const int q = threadIdx.x;
  const bool valid = q < nq;
  const int64_t gq = q0 + q;
  float x0 = 0.f, x1 = 0.f, x2 = 0.f, w0 = 0.f, w1 = 0.f, w2 = 1.f;
  if (valid) {
    x0 = p.x[3 * gq];
    x1 = p.x[3 * gq + 1];
    x2 = p.x[3 * gq + 2];
    w0 = p.omega[3 * gq];
    w1 = p.omega[3 * gq + 1];
    w2 = p.omega[3 * gq + 2];
  }
  float ux, uy;
  octa_fold(w0, w1, w2, ux, uy);
  x0 = clamp01(x0);
  x1 = clamp01(x1);
  x2 = clamp01(x2);
  int node[KP];
  node[0] = valid ? 0 : -1;
  int cp0 = 0, cp1 = 0, cp2 = 0;
#pragma unroll
  for (int l = 1; l < KP; ++l) {
    int nd = -1;
    if (l < sc.K && node[l - 1] >= 0) {
      const int c0 = cell_coord(x0, l), c1 = cell_coord(x1, l), c2 = cell_coord(x2, l);
      const int slot = (c0 - 2 * cp0) | ((c1 - 2 * cp1) << 1) | ((c2 - 2 * cp2) << 2);
      int fc = __ldg(sc.first_child + node[l - 1]);
      if (fc >= 0 && fc > sc.num_nodes - 8) {
        if (p.status) atomicOr(p.status, OCTA_STATUS_BAD_CHILD);
        fc = -1;
      }
      nd = fc >= 0 ? fc + slot : -1;
      cp0 = c0;
      cp1 = c1;
      cp2 = c2;
    }
    node[l] = nd;
  }
  if (node_sm) {
#pragma unroll
    for (int l = 0; l < KP; ++l) node_sm[l * NT + q] = node[l];
    u_sm[q] = ux;
    u_sm[NT + q] = uy;
  }
  if (p.node_idx && valid) {
#pragma unroll
    for (int l = 0; l < KP; ++l)
      if (l < p.kmax_out) p.node_idx[gq * p.kmax_out + l] = node[l];
    for (int l = KP; l < p.kmax_out; ++l) p.node_idx[gq * p.kmax_out + l] = -1;
  }
  int64_t mo[KP];
#pragma unroll
  for (int l = 0; l < KP; ++l) mo[l] = node[l] >= 0 ? f32::map_base(p, sc, node[l], sc.R[l]) : -1;
#pragma unroll
  for (int l0 = 0; l0 < KP; l0 += WIN) {
    TexelRaw<TT, F> t[WIN][4];
    Footprint fp[WIN];
#pragma unroll
    for (int j = 0; j < WIN; ++j) {
      const int l = l0 + j;
      if (l < KP && mo[l] >= 0) {
        fp[j] = footprint(ux, uy, sc.R[l]);
#pragma unroll
        for (int k = 0; k < 4; ++k) t[j][k].load(sc.tables, mo[l] + fp[j].idx[k]);
      }
    }
#pragma unroll
    for (int j = 0; j < WIN; ++j) {
      const int l = l0 + j;
      if (l >= KP) continue;
      float v[F];
      if (mo[l] >= 0) {
#pragma unroll
        for (int f = 0; f < F; ++f) {
          float s = fp[j].w[0] * t[j][0].get(f);
          s = fmaf(fp[j].w[1], t[j][1].get(f), s);
          s = fmaf(fp[j].w[2], t[j][2].get(f), s);
          s = fmaf(fp[j].w[3], t[j][3].get(f), s);
          v[f] = s;
        }
      } else {
#pragma unroll
        for (int f = 0; f < F; ++f) v[f] = 0.f;
      }
      uint8_t* dst = act + kmajor_offset(q, l * F, S::WP);
      if constexpr (F == 8) {
        uint4 o;
        o.x = pack_bf16x2(v[0], v[1]);
        o.y = pack_bf16x2(v[2], v[3]);
        o.z = pack_bf16x2(v[4], v[5]);
        o.w = pack_bf16x2(v[6], v[7]);
        *reinterpret_cast<uint4*>(dst) = o;
      } else {
        uint2 o;
        o.x = pack_bf16x2(v[0], v[1]);
        o.y = pack_bf16x2(v[2], v[3]);
        *reinterpret_cast<uint2*>(dst) = o;
      }
      if (p.texel_addr && valid && l < p.kmax_out) {
        int4 a = make_int4(-1, -1, -1, -1);
        if (mo[l] >= 0)
          a = make_int4(int(mo[l] + fp[j].idx[0]), int(mo[l] + fp[j].idx[1]),
                        int(mo[l] + fp[j].idx[2]), int(mo[l] + fp[j].idx[3]));
        *reinterpret_cast<int4*>(p.texel_addr + (gq * p.kmax_out + l) * 4) = a;
      }
    }
  }
  if (p.texel_addr && valid)
    for (int l = KP; l < p.kmax_out; ++l)
      *reinterpret_cast<int4*>(p.texel_addr + (gq * p.kmax_out + l) * 4) = make_int4(-1, -1, -1, -1);
}

// Issue the MMAs of one layer (single thread) and commit to the mbarrier.
template <class S>
__device__ __forceinline__ void issue_layer(int layer, uint32_t act_sa, uint32_t w_sa, uint32_t tmem,
                                            uint32_t mbar) {
  tc_fence_after_sync();
  const int K = S::kdim(layer);
  const uint32_t idesc = idesc_bf16(128, S::ndim(layer));
  const uint32_t b_sa = w_sa + S::w_off(layer);
#pragma unroll 1
  for (int k0 = 0; k0 < K; k0 += 16)
    mma_bf16(tmem, kmajor_desc(act_sa, k0, K), kmajor_desc(b_sa, k0, K), idesc, k0 > 0 ? 1u : 0u);
  mma_commit(mbar);
}

template <class S, typename TT>
__global__ void __launch_bounds__(NT, 4) fwd_kernel(const __grid_constant__ QueryParams p) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* act = smem + S::OFF_ACT;
  int* node_sm = reinterpret_cast<int*>(smem + S::OFF_NODE);
  float* u_sm = reinterpret_cast<float*>(smem + S::OFF_U);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + S::OFF_BAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + S::OFF_BAR + 8);
  const uint32_t mbar = smem_addr(bar);
  const uint32_t act_sa = smem_addr(act), w_sa = smem_addr(smem);
  const int warp = threadIdx.x >> 5;

  if (threadIdx.x == 0) mbar_init(mbar, 1);
  if (warp == 0) {
    tmem_alloc(smem_addr(tslot), S::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t lane_base = tmem + (static_cast<uint32_t>(warp * 32) << 16);
  uint32_t phase = 0;
  int cur = -1;
  bool failed = false;

  for (int64_t tile = blockIdx.x; tile < p.n_tiles && !failed; tile += gridDim.x) {
    const int s = scene_of_tile(p, tile);
    const DevScene& sc = p.sc[s];
    __syncthreads();
    if (s != cur) {
      load_weights_bf16<S>(sc, smem);
      cur = s;
    }
    const int64_t q0 = sc.q_begin + (tile - sc.tile_begin) * NT;
    const int nq = static_cast<int>(sc.q_end - q0 < NT ? sc.q_end - q0 : int64_t(NT));
    locate_gather_bf16<S, TT>(p, sc, q0, nq, act, nullptr, nullptr);
    fence_proxy_async();
    __syncthreads();

#pragma unroll 1
    for (int layer = 0; layer < S::NL; ++layer) {
      if (threadIdx.x == 0) issue_layer<S>(layer, act_sa, w_sa, tmem, mbar);
      const bool ok = mbar_wait_bounded(mbar, phase);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      tc_fence_after_sync();
      if (layer < S::NL - 1) {
        uint32_t r[S::H];
#pragma unroll
        for (int c = 0; c < S::H; c += 16)
          tmem_ld16(lane_base + c, *reinterpret_cast<uint32_t(*)[16]>(r + c));
        tmem_wait_ld();
        const int q = threadIdx.x;
#pragma unroll
        for (int c = 0; c < S::H; c += 8) {
          uint4 o;
          o.x = pack_bf16x2(fmaxf(__uint_as_float(r[c + 0]), 0.f), fmaxf(__uint_as_float(r[c + 1]), 0.f));
          o.y = pack_bf16x2(fmaxf(__uint_as_float(r[c + 2]), 0.f), fmaxf(__uint_as_float(r[c + 3]), 0.f));
          o.z = pack_bf16x2(fmaxf(__uint_as_float(r[c + 4]), 0.f), fmaxf(__uint_as_float(r[c + 5]), 0.f));
          o.w = pack_bf16x2(fmaxf(__uint_as_float(r[c + 6]), 0.f), fmaxf(__uint_as_float(r[c + 7]), 0.f));
          *reinterpret_cast<uint4*>(act + kmajor_offset(q, c, S::H)) = o;
        }
        fence_proxy_async();
        tc_fence_before_sync();
        __syncthreads();
      } else {
        uint32_t r[16];
        tmem_ld16(lane_base, r);
        tmem_wait_ld();
        tc_fence_before_sync();
        const int q = threadIdx.x;
        if (q < nq) {
          const int64_t gq = q0 + q;
          p.rgb[3 * gq] = expf(__uint_as_float(r[0]));
          p.rgb[3 * gq + 1] = expf(__uint_as_float(r[1]));
          p.rgb[3 * gq + 2] = expf(__uint_as_float(r[2]));
        }
      }
    }
  }
  if (failed && threadIdx.x == 0 && p.status) atomicOr(p.status, OCTA_STATUS_TIMEOUT);
  tc_fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, S::TMEM_COLS);
}

// ---------------------------------------------------------------------------
// Backward (recomputed forward, then the delta chain on the tensor cores)
// ---------------------------------------------------------------------------
// Shared memory: weights | h tile | a_1 .. a_NH tiles | delta_L tile | slack |
// node / u tables | mbarrier.  Tensor memory: a working accumulator of WORK
// columns (every forward layer and every data-gradient GEMM), then the
// transposed weight gradients dW_i^T = a_i^T delta_{i+1} (rows = input
// features, one column per output feature), accumulated over every tile the
// CTA handles and flushed with atomics when the scene changes or at the end.
template <int F_, int WP_, int H_, int NH_>
struct BShape : Shape<F_, WP_, H_, NH_> {
  using B = Shape<F_, WP_, H_, NH_>;
  static constexpr uint32_t H_TILE = NT * WP_ * 2;
  static constexpr uint32_t A_TILE = NT * H_ * 2;
  static constexpr uint32_t DL_TILE = NT * NOUT * 2;
  static constexpr uint32_t OFF_H = B::W_BYTES;
  static constexpr uint32_t OFF_DL = OFF_H + H_TILE + NH_ * A_TILE;
  // MN-major reads with M = 128 rows run past a tile narrower than 128
  // features into the next buffer; the slack keeps the last one in bounds.
  static constexpr uint32_t OFF_NODE = OFF_DL + DL_TILE + 2048;
  static constexpr uint32_t OFF_U = OFF_NODE + B::NODE_BYTES;
  static constexpr uint32_t OFF_BAR = (OFF_U + B::U_BYTES + 15) & ~15u;
  static constexpr size_t SMEM = OFF_BAR + 16;
  static constexpr int WORK = WP_ > H_ ? WP_ : H_;
  static constexpr int COLS = WORK + H_ * NH_ + NOUT;
  static constexpr uint32_t TMEM_COLS = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128
                                        : COLS <= 256 ? 256 : 512;
  static_assert(COLS <= 512, "tensor memory");
  __host__ __device__ static constexpr uint32_t off_act(int i) {
    return i == 0 ? OFF_H : OFF_H + H_TILE + static_cast<uint32_t>(i - 1) * A_TILE;
  }
  __host__ __device__ static constexpr int dw_col(int i) { return WORK + H_ * i; }
};

// Adds the CTA's dW^T accumulators of one scene to its FP32 weight gradient
// (thread r holds row r = input feature r of every matrix).
template <class S>
__device__ void flush_weight_grads(const DevScene& sc, uint32_t lane_base) {
  const int r = threadIdx.x;
  tc_fence_after_sync();
#pragma unroll 1
  for (int i = 0; i < S::NL; ++i) {
    const int n_pad = S::ndim(i);
    const int in = sc.widths[i], out = sc.widths[i + 1];
    float* dW = sc.d_weights + sc.w_offset[i];
#pragma unroll 1
    for (int c = 0; c < n_pad; c += 16) {
      uint32_t v[16];
      tmem_ld16(lane_base + S::dw_col(i) + c, v);
      tmem_wait_ld();
      if (r < in) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c + j < out) atomicAdd(dW + (c + j) * in + r, __uint_as_float(v[j]));
      }
    }
  }
  tc_fence_before_sync();
}

template <class S, typename TT>
__global__ void __launch_bounds__(NT) bwd_kernel(const __grid_constant__ QueryParams p) {
  constexpr int H = S::H, NL = S::NL;
  extern __shared__ __align__(1024) uint8_t smem[];
  int* node_sm = reinterpret_cast<int*>(smem + S::OFF_NODE);
  float* u_sm = reinterpret_cast<float*>(smem + S::OFF_U);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + S::OFF_BAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + S::OFF_BAR + 8);
  const uint32_t mbar = smem_addr(bar);
  const uint32_t base_sa = smem_addr(smem);
  const uint32_t dl_sa = base_sa + S::OFF_DL;
  const int warp = threadIdx.x >> 5;
  const int q = threadIdx.x;

  if (threadIdx.x == 0) mbar_init(mbar, 1);
  if (warp == 0) {
    tmem_alloc(smem_addr(tslot), S::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t lane_base = tmem + (static_cast<uint32_t>(warp * 32) << 16);
  uint32_t phase = 0;
  int cur = -1;
  bool first = true, failed = false;

  for (int64_t tile = blockIdx.x; tile < p.n_tiles && !failed; tile += gridDim.x) {
    const int s = scene_of_tile(p, tile);
    const DevScene& sc = p.sc[s];
    __syncthreads();
    if (s != cur) {
      if (cur >= 0 && !first) flush_weight_grads<S>(p.sc[cur], lane_base);
      load_weights_bf16<S>(sc, smem);
      cur = s;
      first = true;
    }
    const int64_t q0 = sc.q_begin + (tile - sc.tile_begin) * NT;
    const int nq = static_cast<int>(sc.q_end - q0 < NT ? sc.q_end - q0 : int64_t(NT));
    locate_gather_bf16<S, TT>(p, sc, q0, nq, smem + S::OFF_H, node_sm, u_sm);
    fence_proxy_async();
    __syncthreads();

    // ---- forward, keeping a_1 .. a_NH and delta_L
#pragma unroll 1
    for (int layer = 0; layer < NL && !failed; ++layer) {
      if (threadIdx.x == 0) issue_layer<S>(layer, base_sa + S::off_act(layer), base_sa, tmem, mbar);
      const bool ok = mbar_wait_bounded(mbar, phase);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      tc_fence_after_sync();
      if (layer < NL - 1) {
        uint32_t r[H];
#pragma unroll
        for (int c = 0; c < H; c += 16)
          tmem_ld16(lane_base + c, *reinterpret_cast<uint32_t(*)[16]>(r + c));
        tmem_wait_ld();
        uint8_t* dst = smem + S::off_act(layer + 1);
#pragma unroll
        for (int c = 0; c < H; c += 8) {
          uint4 o;
          o.x = pack_bf16x2(fmaxf(__uint_as_float(r[c + 0]), 0.f), fmaxf(__uint_as_float(r[c + 1]), 0.f));
          o.y = pack_bf16x2(fmaxf(__uint_as_float(r[c + 2]), 0.f), fmaxf(__uint_as_float(r[c + 3]), 0.f));
          o.z = pack_bf16x2(fmaxf(__uint_as_float(r[c + 4]), 0.f), fmaxf(__uint_as_float(r[c + 5]), 0.f));
          o.w = pack_bf16x2(fmaxf(__uint_as_float(r[c + 6]), 0.f), fmaxf(__uint_as_float(r[c + 7]), 0.f));
          *reinterpret_cast<uint4*>(dst + kmajor_offset(q, c, H)) = o;
        }
      } else {
        uint32_t r[16];
        tmem_ld16(lane_base, r);
        tmem_wait_ld();
        float d0 = 0.f, d1 = 0.f, d2 = 0.f;
        if (q < nq) {
          const int64_t gq = q0 + q;
          d0 = p.d_rgb[3 * gq];
          d1 = p.d_rgb[3 * gq + 1];
          d2 = p.d_rgb[3 * gq + 2];
        }
        // delta_L = d_rgb * exp(z_L): the derivative of exp is exp
        uint8_t* dst = smem + S::OFF_DL;
        uint4 o0, o1;
        o0.x = pack_bf16x2(d0 * expf(__uint_as_float(r[0])), d1 * expf(__uint_as_float(r[1])));
        o0.y = pack_bf16x2(d2 * expf(__uint_as_float(r[2])), 0.f);
        o0.z = o0.w = 0u;
        o1.x = o1.y = o1.z = o1.w = 0u;
        *reinterpret_cast<uint4*>(dst + kmajor_offset(q, 0, NOUT)) = o0;
        *reinterpret_cast<uint4*>(dst + kmajor_offset(q, 8, NOUT)) = o1;
      }
      fence_proxy_async();
      tc_fence_before_sync();
      __syncthreads();
    }
    if (failed) break;

    // ---- backward through the decoder
#pragma unroll 1
    for (int i = NL - 1; i >= 0; --i) {
      const int out = S::ndim(i), in = S::kdim(i);
      const uint32_t d_sa = i == NL - 1 ? dl_sa : base_sa + S::off_act(i + 1);
      const int dk = out;  // row length of the delta tile
      if (threadIdx.x == 0) {
        tc_fence_after_sync();
        // dW_i^T += a_i^T delta_{i+1}: M = 128 input features, N = out, K = 128 queries
        const uint32_t act_sa = base_sa + S::off_act(i);
        const uint32_t idw = idesc_bf16(128, out, 1, 1);
#pragma unroll 1
        for (int kq = 0; kq < NT; kq += 16)
          mma_bf16(tmem + S::dw_col(i), mnmajor_desc(act_sa, kq, in), mnmajor_desc(d_sa, kq, dk),
                   idw, (!first || kq > 0) ? 1u : 0u);
        // G = delta_{i+1} W_i: M = 128 queries, N = in, K = out
        const uint32_t ig = idesc_bf16(128, in, 0, 1);
        const uint32_t w_sa = base_sa + S::w_off(i);
#pragma unroll 1
        for (int ko = 0; ko < out; ko += 16)
          mma_bf16(tmem, kmajor_desc(d_sa, ko, dk), mnmajor_desc(w_sa, ko, in), ig,
                   ko > 0 ? 1u : 0u);
        mma_commit(mbar);
      }
      const bool ok = mbar_wait_bounded(mbar, phase);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      tc_fence_after_sync();
      if (i > 0) {
        // delta_i = G * 1[a_i > 0], written over a_i (its MMAs have completed)
        uint32_t r[H];
#pragma unroll
        for (int c = 0; c < H; c += 16)
          tmem_ld16(lane_base + c, *reinterpret_cast<uint32_t(*)[16]>(r + c));
        tmem_wait_ld();
        uint8_t* act = smem + S::off_act(i);
#pragma unroll
        for (int c = 0; c < H; c += 8) {
          uint4* pa = reinterpret_cast<uint4*>(act + kmajor_offset(q, c, H));
          const uint4 a = *pa;
          const uint32_t av[4] = {a.x, a.y, a.z, a.w};
          uint32_t ov[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            // a ReLU output in bf16 is > 0 iff its magnitude bits are non-zero
            const float g0 = (av[j] & 0x7FFFu) ? __uint_as_float(r[c + 2 * j]) : 0.f;
            const float g1 = ((av[j] >> 16) & 0x7FFFu) ? __uint_as_float(r[c + 2 * j + 1]) : 0.f;
            ov[j] = pack_bf16x2(g0, g1);
          }
          *pa = make_uint4(ov[0], ov[1], ov[2], ov[3]);
        }
        fence_proxy_async();
        tc_fence_before_sync();
        __syncthreads();
      } else {
        // dh = G; scatter w_k * dh_l into the four texels of every present level
        uint32_t r[S::WP];
#pragma unroll
        for (int c = 0; c < S::WP; c += 16)
          tmem_ld16(lane_base + c, *reinterpret_cast<uint32_t(*)[16]>(r + c));
        tmem_wait_ld();
        tc_fence_before_sync();
#pragma unroll
        for (int l = 0; l < S::KPAD; ++l) {
          const int node = node_sm[l * NT + q];
          if (node < 0) continue;
          const int R = sc.R[l];
          const int64_t mo = f32::map_base(p, sc, node, R);
          if (mo < 0) continue;
          const Footprint fp = footprint(u_sm[q], u_sm[NT + q], R);
#pragma unroll
          for (int c4 = 0; c4 < S::F / 4; ++c4) {
            const float g0 = __uint_as_float(r[l * S::F + 4 * c4 + 0]);
            const float g1 = __uint_as_float(r[l * S::F + 4 * c4 + 1]);
            const float g2 = __uint_as_float(r[l * S::F + 4 * c4 + 2]);
            const float g3 = __uint_as_float(r[l * S::F + 4 * c4 + 3]);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const float w = fp.w[k];
              float4* dst = reinterpret_cast<float4*>(sc.d_tables + (mo + fp.idx[k]) * S::F) + c4;
              atomicAdd(dst, make_float4(w * g0, w * g1, w * g2, w * g3));
            }
          }
        }
      }
    }
    first = false;
  }
  if (!failed && cur >= 0 && !first) {
    __syncthreads();
    flush_weight_grads<S>(p.sc[cur], lane_base);
  }
  if (failed && threadIdx.x == 0 && p.status) atomicOr(p.status, OCTA_STATUS_TIMEOUT);
  tc_fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, S::TMEM_COLS);
}

namespace {

template <class S, typename TT>
int launch_fwd(const QueryParams& p, cudaStream_t stream) {
  if (p.n_tiles == 0) return OCTA_OK;
  auto kern = fwd_kernel<S, TT>;
  int per_sm = 0;
  int rc = launch_cache().get(reinterpret_cast<const void*>(kern), S::SMEM, NT,
                              static_cast<int>(S::TMEM_COLS), &per_sm);
  if (rc) return rc;
  const int64_t grid = std::min<int64_t>(p.n_tiles, int64_t(per_sm) * device_sm_count());
  kern<<<static_cast<unsigned>(grid), NT, S::SMEM, stream>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(OCTA_ECUDA, "tc fwd launch: %s", cudaGetErrorString(e));
  return OCTA_OK;
}

template <class S, typename TT>
int launch_bwd(const QueryParams& p, cudaStream_t stream) {
  if (p.n_tiles == 0) return OCTA_OK;
  auto kern = bwd_kernel<S, TT>;
  int per_sm = 0;
  int rc = launch_cache().get(reinterpret_cast<const void*>(kern), S::SMEM, NT,
                              static_cast<int>(S::TMEM_COLS), &per_sm);
  if (rc) return rc;
  const int64_t grid = std::min<int64_t>(p.n_tiles, int64_t(per_sm) * device_sm_count());
  kern<<<static_cast<unsigned>(grid), NT, S::SMEM, stream>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(OCTA_ECUDA, "tc bwd launch: %s", cudaGetErrorString(e));
  return OCTA_OK;
}

// Common shape selection of the BF16 path.
int select_shape(const octa_scene* scenes, int n_scenes, int* F, int* need, int* H, int* NH,
                 bool* f16) {
  const octa_scene& c0 = scenes[0];
  const int L = c0.n_layers, tdt = c0.table_dtype;
  *F = c0.F;
  *H = c0.widths[1];
  *need = 0;
  for (int s = 0; s < n_scenes; ++s) {
    const octa_scene& c = scenes[s];
    if (c.F != *F || c.n_layers != L || c.table_dtype != tdt || c.weight_dtype != OCTA_BF16)
      return fail(OCTA_EUNSUPPORTED, "scenes of one call must share F, MLP depth and dtypes");
    for (int i = 1; i < L; ++i)
      if (c.widths[i] != *H) return fail(OCTA_EUNSUPPORTED, "BF16 path: hidden widths must match");
    *need = std::max(*need, c.widths[0]);
  }
  *NH = L - 1;
  *f16 = tdt == OCTA_F16;
  return OCTA_OK;
}

}  // namespace

int query_bwd(const octa_scene* scenes, int n_scenes, const QueryParams& p, cudaStream_t stream) {
  int F, need, H, NH;
  bool f16;
  int rc = select_shape(scenes, n_scenes, &F, &need, &H, &NH, &f16);
  if (rc) return rc;
#define OCTA_TC_TRY(F_, WP_, H_, NH_)                                                  \
  if (F == F_ && H == H_ && NH == NH_ && need <= WP_)                                  \
    return f16 ? launch_bwd<BShape<F_, WP_, H_, NH_>, __half>(p, stream)              \
               : launch_bwd<BShape<F_, WP_, H_, NH_>, float>(p, stream);
  OCTA_TC_TRY(4, 32, 32, 2)
  OCTA_TC_TRY(8, 64, 64, 2)
  OCTA_TC_TRY(8, 80, 64, 2)
  OCTA_TC_TRY(8, 80, 64, 3)
#undef OCTA_TC_TRY
  return fail(OCTA_EUNSUPPORTED, "BF16 path: no built shape for F=%d, K*F=%d, hidden %d x %d", F,
              need, NH, H);
}

int query_fwd(const octa_scene* scenes, int n_scenes, const QueryParams& p, cudaStream_t stream) {
  const octa_scene& c0 = scenes[0];
  const int F = c0.F, L = c0.n_layers, H = c0.widths[1], tdt = c0.table_dtype;
  int need = 0;
  for (int s = 0; s < n_scenes; ++s) {
    const octa_scene& c = scenes[s];
    if (c.F != F || c.n_layers != L || c.table_dtype != tdt || c.weight_dtype != OCTA_BF16)
      return fail(OCTA_EUNSUPPORTED, "scenes of one call must share F, MLP depth and dtypes");
    for (int i = 1; i < L; ++i)
      if (c.widths[i] != H) return fail(OCTA_EUNSUPPORTED, "BF16 path: hidden widths must match");
    need = std::max(need, c.widths[0]);
  }
  const int NH = L - 1;
  const bool f16 = tdt == OCTA_F16;
#define OCTA_TC_TRY(F_, WP_, H_, NH_)                                                  \
  if (F == F_ && H == H_ && NH == NH_ && need <= WP_)                                  \
    return f16 ? launch_fwd<Shape<F_, WP_, H_, NH_>, __half>(p, stream)               \
               : launch_fwd<Shape<F_, WP_, H_, NH_>, float>(p, stream);
  OCTA_TC_TRY(4, 32, 32, 2)
  OCTA_TC_TRY(8, 64, 64, 2)
  OCTA_TC_TRY(8, 80, 64, 2)
  OCTA_TC_TRY(8, 80, 64, 3)
#undef OCTA_TC_TRY
  return fail(OCTA_EUNSUPPORTED, "BF16 path: no built shape for F=%d, K*F=%d, hidden %d x %d", F,
              need, NH, H);
}

}  // namespace tc
}  // namespace octa
