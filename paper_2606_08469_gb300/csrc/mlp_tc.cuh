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
//
// The kernels and launchers live in this header; mlp_tc_fwd.cu, mlp_tc_bwd.cu
// and mlp_tc_step.cu each define one group of entry points (OCTA_TC_FWD,
// OCTA_TC_BWD, OCTA_TC_STEP), so the three groups compile in parallel.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "engine_f32.cuh"
#include "gather.cuh"
#include "launch_util.h"
#include "octa_internal.h"
#include "tc_path.h"
#include "tc_ptx.cuh"

namespace octa {
namespace tc {

constexpr int NT = 128;   // threads per CTA = queries per tile
constexpr int NOUT = 16;  // padded output width of the last layer

// Shared memory of an SM and the per-CTA reservation on this GPU family;
// they size the staged octree so that it does not lower the residency the
// rest of a kernel's layout allows (a wrong guess costs residency, never
// correctness: the launcher measures what fits).
constexpr int kSmemPerSM = 233472, kSmemPerCTAReserved = 1024;
constexpr int tree_capacity(uint32_t used, int ctas_per_sm) {
  const int room = kSmemPerSM / ctas_per_sm - kSmemPerCTAReserved - static_cast<int>(used);
  const int n = room > 0 ? (room / 8) & ~15 : 0;
  return n > 2048 ? 2048 : n;
}

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
  static constexpr uint32_t OFF_BAR = (OFF_ACT + ACT_BYTES + 15) & ~15u;
  // staged octree (int2 per node), as large as four CTAs per SM allow
  static constexpr uint32_t OFF_TREE = OFF_BAR + 16;
  static constexpr int TREE_NODES = tree_capacity(OFF_TREE, 4);
  static constexpr size_t SMEM = OFF_TREE + 8u * TREE_NODES;
  static constexpr uint32_t TMEM_COLS = H <= 32 ? 32 : (H <= 64 ? 64 : 128);
  __host__ __device__ static constexpr uint32_t w_off(int layer) {
    return layer == 0 ? 0u : W0_BYTES + static_cast<uint32_t>(layer - 1) * WH_BYTES;
  }
  __host__ __device__ static constexpr int kdim(int layer) { return layer == 0 ? WP : H; }
  __host__ __device__ static constexpr int ndim(int layer) { return layer == NL - 1 ? NOUT : H; }
};

// Weights of one scene into shared memory, canonical K-major, zero padded.
template <class S>
__device__ void load_weights_bf16(const DevScene& sc, uint8_t* smem, int nthreads = NT) {
  const __nv_bfloat16* Wg = static_cast<const __nv_bfloat16*>(sc.weights);
#pragma unroll 1
  for (int l = 0; l < S::NL; ++l) {
    const int K = S::kdim(l), N = S::ndim(l);
    const int in = sc.widths[l], out = sc.widths[l + 1];
    __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(smem + S::w_off(l));
    for (int i = threadIdx.x; i < N * K; i += nthreads) {
      const int n = i / K, k = i % K;
      const __nv_bfloat16 v =
          (n < out && k < in) ? Wg[sc.w_offset[l] + n * in + k] : __float2bfloat16_rn(0.f);
      dst[kmajor_offset(n, k, K) / 2] = v;
    }
  }
}

// Locate and gather of one query per thread into its row of the layer-0
// operand tile (canonical K-major, one 16-byte store per level for F = 8);
// FORM: the query form (the trilinear vertex and shifted forms gather one
// query per thread).  Columns past the K levels take Eq. 12's attributes.
// nrm / disp: the shifted form's normal and disparity arrays of query gq.
template <class S, typename TT, int TPQ = 1, int FORM = OCTA_FORM_CELL_BILINEAR>
__device__ __forceinline__ void locate_gather_bf16(const QueryParams& p, const DevScene& sc,
                                                   const int2* tree, const QueryIn& in, int64_t gq,
                                                   bool valid, int par, uint8_t* act, int* base_sm,
                                                   float* u_sm, int q, const float* nrm = nullptr,
                                                   const float* disp = nullptr) {
  constexpr int F = S::F;
  auto store = [&](int l, const float (&v0)[F]) {
    float v[F];
#pragma unroll
    for (int f = 0; f < F; ++f) v[f] = v0[f];
    if (p.n_attrs > 0 && l >= sc.K) attr_columns<F>(p, sc.K, l, gq, valid, v);
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
  };
  if constexpr (FORM == OCTA_FORM_SHIFTED) {
    static_assert(TPQ == 1, "the shifted form gathers one query per thread");
    gather_shifted_query<F, TT, S::KPAD>(p, sc, tree, in, gq, valid, nrm, disp, store);
  } else if constexpr (FORM == OCTA_FORM_TRILINEAR_VERTEX) {
    static_assert(TPQ == 1, "the full form gathers one query per thread");
    gather_full_query<F, TT, S::KPAD>(p, sc, tree, in, gq, valid, store);
  } else {
    locate_gather_query<F, TT, S::KPAD, true, TPQ>(p, sc, tree, in, gq, valid, par, base_sm, u_sm,
                                                   q, NT, store);
  }
}

// The forward kernel's form that runs the disparity predictor g_psi: its
// input row (hash encoding, omega_r) replaces the octree gather and the
// single output is d = exp(z).
constexpr int FORM_PREDICTOR = 100;

// g_psi's input row of one query (Eq. 7, Section 3.5) into the layer-0
// operand tile: 2 hash features a level, then omega_r; zeros to WP.
template <class S>
__device__ __forceinline__ void predictor_gather(const QueryParams& p, const QueryIn& in,
                                                 int64_t gq, bool valid, uint8_t* act, int q) {
  static_assert(S::WP >= 2 * 14 + 3, "the tensor-core predictor takes up to 14 levels");
  float v[S::WP];
#pragma unroll
  for (int c = 0; c < S::WP; ++c) v[c] = 0.f;
  if (valid) {
    const float xs[3] = {clamp01(in.x0), clamp01(in.x1), clamp01(in.x2)};
#pragma unroll
    for (int l = 0; l < 14; ++l) {
      if (l >= p.pred_levels) break;
      const float2* tab = reinterpret_cast<const float2*>(p.pred_table) + size_t(l) * (p.pred_tmask + 1u);
      const float2 e = hash_level(tab, xs, p.pred_res[l], p.pred_dense[l] != 0, p.pred_tmask);
      v[2 * l] = e.x;
      v[2 * l + 1] = e.y;
    }
    const float w0[3] = {in.w0, in.w1, in.w2};
    const float n0[3] = {p.normal[3 * gq], p.normal[3 * gq + 1], p.normal[3 * gq + 2]};
    float wr[3];
    reflect_f32_rn(w0, n0, wr);
#pragma unroll
    for (int l = 1; l <= 14; ++l)
      if (l == p.pred_levels) {
        v[2 * l] = wr[0];
        v[2 * l + 1] = wr[1];
        v[2 * l + 2] = wr[2];
      }
  }
#pragma unroll
  for (int c = 0; c < S::WP; c += 8) {
    uint4 o;
    o.x = pack_bf16x2(v[c + 0], v[c + 1]);
    o.y = pack_bf16x2(v[c + 2], v[c + 3]);
    o.z = pack_bf16x2(v[c + 4], v[c + 5]);
    o.w = pack_bf16x2(v[c + 6], v[c + 7]);
    *reinterpret_cast<uint4*>(act + kmajor_offset(q, c, S::WP)) = o;
  }
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

// Forward of 128-query tiles: TPQ threads per query (thread par of a row
// gathers the levels l with l % TPQ == par and, in the epilogues, the
// column range par of the hidden layer), all of them waiting on the MMAs of
// the tile; persistent over tiles.
template <class S, typename TT, int TPQ, int FORM = OCTA_FORM_CELL_BILINEAR>
__global__ void __launch_bounds__(NT * TPQ, 4)
    fwd_kernel(const __grid_constant__ QueryParams p) {
  constexpr int NTF = NT * TPQ;         // threads per CTA
  constexpr int HC = S::H / TPQ;        // hidden columns per thread
  static_assert(HC % 16 == 0, "epilogue column split");
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* act = smem + S::OFF_ACT;
  // staged octree: p.tree_cap nodes (sized by the launcher, at most
  // S::TREE_NODES) after the fixed part of the layout
  int2* tree_sm = p.tree_cap > 0 ? reinterpret_cast<int2*>(smem + S::OFF_TREE) : nullptr;
  const int2* tree = nullptr;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + S::OFF_BAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + S::OFF_BAR + 8);
  const uint32_t mbar = smem_addr(bar);
  const uint32_t act_sa = smem_addr(act), w_sa = smem_addr(smem);
  const int warp = threadIdx.x >> 5;
  const int q = threadIdx.x % NT, par = threadIdx.x / NT;  // row, level parity

  if (threadIdx.x == 0) mbar_init(mbar, 1);
  if (warp == 0) {
    tmem_alloc(smem_addr(tslot), S::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem = *tslot;
  // warp w reads the tensor-memory lanes of its subpartition w % 4
  const uint32_t lane_base = tmem + (static_cast<uint32_t>((warp % 4) * 32) << 16);
  uint32_t phase = 0;
  int cur = -1;
  bool failed = false;

  const WorkRange wr = work_range(p.n_tiles, p.order, p.run);
  QueryIn next = wr.begin < wr.end ? load_tile_query(p, wr.begin, q, NT) : QueryIn{};
  for (int64_t tile = wr.begin; tile < wr.end && !failed; tile = wr.next(tile)) {
    const int s = scene_of_tile(p, tile);
    const DevScene& sc = p.sc[s];
    const QueryIn in = next;
    if (wr.next(tile) < wr.end) next = load_tile_query(p, wr.next(tile), q, NT);
    __syncthreads();
    if (s != cur) {
      load_weights_bf16<S>(sc, smem, NTF);
      if constexpr (FORM != FORM_PREDICTOR)
        tree = stage_tree(p, sc, tree_sm, p.tree_cap, threadIdx.x, NTF);
      cur = s;
      __syncthreads();
    }
    const int64_t q0 = sc.q_begin + (tile - sc.tile_begin) * NT;
    const int nq = static_cast<int>(sc.q_end - q0 < NT ? sc.q_end - q0 : int64_t(NT));
    if constexpr (FORM == FORM_PREDICTOR)
      predictor_gather<S>(p, in, q0 + q, q < nq, act, q);
    else
      locate_gather_bf16<S, TT, TPQ, FORM>(p, sc, tree, in, q0 + q, q < nq, par, act, nullptr,
                                           nullptr, q, p.normal, p.disparity);
    fence_proxy_async();
    __syncthreads();

#pragma unroll 1
    for (int layer = 0; layer < S::NL; ++layer) {
      if (threadIdx.x == 0) issue_layer<S>(layer, act_sa, w_sa, tmem, mbar);
      // warp 0 reconverges before its other threads poll the mbarrier:
      // their polls would otherwise interleave with the issue
      __syncwarp();
      const bool ok = mbar_wait_bounded(mbar, phase);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      tc_fence_after_sync();
      if (layer < S::NL - 1) {
        const int c0 = par * HC;
        uint32_t r[HC];
#pragma unroll
        for (int c = 0; c < HC; c += 16)
          tmem_ld16(lane_base + c0 + c, *reinterpret_cast<uint32_t(*)[16]>(r + c));
        tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < HC; c += 8) {
          uint4 o;
          o.x = pack_relu_bf16x2(r[c + 0], r[c + 1]);
          o.y = pack_relu_bf16x2(r[c + 2], r[c + 3]);
          o.z = pack_relu_bf16x2(r[c + 4], r[c + 5]);
          o.w = pack_relu_bf16x2(r[c + 6], r[c + 7]);
          *reinterpret_cast<uint4*>(act + kmajor_offset(q, c0 + c, S::H)) = o;
        }
        fence_proxy_async();
        tc_fence_before_sync();
        __syncthreads();
      } else {
        if (par == 0) {
          uint32_t r[16];
          tmem_ld16(lane_base, r);
          tmem_wait_ld();
          if (q < nq) {
            const int64_t gq = q0 + q;
            if constexpr (FORM == FORM_PREDICTOR) {
              p.disparity_out[gq] = expf(__uint_as_float(r[0]));
            } else {
              p.rgb[3 * gq] = expf(__uint_as_float(r[0]));
              p.rgb[3 * gq + 1] = expf(__uint_as_float(r[1]));
              p.rgb[3 * gq + 2] = expf(__uint_as_float(r[2]));
            }
          }
        }
        tc_fence_before_sync();
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
// A CTA of G = 2 groups of 128 threads works on two tiles of the same scene
// at once; each group runs the per-tile pipeline below on its own shared-
// memory region, mbarrier and tensor-memory working columns, synchronising
// with named barriers.  The groups share the weights (shared memory) and the
// transposed weight gradients dW_i^T = a_i^T delta_{i+1} (tensor memory:
// rows = input features, one column per output feature), which every tile's
// MMAs accumulate into; they are zeroed with tcgen05.st and flushed to the
// FP32 weight gradient with coalesced atomics when the scene changes and at
// the end.
//   per tile: fused locate + gather into h; forward layers keeping the BF16
//   activation tiles a_1..a_NH; delta_L = d_rgb * exp(z_L); then per layer
//   dW_i^T += a_i^T delta (both read MN-major from the forward's K-major
//   tiles) and G = delta W_i (W_i read MN-major); the epilogue masks G with
//   1[a_i > 0] in place; layer 0's G = dh is scattered with float4 atomics.
// TPR (threads per row): 1 or 2 threads per tile row.  With two, a group is
// 256 threads: thread (row, half) takes the levels of parity `half` in the
// gather and the scatter and half of the columns in every epilogue (both
// halves' warps read the same tensor-memory lane quadrant), so a CTA runs 16
// warps and every per-thread chain of the tile is about half as long.
template <int F_, int WP_, int H_, int NH_, int TPR_ = 1>
struct BShape : Shape<F_, WP_, H_, NH_> {
  using B = Shape<F_, WP_, H_, NH_>;
  static constexpr int G = 2;
  static constexpr int TPR = TPR_;
  static_assert(TPR == 1 || TPR == 2, "threads per row");
  static_assert(H_ % (16 * TPR) == 0, "epilogue column split");
  static constexpr int NTG = TPR * NT;  // threads per group
  static constexpr int NTB = G * NTG;
  static constexpr uint32_t H_TILE = NT * WP_ * 2;
  static constexpr uint32_t A_TILE = NT * H_ * 2;
  static constexpr uint32_t DL_TILE = NT * NOUT * 2;
  // group region: h | a_1 .. a_NH | delta_L | slack | map bases | u.  MN-major
  // reads with M = 128 rows run past a tile narrower than 128 features into
  // the next buffer; the slack keeps the last one inside the region.
  static constexpr uint32_t GR_DL = H_TILE + NH_ * A_TILE;
  static constexpr uint32_t GR_NODE = GR_DL + DL_TILE + 2048;
  static constexpr uint32_t GR_U = GR_NODE + B::NODE_BYTES;
  // folded direction of each row, one copy per thread of the row: with two
  // threads per row, one may start the next tile's gather while the other
  // still scatters the current one
  static constexpr uint32_t GR_XCH = GR_U + TPR_ * B::U_BYTES;  // [64][4] floats (fused pass)
  static constexpr uint32_t GR_BYTES = (GR_XCH + 64 * 4 * 4 + 1023) & ~1023u;
  static constexpr uint32_t OFF_GROUP = (B::W_BYTES + 1023) & ~1023u;
  static constexpr uint32_t OFF_BAR = OFF_GROUP + G * GR_BYTES;
  // two mbarriers per group (the backward's dW^T and G MMAs), then the
  // tensor-memory address slot
  static constexpr uint32_t OFF_TREE = (OFF_BAR + 16 * G + 8 + 15) & ~15u;
  static constexpr int TREE_NODES = tree_capacity(OFF_TREE, 1);
  static constexpr size_t SMEM = OFF_TREE + 8u * TREE_NODES;
  static constexpr int WORK = WP_ > H_ ? WP_ : H_;
  static constexpr int DW0 = G * WORK;
  static constexpr int DW_COLS = H_ * NH_ + NOUT;
  static constexpr int COLS = DW0 + DW_COLS;
  static constexpr uint32_t TMEM_COLS = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128
                                        : COLS <= 256 ? 256 : 512;
  static_assert(COLS <= 512, "tensor memory");
  static_assert(DW_COLS % 16 == 0, "dW columns");
  __host__ __device__ static constexpr uint32_t off_act(int g, int i) {
    return OFF_GROUP + static_cast<uint32_t>(g) * GR_BYTES +
           (i == 0 ? 0u : H_TILE + static_cast<uint32_t>(i - 1) * A_TILE);
  }
  __host__ __device__ static constexpr uint32_t off_dl(int g) {
    return OFF_GROUP + static_cast<uint32_t>(g) * GR_BYTES + GR_DL;
  }
  __host__ __device__ static constexpr int dw_col(int i) { return DW0 + H_ * i; }
};

// Adds the dW^T accumulators of the matrices i0, i0 + di, ... below i1 to
// the scene's FP32 weight gradient and zeroes them (thread t holds row t =
// input feature t).
template <class S>
__device__ void flush_weight_grads(const DevScene& sc, uint32_t lane_addr, int i0, int i1,
                                   int di = 1) {
  const int r = threadIdx.x % NT;
  uint32_t zero[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) zero[j] = 0u;
#pragma unroll 1
  for (int i = i0; i < i1; i += di) {
    const int n_pad = S::ndim(i);
    const int in = sc.widths[i], out = sc.widths[i + 1];
    float* dW = sc.d_weights + sc.w_offset[i];
#pragma unroll 1
    for (int c = 0; c < n_pad; c += 16) {
      uint32_t v[16];
      tmem_ld16(lane_addr + S::dw_col(i) + c, v);
      tmem_wait_ld();
      tmem_st16(lane_addr + S::dw_col(i) + c, zero);
      if (r < in) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c + j < out) atomicAdd(dW + (c + j) * in + r, __uint_as_float(v[j]));
      }
    }
  }
  tmem_wait_st();
}

struct BwdParams {
  QueryParams p;
  AdamBlock a;
};

// Grid-wide barrier of a cooperative launch: arrival counter plus a
// generation word, with acquire/release ordering at GPU scope.  Thread 0 of
// each CTA arrives after a CTA barrier (so the CTA's earlier writes precede
// its release); the last arrival resets the counter and releases the next
// generation; the others acquire-load the generation until it changes.  The
// wait is bounded by timeout_ns (globaltimer); on timeout it returns false
// in every thread of the CTA.  (A volatile spin with full fences in its
// place made the compiler slow the whole fused pass down by half.)
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned expected, uint64_t timeout_ns) {
  __shared__ int ok_sm;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned gen, old;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(gen) : "l"(bar + 1) : "memory");
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(bar) : "memory");
    int ok = 1;
    if (old == expected - 1) {
      asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(bar) : "memory");
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar + 1) : "memory");
    } else {
      const uint64_t t0 = globaltimer_ns();
      for (;;) {
        unsigned g;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(bar + 1) : "memory");
        if (g != gen) break;
        if (globaltimer_ns() - t0 > timeout_ns) {
          ok = 0;
          break;
        }
        __nanosleep(256);
      }
    }
    ok_sm = ok;
  }
  __syncthreads();
  return ok_sm != 0;
}

// Block-wide FP64 sum in a fixed order (result in every thread).
__device__ __forceinline__ double block_sum_all(double v) {
  __shared__ double red[32];
  __shared__ double total;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < int(blockDim.x >> 5); ++i) t += red[i];
    total = t;
  }
  __syncthreads();
  return total;
}

__device__ __forceinline__ void adam_elem(float& pm, float& m, float& v, float g, float lr, float b1,
                                          float b2, float eps, float bc1, float bc2) {
  m = b1 * m + (1.f - b1) * g;
  v = b2 * v + (1.f - b2) * g * g;
  pm = pm - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
}

// The optimiser phase of the persistent step (all CTAs, after the fused
// pass): FP64 gradient norm from per-CTA partials, the skip / scale decision
// taken identically in every CTA (same partials, same summation order) from
// the scaler state read after the first barrier, Adam with bias correction over this
// CTA's slice (16-byte accesses where a group allows them), gradients zeroed.
__device__ __forceinline__ void persistent_adam(const AdamBlock& a, int32_t* status) {
  const uint64_t tmo = a.timeout_ns;
  const unsigned expected = gridDim.x + static_cast<unsigned>(a.extra_arrivals);
  if (!grid_barrier(a.bar, expected, tmo)) {  // every gradient is in
    if (threadIdx.x == 0 && status) atomicOr(status, OCTA_STATUS_TIMEOUT);
    return;
  }
  // the scaler state of this step: every CTA reads it here, between the two
  // barriers, and CTA 0 writes the new state only after the second one
  octa_scaler s0;
  {
    const volatile octa_scaler* vs = a.scaler;
    s0.scale = vs->scale;
    s0.good_steps = vs->good_steps;
    s0.growth_interval = vs->growth_interval;
    s0.step = vs->step;
    s0.n_skipped = vs->n_skipped;
  }
  const float inv_s = 1.f / s0.scale;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const int64_t first = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  double acc = 0.0;
  for (int gi = 0; gi < a.n_groups; ++gi) {
    const octa_param_group& G = a.g[gi];
    int64_t done = 0;
    if (a.vec4[gi]) {
      const float4* g4 = reinterpret_cast<const float4*>(G.grad);
      const int64_t n4 = G.n / 4;
      constexpr int UN = 8;  // loads in flight per thread
      for (int64_t i0 = first; i0 < n4; i0 += UN * stride) {
        float4 g[UN];
#pragma unroll
        for (int u = 0; u < UN; ++u) {
          const int64_t i = i0 + u * stride;
          g[u] = i < n4 ? __ldcg(g4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        acc += sum_sq4_batch(g, inv_s);
      }
      done = n4 * 4;
    }
    for (int64_t i = done + first; i < G.n; i += stride) {
      const double v = double(__ldcg(G.grad + i) * inv_s);
      acc += v * v;
    }
  }
  acc = block_sum_all(acc);
  if (threadIdx.x == 0) a.partials[blockIdx.x] = acc;
  if (!grid_barrier(a.bar, expected, tmo)) {
    if (threadIdx.x == 0 && status) atomicOr(status, OCTA_STATUS_TIMEOUT);
    return;
  }
  double part = 0.0;  // thread t takes partials t, t + blockDim, ...: fixed order
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) part += __ldcg(a.partials + b);
  const double total = block_sum_all(part);
  const bool skip = !isfinite(total);
  const int32_t t_new = s0.step + (skip ? 0 : 1);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    octa_scaler* sc = a.scaler;
    sc->inv_scale_used = inv_s;
    sc->grad_norm = sqrt(total);
    if (skip) {
      sc->skipped = 1;
      sc->n_skipped = s0.n_skipped + 1;
      if (s0.growth_interval > 0) {
        sc->scale = s0.scale * 0.5f;
        sc->good_steps = 0;
      }
    } else {
      sc->skipped = 0;
      sc->step = t_new;
      int good = s0.good_steps + 1;
      float scale = s0.scale;
      if (s0.growth_interval > 0 && good >= s0.growth_interval) {
        scale *= 2.f;
        good = 0;
      }
      sc->good_steps = s0.growth_interval > 0 ? good : s0.good_steps;
      sc->scale = scale;
    }
  }
  __shared__ float bc[2];
  if (threadIdx.x == 0) {
    bc[0] = skip ? 1.f : adam_bias_correction(a.beta1, t_new);
    bc[1] = skip ? 1.f : adam_bias_correction(a.beta2, t_new);
  }
  __syncthreads();
  const float bc1 = bc[0], bc2 = bc[1];
  const float b1 = a.beta1, b2 = a.beta2, eps = a.eps;
  for (int gi = 0; gi < a.n_groups; ++gi) {
    const octa_param_group& G = a.g[gi];
    const float lr = G.lr;
    int64_t done = 0;
    if (a.vec4[gi]) {
      const int64_t n4 = G.n / 4;
      float4* P = reinterpret_cast<float4*>(G.param);
      float4* Gr = reinterpret_cast<float4*>(G.grad);
      float4* M = reinterpret_cast<float4*>(G.m);
      float4* V = reinterpret_cast<float4*>(G.v);
      // two elements (float4) per iteration, all their loads issued before
      // any store, so each thread keeps eight 16-byte loads in flight
      auto finish = [&](int64_t i, float4 g, float4 pm, float4 m, float4 v) {
        adam_elem(pm.x, m.x, v.x, g.x * inv_s, lr, b1, b2, eps, bc1, bc2);
        adam_elem(pm.y, m.y, v.y, g.y * inv_s, lr, b1, b2, eps, bc1, bc2);
        adam_elem(pm.z, m.z, v.z, g.z * inv_s, lr, b1, b2, eps, bc1, bc2);
        adam_elem(pm.w, m.w, v.w, g.w * inv_s, lr, b1, b2, eps, bc1, bc2);
        P[i] = pm;
        M[i] = m;
        V[i] = v;
        if (G.work) {
          if (G.work_dtype == OCTA_F16) {
            __half2* w = reinterpret_cast<__half2*>(G.work) + 2 * i;
            w[0] = __floats2half2_rn(pm.x, pm.y);
            w[1] = __floats2half2_rn(pm.z, pm.w);
          } else {
            __nv_bfloat162* w = reinterpret_cast<__nv_bfloat162*>(G.work) + 2 * i;
            w[0] = __floats2bfloat162_rn(pm.x, pm.y);
            w[1] = __floats2bfloat162_rn(pm.z, pm.w);
          }
        }
      };
      // UB elements per iteration, all their loads issued before any store
      constexpr int UB = 4;
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int64_t i0 = first; i0 < n4; i0 += UB * stride) {
        float4 g[UB], pm[UB], m[UB], v[UB];
#pragma unroll
        for (int u = 0; u < UB; ++u) {
          const int64_t i = i0 + u * stride;
          const bool in = i < n4;
          g[u] = in ? __ldcg(Gr + i) : z4;
          pm[u] = in && !skip ? P[i] : z4;
          m[u] = in && !skip ? M[i] : z4;
          v[u] = in && !skip ? V[i] : z4;
        }
#pragma unroll
        for (int u = 0; u < UB; ++u) {
          const int64_t i = i0 + u * stride;
          if (i >= n4) break;
          Gr[i] = z4;
          if (!skip) finish(i, g[u], pm[u], m[u], v[u]);
        }
      }
      done = n4 * 4;
    }
    for (int64_t i = done + first; i < G.n; i += stride) {
      const float g = __ldcg(G.grad + i) * inv_s;
      G.grad[i] = 0.f;
      if (skip) continue;
      float pm = G.param[i], m = G.m[i], v = G.v[i];
      adam_elem(pm, m, v, g, lr, b1, b2, eps, bc1, bc2);
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

// Loss partials of a fused training pass: every thread's FP64 sum of r^2 for
// the current scene is added to loss[s] / (3 n_s) (one atomic per CTA).
__device__ __forceinline__ void flush_loss(double& acc, double* loss, int64_t n_pairs) {
  __shared__ double red[16];
  double v = acc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < int(blockDim.x >> 5); ++i) t += red[i];
    atomicAdd(loss, t / (3.0 * double(n_pairs)));
  }
  __syncthreads();
  acc = 0.0;
}

// TRAIN = false: gradients of sum(d_rgb . L_hat) for the given d_rgb.
// TRAIN = true: the fused training pass over pairs; a tile holds 64 pairs,
// rows 0..63 their primary queries and rows 64..127 their secondary queries,
// and the Eq. 14 gradient of every pair is formed in the tile from the two
// radiances (only the loss value leaves the CTA, as FP64 partials).
// PERSIST (with TRAIN, cooperative launch): after the fused pass the same
// launch applies Adam to every parameter group (persistent_adam).
// FORMS: the kernel also serves the full and shifted query forms (scenes in
// the cell form alone launch the FORMS = false instance, free of their code).
// PRED: the backward of the disparity predictor g_psi instead of the
// decoder (input row = hash encoding and omega_r, one output channel
// d = exp(z) whose upstream gradient is p.d_rgb[q] (one float a query), and
// the input gradient's hash columns scattered into p.pred_dtable).
template <class S, typename TT, bool TRAIN, bool PERSIST = false, bool FORMS = true,
          bool PRED = false>
__global__ void __launch_bounds__(S::NTB, 1) bwd_kernel(const __grid_constant__ BwdParams bp) {
  static_assert(!PRED || (!TRAIN && !FORMS && S::TPR == 1), "the predictor's backward");
  const QueryParams& p = bp.p;
  constexpr int H = S::H, NL = S::NL, TPR = S::TPR, NTG = S::NTG;
  static_assert(!FORMS || TPR == 1, "the full and shifted forms run one thread per row");
  constexpr int ROWS = TRAIN ? NT / 2 : NT;  // pairs or queries per tile
  constexpr int HC = H / TPR;                // epilogue columns of one thread
  extern __shared__ __align__(1024) uint8_t smem[];
  const int g = threadIdx.x / NTG, t = threadIdx.x % NT, warp = threadIdx.x >> 5;
  const int half = (threadIdx.x % NTG) / NT;  // column half / level parity of the row
  uint8_t* gbase = smem + S::OFF_GROUP + g * S::GR_BYTES;
  int* base_sm = reinterpret_cast<int*>(gbase + S::GR_NODE);  // map base per level
  float* u_sm = reinterpret_cast<float*>(gbase + S::GR_U) + half * 2 * NT;  // this thread's copy
  int2* tree_sm = S::TREE_NODES > 0 ? reinterpret_cast<int2*>(smem + S::OFF_TREE) : nullptr;
  const int2* tree = nullptr;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S::OFF_BAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + S::OFF_BAR + 16 * S::G);
  __shared__ int abort_flag;
  const uint32_t mbar = smem_addr(bars + g);
  const uint32_t mbar2 = smem_addr(bars + S::G + g);  // the backward's G MMAs
  const uint32_t base_sa = smem_addr(smem);
  const uint32_t dl_sa = base_sa + S::off_dl(g);
  const int gbar = 1 + g;                         // named barrier of this group
  const int xbar = TPR == 1 ? gbar : 1 + S::G + g;  // its half-0 threads alone
  const bool lead = t == 0 && half == 0;           // issues the group's MMAs

  if (threadIdx.x == 0) {
    for (int i = 0; i < 2 * S::G; ++i) mbar_init(smem_addr(bars + i), 1);
    abort_flag = 0;
  }
  if (warp == 0) {
    tmem_alloc(smem_addr(tslot), S::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t lane_addr = tmem + (static_cast<uint32_t>((warp % 4) * 32) << 16);
  const uint32_t work = tmem + static_cast<uint32_t>(g * S::WORK);           // MMA D address
  const uint32_t lane_work = lane_addr + static_cast<uint32_t>(g * S::WORK);  // epilogue loads
  if (g == 0) {  // zero the shared dW^T accumulators (16-column chunks split by half)
    uint32_t zero[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) zero[j] = 0u;
#pragma unroll 1
    for (int c = 16 * half; c < S::DW_COLS; c += 16 * TPR) tmem_st16(lane_addr + S::DW0 + c, zero);
    tmem_wait_st();
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  uint32_t phase = 0, phase2 = 0;
  int cur = -1;
  double loss_acc = 0.0;
  const float lscale = TRAIN ? (p.scaler ? p.scaler->scale : 1.f) : 1.f;
  float* xch = reinterpret_cast<float*>(gbase + S::GR_XCH);  // radiance exchange (TRAIN)
  // the persistent step's bound on every wait (its test hook makes the
  // first tile's first mbarrier wait run out: no MMA is issued for it)
  const uint64_t wait_ns = PERSIST ? bp.a.timeout_ns : 1000000000ull;
  bool skip_hook = PERSIST && bp.a.skip_first_mma != 0;
  // matrices whose dW^T this thread's set (group, half) flushes
  const int flush_set = g * TPR + half;
  constexpr int FLUSH_SETS = S::G * TPR;

  // query (pair) row of this thread in a tile, and which pair array it reads
  const int row = TRAIN ? (t & (ROWS - 1)) : t;
  const bool primary = !TRAIN || t < ROWS;
  const float* xs = primary ? p.x : p.x2;
  const float* ws = primary ? p.omega : p.omega2;
  const float* nrm = primary ? p.normal : p.normal2;  // the shifted form's inputs
  const float* dsp = primary ? p.disparity : p.disparity2;
  float* d_dsp = primary ? p.d_disparity : p.d_disparity2;  // its dL/dd out (nullable)
  auto item_query = [&](int64_t item) {  // this thread's query of an item, prefetched
    int s = 0;
    while (s + 1 < p.n_scenes && item >= p.item_begin[s + 1]) ++s;
    const DevScene& sc = p.sc[s];
    const int64_t gq = sc.q_begin + (2 * (item - p.item_begin[s]) + g) * ROWS + row;
    return load_query(xs, ws, gq, gq < sc.q_end);
  };
  // Cell form: the two groups run half a tile apart (group 1 starts its
  // first tile of a scene when group 0 has finished that tile's forward),
  // so that one group's gather and scatter (memory) overlap the other's
  // decoder (tensor cores); beyond that they synchronise only at scene
  // changes and at the end.  The full and shifted forms, whose gather and
  // scatter dominate, keep the groups in step (a CTA barrier per item:
  // their gathers overlap each other).  After an abort both groups keep
  // stepping through the items without work, so every barrier sees both.
  constexpr bool SKEW = !FORMS;
  constexpr int SKEW_BAR = 1 + 2 * S::G;
  bool skew_pending = false;
  const WorkRange wr = work_range(p.n_items, p.order, p.run);
  QueryIn next = wr.begin < wr.end ? item_query(wr.begin) : QueryIn{};
  for (int64_t item = wr.begin; item < wr.end; item = wr.next(item)) {
    int s = 0;
    while (s + 1 < p.n_scenes && item >= p.item_begin[s + 1]) ++s;
    const DevScene& sc = p.sc[s];
    const QueryIn in = next;
    if (wr.next(item) < wr.end) next = item_query(wr.next(item));
    if constexpr (!SKEW) {
      tc_fence_before_sync();
      __syncthreads();
    }
    if (s != cur) {
      tc_fence_before_sync();
      __syncthreads();  // both groups are done with the previous scene
      tc_fence_after_sync();
      if (cur >= 0 && !abort_flag) {
        flush_weight_grads<S>(p.sc[cur], lane_addr, flush_set, NL, FLUSH_SETS);
        tc_fence_before_sync();
        if (TRAIN) flush_loss(loss_acc, p.loss + cur, p.sc[cur].norm_pairs);
      }
      for (int l = 0; l < S::NL; ++l) {  // weights, all threads
        const int K = S::kdim(l), N = S::ndim(l);
        const int in = sc.widths[l], out = sc.widths[l + 1];
        const __nv_bfloat16* Wg = static_cast<const __nv_bfloat16*>(sc.weights);
        __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(smem + S::w_off(l));
        for (int i = threadIdx.x; i < N * K; i += S::NTB) {
          const int n = i / K, k = i % K;
          dst[kmajor_offset(n, k, K) / 2] =
              (n < out && k < in) ? Wg[sc.w_offset[l] + n * in + k] : __float2bfloat16_rn(0.f);
        }
      }
      if constexpr (!PRED) tree = stage_tree(p, sc, tree_sm, S::TREE_NODES, threadIdx.x, S::NTB);
      cur = s;
      __syncthreads();
      skew_pending = SKEW;
    }
    if (g == 1 && skew_pending) {  // group 0's first tile of the scene is past its forward
      named_sync(SKEW_BAR, S::NTB);
      skew_pending = false;
    }
    const int64_t tiles_s = (sc.q_end - sc.q_begin + ROWS - 1) / ROWS;
    const int64_t tile_s = 2 * (item - p.item_begin[s]) + g;
    if (tile_s >= tiles_s) continue;  // odd tile count: this group idles
    const int64_t q0 = sc.q_begin + tile_s * ROWS;  // first query (pair) of the tile
    const int nq = static_cast<int>(sc.q_end - q0 < ROWS ? sc.q_end - q0 : int64_t(ROWS));
    const bool valid = row < nq;
    const int64_t gq = q0 + row;
    const bool full = FORMS && sc.query_form == OCTA_FORM_TRILINEAR_VERTEX;  // uniform over the CTA
    const bool shifted = FORMS && sc.query_form == OCTA_FORM_SHIFTED;
    const QueryIn& qry = in;  // the layer loops below reuse the name in
    if constexpr (FORMS) {
      if (full)
        locate_gather_bf16<S, TT, 1, OCTA_FORM_TRILINEAR_VERTEX>(
            p, sc, tree, in, gq, valid, 0, smem + S::off_act(g, 0), nullptr, nullptr, t);
      else if (shifted)
        locate_gather_bf16<S, TT, 1, OCTA_FORM_SHIFTED>(
            p, sc, tree, in, gq, valid, 0, smem + S::off_act(g, 0), nullptr, nullptr, t, nrm, dsp);
      else
        locate_gather_bf16<S, TT>(p, sc, tree, in, gq, valid, 0, smem + S::off_act(g, 0), base_sm,
                                  u_sm, t);
    } else if constexpr (PRED) {
      predictor_gather<S>(p, in, gq, valid, smem + S::off_act(g, 0), t);
    } else {
      locate_gather_bf16<S, TT, TPR>(p, sc, tree, in, gq, valid, half, smem + S::off_act(g, 0),
                                     base_sm, u_sm, t);
    }
    fence_proxy_async();
    // the loss epilogue's per-pair inputs (E, w) or the backward's d_rgb,
    // loaded now so that their latency passes under the forward
    float in3a[3] = {0.f, 0.f, 0.f}, in3b[3] = {0.f, 0.f, 0.f};
    if (valid && half == 0) {
      if (TRAIN) {
        if (primary) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            in3a[c] = __ldcs(p.E + 3 * gq + c);
            in3b[c] = __ldcs(p.w + 3 * gq + c);
          }
        }
      } else if constexpr (PRED) {
        in3a[0] = __ldcs(p.d_rgb + gq);  // the output channel's gradient
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) in3a[c] = __ldcs(p.d_rgb + 3 * gq + c);
      }
    }
    // the previous tile's tensor-memory reads come before this tile's MMAs;
    // an abort (a bounded wait that ran out, in any group) is read here by
    // the whole group at once: the group then steps through its remaining
    // items without MMAs, keeping the skew barrier's count
    tc_fence_before_sync();
    if (named_sync_or(gbar, NTG, abort_flag != 0)) {
      if (g == 0 && skew_pending) {
        named_arrive(SKEW_BAR, S::NTB);
        skew_pending = false;
      }
      continue;
    }

    bool failed = false;
    // ---- forward, keeping a_1 .. a_NH and delta_L
#pragma unroll 1
    for (int layer = 0; layer < NL; ++layer) {
      if (lead && !(skip_hook && layer == 0))
        issue_layer<S>(layer, base_sa + S::off_act(g, layer), base_sa, work, mbar);
      // the issuing warp reconverges before its other threads poll the
      // mbarrier: their polls would otherwise interleave with the issue
      __syncwarp();
      skip_hook = false;
      // a wait that ran out is reported at the barrier that closes the
      // epilogue (the epilogue then reads undefined accumulators, unused)
      const bool ok = mbar_wait_bounded(mbar, phase, wait_ns);
      phase ^= 1u;
      tc_fence_after_sync();
      if (layer < NL - 1) {
        const int c0 = half * HC;
        uint32_t r[HC];
#pragma unroll
        for (int c = 0; c < HC; c += 16)
          tmem_ld16(lane_work + c0 + c, *reinterpret_cast<uint32_t(*)[16]>(r + c));
        tmem_wait_ld();
        uint8_t* dst = smem + S::off_act(g, layer + 1);
#pragma unroll
        for (int c = 0; c < HC; c += 8) {
          uint4 o;
          o.x = pack_relu_bf16x2(r[c + 0], r[c + 1]);
          o.y = pack_relu_bf16x2(r[c + 2], r[c + 3]);
          o.z = pack_relu_bf16x2(r[c + 4], r[c + 5]);
          o.w = pack_relu_bf16x2(r[c + 6], r[c + 7]);
          *reinterpret_cast<uint4*>(dst + kmajor_offset(t, c0 + c, H)) = o;
        }
      } else if (half == 0) {  // warp-uniform: the last layer's 3 outputs
        uint32_t r[16];
        tmem_ld16(lane_work, r);
        tmem_wait_ld();
        const float L0 = expf(__uint_as_float(r[0]));
        const float L1 = expf(__uint_as_float(r[1]));
        const float L2 = expf(__uint_as_float(r[2]));
        float d0 = 0.f, d1 = 0.f, d2 = 0.f;
        if (!TRAIN) {
          d0 = in3a[0];
          d1 = in3a[1];
          d2 = in3a[2];
        } else {
          // Eq. 14 with the one-sample target of Eq. 3, per pair and channel:
          // T = E + w L_s, r = (L_p - T) / (L_p + T + eps) (normaliser
          // detached), d/dL_p = S 2 r / (3 n den), d/dL_s = -w d/dL_p.
          if (!primary) {
            xch[4 * row] = L0;
            xch[4 * row + 1] = L1;
            xch[4 * row + 2] = L2;
          }
          named_sync(xbar, NT);
          if (primary && valid) {
            const float Ls[3] = {xch[4 * row], xch[4 * row + 1], xch[4 * row + 2]};
            const float Lp[3] = {L0, L1, L2};
            const float n3 = 3.f * static_cast<float>(sc.norm_pairs);
            float dp[3], ds[3], r2 = 0.f;  // the pair's three r^2 in binary32
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const float ww = in3b[c];
              const float T = in3a[c] + ww * Ls[c];
              const float den = Lp[c] + T + p.eps;
              const float rr = (Lp[c] - T) / den;
              r2 = fmaf(rr, rr, r2);
              dp[c] = 2.f * lscale * rr / (n3 * den);
              ds[c] = p.rhs_grad ? -dp[c] * ww : 0.f;
            }
            loss_acc += double(r2);  // one FP64 add per pair
            d0 = dp[0];
            d1 = dp[1];
            d2 = dp[2];
            xch[4 * row] = ds[0];
            xch[4 * row + 1] = ds[1];
            xch[4 * row + 2] = ds[2];
          }
          named_sync(xbar, NT);
          if (!primary && valid) {
            d0 = xch[4 * row];
            d1 = xch[4 * row + 1];
            d2 = xch[4 * row + 2];
          }
        }
        // delta_L = d_rgb * exp(z_L): the derivative of exp is exp
        uint8_t* dst = smem + S::off_dl(g);
        uint4 o0, o1;
        o0.x = pack_bf16x2(d0 * L0, d1 * L1);
        o0.y = pack_bf16x2(d2 * L2, 0.f);
        o0.z = o0.w = 0u;
        o1.x = o1.y = o1.z = o1.w = 0u;
        *reinterpret_cast<uint4*>(dst + kmajor_offset(t, 0, NOUT)) = o0;
        *reinterpret_cast<uint4*>(dst + kmajor_offset(t, 8, NOUT)) = o1;
      }
      fence_proxy_async();
      tc_fence_before_sync();
      if (named_sync_or(gbar, NTG, !ok)) {
        failed = true;
        break;
      }
    }
    if (g == 0 && skew_pending) {  // releases group 1 (also after a failed forward)
      named_arrive(SKEW_BAR, S::NTB);
      skew_pending = false;
    }

    // ---- backward through the decoder
#pragma unroll 1
    for (int i = NL - 1; i >= 0 && !failed; --i) {
      const int out = S::ndim(i), in = S::kdim(i);
      const uint32_t d_sa = i == NL - 1 ? dl_sa : base_sa + S::off_act(g, i + 1);
      const int dk = out;  // row length of the delta tile
      if (lead) {
        tc_fence_after_sync();
        // G = delta_{i+1} W_i first (M = 128 queries, N = in, K = out): the
        // epilogue needs it; then dW_i^T += a_i^T delta_{i+1} (M = 128 input
        // features, N = out, K = 128 queries), which runs under the epilogue
        const uint32_t ig = idesc_bf16(128, in, 0, 1);
        const uint32_t w_sa = base_sa + S::w_off(i);
#pragma unroll 1
        for (int ko = 0; ko < out; ko += 16)
          mma_bf16(work, kmajor_desc(d_sa, ko, dk), mnmajor_desc(w_sa, ko, in), ig,
                   ko > 0 ? 1u : 0u);
        mma_commit(mbar2);
        const uint32_t act_sa = base_sa + S::off_act(g, i);
        const uint32_t idw = idesc_bf16(128, out, 1, 1);
#pragma unroll 1
        for (int kq = 0; kq < NT; kq += 16)
          mma_bf16(tmem + S::dw_col(i), mnmajor_desc(act_sa, kq, in), mnmajor_desc(d_sa, kq, dk),
                   idw, 1u);
        mma_commit(mbar);
      }
      __syncwarp();  // as in the forward
      bool ok = mbar_wait_bounded(mbar2, phase2, wait_ns);  // G
      phase2 ^= 1u;
      if (i > 0) {
        // delta_i = G * 1[a_i > 0], formed while dW_i^T still reads a_i and
        // written over a_i once it has completed; a wait that ran out is
        // reported at the closing barrier
        tc_fence_after_sync();
        const int c0 = half * HC;
        uint32_t r[HC];
#pragma unroll
        for (int c = 0; c < HC; c += 16)
          tmem_ld16(lane_work + c0 + c, *reinterpret_cast<uint32_t(*)[16]>(r + c));
        tmem_wait_ld();
        uint8_t* act = smem + S::off_act(g, i);
        uint4 dv[HC / 8];
#pragma unroll
        for (int c = 0; c < HC; c += 8) {
          const uint4 a = *reinterpret_cast<const uint4*>(act + kmajor_offset(t, c0 + c, H));
          const uint32_t av[4] = {a.x, a.y, a.z, a.w};
          uint32_t ov[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            // a ReLU output in bf16 is > 0 iff its magnitude bits are non-zero
            const float g0 = (av[j] & 0x7FFFu) ? __uint_as_float(r[c + 2 * j]) : 0.f;
            const float g1 = ((av[j] >> 16) & 0x7FFFu) ? __uint_as_float(r[c + 2 * j + 1]) : 0.f;
            ov[j] = pack_bf16x2(g0, g1);
          }
          dv[c / 8] = make_uint4(ov[0], ov[1], ov[2], ov[3]);
        }
        ok = mbar_wait_bounded(mbar, phase, wait_ns) && ok;  // dW_i^T
        phase ^= 1u;
#pragma unroll
        for (int c = 0; c < HC; c += 8)
          *reinterpret_cast<uint4*>(act + kmajor_offset(t, c0 + c, H)) = dv[c / 8];
        fence_proxy_async();
        tc_fence_before_sync();
        if (named_sync_or(gbar, NTG, !ok)) {
          failed = true;
          break;
        }
        continue;
      }
      // layer 0: both MMAs complete before the input gradient leaves (the
      // full and shifted forms write dh over h and a_1, and the next tile's
      // gather overwrites h)
      ok = mbar_wait_bounded(mbar, phase, wait_ns) && ok;
      phase ^= 1u;
      if (named_sync_or(gbar, NTG, !ok)) {
        failed = true;
        break;
      }
      tc_fence_after_sync();
      if (PRED) {
        // G = the gradient of g_psi's input row: each level's two hash
        // features go to the 8 vertices of x's cell (trilinear weights)
        uint32_t r[32];
        tmem_ld16(lane_work, *reinterpret_cast<uint32_t(*)[16]>(r));
        tmem_ld16(lane_work + 16, *reinterpret_cast<uint32_t(*)[16]>(r + 16));
        tmem_wait_ld();
        tc_fence_before_sync();
        if (valid) {
          const float xs[3] = {clamp01(qry.x0), clamp01(qry.x1), clamp01(qry.x2)};
#pragma unroll
          for (int l = 0; l < 14; ++l) {
            if (l >= p.pred_levels) break;
            float2* dtab = reinterpret_cast<float2*>(p.pred_dtable) + size_t(l) * (p.pred_tmask + 1u);
            hash_level_scatter(dtab, xs, p.pred_res[l], p.pred_dense[l] != 0, p.pred_tmask,
                               __uint_as_float(r[2 * l]), __uint_as_float(r[2 * l + 1]));
          }
        }
      } else if (!full && !shifted) {
        // dh = G; scatter w_k * dh_l into the four texels of each present
        // level of this thread's parity
        constexpr int KO = (S::KPAD + TPR - 1) / TPR;
        uint32_t r[KO][S::F];
#pragma unroll
        for (int o = 0; o < KO; ++o)
          if (o * TPR + half < S::KPAD)
            tmem_ld_cols<S::F>(lane_work + (o * TPR + half) * S::F, r[o]);
        tmem_wait_ld();
        tc_fence_before_sync();
#pragma unroll
        for (int o = 0; o < KO; ++o) {
          const int l = o * TPR + half;
          if (l >= S::KPAD) continue;
          const int mo = base_sm[l * NT + t];
          if (mo < 0) continue;
          const Footprint fp = footprint(u_sm[t], u_sm[NT + t], sc.R[l]);
#pragma unroll
          for (int c4 = 0; c4 < S::F / 4; ++c4) {
            const float g0 = __uint_as_float(r[o][4 * c4 + 0]);
            const float g1 = __uint_as_float(r[o][4 * c4 + 1]);
            const float g2 = __uint_as_float(r[o][4 * c4 + 2]);
            const float g3 = __uint_as_float(r[o][4 * c4 + 3]);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const float w = fp.w[k];
              float4* dst =
                  reinterpret_cast<float4*>(sc.d_tables + (int64_t(mo) + fp.idx[k]) * S::F) + c4;
              atomicAdd(dst, make_float4(w * g0, w * g1, w * g2, w * g3));
            }
          }
        }
      } else {
        // full and shifted forms (one thread per row): the row's dh is copied
        // once into shared memory -- the group's h, delta_1 and delta_2
        // tiles, whose MMAs have all completed -- and read there level by
        // level (the level loops stay rolled; no register copy of the row)
        constexpr int DHS = S::WP + 4;  // row stride (floats): conflict-free float4 rows
        static_assert(NT * DHS * 4 <= S::H_TILE + 2 * S::A_TILE, "dh rows in h, a_1, a_2");
        float* dh = reinterpret_cast<float*>(smem + S::off_act(g, 0)) + t * DHS;
#pragma unroll
        for (int c = 0; c < S::WP; c += 16) {
          uint32_t r[16];
          tmem_ld16(lane_work + c, r);
          tmem_wait_ld();
#pragma unroll
          for (int k = 0; k < 16; k += 4)
            *reinterpret_cast<uint4*>(dh + c + k) = make_uint4(r[k], r[k + 1], r[k + 2], r[k + 3]);
        }
        tc_fence_before_sync();
        if (full) {  // the 24 vertices of each level (Eq. 10 with Eq. 6)
          if (valid) {
            float ux, uy;
            octa_fold(qry.w0, qry.w1, qry.w2, ux, uy);
            const float xs[3] = {clamp01(qry.x0), clamp01(qry.x1), clamp01(qry.x2)};
            visit_full_levels<S::KPAD, false>(p, sc, tree, xs, ux, uy,
                                              [&](int l, const FullLevel& fl) {
#pragma unroll
              for (int c4 = 0; c4 < S::F / 4; ++c4) {
                const float g0 = dh[l * S::F + 4 * c4 + 0];
                const float g1 = dh[l * S::F + 4 * c4 + 1];
                const float g2 = dh[l * S::F + 4 * c4 + 2];
                const float g3 = dh[l * S::F + 4 * c4 + 3];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                  if (fl.base[j] < 0) continue;
#pragma unroll
                  for (int k = 0; k < 3; ++k) {
                    const float w = fl.wn[j] * fl.b[k];
                    float4* dst = reinterpret_cast<float4*>(
                                      sc.d_tables + int64_t(fl.base[j] + fl.vidx[k]) * S::F) + c4;
                    atomicAdd(dst, make_float4(w * g0, w * g1, w * g2, w * g3));
                  }
                }
              }
            });
          }
        } else {  // shifted: each cell's own triangle (Eq. 7-9 with Eq. 6, 10)
          if (valid) {
            const float xs[3] = {clamp01(qry.x0), clamp01(qry.x1), clamp01(qry.x2)};
            const float w0[3] = {qry.w0, qry.w1, qry.w2};
            const float n0[3] = {nrm[3 * gq], nrm[3 * gq + 1], nrm[3 * gq + 2]};
            float wr[3];
            reflect_f32_rn(w0, n0, wr);
            const float disp = dsp[gq];
            // dL/dd = sum over levels, cells and vertices of
            // wn_j (d b_k / d d) <t_jk, dh_l> (the texels read again)
            float dd = 0.f;
            visit_cell_levels<S::KPAD, false>(p, sc, tree, xs,
                                              [&](int l, const int (&c0)[3], FullLevel& fl) {
#pragma unroll 1
              for (int j = 0; j < 8; ++j) {
                if (fl.base[j] < 0) continue;
                float db[3];
                if (d_dsp)
                  shifted_cell_vertex_dd(sc, xs, wr, disp, l, c0, j, fl, db);
                else
                  shifted_cell_vertex(sc, xs, wr, disp, l, c0, j, fl);
#pragma unroll
                for (int c4 = 0; c4 < S::F / 4; ++c4) {
                  const float g0 = dh[l * S::F + 4 * c4 + 0];
                  const float g1 = dh[l * S::F + 4 * c4 + 1];
                  const float g2 = dh[l * S::F + 4 * c4 + 2];
                  const float g3 = dh[l * S::F + 4 * c4 + 3];
#pragma unroll
                  for (int k = 0; k < 3; ++k) {
                    const float w = fl.wn[j] * fl.b[k];
                    float4* dst = reinterpret_cast<float4*>(
                                      sc.d_tables + int64_t(fl.base[j] + fl.vidx[k]) * S::F) + c4;
                    atomicAdd(dst, make_float4(w * g0, w * g1, w * g2, w * g3));
                  }
                }
                if (d_dsp) {
#pragma unroll
                  for (int k = 0; k < 3; ++k) {
                    TexelRaw<TT, S::F> tx;
                    tx.load(sc.tables, uint32_t(fl.base[j] + fl.vidx[k]));
                    float dot = 0.f;
#pragma unroll
                    for (int f = 0; f < S::F; ++f) dot = fmaf(tx.get(f), dh[l * S::F + f], dot);
                    dd = fmaf(fl.wn[j] * db[k], dot, dd);
                  }
                }
              }
            });
            if (d_dsp) d_dsp[gq] = dd;
          }
        }
      }
    }
    if (failed) {  // read by every group at its next post-gather barrier
      abort_flag = 1;
      if (p.status) atomicOr(p.status, OCTA_STATUS_TIMEOUT);
    }
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  if (cur >= 0 && !abort_flag) {
    flush_weight_grads<S>(p.sc[cur], lane_addr, flush_set, NL, FLUSH_SETS);
    if (TRAIN) flush_loss(loss_acc, p.loss + cur, p.sc[cur].norm_pairs);
  }
  tc_fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, S::TMEM_COLS);
  if constexpr (PERSIST) {
    if (!abort_flag) persistent_adam(bp.a, p.status);
  }
}

namespace {

template <class S, typename TT, int TPQ, int FORM = OCTA_FORM_CELL_BILINEAR>
int launch_fwd_tpq(const QueryParams& p, const octa_tuning& tu, cudaStream_t stream) {
  auto kern = fwd_kernel<S, TT, TPQ, FORM>;
  // the staged tree holds the largest scene that fits S::TREE_NODES, in
  // granules of 16 nodes; shared memory past it can stay L1 cache
  int nodes = 0;
  if constexpr (FORM != FORM_PREDICTOR)
    for (int s = 0; s < p.n_scenes; ++s)
      if (p.sc[s].num_nodes <= S::TREE_NODES) nodes = std::max(nodes, p.sc[s].num_nodes);
  const int cap = std::min(S::TREE_NODES, (nodes + 15) & ~15);
  const size_t smem = S::OFF_TREE + 8u * static_cast<size_t>(cap);
  int per_sm = 0;
  int rc = launch_cache().get(reinterpret_cast<const void*>(kern), smem, NT * TPQ,
                              static_cast<int>(S::TMEM_COLS), &per_sm, carve_mode(tu),
                              tu.fwd_ctas_per_sm);
  if (rc) return rc;
  per_sm = apply_cap(per_sm, tu.fwd_ctas_per_sm);
  QueryParams pp = p;
  pp.order = tu.fwd_order == 1 ? 1 : 0;
  pp.run = tu.fwd_run > 1 ? tu.fwd_run : 1;
  pp.tree_cap = cap;
  const int64_t grid = std::min<int64_t>(p.n_tiles, int64_t(per_sm) * device_sm_count());
  kern<<<static_cast<unsigned>(grid), NT * TPQ, smem, stream>>>(pp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(OCTA_ECUDA, "tc fwd launch: %s", cudaGetErrorString(e));
  return OCTA_OK;
}

template <class S, typename TT>
int launch_fwd(const QueryParams& p, cudaStream_t stream) {
  if (p.n_tiles == 0) return OCTA_OK;
  const octa_tuning tu = tuning_snapshot();
  if (p.sc[0].query_form == OCTA_FORM_TRILINEAR_VERTEX)  // all scenes of a call share it
    return launch_fwd_tpq<S, TT, 1, OCTA_FORM_TRILINEAR_VERTEX>(p, tu, stream);
  if (p.sc[0].query_form == OCTA_FORM_SHIFTED)
    return launch_fwd_tpq<S, TT, 1, OCTA_FORM_SHIFTED>(p, tu, stream);
  return tu.fwd_threads_per_query == 2 && p.n_attrs == 0 ? launch_fwd_tpq<S, TT, 2>(p, tu, stream)
                                                         : launch_fwd_tpq<S, TT, 1>(p, tu, stream);
}

template <class S, typename TT, bool TRAIN, bool PERSIST, bool FORMS, bool PRED = false>
int launch_bwd(const QueryParams& p0, const AdamBlock* adam, cudaStream_t stream) {
  if (p0.n_tiles == 0 && !PERSIST) return OCTA_OK;
  constexpr int ROWS = TRAIN ? NT / 2 : NT;
  BwdParams bp{};
  bp.p = p0;  // work items: pairs of tiles of one scene
  QueryParams& p = bp.p;
  if (adam) bp.a = *adam;
  int64_t items = 0;
  for (int s = 0; s < p.n_scenes; ++s) {
    p.item_begin[s] = items;
    const int64_t tiles = (p.sc[s].q_end - p.sc[s].q_begin + ROWS - 1) / ROWS;
    items += (tiles + S::G - 1) / S::G;
  }
  p.item_begin[p.n_scenes] = items;
  p.n_items = items;
  const octa_tuning tu = tuning_snapshot();
  p.order = tu.train_order == 1 ? 1 : 0;
  p.run = tu.train_run > 1 ? tu.train_run : 1;
  if (items == 0 && !PERSIST) return OCTA_OK;
  auto kern = bwd_kernel<S, TT, TRAIN, PERSIST, FORMS, PRED>;
  int per_sm = 0;
  // the cooperative launch keeps the largest carveout: all CTAs co-resident
  int rc = launch_cache().get(reinterpret_cast<const void*>(kern), S::SMEM, S::NTB,
                              static_cast<int>(S::TMEM_COLS), &per_sm,
                              PERSIST ? kCarveMaxShared : carve_mode(tu));
  if (rc) return rc;
  cudaError_t e;
  if (PERSIST) {  // every CTA co-resident: the grid barriers need it
    const int grid = per_sm * device_sm_count();
    void* args[] = {&bp};
    e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kern), dim3(grid), dim3(S::NTB),
                                    args, S::SMEM, stream);
  } else {
    const int64_t grid = std::min<int64_t>(items, int64_t(per_sm) * device_sm_count());
    kern<<<static_cast<unsigned>(grid), S::NTB, S::SMEM, stream>>>(bp);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return fail(OCTA_ECUDA, "tc %s launch: %s", TRAIN ? "train" : "bwd",
                                    cudaGetErrorString(e));
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

template <bool TRAIN, bool PERSIST>
int dispatch_bwd(const octa_scene* scenes, int n_scenes, const QueryParams& p, const AdamBlock* adam,
                 cudaStream_t stream) {
  int F, need, H, NH;
  bool f16;
  int rc = select_shape(scenes, n_scenes, &F, &need, &H, &NH, &f16);
  if (rc) return rc;
  bool forms = false;  // any scene in the full or shifted form
  for (int s = 0; s < n_scenes; ++s) forms = forms || scenes[s].query_form != OCTA_FORM_CELL_BILINEAR;
  // cell form: two threads per tile row unless the tuning asks for one
  const bool tpr1 = tuning_snapshot().train_threads_per_row == 1;
#define OCTA_TC_TRY(F_, WP_, H_, NH_)                                                         \
  if (F == F_ && H == H_ && NH == NH_ && need <= WP_) {                                       \
    if (forms)                                                                                \
      return f16 ? launch_bwd<BShape<F_, WP_, H_, NH_, 1>, __half, TRAIN, PERSIST, true>(      \
                       p, adam, stream)                                                       \
                 : launch_bwd<BShape<F_, WP_, H_, NH_, 1>, float, TRAIN, PERSIST, true>(       \
                       p, adam, stream);                                                      \
    if (tpr1)                                                                                 \
      return f16 ? launch_bwd<BShape<F_, WP_, H_, NH_, 1>, __half, TRAIN, PERSIST, false>(     \
                       p, adam, stream)                                                       \
                 : launch_bwd<BShape<F_, WP_, H_, NH_, 1>, float, TRAIN, PERSIST, false>(      \
                       p, adam, stream);                                                      \
    return f16 ? launch_bwd<BShape<F_, WP_, H_, NH_, 2>, __half, TRAIN, PERSIST, false>(       \
                     p, adam, stream)                                                         \
               : launch_bwd<BShape<F_, WP_, H_, NH_, 2>, float, TRAIN, PERSIST, false>(        \
                     p, adam, stream);                                                        \
  }
  OCTA_TC_TRY(4, 32, 32, 2)
  OCTA_TC_TRY(8, 64, 64, 2)
  OCTA_TC_TRY(8, 80, 64, 2)
  OCTA_TC_TRY(8, 80, 64, 3)
#undef OCTA_TC_TRY
  return fail(OCTA_EUNSUPPORTED, "BF16 path: no built shape for F=%d, K*F=%d, hidden %d x %d", F,
              need, NH, H);
}

#ifdef OCTA_TC_BWD
int query_bwd(const octa_scene* scenes, int n_scenes, const QueryParams& p, cudaStream_t stream) {
  return dispatch_bwd<false, false>(scenes, n_scenes, p, nullptr, stream);
}

int train_fused(const octa_scene* scenes, int n_scenes, const QueryParams& p, cudaStream_t stream) {
  return dispatch_bwd<true, false>(scenes, n_scenes, p, nullptr, stream);
}

// g_psi's backward on the tensor cores: the decoder's backward kernel with the
// predictor's input row, one output channel and the hash-table scatter.
int predictor_bwd(const octa_predictor* pred, const octa_queries* q, const float* d_disp,
                  float* d_table, float* d_weights, cudaStream_t stream) {
  QueryParams p;
  std::memset(&p, 0, sizeof(p));
  const int L = pred->levels;
  DevScene& d = p.sc[0];
  d.weights = pred->weights_bf16;
  d.d_weights = d_weights;
  d.n_layers = 3;
  d.K = 1;
  d.widths[0] = 2 * L + 3;
  d.widths[1] = OCTA_PRED_HIDDEN;
  d.widths[2] = OCTA_PRED_HIDDEN;
  d.widths[3] = 1;
  int off = 0;
  for (int i = 0; i <= 3; ++i) {
    d.w_offset[i] = off;
    if (i < 3) off += d.widths[i] * d.widths[i + 1];
  }
  d.q_begin = 0;
  d.q_end = q->n;
  d.norm_pairs = q->n;
  p.n_scenes = 1;
  p.n_tiles = (q->n + NT - 1) / NT;
  p.x = q->x;
  p.omega = q->omega;
  p.normal = q->normal;
  p.d_rgb = d_disp;
  p.pred_table = pred->table;
  p.pred_dtable = d_table;
  p.pred_levels = L;
  const int64_t T = int64_t(1) << pred->log2_T;
  p.pred_tmask = static_cast<uint32_t>(T - 1);
  for (int l = 0; l < L; ++l) {
    p.pred_res[l] = pred->res[l];
    const int64_t side = pred->res[l] + 1;
    p.pred_dense[l] = side * side * side <= T ? 1 : 0;
  }
  if (p.n_tiles == 0) return OCTA_OK;
  return launch_bwd<BShape<8, 32, 64, 2, 1>, __half, false, false, false, true>(p, nullptr,
                                                                                 stream);
}
#endif  // OCTA_TC_BWD

#ifdef OCTA_TC_STEP
int train_step_persistent(const octa_scene* scenes, int n_scenes, const QueryParams& p,
                          const AdamBlock& adam, cudaStream_t stream) {
  return dispatch_bwd<true, true>(scenes, n_scenes, p, &adam, stream);
}
#endif  // OCTA_TC_STEP

#ifdef OCTA_TC_FWD
int predictor_fwd(const octa_predictor* pred, const octa_queries* q, float* disparity,
                  cudaStream_t stream) {
  QueryParams p;
  std::memset(&p, 0, sizeof(p));
  const int L = pred->levels;
  DevScene& d = p.sc[0];
  d.weights = pred->weights_bf16;
  d.n_layers = 3;
  d.K = 1;
  d.widths[0] = 2 * L + 3;
  d.widths[1] = OCTA_PRED_HIDDEN;
  d.widths[2] = OCTA_PRED_HIDDEN;
  d.widths[3] = 1;
  int off = 0;
  for (int i = 0; i <= 3; ++i) {
    d.w_offset[i] = off;
    if (i < 3) off += d.widths[i] * d.widths[i + 1];
  }
  d.q_begin = 0;
  d.q_end = q->n;
  d.tile_begin = 0;
  p.n_scenes = 1;
  p.n_tiles = (q->n + NT - 1) / NT;
  p.x = q->x;
  p.omega = q->omega;
  p.normal = q->normal;
  p.pred_table = pred->table;
  p.pred_levels = L;
  const int64_t T = int64_t(1) << pred->log2_T;
  p.pred_tmask = static_cast<uint32_t>(T - 1);
  for (int l = 0; l < L; ++l) {
    p.pred_res[l] = pred->res[l];
    const int64_t side = pred->res[l] + 1;
    p.pred_dense[l] = side * side * side <= T ? 1 : 0;
  }
  p.disparity_out = disparity;
  if (p.n_tiles == 0) return OCTA_OK;
  return launch_fwd_tpq<Shape<8, 32, 64, 2>, __half, 1, FORM_PREDICTOR>(p, tuning_snapshot(),
                                                                          stream);
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
  OCTA_TC_TRY(8, 96, 64, 2)  // K*F + Eq. 12's attributes
#undef OCTA_TC_TRY
  return fail(OCTA_EUNSUPPORTED, "BF16 path: no built shape for F=%d, K*F=%d, hidden %d x %d", F,
              need, NH, H);
}
#endif  // OCTA_TC_FWD

}  // namespace tc
}  // namespace octa
