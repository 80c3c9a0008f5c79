// C ABI of the query path: octa_encode, octa_query_fwd, octa_query_bwd.
// Host-side validation, the kernel parameter block, dispatch to the FP32
// engine (CUDA cores) or the BF16 tensor-core kernels, and the standalone
// encoding kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "engine_path.h"
#include "gather.cuh"
#include "launch_persistent.cuh"
#include "octa_internal.h"
#include "tc_path.h"

namespace octa {

// ---------------------------------------------------------------------------
// Standalone encoding kernel (Eq. 10 single-cell bilinear form + Eq. 11)
// ---------------------------------------------------------------------------
// One query per thread (fold, walk, gather; see gather.cuh), its K*F
// features written into a shared-memory staging row in the output type.
// When the output rows are packed, the rows leave in bulk asynchronous
// copies (each warp's 32 rows by its lane 0 at one thread per query, the
// whole tile by thread 0 at two); otherwise as element stores at the row
// stride.  Either way the feature stream is written coalesced.
constexpr int ENC_NT = 128;

// Bulk asynchronous copy of `bytes` (multiple of 16) from shared to global
// memory (both addresses 16-byte aligned), committed as one bulk group; the
// waits for the source to have been read, and for the copy to have landed.
__device__ __forceinline__ void bulk_copy_s2g(void* dst, uint32_t src, uint32_t bytes) {
  asm volatile(
      "cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n\t"
      "cp.async.bulk.commit_group;\n" ::"l"(dst),
      "r"(src), "r"(bytes)
      : "memory");
}
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// NS > 0: the cell form's texels staged through a ring of NS levels in
// shared memory (locate_gather_query_staged) at p.ring_off.
template <int F, typename TT, typename OT, int KP, int FORM = OCTA_FORM_CELL_BILINEAR,
          int TPQ = 1, int NS = 0>
__global__ void __launch_bounds__(ENC_NT * TPQ) encode_kernel(const __grid_constant__ QueryParams p) {
  static_assert(TPQ == 1 || FORM == OCTA_FORM_CELL_BILINEAR, "threads per query: cell form");
  static_assert(NS == 0 || (TPQ == 1 && FORM == OCTA_FORM_CELL_BILINEAR), "staged: cell form");
  constexpr int NTH = ENC_NT * TPQ;  // TPQ threads per query, thread par gathers levels l % TPQ
  extern __shared__ __align__(16) uint8_t stage[];
  const int q = threadIdx.x % ENC_NT, par = threadIdx.x / ENC_NT;
  OT* out = static_cast<OT*>(p.features);
  int2* tree_sm = p.tree_cap > 0 ? reinterpret_cast<int2*>(stage + p.tree_off) : nullptr;
  const int2* tree = nullptr;
  int cur = -1;
  const WorkRange wr = work_range(p.n_tiles, p.order, p.run);
  QueryIn next = wr.begin < wr.end ? load_tile_query(p, wr.begin, q, ENC_NT) : QueryIn{};
  // a bulk copy of staging rows in flight (thread 0 of the CTA, or lane 0
  // of a warp that copies its own rows)
  bool bulk_pending = false;
  // the previous tile's rows were read out warp by warp (no CTA-wide reads
  // of them can be in flight)
  bool prev_warp_rows = true;
  const int lane = threadIdx.x & 31;
  for (int64_t tile = wr.begin; tile < wr.end; tile = wr.next(tile)) {
    const int s = scene_of_tile(p, tile);
    const DevScene& sc = p.sc[s];
    const QueryIn in = next;
    if (wr.next(tile) < wr.end) next = load_tile_query(p, wr.next(tile), q, ENC_NT);
    if (s != cur) {
      __syncthreads();  // no thread walks the previous scene's tree any more
      tree = stage_tree(p, sc, tree_sm, p.tree_cap, threadIdx.x, NTH);
      cur = s;
      __syncthreads();
    }
    const int64_t q0 = sc.q_begin + (tile - sc.tile_begin) * ENC_NT;
    const int nq = static_cast<int>(sc.q_end - q0 < ENC_NT ? sc.q_end - q0 : int64_t(ENC_NT));
    const int W = sc.K * F;
    const int row_bytes = W * int(sizeof(OT));
    const int rb = (row_bytes + 15) & ~15;  // staging row stride
    const bool packed = p.row_stride == W && rb == row_bytes &&
                        (reinterpret_cast<uintptr_t>(out) & 15u) == 0;
    // one thread per query with packed rows: each warp writes, copies out
    // and rewrites only its own 32 rows, so the warps need no CTA barrier
    const bool warp_rows = TPQ == 1 && packed;
    if (bulk_pending) {  // the previous tile's rows have been read out before they are rewritten
      bulk_wait_read_all();
      bulk_pending = false;
    }
    if (warp_rows && prev_warp_rows)
      __syncwarp();
    else
      __syncthreads();
    prev_warp_rows = warp_rows;
    auto stage_row = [&](int l, const float (&v)[F]) {
      if (l >= sc.K) return;
      uint8_t* dst = stage + q * rb + l * F * int(sizeof(OT));
      if constexpr (sizeof(OT) == 2) {
        uint32_t w[F / 2];
#pragma unroll
        for (int i = 0; i < F / 2; ++i) w[i] = pack_bf16x2_rn(v[2 * i], v[2 * i + 1]);
        if constexpr (F == 8)
          *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
        else
          *reinterpret_cast<uint2*>(dst) = make_uint2(w[0], w[1]);
      } else {
#pragma unroll
        for (int i = 0; i < F / 4; ++i)
          reinterpret_cast<float4*>(dst)[i] =
              make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
      }
    };
    if constexpr (FORM == OCTA_FORM_SHIFTED)
      gather_shifted_query<F, TT, KP>(p, sc, tree, in, q0 + q, q < nq, p.normal, p.disparity,
                                      stage_row);
    else if constexpr (FORM == OCTA_FORM_TRILINEAR_VERTEX)
      gather_full_query<F, TT, KP>(p, sc, tree, in, q0 + q, q < nq, stage_row);
    else if constexpr (NS > 0)
      locate_gather_query_staged<F, TT, KP, sizeof(OT) == 2, NS>(
          p, sc, tree, in, q0 + q, q < nq,
          static_cast<uint32_t>(__cvta_generic_to_shared(stage + p.ring_off)), q, ENC_NT, stage_row);
    else
      locate_gather_query<F, TT, KP, sizeof(OT) == 2, TPQ>(p, sc, tree, in, q0 + q, q < nq, par,
                                                            nullptr, nullptr, q, ENC_NT, stage_row);
    if (packed) fence_proxy_async_smem();  // the rows' generic writes, before the bulk copy reads them
    if (warp_rows) {  // this warp's rows: one bulk copy by its lane 0
      __syncwarp();
      const int r0 = threadIdx.x & ~31;
      const int nr = nq - r0 < 32 ? nq - r0 : 32;
      if (lane == 0 && nr > 0) {
        bulk_copy_s2g(reinterpret_cast<uint8_t*>(out + (q0 + r0) * W),
                      static_cast<uint32_t>(__cvta_generic_to_shared(stage + r0 * rb)),
                      static_cast<uint32_t>(nr * row_bytes));
        bulk_pending = true;
      }
      continue;
    }
    __syncthreads();
    if (packed) {
      // the tile's rows are one contiguous block in global memory: one bulk
      // asynchronous copy (nq * row_bytes bytes, a multiple of 16; both
      // addresses 16-byte aligned), issued by thread 0 while the others
      // start the next tile's walk
      if (threadIdx.x == 0) {
        bulk_copy_s2g(reinterpret_cast<uint8_t*>(out + q0 * W),
                      static_cast<uint32_t>(__cvta_generic_to_shared(stage)),
                      static_cast<uint32_t>(nq * row_bytes));
        bulk_pending = true;
      }
    } else {
      for (int i = threadIdx.x; i < nq * W; i += NTH) {
        const int r = i / W, k = i % W;
        out[(q0 + r) * p.row_stride + k] =
            *reinterpret_cast<const OT*>(stage + r * rb + k * int(sizeof(OT)));
      }
    }
  }
  if (bulk_pending) bulk_wait_all();  // the last copy has landed before the CTA's memory is freed
}

namespace {

bool aligned16(const void* ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15u) == 0; }

}  // namespace

// Texel-ring depth of the staged cell-form gathers (16-byte texels, one
// thread per query): the gather_stages knob, 0 = the default.
constexpr int kDefaultGatherStages = 1;
int gather_stages(const octa_tuning& tu) {
  return tu.gather_stages > 0 ? tu.gather_stages : kDefaultGatherStages;
}

// The cell-form encoding at one thread per query: texel loads into
// registers (ns < 2) or a shared-memory ring of ns (2..4) levels (16-byte
// texels only); smem: the staging rows and the tree, the ring after them.
template <int F, typename TT, typename OT, int KP, int NS>
int launch_encode_cell_ns(size_t smem, QueryParams& p, cudaStream_t st, const octa_tuning& tu) {
  return launch_persistent(encode_kernel<F, TT, OT, KP, OCTA_FORM_CELL_BILINEAR, 1, NS>, smem, p,
                           st, ENC_NT, tu.encode_ctas_per_sm, tu.fwd_order, tu.fwd_run);
}

template <int F, typename TT, typename OT, int KP>
int launch_encode_cell(int ns, size_t smem, QueryParams& p, cudaStream_t st,
                       const octa_tuning& tu) {
  if constexpr (F * sizeof(TT) == 16) {
    if (ns >= 2) {
      p.ring_off = static_cast<int32_t>((smem + 15) & ~size_t(15));
      smem = size_t(p.ring_off) + size_t(ns) * 4 * ENC_NT * 16;
      if (ns == 2) return launch_encode_cell_ns<F, TT, OT, KP, 2>(smem, p, st, tu);
      if (ns == 3) return launch_encode_cell_ns<F, TT, OT, KP, 3>(smem, p, st, tu);
      return launch_encode_cell_ns<F, TT, OT, KP, 4>(smem, p, st, tu);
    }
  }
  return launch_encode_cell_ns<F, TT, OT, KP, 0>(smem, p, st, tu);
}

// Validates scenes + queries and fills the kernel parameter block.
int build_query_params(const octa_scene* scenes, int32_t n_scenes, const octa_queries* q,
                       const octa_scene_grads* grads, QueryParams& p) {
  std::memset(&p, 0, sizeof(p));
  if (!scenes || !q) return fail(OCTA_EINVAL, "scenes and queries must be non-NULL");
  if (n_scenes < 1 || n_scenes > OCTA_MAX_SCENES)
    return fail(OCTA_ERANGE, "n_scenes %d outside [1, %d]", n_scenes, OCTA_MAX_SCENES);
  if (q->n < 0) return fail(OCTA_EINVAL, "negative query count");
  if (q->n_attrs < 0 || q->n_attrs > OCTA_MAX_ATTRS)
    return fail(OCTA_ERANGE, "n_attrs %d outside [0, %d]", q->n_attrs, OCTA_MAX_ATTRS);
  if (q->n_attrs > 0 && q->n > 0 && !q->attrs) return fail(OCTA_EINVAL, "attrs must be non-NULL");
  if (q->n > 0 && (!q->x || !q->omega)) return fail(OCTA_EINVAL, "x / omega must be non-NULL");
  if (q->scene_start[0] != 0 || q->scene_start[n_scenes] != q->n)
    return fail(OCTA_EINVAL, "scene_start must run from 0 to n");
  p.n_scenes = n_scenes;
  p.attrs = q->n_attrs > 0 ? q->attrs : nullptr;
  p.n_attrs = q->n_attrs;
  int64_t tiles = 0;
  for (int s = 0; s < n_scenes; ++s) {
    const octa_scene& c = scenes[s];
    DevScene& d = p.sc[s];
    if (q->scene_start[s + 1] < q->scene_start[s])
      return fail(OCTA_EINVAL, "scene_start must be non-decreasing");
    if (!c.first_child || !c.map_offset || !c.tables || !c.weights)
      return fail(OCTA_EINVAL, "scene %d: NULL tree, table or weight pointer", s);
    if (c.num_levels < 1 || c.num_levels > OCTA_MAX_LEVELS)
      return fail(OCTA_ERANGE, "scene %d: num_levels %d outside [1, %d]", s, c.num_levels,
                  OCTA_MAX_LEVELS);
    if (c.num_nodes < 1) return fail(OCTA_EINVAL, "scene %d: empty tree", s);
    if (c.num_texels < 1 || c.num_texels > 2147483647LL)
      return fail(OCTA_ERANGE, "scene %d: num_texels outside [1, 2^31)", s);
    if (c.F != 4 && c.F != 8) return fail(OCTA_EINVAL, "scene %d: F must be 4 or 8", s);
    if (c.table_dtype != OCTA_F32 && c.table_dtype != OCTA_F16)
      return fail(OCTA_EINVAL, "scene %d: table dtype must be F32 or F16", s);
    if (c.weight_dtype != OCTA_F32 && c.weight_dtype != OCTA_BF16)
      return fail(OCTA_EINVAL, "scene %d: weight dtype must be F32 or BF16", s);
    if (c.n_layers < 2 || c.n_layers > OCTA_MAX_LAYERS)
      return fail(OCTA_ERANGE, "scene %d: n_layers %d outside [2, %d]", s, c.n_layers,
                  OCTA_MAX_LAYERS);
    if (c.widths[0] != c.num_levels * c.F + q->n_attrs)
      return fail(OCTA_EINVAL, "scene %d: widths[0] must equal K*F + n_attrs", s);
    if (c.widths[c.n_layers] != 3) return fail(OCTA_EINVAL, "scene %d: output width must be 3", s);
    if (!aligned16(c.tables)) return fail(OCTA_EINVAL, "scene %d: tables not 16-byte aligned", s);
    for (int l = 0; l < c.num_levels; ++l)
      if (c.R[l] < 2 || c.R[l] > 4096)
        return fail(OCTA_ERANGE, "scene %d: R[%d] = %d outside [2, 4096]", s, l, c.R[l]);
    d.first_child = c.first_child;
    d.map_offset = c.map_offset;
    d.tables = c.tables;
    d.weights = c.weights;
    d.num_texels = c.num_texels;
    d.num_nodes = c.num_nodes;
    d.K = c.num_levels;
    d.n_layers = c.n_layers;
    for (int l = 0; l < c.num_levels; ++l) d.R[l] = c.R[l];
    d.query_form = c.query_form;
    if (c.query_form != OCTA_FORM_CELL_BILINEAR && c.query_form != OCTA_FORM_TRILINEAR_VERTEX &&
        c.query_form != OCTA_FORM_SHIFTED)
      return fail(OCTA_EINVAL, "scene %d: unknown query_form %d", s, c.query_form);
    if (c.query_form != OCTA_FORM_CELL_BILINEAR) {
      for (int l = 0; l < c.num_levels; ++l) {
        const int n = c.R[l] - 1;  // cells a side: a power of two >= 2
        if (n < 2 || (n & (n - 1)))
          return fail(OCTA_EINVAL, "scene %d: vertex map side R[%d] = %d is not 2^k + 1", s, l,
                      c.R[l]);
      }
    }
    int off = 0;
    for (int i = 0; i <= c.n_layers; ++i) {
      if (c.widths[i] < 1) return fail(OCTA_EINVAL, "scene %d: width %d < 1", s, i);
      d.widths[i] = c.widths[i];
      d.w_offset[i] = off;
      if (i < c.n_layers) off += c.widths[i] * c.widths[i + 1];
    }
    if (grads) {
      if (!grads[s].d_tables || !grads[s].d_weights)
        return fail(OCTA_EINVAL, "scene %d: NULL gradient buffer", s);
      if (!aligned16(grads[s].d_tables))
        return fail(OCTA_EINVAL, "scene %d: d_tables not 16-byte aligned", s);
      d.d_tables = grads[s].d_tables;
      d.d_weights = grads[s].d_weights;
    }
    d.q_begin = q->scene_start[s];
    d.q_end = q->scene_start[s + 1];
    d.norm_pairs = d.q_end - d.q_begin;
    d.tile_begin = tiles;
    tiles += (d.q_end - d.q_begin + QT - 1) / QT;
  }
  p.n_tiles = tiles;
  p.x = q->x;
  p.omega = q->omega;
  return OCTA_OK;
}


// Loss normalisation of the training passes: pairs->norm_pairs[s] when set.
int apply_norm_pairs(const octa_pairs* pairs, int n_scenes, QueryParams& p) {
  for (int s = 0; s < n_scenes; ++s) {
    const int64_t m = pairs->norm_pairs[s];
    if (m < 0) return fail(OCTA_EINVAL, "norm_pairs[%d] < 0", s);
    if (m > 0) p.sc[s].norm_pairs = m;
  }
  return OCTA_OK;
}
}  // namespace octa

using namespace octa;

namespace {
// The one-launch step does not evaluate the shifted form.
int reject_shifted(const octa_scene* scenes, int32_t n_scenes) {
  for (int s = 0; s < n_scenes; ++s)
    if (scenes[s].query_form == OCTA_FORM_SHIFTED)
      return fail(OCTA_EUNSUPPORTED,
                  "scene %d: the one-launch step does not evaluate the shifted form", s);
  return 0;
}

// One query form per call (texel_addr's row layout depends on it); node_idx
// has no meaning in the trilinear vertex form (eight cells per level).
int check_one_form(const octa_scene* scenes, int32_t n_scenes, const int32_t* node_idx) {
  for (int s = 1; s < n_scenes; ++s)
    if (scenes[s].query_form != scenes[0].query_form)
      return fail(OCTA_EUNSUPPORTED, "scenes of one call must share the query form");
  if (node_idx && scenes[0].query_form != OCTA_FORM_CELL_BILINEAR)
    return fail(OCTA_EINVAL, "node_idx is not defined for the trilinear vertex form");
  return 0;
}
}  // namespace

extern "C" int octa_encode(const octa_scene* scenes, int32_t n_scenes, const octa_queries* q,
                           void* features, int32_t feat_dtype, int64_t row_stride,
                           int32_t* node_idx, int32_t* texel_addr, int32_t* status,
                           void* stream) {
  clear_error();
  QueryParams p;
  int rc = build_query_params(scenes, n_scenes, q, nullptr, p);
  if (rc) return rc;
  if (q->n > 0 && !features) return fail(OCTA_EINVAL, "features must be non-NULL");
  rc = check_one_form(scenes, n_scenes, node_idx);
  if (rc) return rc;
  if (scenes[0].query_form == OCTA_FORM_SHIFTED && q->n > 0 && (!q->normal || !q->disparity))
    return fail(OCTA_EINVAL, "the shifted form needs normal and disparity");
  if (feat_dtype != OCTA_F32 && feat_dtype != OCTA_BF16)
    return fail(OCTA_EINVAL, "feature dtype must be F32 or BF16");
  int kmax = 0, F = scenes[0].F, tdt = scenes[0].table_dtype;
  for (int s = 0; s < n_scenes; ++s) {
    kmax = std::max(kmax, scenes[s].num_levels);
    if (row_stride < scenes[s].num_levels * scenes[s].F)
      return fail(OCTA_EINVAL, "row_stride smaller than K*F of scene %d", s);
    if (scenes[s].F != F || scenes[s].table_dtype != tdt)
      return fail(OCTA_EUNSUPPORTED, "scenes of one call must share F and table dtype");
  }
  if (texel_addr && (reinterpret_cast<uintptr_t>(texel_addr) & 15u))
    return fail(OCTA_EINVAL, "texel_addr not 16-byte aligned");
  p.features = features;
  p.row_stride = row_stride;
  p.feat_dtype = feat_dtype;
  p.node_idx = node_idx;
  p.texel_addr = texel_addr;
  p.kmax_out = kmax;
  p.status = status;
  const size_t ot = feat_dtype == OCTA_BF16 ? 2 : 4;
  size_t smem = size_t(ENC_NT) * ((size_t(kmax) * F * ot + 15) & ~size_t(15));
  // staged octree: the largest scene's nodes in granules of 16, at most 2048
  int max_nodes = 0;
  for (int s = 0; s < n_scenes; ++s) max_nodes = std::max(max_nodes, scenes[s].num_nodes);
  if (max_nodes <= 2048) {
    p.tree_cap = (max_nodes + 15) & ~15;
    p.tree_off = static_cast<int32_t>(smem);
    smem += size_t(p.tree_cap) * 8;
  }
  // the encode kernel tiles ENC_NT queries; QT-sized tiles were counted above
  static_assert(ENC_NT == QT, "tile size");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool f16 = tdt == OCTA_F16, bf = feat_dtype == OCTA_BF16;
  const int form = scenes[0].query_form;
  p.normal = q->normal;
  p.disparity = q->disparity;
  const octa_tuning tu = tuning_snapshot();
#define OCTA_ENC_FORM(F_, TT_, KP_, FORM_)                                                       \
  return bf ? launch_persistent(encode_kernel<F_, TT_, __nv_bfloat16, KP_, FORM_>, smem, p, st,  \
                                ENC_NT, tu.encode_ctas_per_sm, tu.fwd_order, tu.fwd_run)                     \
            : launch_persistent(encode_kernel<F_, TT_, float, KP_, FORM_>, smem, p, st, ENC_NT,  \
                                tu.encode_ctas_per_sm, tu.fwd_order, tu.fwd_run);
#define OCTA_ENC(F_, TT_, KP_)                                    \
  if (form == OCTA_FORM_SHIFTED) {                                \
    OCTA_ENC_FORM(F_, TT_, KP_, OCTA_FORM_SHIFTED)                \
  }                                                               \
  if (form == OCTA_FORM_TRILINEAR_VERTEX) {                       \
    OCTA_ENC_FORM(F_, TT_, KP_, OCTA_FORM_TRILINEAR_VERTEX)       \
  }                                                               \
  if (tu.encode_threads_per_query != 2)                            \
    return bf ? launch_encode_cell<F_, TT_, __nv_bfloat16, KP_>(gather_stages(tu), smem, p, st, \
                                                                tu)                         \
              : launch_encode_cell<F_, TT_, float, KP_>(gather_stages(tu), smem, p, st, tu);  \
  return bf ? launch_persistent(                                  \
                  encode_kernel<F_, TT_, __nv_bfloat16, KP_, OCTA_FORM_CELL_BILINEAR, 2>, smem, p, \
                  st, 2 * ENC_NT, tu.encode_ctas_per_sm, tu.fwd_order, tu.fwd_run)         \
            : launch_persistent(encode_kernel<F_, TT_, float, KP_, OCTA_FORM_CELL_BILINEAR, 2>, \
                                smem, p, st, 2 * ENC_NT, tu.encode_ctas_per_sm, tu.fwd_order, \
                                tu.fwd_run);
#define OCTA_ENC_KP(F_, TT_)      \
  if (kmax <= 10) {               \
    OCTA_ENC(F_, TT_, 10)         \
  } else {                        \
    OCTA_ENC(F_, TT_, OCTA_MAX_LEVELS) \
  }
  if (F == 4) {
    if (f16) {
      OCTA_ENC_KP(4, __half)
    } else {
      OCTA_ENC_KP(4, float)
    }
  }
  if (f16) {
    OCTA_ENC_KP(8, __half)
  }
  OCTA_ENC_KP(8, float)
#undef OCTA_ENC_KP
#undef OCTA_ENC
#undef OCTA_ENC_FORM
}

extern "C" int octa_query_fwd(const octa_scene* scenes, int32_t n_scenes, const octa_queries* q,
                              float* rgb, int32_t* node_idx, int32_t* texel_addr,
                              int32_t* status, void* stream) {
  clear_error();
  QueryParams p;
  int rc = build_query_params(scenes, n_scenes, q, nullptr, p);
  if (rc) return rc;
  if (scenes[0].query_form == OCTA_FORM_SHIFTED && q->n > 0 && (!q->normal || !q->disparity))
    return fail(OCTA_EINVAL, "the shifted form needs normal and disparity");
  rc = check_one_form(scenes, n_scenes, node_idx);
  if (rc) return rc;
  if (q->n > 0 && !rgb) return fail(OCTA_EINVAL, "rgb must be non-NULL");
  if (texel_addr && (reinterpret_cast<uintptr_t>(texel_addr) & 15u))
    return fail(OCTA_EINVAL, "texel_addr not 16-byte aligned");
  int kmax = 0;
  for (int s = 0; s < n_scenes; ++s) kmax = std::max(kmax, scenes[s].num_levels);
  p.rgb = rgb;
  p.node_idx = node_idx;
  p.texel_addr = texel_addr;
  p.kmax_out = kmax;
  p.status = status;
  p.normal = q->normal;
  p.disparity = q->disparity;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (scenes[0].weight_dtype == OCTA_BF16) return tc::query_fwd(scenes, n_scenes, p, st);
  return f32::dispatch(scenes, n_scenes, p, f32::Mode::kForward, st);
}

extern "C" int octa_query_bwd(const octa_scene* scenes, int32_t n_scenes, const octa_queries* q,
                              const float* d_rgb, const octa_scene_grads* grads,
                              int32_t* status, void* stream) {
  clear_error();
  if (!grads) return fail(OCTA_EINVAL, "grads must be non-NULL");
  QueryParams p;
  int rc = build_query_params(scenes, n_scenes, q, grads, p);
  if (rc) return rc;
  const bool shifted = scenes[0].query_form == OCTA_FORM_SHIFTED;
  if (shifted && q->n > 0 && (!q->normal || !q->disparity))
    return fail(OCTA_EINVAL, "the shifted form needs normal and disparity");
  if (q->d_disparity && !shifted)
    return fail(OCTA_EINVAL, "d_disparity is defined for the shifted form only");
  rc = check_one_form(scenes, n_scenes, nullptr);
  if (rc) return rc;
  if (q->n > 0 && !d_rgb) return fail(OCTA_EINVAL, "d_rgb must be non-NULL");
  p.d_rgb = d_rgb;
  p.status = status;
  p.normal = q->normal;
  p.disparity = q->disparity;
  p.d_disparity = q->d_disparity;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (scenes[0].weight_dtype == OCTA_BF16) return tc::query_bwd(scenes, n_scenes, p, st);
  return f32::dispatch(scenes, n_scenes, p, f32::Mode::kBackward, st);
}

extern "C" int octa_train_fused(const octa_scene* scenes, int32_t n_scenes, const octa_pairs* pairs,
                                float eps, int32_t rhs_grad, const octa_scaler* scaler,
                                double* loss_dev, const octa_scene_grads* grads, int32_t* status,
                                void* stream) {
  clear_error();
  if (!pairs || !grads || !loss_dev) return fail(OCTA_EINVAL, "pairs, grads and loss_dev must be non-NULL");
  if (pairs->n > 0 && (!pairs->x2 || !pairs->omega2 || !pairs->E || !pairs->w))
    return fail(OCTA_EINVAL, "pair arrays must be non-NULL");
  if (!(eps > 0.f)) return fail(OCTA_EINVAL, "eps must be > 0");
  octa_queries q;
  std::memset(&q, 0, sizeof(q));
  q.x = pairs->x;
  q.omega = pairs->omega;
  q.n = pairs->n;
  for (int s = 0; s <= OCTA_MAX_SCENES; ++s) q.scene_start[s] = pairs->scene_start[s];
  QueryParams p;
  int rc = build_query_params(scenes, n_scenes, &q, grads, p);
  if (rc) return rc;
  rc = check_one_form(scenes, n_scenes, nullptr);
  if (rc) return rc;
  const bool shifted = scenes[0].query_form == OCTA_FORM_SHIFTED;
  if (shifted && pairs->n > 0 &&
      (!pairs->normal || !pairs->normal2 || !pairs->disparity || !pairs->disparity2))
    return fail(OCTA_EINVAL, "the shifted form needs both queries' normals and disparities");
  if ((pairs->d_disparity || pairs->d_disparity2) && !shifted)
    return fail(OCTA_EINVAL, "d_disparity is defined for the shifted form only");
  if (shifted) {
    p.normal = pairs->normal;
    p.normal2 = pairs->normal2;
    p.disparity = pairs->disparity;
    p.disparity2 = pairs->disparity2;
    p.d_disparity = pairs->d_disparity;
    p.d_disparity2 = pairs->d_disparity2;
  }
  const bool bf16 = scenes[0].weight_dtype == OCTA_BF16;
  for (int s = 0; s < n_scenes; ++s)
    if ((scenes[s].weight_dtype == OCTA_BF16) != bf16)
      return fail(OCTA_EUNSUPPORTED, "scenes of one call must share the decoder dtype");
  rc = apply_norm_pairs(pairs, n_scenes, p);
  if (rc) return rc;
  p.x2 = pairs->x2;
  p.omega2 = pairs->omega2;
  p.E = pairs->E;
  p.w = pairs->w;
  p.scaler = scaler;
  p.loss = loss_dev;
  p.eps = eps;
  p.rhs_grad = rhs_grad;
  p.status = status;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(loss_dev, 0, sizeof(double) * n_scenes, st);
  if (e != cudaSuccess) return fail(OCTA_ECUDA, "clearing loss_dev: %s", cudaGetErrorString(e));
  return bf16 ? tc::train_fused(scenes, n_scenes, p, st)
              : f32::dispatch(scenes, n_scenes, p, f32::Mode::kTrain, st);
}

extern "C" int octa_train_step_batched(const octa_scene* scenes, int32_t n_scenes,
                                       const octa_pairs* pairs, const octa_scene_grads* grads,
                                       const octa_param_group* groups, int32_t n_groups, float eps,
                                       int32_t rhs_grad, const octa_adam_cfg* adam,
                                       octa_scaler* scaler, double* loss_dev,
                                       const octa_step_options* options, void* workspace,
                                       size_t workspace_bytes, int32_t* status, void* stream) {
  clear_error();
  if (!pairs || !grads || !loss_dev || !groups || !adam || !scaler || !workspace)
    return fail(OCTA_EINVAL, "NULL argument");
  if (n_groups < 1 || n_groups > OCTA_MAX_GROUPS)
    return fail(OCTA_ERANGE, "n_groups %d outside [1, %d]", n_groups, OCTA_MAX_GROUPS);
  if (reinterpret_cast<uintptr_t>(workspace) & 255u)
    return fail(OCTA_EINVAL, "workspace must be 256-byte aligned");
  if (workspace_bytes < octa_workspace_bytes(OCTA_OP_STEP, 0))
    return fail(OCTA_EINVAL, "workspace too small for the persistent step");
  if (!(eps > 0.f)) return fail(OCTA_EINVAL, "eps must be > 0");
  octa_queries q;
  std::memset(&q, 0, sizeof(q));
  q.x = pairs->x;
  q.omega = pairs->omega;
  q.n = pairs->n;
  for (int s = 0; s <= OCTA_MAX_SCENES; ++s) q.scene_start[s] = pairs->scene_start[s];
  QueryParams p;
  int rc = build_query_params(scenes, n_scenes, &q, grads, p);
  if (rc) return rc;
  rc = reject_shifted(scenes, n_scenes);
  if (rc) return rc;
  for (int s = 0; s < n_scenes; ++s)
    if (scenes[s].weight_dtype != OCTA_BF16)
      return fail(OCTA_EUNSUPPORTED, "the persistent step needs BF16 decoders");
  rc = apply_norm_pairs(pairs, n_scenes, p);
  if (rc) return rc;
  p.x2 = pairs->x2;
  p.omega2 = pairs->omega2;
  p.E = pairs->E;
  p.w = pairs->w;
  p.scaler = scaler;
  p.loss = loss_dev;
  p.eps = eps;
  p.rhs_grad = rhs_grad;
  p.status = status;
  tc::AdamBlock a{};
  for (int i = 0; i < n_groups; ++i) {
    const octa_param_group& g = groups[i];
    if (g.n < 0 || (g.n > 0 && (!g.param || !g.grad || !g.m || !g.v)))
      return fail(OCTA_EINVAL, "group %d: bad arrays", i);
    if (g.work && g.work_dtype != OCTA_F16 && g.work_dtype != OCTA_BF16)
      return fail(OCTA_EINVAL, "group %d: working copy dtype must be F16 or BF16", i);
    a.g[i] = g;
    const uintptr_t mask = reinterpret_cast<uintptr_t>(g.param) | reinterpret_cast<uintptr_t>(g.grad) |
                           reinterpret_cast<uintptr_t>(g.m) | reinterpret_cast<uintptr_t>(g.v);
    a.vec4[i] = (mask & 15u) == 0 && (!g.work || (reinterpret_cast<uintptr_t>(g.work) & 7u) == 0);
  }
  a.n_groups = n_groups;
  a.beta1 = adam->beta1;
  a.beta2 = adam->beta2;
  a.eps = adam->eps;
  a.scaler = scaler;
  a.bar = static_cast<unsigned*>(workspace);
  a.partials = reinterpret_cast<double*>(static_cast<char*>(workspace) + 256);
  a.timeout_ns = options && options->barrier_timeout_ns ? options->barrier_timeout_ns : 1000000000ull;
  a.extra_arrivals = options ? options->extra_barrier_arrivals : 0;
  a.skip_first_mma = options ? options->skip_first_mma : 0;
  if (a.extra_arrivals < 0) return fail(OCTA_EINVAL, "extra_barrier_arrivals must be >= 0");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(loss_dev, 0, sizeof(double) * n_scenes, st);
  if (e != cudaSuccess) return fail(OCTA_ECUDA, "clearing loss_dev: %s", cudaGetErrorString(e));
  // the barrier's arrival counter and generation word start at zero on every
  // call, so a step that timed out (arrivals left behind) does not make the
  // next step's barriers miscount
  e = cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned), st);
  if (e != cudaSuccess) return fail(OCTA_ECUDA, "clearing the barrier: %s", cudaGetErrorString(e));
  return tc::train_step_persistent(scenes, n_scenes, p, a, st);
}

extern "C" int octa_set_tuning(const octa_tuning* t) {
  clear_error();
  std::lock_guard<std::mutex> lock(tuning_mutex());
  if (!t) {
    tuning() = octa_tuning{};
    return OCTA_OK;
  }
  if (t->fwd_ctas_per_sm < 0 || t->encode_ctas_per_sm < 0 || t->engine_ctas_per_sm < 0 ||
      t->fwd_order < 0 || t->fwd_order > 2 || t->train_order < 0 || t->train_order > 2 ||
      t->fwd_threads_per_query < 0 || t->fwd_threads_per_query > 2 ||
      t->encode_threads_per_query < 0 || t->encode_threads_per_query > 2 ||
      t->train_threads_per_row < 0 || t->train_threads_per_row > 2 || t->fwd_run < 0 ||
      t->fwd_run > 64 || t->train_run < 0 || t->train_run > 64 || t->gather_stages < 0 ||
      t->gather_stages > 4 || t->l1_carveout < 0 || t->l1_carveout > 2)
    return fail(OCTA_EINVAL, "tuning values out of range");
  tuning() = *t;
  return OCTA_OK;
}

extern "C" int octa_get_tuning(octa_tuning* t) {
  clear_error();
  if (!t) return fail(OCTA_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lock(tuning_mutex());
  *t = tuning();
  return OCTA_OK;
}
