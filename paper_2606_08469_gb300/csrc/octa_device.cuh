// Device-side building blocks of the OctaOctree query shared by the FP32 and
// the tensor-core kernels: kernel parameter blocks, the canonical binary32
// octahedral encoding, the texel wrap and the tree descent.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "octaoctree.h"

namespace octa {

// Queries per tile: one CTA works on QT queries at a time.
constexpr int QT = 128;

// Per-scene descriptor, passed by value inside the kernel parameter block.
struct DevScene {
  const int32_t* first_child;
  const int32_t* map_offset;
  const void* tables;
  const void* weights;
  float* d_tables;
  float* d_weights;
  int64_t num_texels;
  int64_t q_begin, q_end;  // query range of this scene
  int64_t norm_pairs;      // training passes: pairs the loss is a mean over
  int32_t query_form;      // OCTA_FORM_*
  int64_t tile_begin;      // first global tile of this scene
  int32_t num_nodes;
  int32_t K;
  int32_t n_layers;
  int32_t R[OCTA_MAX_LEVELS];
  int32_t widths[OCTA_MAX_LAYERS + 1];
  int32_t w_offset[OCTA_MAX_LAYERS + 1];  // element offset of W_i; [L] = total
};

struct QueryParams {
  DevScene sc[OCTA_MAX_SCENES];
  int32_t n_scenes;
  int32_t kmax_out;        // columns of node_idx / texel_addr
  int64_t n_tiles;
  const float* x;
  const float* omega;
  float* rgb;
  const float* d_rgb;
  int32_t* node_idx;
  int32_t* texel_addr;
  int32_t* status;
  void* features;
  int64_t row_stride;
  int32_t feat_dtype;
  // work items of kernels that take several tiles of one scene at a time:
  // scene s owns items [item_begin[s], item_begin[s+1])
  int64_t n_items;
  int64_t item_begin[OCTA_MAX_SCENES + 1];
  // fused training pass: pairs of scene s are [q_begin, q_end) of the pair
  // arrays; x / omega hold the primaries, x2 / omega2 the secondary queries
  const float* x2;
  const float* omega2;
  const float* E;
  const float* w;
  const octa_scaler* scaler;
  double* loss;  // [n_scenes], accumulated
  float eps;
  int32_t rhs_grad;
  int32_t order;  // how persistent CTAs take work: 0 interleaved, 1 contiguous chunks
  int32_t run;    // interleaved order: consecutive work units a CTA takes at a time
  // staged octree of kernels with a run-time shared-memory layout: capacity
  // in nodes (0: walk in global memory) and byte offset in dynamic memory
  int32_t tree_cap;
  int32_t tree_off;
  // byte offset in dynamic shared memory of the staged gather's texel ring
  int32_t ring_off;
  // the shifted form's per-query inputs (normal [n][3], disparity [n]); in
  // the fused training pass those of the primaries, the secondaries' in
  // normal2 / disparity2
  const float* normal;
  const float* disparity;
  const float* normal2;
  const float* disparity2;
  // the shifted form's backward: dL/dd per query (nullable), the fused
  // training pass's secondaries in d_disparity2
  float* d_disparity;
  float* d_disparity2;
  // Eq. 12's attributes [n][n_attrs], decoder input columns K*F .. K*F+n_attrs-1
  const float* attrs;
  int32_t n_attrs;
  // the predictor g_psi on the tensor-core path: hash tables, levels, and the
  // disparity it writes
  const float* pred_table;
  uint32_t pred_tmask;
  int32_t pred_levels;
  int32_t pred_res[OCTA_PRED_MAX_LEVELS];
  int32_t pred_dense[OCTA_PRED_MAX_LEVELS];
  float* disparity_out;
  float* pred_dtable;  // g_psi's backward: the hash tables' gradient (float2 entries)
};

// Decoder-input columns of level l >= K (past the features): Eq. 12's
// attributes of query gq where they fall, else zeros.
template <int F>
__device__ __forceinline__ void attr_columns(const QueryParams& p, int K, int l, int64_t gq,
                                             bool valid, float (&v)[F]) {
#pragma unroll
  for (int f = 0; f < F; ++f) {
    const int c = (l - K) * F + f;
    v[f] = (valid && c < p.n_attrs) ? p.attrs[gq * p.n_attrs + c] : 0.f;
  }
}

// Work units [0, n) of this CTA, visited begin, next(begin), ... while < end:
// interleaved in runs of `run` consecutive units (the CTA's run k starts at
// (block + k grid) run; run = 1: u = block + k grid), or one contiguous chunk
// per CTA (order 1: fewer scene switches in a multi-scene launch).
struct WorkRange {
  int64_t begin, end, step, run;
  __device__ __forceinline__ int64_t next(int64_t u) const {
    return ((u + 1) % run) ? u + 1 : u + 1 + step - run;
  }
};
__device__ __forceinline__ WorkRange work_range(int64_t n, int order, int run = 1) {
  if (order == 1) {
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b = int64_t(blockIdx.x) * chunk;
    return WorkRange{b, b + chunk < n ? b + chunk : n, 1, 1};
  }
  const int64_t r = run > 1 ? run : 1;
  return WorkRange{int64_t(blockIdx.x) * r, n, int64_t(gridDim.x) * r, r};
}

// Scene owning global tile t (tiles never straddle scenes).
__device__ __forceinline__ int scene_of_tile(const QueryParams& p, int64_t t) {
  int s = 0;
#pragma unroll 1
  while (s + 1 < p.n_scenes && t >= p.sc[s + 1].tile_begin) ++s;
  return s;
}

// Position and direction of one query, loaded a tile ahead of its walk so
// that the HBM latency overlaps the previous tile's work.
struct QueryIn {
  float x0, x1, x2, w0, w1, w2;
};
__device__ __forceinline__ QueryIn load_query(const float* __restrict__ xs,
                                              const float* __restrict__ ws, int64_t gq,
                                              bool valid) {
  QueryIn in{0.f, 0.f, 0.f, 0.f, 0.f, 1.f};
  if (valid) {
    in.x0 = __ldcs(xs + 3 * gq);
    in.x1 = __ldcs(xs + 3 * gq + 1);
    in.x2 = __ldcs(xs + 3 * gq + 2);
    in.w0 = __ldcs(ws + 3 * gq);
    in.w1 = __ldcs(ws + 3 * gq + 1);
    in.w2 = __ldcs(ws + 3 * gq + 2);
  }
  return in;
}

// Query row of one tile of tile_rows queries (persistent tile loops).
__device__ __forceinline__ QueryIn load_tile_query(const QueryParams& p, int64_t tile, int row,
                                                   int tile_rows) {
  const DevScene& sc = p.sc[scene_of_tile(p, tile)];
  const int64_t gq = sc.q_begin + (tile - sc.tile_begin) * tile_rows + row;
  return load_query(p.x, p.omega, gq, row < tile_rows && gq < sc.q_end);
}

// Eq. 4 and Eq. 5 in the canonical binary32 order (one IEEE rounding per
// operation, no contraction), so the integer texel coordinates agree
// bit-exactly with any other implementation of the same sequence:
// s = (|wx| + |wy|) + |wz|; u = (wx / s, wy / s); if wz < 0 fold with
// sign(0) = +1.
__device__ __forceinline__ void octa_fold(float wx, float wy, float wz, float& ux, float& uy) {
  const float s = __fadd_rn(__fadd_rn(fabsf(wx), fabsf(wy)), fabsf(wz));
  float a = __fdiv_rn(wx, s);
  float b = __fdiv_rn(wy, s);
  if (wz < 0.f) {
    const float sa = a >= 0.f ? 1.f : -1.f;
    const float sb = b >= 0.f ? 1.f : -1.f;
    const float na = __fmul_rn(__fsub_rn(1.f, fabsf(b)), sa);
    const float nb = __fmul_rn(__fsub_rn(1.f, fabsf(a)), sb);
    a = na;
    b = nb;
  }
  ux = a;
  uy = b;
}

// Continuous texel coordinate p = (u * 0.5 + 0.5) * R - 0.5 (texel (i, j) is
// centred at uv = ((i + 1/2)/R, (j + 1/2)/R)).
__device__ __forceinline__ float octa_texel_coord(float u, float R) {
  return __fsub_rn(__fmul_rn(__fadd_rn(__fmul_rn(u, 0.5f), 0.5f), R), 0.5f);
}

// Bilinear footprint of one direction on an R x R map: texel indices (within
// the node's map) of the 4 corners (i0+a, j0+b), k = a + 2b, after the
// octahedral wrap, and their weights.
struct Footprint {
  int idx[4];
  float w[4];
};

// Octahedral wrap of a corner in [-1, R]^2: across u_x = +-1 the map
// continues mirrored in u_y, across u_y = +-1 mirrored in u_x (i first).
__device__ __forceinline__ int wrap_index(int i, int j, int R) {
  if (i < 0) {
    i = 0;
    j = R - 1 - j;
  } else if (i >= R) {
    i = R - 1;
    j = R - 1 - j;
  }
  if (j < 0) {
    j = 0;
    i = R - 1 - i;
  } else if (j >= R) {
    j = R - 1;
    i = R - 1 - i;
  }
  return j * R + i;
}

__device__ __forceinline__ Footprint footprint(float ux, float uy, int R) {
  const float Rf = static_cast<float>(R);
  const float px = octa_texel_coord(ux, Rf);
  const float py = octa_texel_coord(uy, Rf);
  const float flx = floorf(px), fly = floorf(py);
  // p lies in [-1/2, R - 1/2] for any finite direction; the clamp only
  // guards non-finite input (zero direction) against out-of-map indices.
  const int i0 = min(max(static_cast<int>(flx), -1), R - 1);
  const int j0 = min(max(static_cast<int>(fly), -1), R - 1);
  const float fx = __fsub_rn(px, flx);
  const float fy = __fsub_rn(py, fly);
  Footprint f;
  if (i0 >= 0 && j0 >= 0 && i0 + 1 < R && j0 + 1 < R) {  // interior: no wrap
    f.idx[0] = j0 * R + i0;
    f.idx[1] = f.idx[0] + 1;
    f.idx[2] = f.idx[0] + R;
    f.idx[3] = f.idx[2] + 1;
  } else {
    f.idx[0] = wrap_index(i0, j0, R);
    f.idx[1] = wrap_index(i0 + 1, j0, R);
    f.idx[2] = wrap_index(i0, j0 + 1, R);
    f.idx[3] = wrap_index(i0 + 1, j0 + 1, R);
  }
  const float gx = 1.f - fx, gy = 1.f - fy;
  f.w[0] = gx * gy;
  f.w[1] = fx * gy;
  f.w[2] = gx * fy;
  f.w[3] = fx * fy;
  return f;
}

__device__ __forceinline__ float clamp01(float v) { return fminf(fmaxf(v, 0.f), 1.f); }

// Sum of squares of four unscaled gradient components for the gradient-norm
// reductions: the products and their sum in binary32 (GB300's FP64 rate is a
// small fraction of its FP32 rate), widened to FP64 once per four elements
// for the accumulation; recomputed in FP64 when the binary32 sum is not
// finite, so a finite gradient never reads as an overflow and a non-finite
// one stays non-finite.
__device__ __forceinline__ double sum_sq4(float4 g, float inv_s) {
  const float x = g.x * inv_s, y = g.y * inv_s, z = g.z * inv_s, w = g.w * inv_s;
  const float s = fmaf(x, x, fmaf(y, y, fmaf(z, z, w * w)));
  if (fabsf(s) <= 3.4028235e38f) return static_cast<double>(s);
  return double(x) * x + double(y) * y + double(z) * z + double(w) * w;
}

// Binary32 sum of squares of n unscaled float4 gradients, widened to FP64
// once; recomputed in FP64 when the binary32 sum is not finite (same
// guarantees as sum_sq4).
template <int N>
__device__ __forceinline__ double sum_sq4_batch(const float4 (&g)[N], float inv_s) {
  float s = 0.f;
#pragma unroll
  for (int u = 0; u < N; ++u) {
    const float x = g[u].x * inv_s, y = g[u].y * inv_s, z = g[u].z * inv_s, w = g[u].w * inv_s;
    s = fmaf(x, x, fmaf(y, y, fmaf(z, z, fmaf(w, w, s))));
  }
  if (fabsf(s) <= 3.4028235e38f) return static_cast<double>(s);
  double d = 0.0;
#pragma unroll
  for (int u = 0; u < N; ++u) d += sum_sq4(g[u], inv_s);
  return d;
}

// Adam's bias correction 1 - beta^t (Kingma and Ba 2015) in binary32 without
// cancellation: beta^t = exp(t log(1 - (1 - beta))), so 1 - beta^t =
// -expm1(t log1p(-(1 - beta))); 1 - beta is exact for beta in [1/2, 1).
__device__ __forceinline__ float adam_bias_correction(float beta, int64_t t) {
  return -expm1f(static_cast<float>(t) * log1pf(-(1.f - beta)));
}

// Node records {first_child, map_offset} of scene sc in shared memory for the
// walk of Section 3.4: one int2 per node, first_child validated here (a child
// block running past the node array is reported and cut).  Returns the staged
// view, or nullptr when there is no room (tree larger than cap nodes); the
// caller synchronises the CTA before the first walk.
__device__ __forceinline__ const int2* stage_tree(const QueryParams& p, const DevScene& sc,
                                                  int2* tree_sm, int cap, int tid, int nthr) {
  if (tree_sm == nullptr || sc.num_nodes > cap) return nullptr;
  for (int n = tid; n < sc.num_nodes; n += nthr) {
    int fc = __ldg(sc.first_child + n);
    if (fc >= 0 && fc > sc.num_nodes - 8) {
      if (p.status) atomicOr(p.status, OCTA_STATUS_BAD_CHILD);
      fc = -1;
    }
    tree_sm[n] = make_int2(fc, __ldg(sc.map_offset + n));
  }
  return tree_sm;
}

// Map base of a level-l node, or -1 (reported) when its R x R map starts
// before the table or runs past its end.  mo < 0 is rejected on its own: in
// 32-bit unsigned arithmetic a base in [-R^2, -1] would wrap the sum back
// into range.  With 0 <= mo < 2^31, R <= 4096 and num_texels < 2^31 the
// unsigned sum cannot wrap.
__device__ __forceinline__ int checked_map_base(const QueryParams& p, const DevScene& sc, int mo,
                                                int R) {
  if (mo < 0 ||
      static_cast<uint32_t>(mo) + static_cast<uint32_t>(R * R) > static_cast<uint32_t>(sc.num_texels)) {
    if (p.status) atomicOr(p.status, OCTA_STATUS_BAD_MAP);
    return -1;
  }
  return mo;
}

// One level of the full query form (Eq. 10 with the directional lookup of
// Eq. 6, the same direction in every cell):
//   direction  the folded direction (ux, uy), p = uv N on the V x V vertex
//              map (N = V - 1, vertex (i, j) at uv = (i, j) / N), the grid
//              cell (i0, j0) = min(floor(p), N - 1) and the triangle of it
//              holding p: cells split along the diagonal parallel to their
//              quadrant's face edge (anti-diagonal where u_x and u_y share a
//              sign), the side decided in binary32 (fx + fy <= 1, fy <= fx);
//              barycentric weights b of the three vertices, whose entries
//              vidx fold mirrored vertices of the map's edges onto one;
//   space      the eight cells around x: c0 = floor(x 2^l - 1/2) (binary32),
//              neighbour j = c0 + (j & 1, j >> 1 & 1, j >> 2), trilinear
//              weights, each cell found by a descent from the root, the
//              weights renormalised over the cells present (base[j] = their
//              map base, -1 for absent cells; all weights 0 when none is).
struct FullLevel {
  int base[8];
  float wn[8];
  int vidx[3];
  float b[3];
  int tri;  // which of the four triangle shapes holds the point (see full_vertex)
};

// Direction part of one level: the triangle of the vertex map holding u and
// its barycentric weights (vidx, b of o).
__device__ __forceinline__ void full_vertex(float ux, float uy, int V, FullLevel& o) {
  const int N = V - 1;
  const float fN = static_cast<float>(N);
  const float px = __fmul_rn(__fadd_rn(__fmul_rn(ux, 0.5f), 0.5f), fN);
  const float py = __fmul_rn(__fadd_rn(__fmul_rn(uy, 0.5f), 0.5f), fN);
  const int i0 = min(max(static_cast<int>(floorf(px)), 0), N - 1);
  const int j0 = min(max(static_cast<int>(floorf(py)), 0), N - 1);
  const float fx = __fsub_rn(px, static_cast<float>(i0));
  const float fy = __fsub_rn(py, static_cast<float>(j0));
  int oi[3], oj[3];
  // tri: 0 / 1 the lower-left / upper-right triangle of an anti-diagonal
  // split, 2 / 3 the lower-right / upper-left one of a main-diagonal split
  if ((i0 >= N / 2) == (j0 >= N / 2)) {  // anti-diagonal split
    if (__fadd_rn(fx, fy) <= 1.f) {
      oi[0] = 0, oj[0] = 0, oi[1] = 1, oj[1] = 0, oi[2] = 0, oj[2] = 1;
      o.b[0] = 1.f - fx - fy, o.b[1] = fx, o.b[2] = fy;
      o.tri = 0;
    } else {
      oi[0] = 1, oj[0] = 1, oi[1] = 1, oj[1] = 0, oi[2] = 0, oj[2] = 1;
      o.b[0] = fx + fy - 1.f, o.b[1] = 1.f - fy, o.b[2] = 1.f - fx;
      o.tri = 1;
    }
  } else {  // main-diagonal split
    if (fy <= fx) {
      oi[0] = 0, oj[0] = 0, oi[1] = 1, oj[1] = 0, oi[2] = 1, oj[2] = 1;
      o.b[0] = 1.f - fx, o.b[1] = fx - fy, o.b[2] = fy;
      o.tri = 2;
    } else {
      oi[0] = 0, oj[0] = 0, oi[1] = 0, oj[1] = 1, oi[2] = 1, oj[2] = 1;
      o.b[0] = 1.f - fy, o.b[1] = fy - fx, o.b[2] = fx;
      o.tri = 3;
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    int vi = i0 + oi[k], vj = j0 + oj[k];
    if (vi == 0 || vi == N) vj = min(vj, N - vj);  // the fold glues each edge to itself
    if (vj == 0 || vj == N) vi = min(vi, N - vi);
    o.vidx[k] = vj * V + vi;
  }
}

// Spatial part of one level: the lower cell c0 = floor(x 2^l - 1/2) per axis
// (binary32) and the fractions t.
__device__ __forceinline__ void full_cells(const float (&xs)[3], int l, int (&c0)[3],
                                           float (&t)[3]) {
  const float fn = static_cast<float>(1 << l);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float pa = __fsub_rn(__fmul_rn(xs[a], fn), 0.5f);
    const float fl = floorf(pa);
    c0[a] = static_cast<int>(fl);
    t[a] = __fsub_rn(pa, fl);
  }
}

// First child of node nd (staged tree, else global memory with the child
// range check), -1 for a leaf.
__device__ __forceinline__ int full_first_child(const QueryParams& p, const DevScene& sc,
                                                const int2* tree, int nd) {
  if (tree) return tree[nd].x;
  int fc = __ldg(sc.first_child + nd);
  if (fc >= 0 && fc > sc.num_nodes - 8) {
    if (p.status) atomicOr(p.status, OCTA_STATUS_BAD_CHILD);
    fc = -1;
  }
  return fc;
}

// Map bases and renormalised trilinear weights of the eight cells whose
// nodes are nd (-1: absent or outside the cube).
__device__ __forceinline__ void full_finish(const QueryParams& p, const DevScene& sc,
                                            const int2* tree, const int (&nd)[8],
                                            const float (&t)[3], int V, FullLevel& o) {
  float wsum = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    o.base[j] = -1;
    o.wn[j] = 0.f;
    if (nd[j] < 0) continue;
    const int mo = checked_map_base(p, sc, tree ? tree[nd[j]].y : __ldg(sc.map_offset + nd[j]), V);
    if (mo < 0) continue;
    o.base[j] = mo;
    o.wn[j] = ((j & 1) ? t[0] : 1.f - t[0]) * (((j >> 1) & 1) ? t[1] : 1.f - t[1]) *
              ((j >> 2) ? t[2] : 1.f - t[2]);
    wsum += o.wn[j];
  }
  const float inv = wsum > 0.f ? 1.f / wsum : 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) o.wn[j] *= inv;
}

// Spatial part of one level from scratch (the cells' map bases and weights
// of o, the lower cell in c0): the eight descents from the root advance
// together, one level per step (eight independent node reads in flight).
__device__ __forceinline__ void cells_form_level(const QueryParams& p, const DevScene& sc,
                                                 const int2* tree, const float (&xs)[3], int l,
                                                 int (&c0)[3], FullLevel& o) {
  const int V = sc.R[l];
  float t[3];
  full_cells(xs, l, c0, t);
  const int n = 1 << l;
  int nd[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int cx = c0[0] + (j & 1), cy = c0[1] + ((j >> 1) & 1), cz = c0[2] + (j >> 2);
    nd[j] = (cx < 0 || cy < 0 || cz < 0 || cx >= n || cy >= n || cz >= n) ? -1 : 0;
  }
  for (int m = 1; m <= l; ++m) {
    const int sh = l - m;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (nd[j] < 0) continue;
      const int fc = full_first_child(p, sc, tree, nd[j]);
      const int slot = (((c0[0] + (j & 1)) >> sh) & 1) | ((((c0[1] + ((j >> 1) & 1)) >> sh) & 1) << 1) |
                       ((((c0[2] + (j >> 2)) >> sh) & 1) << 2);
      nd[j] = fc >= 0 ? fc + slot : -1;
    }
  }
  full_finish(p, sc, tree, nd, t, V, o);
}

// One level of the full form from scratch: the direction's triangle and the
// eight cells.
__device__ __forceinline__ void full_form_level(const QueryParams& p, const DevScene& sc,
                                                const int2* tree, const float (&xs)[3], float ux,
                                                float uy, int l, FullLevel& o) {
  full_vertex(ux, uy, sc.R[l], o);
  int c0[3];
  cells_form_level(p, sc, tree, xs, l, c0, o);
}

// Level-to-level step of the eight cells' nodes: nd holds the nodes of level
// l - 1's cells (lower cell pc), and on return those of level l's (lower
// cell c0).  The parent of a level-l cell c is c >> 1, and since
// floor(x 2^l - 1/2) >> 1 and (floor(x 2^l - 1/2) + 1) >> 1 both lie in
// {pc, pc + 1} per axis, every parent is one of level l - 1's eight cells.
__device__ __forceinline__ void full_descend(const QueryParams& p, const DevScene& sc,
                                             const int2* tree, const int (&pc)[3],
                                             const int (&c0)[3], int l, int (&nd)[8]) {
  const int n = 1 << l;
  int par[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) par[j] = nd[j];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int cx = c0[0] + (j & 1), cy = c0[1] + ((j >> 1) & 1), cz = c0[2] + (j >> 2);
    if (cx < 0 || cy < 0 || cz < 0 || cx >= n || cy >= n || cz >= n) {
      nd[j] = -1;
      continue;
    }
    const int pj = ((cx >> 1) - pc[0]) | (((cy >> 1) - pc[1]) << 1) | (((cz >> 1) - pc[2]) << 2);
    int pn = par[0];
#pragma unroll
    for (int i = 1; i < 8; ++i) pn = pj == i ? par[i] : pn;
    const int fc = pn >= 0 ? full_first_child(p, sc, tree, pn) : -1;
    nd[j] = fc >= 0 ? fc + ((cx & 1) | ((cy & 1) << 1) | ((cz & 1) << 2)) : -1;
  }
}

// Loads of one texel's F features as FP32.
template <typename TT, int F>
struct TexelLoad;

template <>
struct TexelLoad<float, 4> {
  static __device__ __forceinline__ void load(const void* t, int64_t texel, float (&v)[4]) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(t) + texel);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
};

template <>
struct TexelLoad<float, 8> {
  static __device__ __forceinline__ void load(const void* t, int64_t texel, float (&v)[8]) {
    const float4* p = reinterpret_cast<const float4*>(t) + 2 * texel;
    const float4 a = __ldg(p), b = __ldg(p + 1);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  }
};

template <>
struct TexelLoad<__half, 8> {
  static __device__ __forceinline__ void load(const void* t, int64_t texel, float (&v)[8]) {
    const uint4 a = __ldg(reinterpret_cast<const uint4*>(t) + texel);
    const __half2* h = reinterpret_cast<const __half2*>(&a);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = __half22float2(h[i]);
      v[2 * i] = f.x;
      v[2 * i + 1] = f.y;
    }
  }
};

template <>
struct TexelLoad<__half, 4> {
  static __device__ __forceinline__ void load(const void* t, int64_t texel, float (&v)[4]) {
    const uint2 a = __ldg(reinterpret_cast<const uint2*>(t) + texel);
    const __half2* h = reinterpret_cast<const __half2*>(&a);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const float2 f = __half22float2(h[i]);
      v[2 * i] = f.x;
      v[2 * i + 1] = f.y;
    }
  }
};

// Raw texel record kept in registers until the blend: the F features as
// stored (8, 16 or 32 bytes), loaded with the matching vector width.
template <typename TT, int F>
struct TexelRaw {
  static constexpr int BYTES = F * int(sizeof(TT));
  static_assert(BYTES == 8 || BYTES == 16 || BYTES == 32, "texel size");
  static constexpr int WORDS = BYTES / 4;
  uint32_t w[WORDS];
  // texel index < 2^31 (the table limit): 32-bit index arithmetic, one
  // widening multiply-add for the address
  __device__ __forceinline__ void load(const void* t, uint32_t texel) {
    if constexpr (BYTES == 8) {
      const uint2 a = __ldg(reinterpret_cast<const uint2*>(t) + texel);
      w[0] = a.x;
      w[1] = a.y;
    } else {
      const uint4* p = reinterpret_cast<const uint4*>(t) + texel * (BYTES / 16);
#pragma unroll
      for (int i = 0; i < BYTES / 16; ++i) {
        const uint4 a = __ldg(p + i);
        w[4 * i] = a.x;
        w[4 * i + 1] = a.y;
        w[4 * i + 2] = a.z;
        w[4 * i + 3] = a.w;
      }
    }
  }
  __device__ __forceinline__ float get(int f) const {
    if constexpr (sizeof(TT) == 2) {
      const uint32_t v = w[f >> 1];
      return __half2float(__ushort_as_half(static_cast<unsigned short>((f & 1) ? (v >> 16) : (v & 0xFFFFu))));
    } else {
      return __uint_as_float(w[f]);
    }
  }
};

}  // namespace octa
