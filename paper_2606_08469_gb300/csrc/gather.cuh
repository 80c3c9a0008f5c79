// Per-thread walk and gather of one query, shared by the tensor-core kernels
// and the standalone encoding kernel.
#pragma once
#include "octa_device.cuh"

namespace octa {

// s0 += w * lo(t), s1 += w * hi(t): FP16 weight times the two FP16 features
// packed in t, accumulated in FP32 (mixed-precision fma, one rounding each).
__device__ __forceinline__ void fma_f16x2_f32(float& s0, float& s1, uint16_t w, uint32_t t) {
  asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\t"
      "fma.rn.f32.f16 %0, %3, lo, %0;\n\tfma.rn.f32.f16 %1, %3, hi, %1;\n\t}\n"
      : "+f"(s0), "+f"(s1)
      : "r"(t), "h"(w));
}

// The fold of omega (Eq. 4, 5) and the walk of one query down the octree
// (Section 3.4): mo[o] = map base of level o * TPQ + par on the query's path
// (-1: absent or not this thread's level); returns the path's depth (0 for
// an invalid row).  Node records come from the staged tree (global memory
// when tree is nullptr); thread par 0 writes node_idx when requested.
template <int KP, int TPQ>
__device__ __forceinline__ int walk_query(const QueryParams& p, const DevScene& sc, const int2* tree,
                                          const QueryIn& in, int64_t gq, bool valid, int par,
                                          int (&mo)[(KP + TPQ - 1) / TPQ], float& ux, float& uy) {
  constexpr int KO = (KP + TPQ - 1) / TPQ;
  octa_fold(in.w0, in.w1, in.w2, ux, uy);
  const int cx = min(static_cast<int>(clamp01(in.x0) * 32768.f), 32767);
  const int cy = min(static_cast<int>(clamp01(in.x1) * 32768.f), 32767);
  const int cz = min(static_cast<int>(clamp01(in.x2) * 32768.f), 32767);
  const bool out_nodes = p.node_idx != nullptr && valid && par == 0;
#pragma unroll
  for (int o = 0; o < KO; ++o) mo[o] = -1;
  int depth = 0;
  int nd = valid ? 0 : -1;
#pragma unroll
  for (int l = 0; l < KP; ++l) {
    if (nd < 0) break;
    depth = l + 1;
    if (out_nodes && l < p.kmax_out) p.node_idx[gq * p.kmax_out + l] = nd;
    int2 rec;
    if (tree) {
      rec = tree[nd];
    } else {
      rec = make_int2(__ldg(sc.first_child + nd), __ldg(sc.map_offset + nd));
      if (rec.x >= 0 && rec.x > sc.num_nodes - 8) {
        if (p.status) atomicOr(p.status, OCTA_STATUS_BAD_CHILD);
        rec.x = -1;
      }
    }
    if (l % TPQ == par) mo[l / TPQ] = checked_map_base(p, sc, rec.y, sc.R[l]);
    if (l + 1 >= KP || l + 1 >= sc.K || rec.x < 0) break;
    const int sh = 14 - l;  // level l + 1
    nd = rec.x + (((cx >> sh) & 1) | (((cy >> sh) & 1) << 1) | (((cz >> sh) & 1) << 2));
  }
  if (out_nodes)
    for (int l = depth; l < p.kmax_out; ++l) p.node_idx[gq * p.kmax_out + l] = -1;
  return depth;
}

// One query per TPQ threads: each folds omega (Eq. 4, 5, canonical
// binary32) and walks the query's path down the octree (Section 3.4),
// reading node records from the staged tree (global memory when tree is
// nullptr); thread par (0 <= par < TPQ) then gathers the levels l with
// l % TPQ == par, WIN of its levels at a time (their texel loads in flight
// together; one at a time for 32-byte texels), handing the F blended
// features of level l to store(l, v) (absent levels: zeros).  The cells of
// all levels come from one integer per axis: with c = min(floor(x * 2^15),
// 2^15 - 1), level l's cell is c >> (15 - l), since x * 2^l is exact in
// binary32 and the floor commutes with the shift.  Windows stop at the
// deepest path of the warp (all lanes of a warp share par and call this
// converged); deeper levels only get zero features.  base_sm / u_sm
// (nullable, row stride nt) keep the map base of the thread's levels (-1:
// absent) and the folded direction for a later scatter; node_idx (thread
// par 0) and texel_addr (the level's thread) outputs of p are written for
// query gq when requested.  F16W (FP16 tables only): blend with the four
// weights rounded to FP16 and FP32 accumulation, for consumers that round
// the features to BF16 anyway (the weight rounding, 2^-12 relative, is 8x
// below that of the BF16 result).
template <int F, typename TT, int KP, bool F16W = false, int TPQ = 1, class Store>
__device__ __forceinline__ void locate_gather_query(const QueryParams& p, const DevScene& sc,
                                                    const int2* tree, const QueryIn& in,
                                                    int64_t gq, bool valid, int par, int* base_sm,
                                                    float* u_sm, int q, int nt, Store&& store) {
  static_assert(KP <= 16, "levels");
  static_assert(TPQ == 1 || TPQ == 2, "threads per query");
  // two levels per window for 16-byte texels at one thread per query; one
  // when the levels are split over two threads (register budget)
  constexpr int WIN = (TexelRaw<TT, F>::BYTES <= 16 && TPQ == 1) ? 2 : 1;
  constexpr int KO = (KP + TPQ - 1) / TPQ;  // level slots of one thread
  float ux, uy;
  int mo[KO];  // map base of level o * TPQ + par, -1 when absent
  const int depth = walk_query<KP, TPQ>(p, sc, tree, in, gq, valid, par, mo, ux, uy);
  if (base_sm) {
#pragma unroll
    for (int o = 0; o < KO; ++o)
      if (o * TPQ + par < KP) base_sm[(o * TPQ + par) * nt + q] = mo[o];
    u_sm[q] = ux;
    u_sm[nt + q] = uy;
  }
  const int dw = __reduce_max_sync(0xffffffffu, depth);
  auto addr_out = [&](int l, int4 a) {
    if (p.texel_addr && valid && l < p.kmax_out)
      *reinterpret_cast<int4*>(p.texel_addr + (gq * p.kmax_out + l) * 4) = a;
  };
#pragma unroll
  for (int o0 = 0; o0 < KO; o0 += WIN) {
    if (o0 * TPQ >= dw) {  // warp-uniform: no lane has these levels
#pragma unroll
      for (int o = o0; o < KO; ++o) {
        const int l = o * TPQ + par;
        if (l >= KP) continue;
        float v[F];
#pragma unroll
        for (int f = 0; f < F; ++f) v[f] = 0.f;
        store(l, v);
        addr_out(l, make_int4(-1, -1, -1, -1));
      }
      break;
    }
    TexelRaw<TT, F> t[WIN][4];
    Footprint fp[WIN];
#pragma unroll
    for (int j = 0; j < WIN; ++j) {
      const int o = o0 + j;
      if (o < KO && mo[o] >= 0) {
        fp[j] = footprint(ux, uy, sc.R[o * TPQ + par]);
#pragma unroll
        for (int k = 0; k < 4; ++k) t[j][k].load(sc.tables, uint32_t(mo[o] + fp[j].idx[k]));
      }
    }
#pragma unroll
    for (int j = 0; j < WIN; ++j) {
      const int o = o0 + j;
      const int l = o * TPQ + par;
      if (o >= KO || l >= KP) continue;
      float v[F];
      if (mo[o] >= 0) {
        if constexpr (F16W && sizeof(TT) == 2) {
          uint16_t w16[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) w16[k] = __half_as_ushort(__float2half_rn(fp[j].w[k]));
#pragma unroll
          for (int i = 0; i < F / 2; ++i) {
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int k = 0; k < 4; ++k) fma_f16x2_f32(s0, s1, w16[k], t[j][k].w[i]);
            v[2 * i] = s0;
            v[2 * i + 1] = s1;
          }
        } else {
#pragma unroll
          for (int f = 0; f < F; ++f) {
            float s = fp[j].w[0] * t[j][0].get(f);
            s = fmaf(fp[j].w[1], t[j][1].get(f), s);
            s = fmaf(fp[j].w[2], t[j][2].get(f), s);
            s = fmaf(fp[j].w[3], t[j][3].get(f), s);
            v[f] = s;
          }
        }
      } else {
#pragma unroll
        for (int f = 0; f < F; ++f) v[f] = 0.f;
      }
      store(l, v);
      int4 a = make_int4(-1, -1, -1, -1);
      if (mo[o] >= 0)
        a = make_int4(mo[o] + fp[j].idx[0], mo[o] + fp[j].idx[1], mo[o] + fp[j].idx[2],
                      mo[o] + fp[j].idx[3]);
      addr_out(l, a);
    }
  }
  if (p.texel_addr && valid && par == 0)
    for (int l = KP; l < p.kmax_out; ++l)
      *reinterpret_cast<int4*>(p.texel_addr + (gq * p.kmax_out + l) * 4) = make_int4(-1, -1, -1, -1);
}

// Asynchronous 16-byte global -> shared copies (cp.async, allocating in L1),
// their commit groups and the wait for all but the N newest groups.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ uint4 ld_shared_v4(uint32_t a) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(a)
               : "memory");
  return v;
}

// locate_gather_query for 16-byte texels at one thread per query with the
// texel loads landing in shared memory instead of registers: after the walk,
// the four texels of NS levels are in flight at once (one cp.async group a
// level); level o is blended when its group has arrived, handed to
// store(o, v), and its slot then refilled with level o + NS.  ring: the
// CTA's [NS][4][nt] staging area of 16-byte chunks (16-byte aligned shared
// address); thread q owns chunk q of each (slot, corner) row, so a warp's
// copies and reads of one corner are 512 contiguous bytes.  store must write
// shared memory (it orders the slot's reads before the refill).  Results are
// those of locate_gather_query<F, TT, KP, F16W, 1>.
template <int F, typename TT, int KP, bool F16W, int NS, class Store>
__device__ __forceinline__ void locate_gather_query_staged(const QueryParams& p, const DevScene& sc,
                                                           const int2* tree, const QueryIn& in,
                                                           int64_t gq, bool valid, uint32_t ring,
                                                           int q, int nt, Store&& store) {
  static_assert(TexelRaw<TT, F>::BYTES == 16, "16-byte texels");
  static_assert(NS >= 2 && NS <= KP, "stages");
  float ux, uy;
  int mo[KP];
  const int depth = walk_query<KP, 1>(p, sc, tree, in, gq, valid, 0, mo, ux, uy);
  const int dw = __reduce_max_sync(0xffffffffu, depth);
  const uint4* tab = static_cast<const uint4*>(sc.tables);
  float wt[NS][4];
  auto chunk = [&](int slot, int k) {
    return ring + static_cast<uint32_t>(((slot * 4 + k) * nt + q) * 16);
  };
  auto issue = [&](int o) {
    if (o < KP && mo[o] >= 0) {
      const Footprint fp = footprint(ux, uy, sc.R[o]);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        wt[o % NS][k] = fp.w[k];
        cp_async16(chunk(o % NS, k), tab + static_cast<uint32_t>(mo[o] + fp.idx[k]));
      }
    }
    cp_async_commit();  // an empty group past the path keeps the count
  };
#pragma unroll
  for (int o = 0; o < NS; ++o) issue(o);
#pragma unroll
  for (int o = 0; o < KP; ++o) {
    float v[F];
    if (o >= dw) {  // warp-uniform: no lane has these levels
#pragma unroll
      for (int f = 0; f < F; ++f) v[f] = 0.f;
      store(o, v);
      if (p.texel_addr && valid && o < p.kmax_out)
        *reinterpret_cast<int4*>(p.texel_addr + (gq * p.kmax_out + o) * 4) =
            make_int4(-1, -1, -1, -1);
      continue;
    }
    cp_async_wait<NS - 1>();  // level o's group has landed
    if (mo[o] >= 0) {
      TexelRaw<TT, F> t[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint4 a = ld_shared_v4(chunk(o % NS, k));
        t[k].w[0] = a.x;
        t[k].w[1] = a.y;
        t[k].w[2] = a.z;
        t[k].w[3] = a.w;
      }
      if constexpr (F16W && sizeof(TT) == 2) {
        uint16_t w16[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) w16[k] = __half_as_ushort(__float2half_rn(wt[o % NS][k]));
#pragma unroll
        for (int i = 0; i < F / 2; ++i) {
          float s0 = 0.f, s1 = 0.f;
#pragma unroll
          for (int k = 0; k < 4; ++k) fma_f16x2_f32(s0, s1, w16[k], t[k].w[i]);
          v[2 * i] = s0;
          v[2 * i + 1] = s1;
        }
      } else {
#pragma unroll
        for (int f = 0; f < F; ++f) {
          float s = wt[o % NS][0] * t[0].get(f);
          s = fmaf(wt[o % NS][1], t[1].get(f), s);
          s = fmaf(wt[o % NS][2], t[2].get(f), s);
          s = fmaf(wt[o % NS][3], t[3].get(f), s);
          v[f] = s;
        }
      }
    } else {
#pragma unroll
      for (int f = 0; f < F; ++f) v[f] = 0.f;
    }
    store(o, v);
    if (p.texel_addr && valid && o < p.kmax_out) {
      int4 a = make_int4(-1, -1, -1, -1);
      if (mo[o] >= 0) {
        const Footprint fp = footprint(ux, uy, sc.R[o]);
        a = make_int4(mo[o] + fp.idx[0], mo[o] + fp.idx[1], mo[o] + fp.idx[2], mo[o] + fp.idx[3]);
      }
      *reinterpret_cast<int4*>(p.texel_addr + (gq * p.kmax_out + o) * 4) = a;
    }
    issue(o + NS);
  }
  cp_async_wait<0>();
  if (p.texel_addr && valid)
    for (int l = KP; l < p.kmax_out; ++l)
      *reinterpret_cast<int4*>(p.texel_addr + (gq * p.kmax_out + l) * 4) = make_int4(-1, -1, -1, -1);
}

// The levels 0 .. min(K, KP) - 1 of one query in the full form, the eight
// cells' nodes carried from each level to the next (full_descend): per level
// the lower cell c0 and the cells' map bases and renormalised weights (base,
// wn of fl), handed to fn(l, c0, fl).  UNROLL unrolls the level loop (fn may
// then index register arrays by l).
template <int KP, bool UNROLL, class Fn>
__device__ __forceinline__ void visit_cell_levels(const QueryParams& p, const DevScene& sc,
                                                  const int2* tree, const float (&xs)[3],
                                                  Fn&& fn) {
  int nd[8];
  int pc[3] = {0, 0, 0};
#pragma unroll(UNROLL ? KP : 1)
  for (int l = 0; l < KP; ++l) {
    if (l >= sc.K) break;
    FullLevel fl;
    int c0[3];
    float t[3];
    full_cells(xs, l, c0, t);
    if (l == 0) {
#pragma unroll
      for (int j = 0; j < 8; ++j)  // the root is the one cell of level 0
        nd[j] = (c0[0] + (j & 1) == 0 && c0[1] + ((j >> 1) & 1) == 0 && c0[2] + (j >> 2) == 0)
                    ? 0 : -1;
    } else {
      full_descend(p, sc, tree, pc, c0, l, nd);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) pc[a] = c0[a];
    full_finish(p, sc, tree, nd, t, sc.R[l], fl);
    fn(l, c0, fl);
  }
}

// visit_cell_levels with one direction for all cells: fl also carries the
// triangle (vidx, b) of the folded direction (ux, uy) on the level's map.
template <int KP, bool UNROLL, class Fn>
__device__ __forceinline__ void visit_full_levels(const QueryParams& p, const DevScene& sc,
                                                  const int2* tree, const float (&xs)[3], float ux,
                                                  float uy, Fn&& fn) {
  visit_cell_levels<KP, UNROLL>(p, sc, tree, xs, [&](int l, const int (&)[3], FullLevel& fl) {
    full_vertex(ux, uy, sc.R[l], fl);
    fn(l, fl);
  });
}

// ((a0 b0 + a1 b1) + a2 b2), one rounding per operation.
__device__ __forceinline__ float dot3_f32_rn(const float (&a)[3], const float (&b)[3]) {
  return __fadd_rn(__fadd_rn(__fmul_rn(a[0], b[0]), __fmul_rn(a[1], b[1])), __fmul_rn(a[2], b[2]));
}

// The mirror reflection of Eq. 7: w and n normalised (v / sqrt(v.v)), then
// r = (2 (n.w)) n - w, one rounding per operation.
__device__ __forceinline__ void reflect_f32_rn(const float (&w0)[3], const float (&n0)[3],
                                               float (&r)[3]) {
  const float sw = __fsqrt_rn(dot3_f32_rn(w0, w0)), sn = __fsqrt_rn(dot3_f32_rn(n0, n0));
  const float w[3] = {__fdiv_rn(w0[0], sw), __fdiv_rn(w0[1], sw), __fdiv_rn(w0[2], sw)};
  const float n[3] = {__fdiv_rn(n0[0], sn), __fdiv_rn(n0[1], sn), __fdiv_rn(n0[2], sn)};
  const float d2 = __fmul_rn(2.f, dot3_f32_rn(n, w));
#pragma unroll
  for (int a = 0; a < 3; ++a) r[a] = __fsub_rn(__fmul_rn(d2, n[a]), w[a]);
}

// One level of g_psi's hash encoding at x (Mueller et al. 2022): p = x N in
// binary32, cell i0 = min(floor(p), N - 1) per axis, the trilinear blend of
// the 2 features of the cell's 8 vertices; vertex (i, j, k) is entry
// i + (N+1) (j + (N+1) k) of a dense level, else (i ^ j pi_2 ^ k pi_3) mod T.
__device__ __forceinline__ float2 hash_level(const float2* __restrict__ tab, const float (&xs)[3],
                                             int N, bool dense, uint32_t tmask) {
  const float fN = static_cast<float>(N);
  int i0[3];
  float f[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float pa = __fmul_rn(xs[a], fN);
    i0[a] = min(static_cast<int>(floorf(pa)), N - 1);
    f[a] = __fsub_rn(pa, static_cast<float>(i0[a]));
  }
  const uint32_t side = static_cast<uint32_t>(N + 1);
  float2 t[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const uint32_t i = i0[0] + (c & 1), j = i0[1] + ((c >> 1) & 1), k = i0[2] + (c >> 2);
    const uint32_t e = dense ? i + side * (j + side * k)
                             : (i ^ (j * 2654435761u) ^ (k * 805459861u)) & tmask;
    t[c] = __ldg(tab + e);
  }
  float s0 = 0.f, s1 = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float w = ((c & 1) ? f[0] : 1.f - f[0]) * (((c >> 1) & 1) ? f[1] : 1.f - f[1]) *
                    ((c >> 2) ? f[2] : 1.f - f[2]);
    s0 = fmaf(w, t[c].x, s0);
    s1 = fmaf(w, t[c].y, s1);
  }
  return make_float2(s0, s1);
}

// The trilinear scatter of one level's two feature gradients (g0, g1) into
// the 8 vertices of x's cell, with the forward's cell, weights and entries.
__device__ __forceinline__ void hash_level_scatter(float2* __restrict__ dtab, const float (&xs)[3],
                                                   int N, bool dense, uint32_t tmask, float g0,
                                                   float g1) {
  const float fN = static_cast<float>(N);
  uint32_t i0[3];
  float f[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float pa = __fmul_rn(xs[a], fN);
    const int c = min(static_cast<int>(floorf(pa)), N - 1);
    i0[a] = static_cast<uint32_t>(c);
    f[a] = __fsub_rn(pa, static_cast<float>(c));
  }
  const uint32_t side = static_cast<uint32_t>(N + 1);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const uint32_t i = i0[0] + (c & 1), j = i0[1] + ((c >> 1) & 1), k = i0[2] + (c >> 2);
    const uint32_t e = dense ? i + side * (j + side * k)
                             : (i ^ (j * 2654435761u) ^ (k * 805459861u)) & tmask;
    const float w = ((c & 1) ? f[0] : 1.f - f[0]) * (((c >> 1) & 1) ? f[1] : 1.f - f[1]) *
                    ((c >> 2) ? f[2] : 1.f - f[2]);
    atomicAdd(dtab + e, make_float2(w * g0, w * g1));
  }
}

// Cell j's shifted direction v_j = (x - c_j) d + omega_r (Eq. 9; c_j =
// (c0 + offset_j + 1/2) 2^-l, exact) and e = x - c_j, one rounding per
// operation.
__device__ __forceinline__ void shifted_dir(const float (&xs)[3], const float (&wr)[3], float disp,
                                            int l, const int (&c0)[3], int j, float (&dir)[3],
                                            float (&e)[3]) {
  const float scale = __int_as_float((127 - l) << 23);  // 2^-l
  const int cj[3] = {c0[0] + (j & 1), c0[1] + ((j >> 1) & 1), c0[2] + (j >> 2)};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float c = __fmul_rn(__fadd_rn(static_cast<float>(cj[a]), 0.5f), scale);
    e[a] = __fsub_rn(xs[a], c);
    dir[a] = __fadd_rn(__fmul_rn(e[a], disp), wr[a]);
  }
}

// Cell j's triangle in the shifted form: the direction v_j, folded, and its
// triangle and barycentric weights on the level's vertex map (vidx, b of fl).
__device__ __forceinline__ void shifted_cell_vertex(const DevScene& sc, const float (&xs)[3],
                                                    const float (&wr)[3], float disp, int l,
                                                    const int (&c0)[3], int j, FullLevel& fl) {
  float dir[3], e[3];
  shifted_dir(xs, wr, disp, l, c0, j, dir, e);
  float ux, uy;
  octa_fold(dir[0], dir[1], dir[2], ux, uy);
  full_vertex(ux, uy, sc.R[l], fl);
}

// shifted_cell_vertex, and the derivative of its barycentric weights in the
// disparity (Eq. 9 differentiated on the triangle the lookup chose):
// dv/dd = x - c_j; the octahedral map u = (v_x, v_y) / |v|_1 (Eq. 4) has
// du_a/dv = (e_a - u_a sgn(v)) / |v|_1, and the fold of Eq. 5 (v_z < 0)
// turns (u_x, u_y) into ((1 - |u_y|) sgn u_x, (1 - |u_x|) sgn u_y), whose
// derivatives are those of (u_y, u_x) times -sgn(u_x) sgn(u_y); the map
// position is p = (u / 2 + 1 / 2) N, and each triangle's weights are
// affine in p's fractions (full_vertex) with the constant gradients used
// below.  db[k] = d b_k / d d, in binary32.
__device__ __forceinline__ void shifted_cell_vertex_dd(const DevScene& sc, const float (&xs)[3],
                                                       const float (&wr)[3], float disp, int l,
                                                       const int (&c0)[3], int j, FullLevel& fl,
                                                       float (&db)[3]) {
  float dir[3], e[3];
  shifted_dir(xs, wr, disp, l, c0, j, dir, e);
  float ux, uy;
  octa_fold(dir[0], dir[1], dir[2], ux, uy);
  full_vertex(ux, uy, sc.R[l], fl);
  const float s = fabsf(dir[0]) + fabsf(dir[1]) + fabsf(dir[2]);
  const float is = s > 0.f ? 1.f / s : 0.f;
  const float a = dir[0] * is, b = dir[1] * is;
  const float g = (dir[0] >= 0.f ? e[0] : -e[0]) + (dir[1] >= 0.f ? e[1] : -e[1]) +
                  (dir[2] >= 0.f ? e[2] : -e[2]);
  float dux = (e[0] - a * g) * is, duy = (e[1] - b * g) * is;
  if (dir[2] < 0.f) {  // the fold: swapped rows, factor -sgn(a) sgn(b)
    const float m = ((a >= 0.f) == (b >= 0.f)) ? -1.f : 1.f;
    const float t = dux;
    dux = m * duy;
    duy = m * t;
  }
  const float hN = 0.5f * static_cast<float>(sc.R[l] - 1);
  const float px = hN * dux, py = hN * duy;
  switch (fl.tri) {
    case 0:  // b = (1 - fx - fy, fx, fy)
      db[0] = -px - py, db[1] = px, db[2] = py;
      break;
    case 1:  // b = (fx + fy - 1, 1 - fy, 1 - fx)
      db[0] = px + py, db[1] = -py, db[2] = -px;
      break;
    case 2:  // b = (1 - fx, fx - fy, fy)
      db[0] = -px, db[1] = px - py, db[2] = py;
      break;
    default:  // b = (1 - fy, fy - fx, fx)
      db[0] = -py, db[1] = py - px, db[2] = px;
      break;
  }
}

// The shifted form of one query per thread (encoding kernel): per level the
// eight cells' nodes, then in each present cell j its own direction
// v_j = (x - c_j) d + omega_r (Eq. 9; c_j = (c + 1/2) 2^-l exact), the
// triangle of v_j on the cell's vertex map and the blend of its 3 vertices
// (Eq. 6) with the renormalised trilinear weight (Eq. 10); store(l, v) for
// every l < KP as gather_full_query, texel_addr rows of 24 entries.
// nrm / disp: the normal and disparity arrays query gq indexes.
template <int F, typename TT, int KP, class Store>
__device__ __forceinline__ void gather_shifted_query(const QueryParams& p, const DevScene& sc,
                                                     const int2* tree, const QueryIn& in,
                                                     int64_t gq, bool valid, const float* nrm,
                                                     const float* disparity, Store&& store) {
  const float xs[3] = {clamp01(in.x0), clamp01(in.x1), clamp01(in.x2)};
  const bool want_addr = p.texel_addr != nullptr && valid;
  int done = 0;
  if (valid) {
    const float w0[3] = {in.w0, in.w1, in.w2};
    const float n0[3] = {nrm[3 * gq], nrm[3 * gq + 1], nrm[3 * gq + 2]};
    float wr[3];
    reflect_f32_rn(w0, n0, wr);
    const float disp = disparity[gq];
    visit_cell_levels<KP, false>(p, sc, tree, xs, [&](int l, const int (&c0)[3], FullLevel& fl) {
      float v[F];
#pragma unroll
      for (int f = 0; f < F; ++f) v[f] = 0.f;
      int32_t* aout = (want_addr && l < p.kmax_out) ? p.texel_addr + (gq * p.kmax_out + l) * 24
                                                    : nullptr;
#pragma unroll 1
      for (int j = 0; j < 8; ++j) {
        if (fl.base[j] < 0) {
          if (aout)
            for (int k = 0; k < 3; ++k) aout[3 * j + k] = -1;
          continue;
        }
        shifted_cell_vertex(sc, xs, wr, disp, l, c0, j, fl);
        TexelRaw<TT, F> tx[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) tx[k].load(sc.tables, uint32_t(fl.base[j] + fl.vidx[k]));
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float w = fl.wn[j] * fl.b[k];
#pragma unroll
          for (int f = 0; f < F; ++f) v[f] = fmaf(w, tx[k].get(f), v[f]);
          if (aout) aout[3 * j + k] = fl.base[j] + fl.vidx[k];
        }
      }
      store(l, v);
      done = l + 1;
    });
  }
#pragma unroll 1
  for (int l = done; l < KP; ++l) {
    float v[F];
#pragma unroll
    for (int f = 0; f < F; ++f) v[f] = 0.f;
    store(l, v);
    if (want_addr && l < p.kmax_out)
      for (int k = 0; k < 24; ++k) p.texel_addr[(gq * p.kmax_out + l) * 24 + k] = -1;
  }
  if (want_addr)
    for (int l = KP; l < p.kmax_out; ++l)
      for (int k = 0; k < 24; ++k) p.texel_addr[(gq * p.kmax_out + l) * 24 + k] = -1;
}

// The full query form of one query per thread (encoding and tensor-core
// kernels): the 8 x 3 vertex features of each level blended into its F
// features, handed to store(l, v) for every l < KP (zeros for absent levels
// and levels beyond the scene's K).  texel_addr (when requested) receives
// the 24 entries of each level (neighbour-major, -1 where absent).
template <int F, typename TT, int KP, class Store>
__device__ __forceinline__ void gather_full_query(const QueryParams& p, const DevScene& sc,
                                                  const int2* tree, const QueryIn& in, int64_t gq,
                                                  bool valid, Store&& store) {
  float ux, uy;
  octa_fold(in.w0, in.w1, in.w2, ux, uy);
  const float xs[3] = {clamp01(in.x0), clamp01(in.x1), clamp01(in.x2)};
  const bool want_addr = p.texel_addr != nullptr && valid;
  int done = 0;  // levels handed over
  if (valid) {
    visit_full_levels<KP, false>(p, sc, tree, xs, ux, uy, [&](int l, const FullLevel& fl) {
      float v[F];
#pragma unroll
      for (int f = 0; f < F; ++f) v[f] = 0.f;
      int32_t* aout = (want_addr && l < p.kmax_out) ? p.texel_addr + (gq * p.kmax_out + l) * 24
                                                    : nullptr;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (fl.base[j] < 0) {
          if (aout)
            for (int k = 0; k < 3; ++k) aout[3 * j + k] = -1;
          continue;
        }
        TexelRaw<TT, F> tx[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) tx[k].load(sc.tables, uint32_t(fl.base[j] + fl.vidx[k]));
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float w = fl.wn[j] * fl.b[k];
#pragma unroll
          for (int f = 0; f < F; ++f) v[f] = fmaf(w, tx[k].get(f), v[f]);
          if (aout) aout[3 * j + k] = fl.base[j] + fl.vidx[k];
        }
      }
      store(l, v);
      done = l + 1;
    });
  }
#pragma unroll 1
  for (int l = done; l < KP; ++l) {
    float v[F];
#pragma unroll
    for (int f = 0; f < F; ++f) v[f] = 0.f;
    store(l, v);
    if (want_addr && l < p.kmax_out)
      for (int k = 0; k < 24; ++k) p.texel_addr[(gq * p.kmax_out + l) * 24 + k] = -1;
  }
  if (want_addr)
    for (int l = KP; l < p.kmax_out; ++l)
      for (int k = 0; k < 24; ++k) p.texel_addr[(gq * p.kmax_out + l) * 24 + k] = -1;
}

__device__ __forceinline__ uint32_t pack_bf16x2_rn(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

}  // namespace octa
