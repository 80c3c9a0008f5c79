// Per-thread walk and gather of one query, shared by the tensor-core kernels
// and the standalone encoding kernel.
#pragma once
#include "engine_f32.cuh"
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

// One query per thread: fold omega (Eq. 4, 5, canonical binary32), walk the
// query's path down the octree (Section 3.4), load the map base of every
// present level, then gather KP levels, two at a time (both levels' texel
// loads in flight together; one at a time for 32-byte texels), handing the
// F blended features of level l to store(l, v) (absent levels: zeros).
// node_sm / u_sm (nullable, row stride nt) keep the path and the folded
// direction for a later scatter; node_idx / texel_addr outputs of p are
// written for query gq when requested.  F16W (FP16 tables only): blend with
// the four weights rounded to FP16 and FP32 accumulation, for consumers that
// round the features to BF16 anyway (the weight rounding, 2^-12 relative, is
// 8x below that of the BF16 result).
template <int F, typename TT, int KP, bool F16W = false, class Store>
__device__ __forceinline__ void locate_gather_query(const QueryParams& p, const DevScene& sc,
                                                    const float* __restrict__ xs,
                                                    const float* __restrict__ ws, int64_t gq,
                                                    bool valid, int* node_sm, float* u_sm, int q,
                                                    int nt, Store&& store) {
  constexpr int WIN = TexelRaw<TT, F>::BYTES <= 16 ? 2 : 1;
  float x0 = 0.f, x1 = 0.f, x2 = 0.f, w0 = 0.f, w1 = 0.f, w2 = 1.f;
  if (valid) {
    x0 = xs[3 * gq];
    x1 = xs[3 * gq + 1];
    x2 = xs[3 * gq + 2];
    w0 = ws[3 * gq];
    w1 = ws[3 * gq + 1];
    w2 = ws[3 * gq + 2];
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
    for (int l = 0; l < KP; ++l) node_sm[l * nt + q] = node[l];
    u_sm[q] = ux;
    u_sm[nt + q] = uy;
  }
  if (p.node_idx && valid) {
#pragma unroll
    for (int l = 0; l < KP; ++l)
      if (l < p.kmax_out) p.node_idx[gq * p.kmax_out + l] = node[l];
    for (int l = KP; l < p.kmax_out; ++l) p.node_idx[gq * p.kmax_out + l] = -1;
  }
  int mo[KP];  // map base per level (texel index < 2^31), -1 when absent
#pragma unroll
  for (int l = 0; l < KP; ++l)
    mo[l] = node[l] >= 0 ? static_cast<int>(f32::map_base(p, sc, node[l], sc.R[l])) : -1;
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
        for (int k = 0; k < 4; ++k) t[j][k].load(sc.tables, int64_t(mo[l]) + fp[j].idx[k]);
      }
    }
#pragma unroll
    for (int j = 0; j < WIN; ++j) {
      const int l = l0 + j;
      if (l >= KP) continue;
      float v[F];
      if (mo[l] >= 0) {
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
      if (p.texel_addr && valid && l < p.kmax_out) {
        int4 a = make_int4(-1, -1, -1, -1);
        if (mo[l] >= 0)
          a = make_int4(mo[l] + fp[j].idx[0], mo[l] + fp[j].idx[1], mo[l] + fp[j].idx[2],
                        mo[l] + fp[j].idx[3]);
        *reinterpret_cast<int4*>(p.texel_addr + (gq * p.kmax_out + l) * 4) = a;
      }
    }
  }
  if (p.texel_addr && valid)
    for (int l = KP; l < p.kmax_out; ++l)
      *reinterpret_cast<int4*>(p.texel_addr + (gq * p.kmax_out + l) * 4) = make_int4(-1, -1, -1, -1);
}

__device__ __forceinline__ uint32_t pack_bf16x2_rn(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

}  // namespace octa
