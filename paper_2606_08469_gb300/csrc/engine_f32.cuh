// FP32 path of the OctaOctree query (forward and backward) on the CUDA cores.
//
// One persistent CTA of 256 threads works on tiles of QT = 128 queries of
// one scene.  Per tile:
//   1. locate   one thread per query: octahedral fold of omega (Eq. 4, 5) and
//               the descent from the root to the containing node of every
//               level (Section 3.4);
//   2. gather   one thread per (query, level): bilinear blend of the 4
//               wrapped texels of that node's map, written feature-major into
//               shared memory (the concatenation of Eq. 11 is the row index);
//   3. decoder  Eq. 13 as register-blocked FP32 GEMMs over the tile, weights
//               and activations in shared memory;
//   4. backward (BWD) delta chain, dW accumulated in registers across all
//               tiles the CTA handles, dh, then float4 atomics into the FP32
//               table gradient.
// Shared-memory activations are stored [feature][query] with row stride
// LDA = QT + 4 floats, so every GEMM operand read is a 16-byte vector and
// rows of neighbouring features fall into different banks.
#pragma once
#include "gather.cuh"

namespace octa {
namespace f32 {

constexpr int NT = 256;        // threads per CTA

// Two independent binary32 fused multiply-adds in one instruction (the
// packed FP32 pair form of sm_100 and later): d.x = a.x*b.x + c.x, d.y =
// a.y*b.y + c.y, each rounded once, exactly as two fmaf calls.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long A, B, Cc, D;
  asm("mov.b64 %0, {%1, %2};" : "=l"(A) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(B) : "f"(b.x), "f"(b.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(Cc) : "f"(c.x), "f"(c.y));
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(D) : "l"(A), "l"(B), "l"(Cc));
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(D));
  return d;
}
constexpr int LDA = QT + 4;    // activation row stride (floats)

template <int F_, int WP_, int H_, int NH_, bool BWD_>
struct Shape {
  static constexpr int F = F_, WP = WP_, H = H_, NH = NH_;
  static constexpr bool BWD = BWD_;
  static constexpr int KMAX = WP / F;
  static_assert(WP % F == 0 && WP % 4 == 0, "padded input width");
  static_assert(H % 16 == 0, "hidden width");
  // weights: W_0 [H][WP], W_1..W_{NH-1} [H][H], W_L [4][H] (row 3 zero)
  static constexpr int WSM = H * WP + (NH - 1) * H * H + 4 * H;
  static constexpr int MAXW = WP > H ? WP : H;
  // BWD keeps h, a_1..a_NH and delta_L; FWD ping-pongs two buffers
  static constexpr int ACT_ROWS = BWD ? (WP + NH * H + 4) : 2 * MAXW;
  static constexpr int TREE_NODES = 1280;  // staged octree, int2 per node
  static constexpr size_t bytes_before_tree(int wdup) {
    return sizeof(float) * (size_t(WSM) * wdup + size_t(ACT_ROWS) * LDA) +
           sizeof(int) * KMAX * QT + sizeof(float) * 2 * QT;
  }
  // the backward kernels keep every weight twice in a row (w, w) where the
  // shared memory allows (one 16-byte broadcast load then yields two ready
  // operand pairs of ffma2); 227 KB per CTA less 1 KB of static memory
  static constexpr int WDUP =
      BWD && bytes_before_tree(2) + 8 * size_t(TREE_NODES) <= 232448 - 1024 ? 2 : 1;
  static constexpr bool DUP = WDUP == 2;
  static constexpr size_t TREE_OFF = bytes_before_tree(WDUP);
  static constexpr size_t SMEM = TREE_OFF + 8 * size_t(TREE_NODES);
};

// ---------------------------------------------------------------------------
// Tile GEMMs (all operands in shared memory)
// ---------------------------------------------------------------------------

// Y[m][q] = relu(sum_k W[m][k] X[k][q]);  W row-major [M][KD].
// Warp w owns rows [w*M/8, (w+1)*M/8) (weight reads are warp-uniform
// broadcasts); lane owns queries [4 lane, 4 lane + 4).
template <int M, int KD, bool DUP = false>
__device__ __forceinline__ void gemm_fwd_relu(const float* __restrict__ W,
                                              const float* __restrict__ X,
                                              float* __restrict__ Y) {
  constexpr int TM = M / 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = warp * TM, q0 = lane * 4;
  if constexpr (DUP) {  // W holds each weight twice; two query columns per ffma2
    float2 lo[TM], hi[TM];
#pragma unroll
    for (int i = 0; i < TM; ++i) lo[i] = hi[i] = make_float2(0.f, 0.f);
#pragma unroll 2
    for (int k = 0; k < KD; k += 4) {
      float4 x[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) x[c] = *reinterpret_cast<const float4*>(X + (k + c) * LDA + q0);
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        const float4* wr = reinterpret_cast<const float4*>(W + 2 * ((m0 + i) * KD + k));
        const float4 wa = wr[0], wb = wr[1];
        const float2 w2[4] = {make_float2(wa.x, wa.y), make_float2(wa.z, wa.w),
                              make_float2(wb.x, wb.y), make_float2(wb.z, wb.w)};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          lo[i] = ffma2(w2[c], make_float2(x[c].x, x[c].y), lo[i]);
          hi[i] = ffma2(w2[c], make_float2(x[c].z, x[c].w), hi[i]);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < TM; ++i)
      *reinterpret_cast<float4*>(Y + (m0 + i) * LDA + q0) =
          make_float4(fmaxf(lo[i].x, 0.f), fmaxf(lo[i].y, 0.f), fmaxf(hi[i].x, 0.f),
                      fmaxf(hi[i].y, 0.f));
    return;
  }
  float acc[TM][4];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll 2
  for (int k = 0; k < KD; k += 4) {
    float4 x[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) x[c] = *reinterpret_cast<const float4*>(X + (k + c) * LDA + q0);
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const float4 w = *reinterpret_cast<const float4*>(W + (m0 + i) * KD + k);
      const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        acc[i][0] = fmaf(wv[c], x[c].x, acc[i][0]);
        acc[i][1] = fmaf(wv[c], x[c].y, acc[i][1]);
        acc[i][2] = fmaf(wv[c], x[c].z, acc[i][2]);
        acc[i][3] = fmaf(wv[c], x[c].w, acc[i][3]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    float4 o;
    o.x = fmaxf(acc[i][0], 0.f);
    o.y = fmaxf(acc[i][1], 0.f);
    o.z = fmaxf(acc[i][2], 0.f);
    o.w = fmaxf(acc[i][3], 0.f);
    *reinterpret_cast<float4*>(Y + (m0 + i) * LDA + q0) = o;
  }
}

// Y[k][q] = (sum_m W[m][k] D[m][q]) * (MASK ? 1[Y[k][q] > 0] : 1), W
// row-major [M][KD].  Rows k come in chunks of 4; chunk c goes to warp c % 8.
// With MASK the result overwrites the activation it is masked with (each
// element is read and written by the same thread).
template <int M, int KD, bool MASK, bool DUP = false>
__device__ __forceinline__ void gemm_bwd_data(const float* __restrict__ W,
                                              const float* __restrict__ D, float* Y) {
  constexpr int NCH = KD / 4;
  constexpr int CPW = (NCH + 7) / 8;
  static_assert(KD % 4 == 0, "KD");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q0 = lane * 4;
  if constexpr (DUP) {  // W holds each weight twice; two query columns per ffma2
    float2 lo[CPW][4], hi[CPW][4];
#pragma unroll
    for (int j = 0; j < CPW; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) lo[j][r] = hi[j][r] = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int m = 0; m < M; ++m) {
      const float4 d = *reinterpret_cast<const float4*>(D + m * LDA + q0);
      const float2 dlo = make_float2(d.x, d.y), dhi = make_float2(d.z, d.w);
#pragma unroll
      for (int j = 0; j < CPW; ++j) {
        const int ch = warp + 8 * j;
        if (ch < NCH) {
          const float4* wr = reinterpret_cast<const float4*>(W + 2 * (m * KD + 4 * ch));
          const float4 wa = wr[0], wb = wr[1];
          const float2 w2[4] = {make_float2(wa.x, wa.y), make_float2(wa.z, wa.w),
                                make_float2(wb.x, wb.y), make_float2(wb.z, wb.w)};
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            lo[j][r] = ffma2(w2[r], dlo, lo[j][r]);
            hi[j][r] = ffma2(w2[r], dhi, hi[j][r]);
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < CPW; ++j) {
      const int ch = warp + 8 * j;
      if (ch < NCH) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          float* y = Y + (4 * ch + r) * LDA + q0;
          float4 o = make_float4(lo[j][r].x, lo[j][r].y, hi[j][r].x, hi[j][r].y);
          if (MASK) {
            const float4 a = *reinterpret_cast<const float4*>(y);
            o.x = a.x > 0.f ? o.x : 0.f;
            o.y = a.y > 0.f ? o.y : 0.f;
            o.z = a.z > 0.f ? o.z : 0.f;
            o.w = a.w > 0.f ? o.w : 0.f;
          }
          *reinterpret_cast<float4*>(y) = o;
        }
      }
    }
    return;
  }
  float acc[CPW][4][4];
#pragma unroll
  for (int j = 0; j < CPW; ++j)
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[j][r][c] = 0.f;
#pragma unroll 4
  for (int m = 0; m < M; ++m) {
    const float4 d = *reinterpret_cast<const float4*>(D + m * LDA + q0);
#pragma unroll
    for (int j = 0; j < CPW; ++j) {
      const int ch = warp + 8 * j;
      if (ch < NCH) {
        const float4 w = *reinterpret_cast<const float4*>(W + m * KD + 4 * ch);
        const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          acc[j][r][0] = fmaf(wv[r], d.x, acc[j][r][0]);
          acc[j][r][1] = fmaf(wv[r], d.y, acc[j][r][1]);
          acc[j][r][2] = fmaf(wv[r], d.z, acc[j][r][2]);
          acc[j][r][3] = fmaf(wv[r], d.w, acc[j][r][3]);
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < CPW; ++j) {
    const int ch = warp + 8 * j;
    if (ch < NCH) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        float* y = Y + (4 * ch + r) * LDA + q0;
        float4 o = make_float4(acc[j][r][0], acc[j][r][1], acc[j][r][2], acc[j][r][3]);
        if (MASK) {
          const float4 a = *reinterpret_cast<const float4*>(y);
          o.x = a.x > 0.f ? o.x : 0.f;
          o.y = a.y > 0.f ? o.y : 0.f;
          o.z = a.z > 0.f ? o.z : 0.f;
          o.w = a.w > 0.f ? o.w : 0.f;
        }
        *reinterpret_cast<float4*>(y) = o;
      }
    }
  }
}

// Weight-gradient tile of one thread: rows m = mb + 16 r, columns
// k = kb + 16 c with (mb, kb) = (tid % 16, tid / 16).
template <int M, int KD>
struct WGrad {
  static constexpr int TMW = M / 16;
  static constexpr int TKW = (KD + 15) / 16;
  float a[TMW][TKW];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int r = 0; r < TMW; ++r)
#pragma unroll
      for (int c = 0; c < TKW; ++c) a[r][c] = 0.f;
  }
  // a[r][c] += sum_q D[m_r][q] X[k_c][q]: the tile's sum is kept as two
  // partial sums over even and odd queries (one ffma2 per query pair) and
  // folded into a once per tile.
  __device__ __forceinline__ void accumulate(const float* __restrict__ D,
                                             const float* __restrict__ X) {
    const int mb = threadIdx.x & 15, kb = threadIdx.x >> 4;
    float2 t[TMW][TKW];
#pragma unroll
    for (int r = 0; r < TMW; ++r)
#pragma unroll
      for (int c = 0; c < TKW; ++c) t[r][c] = make_float2(0.f, 0.f);
#pragma unroll 2
    for (int q = 0; q < QT; q += 4) {
      float4 d[TMW], x[TKW];
#pragma unroll
      for (int r = 0; r < TMW; ++r)
        d[r] = *reinterpret_cast<const float4*>(D + (mb + 16 * r) * LDA + q);
#pragma unroll
      for (int c = 0; c < TKW; ++c)
        x[c] = (kb + 16 * c < KD) ? *reinterpret_cast<const float4*>(X + (kb + 16 * c) * LDA + q)
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int r = 0; r < TMW; ++r)
#pragma unroll
        for (int c = 0; c < TKW; ++c) {
          t[r][c] = ffma2(make_float2(d[r].x, d[r].y), make_float2(x[c].x, x[c].y), t[r][c]);
          t[r][c] = ffma2(make_float2(d[r].z, d[r].w), make_float2(x[c].z, x[c].w), t[r][c]);
        }
    }
#pragma unroll
    for (int r = 0; r < TMW; ++r)
#pragma unroll
      for (int c = 0; c < TKW; ++c) a[r][c] += t[r][c].x + t[r][c].y;
  }
  // d_weights[off + m * in + k] += a (k < in only: padded columns are zero)
  __device__ __forceinline__ void flush(float* dW, int in) const {
    const int mb = threadIdx.x & 15, kb = threadIdx.x >> 4;
#pragma unroll
    for (int r = 0; r < TMW; ++r)
#pragma unroll
      for (int c = 0; c < TKW; ++c) {
        const int k = kb + 16 * c;
        if (k < KD && k < in) atomicAdd(dW + (mb + 16 * r) * in + k, a[r][c]);
      }
  }
};

// ---------------------------------------------------------------------------
// The engine
// ---------------------------------------------------------------------------

template <class S>
struct Grads {
  WGrad<S::H, S::WP> w0;
  WGrad<S::H, S::H> wh[S::NH > 1 ? S::NH - 1 : 1];
  float wl;
  __device__ __forceinline__ void zero() {
    w0.zero();
#pragma unroll
    for (int i = 0; i < S::NH - 1; ++i) wh[i].zero();
    wl = 0.f;
  }
  __device__ __forceinline__ void flush(const DevScene& sc) const {
    float* dW = sc.d_weights;
    w0.flush(dW + sc.w_offset[0], sc.widths[0]);
#pragma unroll
    for (int i = 0; i < S::NH - 1; ++i) wh[i].flush(dW + sc.w_offset[i + 1], S::H);
    if (threadIdx.x < 3 * S::H) atomicAdd(dW + sc.w_offset[S::NH] + threadIdx.x, wl);
  }
};

// Weight element i of the padded layout (W_0 [H][WP], W_1.. [H][H], W_L
// [4][H] with row 3 zero), stored once or, for the backward kernels, twice
// in a row.
template <class S>
__device__ __forceinline__ void put_weight(float* wsm, int i, float v) {
  if constexpr (S::WDUP == 2)
    reinterpret_cast<float2*>(wsm)[i] = make_float2(v, v);
  else
    wsm[i] = v;
}

template <class S>
__device__ __forceinline__ void load_weights(const DevScene& sc, float* wsm) {
  const float* Wg = static_cast<const float*>(sc.weights);
  const int in0 = sc.widths[0];
  for (int i = threadIdx.x; i < S::H * S::WP; i += NT) {
    const int m = i / S::WP, k = i % S::WP;
    put_weight<S>(wsm, i, k < in0 ? Wg[sc.w_offset[0] + m * in0 + k] : 0.f);
  }
  int dst = S::H * S::WP;
  for (int l = 1; l < S::NH; ++l, dst += S::H * S::H)
    for (int i = threadIdx.x; i < S::H * S::H; i += NT)
      put_weight<S>(wsm, dst + i, Wg[sc.w_offset[l] + i]);
  for (int i = threadIdx.x; i < 4 * S::H; i += NT)
    put_weight<S>(wsm, dst + i, i < 3 * S::H ? Wg[sc.w_offset[S::NH] + i] : 0.f);
}

// Phase 1: fold omega and walk the tree (one thread per query), reading node
// records from the staged tree (global memory when tree is nullptr).  Level
// l's cell is c >> (15 - l) with c = min(floor(x * 2^15), 2^15 - 1) per axis.
// In the trilinear vertex form (Eq. 10) every level needs eight cells, so the
// walk is left to the (query, level) items: rows 0-2 of node_sm then hold the
// clamped position (as floats) and row 3 the query's validity (0 / -1).  The
// shifted form (Eq. 7-9) also keeps omega_r (rows 4-5 of node_sm and row 0
// of u_sm) and the disparity (row 1 of u_sm), read from nrm / dsp at index
// gqs, the query's row of those arrays.
template <int KMAX, bool SHIFT>
__device__ __forceinline__ void locate_tile(const QueryParams& p, const DevScene& sc,
                                            const int2* tree, const QueryIn& in, int64_t q0,
                                            int nq, int* node_sm, float* u_sm,
                                            const float* nrm = nullptr, const float* dsp = nullptr,
                                            int64_t gqs = 0) {
  static_assert(KMAX >= 6, "the shifted form keeps positions, validity and omega_r in six rows");
  const int q = threadIdx.x;
  if (q >= QT) return;
  const bool valid = q < nq;
  const int64_t gq = q0 + q;
  if (sc.query_form != OCTA_FORM_CELL_BILINEAR) {  // the items look up their own cells
    float* xs = reinterpret_cast<float*>(node_sm);  // [3][QT] positions
    xs[q] = clamp01(in.x0);
    xs[QT + q] = clamp01(in.x1);
    xs[2 * QT + q] = clamp01(in.x2);
    node_sm[3 * QT + q] = valid ? 0 : -1;           // validity of the query
    if (SHIFT && sc.query_form == OCTA_FORM_SHIFTED) {
      float wr[3] = {0.f, 0.f, 1.f}, disp = 0.f;
      if (valid) {
        const float w0[3] = {in.w0, in.w1, in.w2};
        const float n0[3] = {nrm[3 * gqs], nrm[3 * gqs + 1], nrm[3 * gqs + 2]};
        reflect_f32_rn(w0, n0, wr);
        disp = dsp[gqs];
      }
      xs[4 * QT + q] = wr[0];
      xs[5 * QT + q] = wr[1];
      u_sm[q] = wr[2];
      u_sm[QT + q] = disp;
      return;
    }
    float ux, uy;
    octa_fold(in.w0, in.w1, in.w2, ux, uy);
    u_sm[q] = ux;
    u_sm[QT + q] = uy;
    return;
  }
  float ux, uy;
  octa_fold(in.w0, in.w1, in.w2, ux, uy);
  u_sm[q] = ux;
  u_sm[QT + q] = uy;
  const int cx = min(static_cast<int>(clamp01(in.x0) * 32768.f), 32767);
  const int cy = min(static_cast<int>(clamp01(in.x1) * 32768.f), 32767);
  const int cz = min(static_cast<int>(clamp01(in.x2) * 32768.f), 32767);
  int node = valid ? 0 : -1;
  node_sm[q] = node;
#pragma unroll
  for (int l = 1; l < KMAX; ++l) {
    if (l < sc.K && node >= 0) {
      const int sh = 15 - l;
      const int slot = ((cx >> sh) & 1) | (((cy >> sh) & 1) << 1) | (((cz >> sh) & 1) << 2);
      int fc;
      if (tree) {
        fc = tree[node].x;
      } else {
        fc = __ldg(sc.first_child + node);
        if (fc >= 0 && fc > sc.num_nodes - 8) {
          if (p.status) atomicOr(p.status, OCTA_STATUS_BAD_CHILD);
          fc = -1;
        }
      }
      node = fc >= 0 ? fc + slot : -1;
    } else {
      node = -1;
    }
    node_sm[l * QT + q] = node;
  }
  if (p.node_idx && valid) {
    for (int l = 0; l < p.kmax_out; ++l)
      p.node_idx[gq * p.kmax_out + l] = l < KMAX ? node_sm[l * QT + q] : -1;
  }
}

// Base texel of a node's map, or -1 if the map would leave the table.
__device__ __forceinline__ int64_t map_base(const QueryParams& p, const DevScene& sc,
                                            const int2* tree, int node, int R) {
  return checked_map_base(p, sc, tree ? tree[node].y : __ldg(sc.map_offset + node), R);
}

// Phase 2: one thread per (query, level) item for levels [0, nlev); writes
// feature f of level l for query q to h[(l*F + f) * ld_feat + q * ld_q]
// (levels past the scene's K: Eq. 12's attributes, else zeros).  In
// the trilinear vertex form the item blends the 8 x 3 vertex features of
// full_form_level (Eq. 6, 10; texel_addr rows of 24 entries a level).
template <int F, typename TT, bool SHIFT>
__device__ __forceinline__ void gather_tile(const QueryParams& p, const DevScene& sc,
                                            const int2* tree, int64_t q0, int nq, int nlev,
                                            const int* node_sm,
                                            const float* u_sm, float* h, int ld_feat, int ld_q) {
  if (sc.query_form != OCTA_FORM_CELL_BILINEAR) {
    const float* xsm = reinterpret_cast<const float*>(node_sm);
    const bool shifted = SHIFT && sc.query_form == OCTA_FORM_SHIFTED;
    for (int it = threadIdx.x; it < nlev * QT; it += NT) {
      const int l = it / QT, q = it % QT;
      float v[F];
#pragma unroll
      for (int f = 0; f < F; ++f) v[f] = 0.f;
      const bool on = node_sm[3 * QT + q] >= 0 && l < sc.K;
      int32_t* aout = (p.texel_addr && q < nq && l < p.kmax_out)
                          ? p.texel_addr + ((q0 + q) * p.kmax_out + l) * 24 : nullptr;
      if (on) {
        const float xs[3] = {xsm[q], xsm[QT + q], xsm[2 * QT + q]};
        const float wr[3] = {xsm[4 * QT + q], xsm[5 * QT + q], u_sm[q]};
        const float disp = u_sm[QT + q];
        FullLevel fl;
        int c0[3];
        if (shifted)
          cells_form_level(p, sc, tree, xs, l, c0, fl);
        else
          full_form_level(p, sc, tree, xs, u_sm[q], u_sm[QT + q], l, fl);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (fl.base[j] < 0) {
            if (aout)
              for (int k = 0; k < 3; ++k) aout[3 * j + k] = -1;
            continue;
          }
          if (shifted) shifted_cell_vertex(sc, xs, wr, disp, l, c0, j, fl);
          float t[3][F];
#pragma unroll
          for (int k = 0; k < 3; ++k)
            TexelLoad<TT, F>::load(sc.tables, int64_t(fl.base[j] + fl.vidx[k]), t[k]);
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const float w = fl.wn[j] * fl.b[k];
#pragma unroll
            for (int f = 0; f < F; ++f) v[f] = fmaf(w, t[k][f], v[f]);
            if (aout) aout[3 * j + k] = fl.base[j] + fl.vidx[k];
          }
        }
      } else {
        if (aout)
          for (int k = 0; k < 24; ++k) aout[k] = -1;
        if (p.n_attrs > 0 && l >= sc.K) attr_columns<F>(p, sc.K, l, q0 + q, q < nq, v);
      }
#pragma unroll
      for (int f = 0; f < F; ++f) h[(l * F + f) * ld_feat + q * ld_q] = v[f];
    }
    if (p.texel_addr && p.kmax_out > nlev)
      for (int it = threadIdx.x; it < (p.kmax_out - nlev) * QT; it += NT) {
        const int l = nlev + it / QT, q = it % QT;
        if (q < nq)
          for (int k = 0; k < 24; ++k) p.texel_addr[((q0 + q) * p.kmax_out + l) * 24 + k] = -1;
      }
    return;
  }
  for (int it = threadIdx.x; it < nlev * QT; it += NT) {
    const int l = it / QT, q = it % QT;
    const int node = node_sm[l * QT + q];
    float v[F];
#pragma unroll
    for (int f = 0; f < F; ++f) v[f] = 0.f;
    int64_t a4[4] = {-1, -1, -1, -1};
    if (node >= 0) {
      const int R = sc.R[l];
      const int64_t mo = map_base(p, sc, tree, node, R);
      if (mo >= 0) {
        const Footprint fp = footprint(u_sm[q], u_sm[QT + q], R);
        float t[4][F];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          a4[k] = mo + fp.idx[k];
          TexelLoad<TT, F>::load(sc.tables, a4[k], t[k]);
        }
#pragma unroll
        for (int f = 0; f < F; ++f) {
          float s = fp.w[0] * t[0][f];
          s = fmaf(fp.w[1], t[1][f], s);
          s = fmaf(fp.w[2], t[2][f], s);
          s = fmaf(fp.w[3], t[3][f], s);
          v[f] = s;
        }
      }
    } else if (p.n_attrs > 0 && l >= sc.K) {  // Eq. 12's attributes past the features
      attr_columns<F>(p, sc.K, l, q0 + q, q < nq, v);
    }
#pragma unroll
    for (int f = 0; f < F; ++f) h[(l * F + f) * ld_feat + q * ld_q] = v[f];
    if (p.texel_addr && q < nq && l < p.kmax_out) {
      int4 o = make_int4(int(a4[0]), int(a4[1]), int(a4[2]), int(a4[3]));
      *reinterpret_cast<int4*>(p.texel_addr + ((q0 + q) * p.kmax_out + l) * 4) = o;
    }
  }
  // texel_addr columns of levels this scene does not have
  if (p.texel_addr && p.kmax_out > nlev) {
    for (int it = threadIdx.x; it < (p.kmax_out - nlev) * QT; it += NT) {
      const int l = nlev + it / QT, q = it % QT;
      if (q < nq)
        *reinterpret_cast<int4*>(p.texel_addr + ((q0 + q) * p.kmax_out + l) * 4) =
            make_int4(-1, -1, -1, -1);
    }
  }
}

// Phase 4 (BWD): d_tables[texel] += w_k * dh_l for the 4 corners of every
// present level (float4 vector atomics); in the trilinear vertex form for the
// 24 vertices of a level, weight = renormalised cell weight x barycentric.
// In the shifted form with dd_sm non-NULL, every item also adds its level's
// share of dL/dd, sum over cells and vertices of wn_j (d b_k / d d)
// <t_jk, dh_l>, into dd_sm[q] (shared memory, zeroed by the caller).
template <int KMAX, int F, typename TT, bool SHIFT>
__device__ __forceinline__ void scatter_tile(const QueryParams& p, const DevScene& sc,
                                             const int2* tree, const int* node_sm, const float* u_sm,
                                             const float* dh, float* dd_sm = nullptr) {
  if (sc.query_form == OCTA_FORM_TRILINEAR_VERTEX) {
    const float* xsm = reinterpret_cast<const float*>(node_sm);
    for (int it = threadIdx.x; it < KMAX * QT; it += NT) {
      const int l = it / QT, q = it % QT;
      if (node_sm[3 * QT + q] < 0 || l >= sc.K) continue;
      const float xs[3] = {xsm[q], xsm[QT + q], xsm[2 * QT + q]};
      FullLevel fl;
      full_form_level(p, sc, tree, xs, u_sm[q], u_sm[QT + q], l, fl);
      for (int c = 0; c < F / 4; ++c) {
        const float g0 = dh[(l * F + 4 * c + 0) * LDA + q];
        const float g1 = dh[(l * F + 4 * c + 1) * LDA + q];
        const float g2 = dh[(l * F + 4 * c + 2) * LDA + q];
        const float g3 = dh[(l * F + 4 * c + 3) * LDA + q];
        for (int j = 0; j < 8; ++j) {
          if (fl.base[j] < 0) continue;
          for (int k = 0; k < 3; ++k) {
            const float w = fl.wn[j] * fl.b[k];
            float4* dst =
                reinterpret_cast<float4*>(sc.d_tables + int64_t(fl.base[j] + fl.vidx[k]) * F) + c;
            atomicAdd(dst, make_float4(w * g0, w * g1, w * g2, w * g3));
          }
        }
      }
    }
    return;
  }
  if (SHIFT && sc.query_form == OCTA_FORM_SHIFTED) {
    const float* xsm = reinterpret_cast<const float*>(node_sm);
    for (int it = threadIdx.x; it < KMAX * QT; it += NT) {
      const int l = it / QT, q = it % QT;
      if (node_sm[3 * QT + q] < 0 || l >= sc.K) continue;
      const float xs[3] = {xsm[q], xsm[QT + q], xsm[2 * QT + q]};
      const float wr[3] = {xsm[4 * QT + q], xsm[5 * QT + q], u_sm[q]};
      const float disp = u_sm[QT + q];
      float g[F];
#pragma unroll
      for (int f = 0; f < F; ++f) g[f] = dh[(l * F + f) * LDA + q];
      FullLevel fl;
      int c0[3];
      cells_form_level(p, sc, tree, xs, l, c0, fl);
      float dd = 0.f;
#pragma unroll 1
      for (int j = 0; j < 8; ++j) {
        if (fl.base[j] < 0) continue;
        float db[3];
        if (dd_sm)
          shifted_cell_vertex_dd(sc, xs, wr, disp, l, c0, j, fl, db);
        else
          shifted_cell_vertex(sc, xs, wr, disp, l, c0, j, fl);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float w = fl.wn[j] * fl.b[k];
          const int64_t e = int64_t(fl.base[j] + fl.vidx[k]);
#pragma unroll
          for (int c = 0; c < F / 4; ++c)
            atomicAdd(reinterpret_cast<float4*>(sc.d_tables + e * F) + c,
                      make_float4(w * g[4 * c], w * g[4 * c + 1], w * g[4 * c + 2],
                                  w * g[4 * c + 3]));
          if (dd_sm) {
            float t[F];
            TexelLoad<TT, F>::load(sc.tables, e, t);
            float dot = 0.f;
#pragma unroll
            for (int f = 0; f < F; ++f) dot = fmaf(t[f], g[f], dot);
            dd = fmaf(fl.wn[j] * db[k], dot, dd);
          }
        }
      }
      if (dd_sm) atomicAdd(dd_sm + q, dd);
    }
    return;
  }
  for (int it = threadIdx.x; it < KMAX * QT; it += NT) {
    const int l = it / QT, q = it % QT;
    const int node = node_sm[l * QT + q];
    if (node < 0) continue;
    const int R = sc.R[l];
    const int64_t mo = map_base(p, sc, tree, node, R);
    if (mo < 0) continue;
    const Footprint fp = footprint(u_sm[q], u_sm[QT + q], R);
#pragma unroll
    for (int c = 0; c < F / 4; ++c) {
      const float g0 = dh[(l * F + 4 * c + 0) * LDA + q];
      const float g1 = dh[(l * F + 4 * c + 1) * LDA + q];
      const float g2 = dh[(l * F + 4 * c + 2) * LDA + q];
      const float g3 = dh[(l * F + 4 * c + 3) * LDA + q];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float w = fp.w[k];
        float4* dst = reinterpret_cast<float4*>(sc.d_tables + (mo + fp.idx[k]) * F) + c;
        atomicAdd(dst, make_float4(w * g0, w * g1, w * g2, w * g3));
      }
    }
  }
}

// Sum of every thread's FP64 loss partial, added once per CTA to loss as
// a mean over 3 n_pairs elements (all threads of the CTA call it).
__device__ __forceinline__ void flush_loss_f64(double& acc, double* loss, int64_t n_pairs) {
  __shared__ double red[NT / 32];
  double v = acc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < NT / 32; ++i) t += red[i];
    atomicAdd(loss, t / (3.0 * double(n_pairs)));
  }
  __syncthreads();
  acc = 0.0;
}

// TRAIN (with BWD): the fused training pass.  A tile holds PR = QT / 2 pairs:
// rows 0..PR-1 their primary queries (x, omega) and rows PR..QT-1 their
// secondary queries (x2, omega2); after the forward the Eq. 14 gradient of
// every pair is formed in the tile from the two radiances, and the backward
// runs on it directly (only the loss value leaves the CTA, as FP64 partials).
template <class S, typename TT, bool TRAIN = false, bool SHIFT = false>
__global__ void __launch_bounds__(NT, 1) engine_kernel(const __grid_constant__ QueryParams p) {
  static_assert(!TRAIN || S::BWD, "the training pass runs the backward");
  constexpr int PR = QT / 2;            // pairs per tile (TRAIN)
  constexpr int ROWS = TRAIN ? PR : QT;  // work units (pairs or queries) per tile
  constexpr int H = S::H, WP = S::WP, NH = S::NH;
  extern __shared__ __align__(16) float smem[];
  float* wsm = smem;
  float* act = wsm + S::WSM * S::WDUP;
  constexpr int WD = S::WDUP;  // weight element i sits at wsm[WD * i]
  int* node_sm = reinterpret_cast<int*>(act + S::ACT_ROWS * LDA);
  float* u_sm = reinterpret_cast<float*>(node_sm + S::KMAX * QT);
  int2* tree_sm = reinterpret_cast<int2*>(reinterpret_cast<uint8_t*>(smem) + S::TREE_OFF);
  const int2* tree = nullptr;
  // activation buffers
  auto act_bwd = [&](int i) { return i == 0 ? act : act + (WP + (i - 1) * H) * LDA; };
  float* dL = act + (WP + NH * H) * LDA;  // delta_L (BWD)
  float* buf[2] = {act, act + S::MAXW * LDA};

  Grads<S> g;
  if (S::BWD) g.zero();
  int cur = -1;
  double loss_acc = 0.0;
  const float lscale = TRAIN ? (p.scaler ? p.scaler->scale : 1.f) : 1.f;
  // the locate threads' row in a tile and the array it reads (TRAIN:
  // primaries in rows 0..PR-1, secondaries in PR..QT-1)
  const int qrow = threadIdx.x < QT ? (TRAIN ? int(threadIdx.x) % PR : int(threadIdx.x)) : ROWS;
  const bool primary = !TRAIN || threadIdx.x < PR;
  const float* xs = primary ? p.x : p.x2;
  const float* ws = primary ? p.omega : p.omega2;
  const float* nrm = primary ? p.normal : p.normal2;  // the shifted form's inputs
  const float* dsp = primary ? p.disparity : p.disparity2;
  float* d_dsp = primary ? p.d_disparity : p.d_disparity2;  // its dL/dd out (nullable)
  __shared__ float dd_sm[QT];
  auto tile_query = [&](int64_t tile) {
    const DevScene& sc = p.sc[scene_of_tile(p, tile)];
    const int64_t gq = sc.q_begin + (tile - sc.tile_begin) * ROWS + qrow;
    return load_query(xs, ws, gq, qrow < ROWS && gq < sc.q_end);
  };
  const WorkRange wr = work_range(p.n_tiles, p.order, p.run);
  QueryIn next = wr.begin < wr.end ? tile_query(wr.begin) : QueryIn{};
  for (int64_t tile = wr.begin; tile < wr.end; tile = wr.next(tile)) {
    const int s = scene_of_tile(p, tile);
    const DevScene& sc = p.sc[s];
    const QueryIn in = next;
    if (wr.next(tile) < wr.end) next = tile_query(wr.next(tile));
    __syncthreads();  // previous tile finished with shared memory
    if (s != cur) {
      if (S::BWD && cur >= 0) {
        g.flush(p.sc[cur]);
        g.zero();
        if (TRAIN) flush_loss_f64(loss_acc, p.loss + cur, p.sc[cur].norm_pairs);
      }
      load_weights<S>(sc, wsm);
      tree = stage_tree(p, sc, tree_sm, S::TREE_NODES, threadIdx.x, NT);
      cur = s;
      __syncthreads();
    }
    const int64_t q0 = sc.q_begin + (tile - sc.tile_begin) * ROWS;
    const int nq = static_cast<int>(sc.q_end - q0 < ROWS ? sc.q_end - q0 : int64_t(ROWS));
    float* h = S::BWD ? act_bwd(0) : buf[0];
    const bool want_dd = SHIFT && S::BWD && sc.query_form == OCTA_FORM_SHIFTED &&
                         (p.d_disparity || p.d_disparity2);
    if (want_dd && threadIdx.x < QT) dd_sm[threadIdx.x] = 0.f;
    if (TRAIN)  // rows of both halves are valid for the tile's nq pairs
      locate_tile<S::KMAX, SHIFT>(p, sc, tree, in, q0, threadIdx.x < PR ? nq : PR + nq, node_sm, u_sm,
                           nrm, dsp, q0 + qrow);
    else
      locate_tile<S::KMAX, SHIFT>(p, sc, tree, in, q0, nq, node_sm, u_sm, nrm, dsp, q0 + qrow);
    __syncthreads();
    gather_tile<S::F, TT, SHIFT>(p, sc, tree, q0, nq, S::KMAX, node_sm, u_sm, h, LDA, 1);
    __syncthreads();

    // ---- decoder forward (Eq. 13)
    const float* Wl = wsm + WD * (H * WP + (NH - 1) * H * H);  // last layer [4][H]
    float* a_last;
    if (S::BWD) {
      gemm_fwd_relu<H, WP, S::DUP>(wsm, act_bwd(0), act_bwd(1));
      __syncthreads();
#pragma unroll
      for (int i = 1; i < NH; ++i) {
        gemm_fwd_relu<H, H, S::DUP>(wsm + WD * (H * WP + (i - 1) * H * H), act_bwd(i),
                                  act_bwd(i + 1));
        __syncthreads();
      }
      a_last = act_bwd(NH);
    } else {
      gemm_fwd_relu<H, WP>(wsm, buf[0], buf[1]);
      __syncthreads();
#pragma unroll
      for (int i = 1; i < NH; ++i) {
        gemm_fwd_relu<H, H>(wsm + H * WP + (i - 1) * H * H, buf[i & 1], buf[(i + 1) & 1]);
        __syncthreads();
      }
      a_last = buf[NH & 1];
    }
    if (threadIdx.x < QT) {
      const int q = threadIdx.x;
      float z0 = 0.f, z1 = 0.f, z2 = 0.f;
#pragma unroll 8
      for (int k = 0; k < H; ++k) {
        const float a = a_last[k * LDA + q];
        z0 = fmaf(Wl[WD * k], a, z0);
        z1 = fmaf(Wl[WD * (H + k)], a, z1);
        z2 = fmaf(Wl[WD * (2 * H + k)], a, z2);
      }
      const float r0 = expf(z0), r1 = expf(z1), r2 = expf(z2);
      const int64_t gq = q0 + q;
      if (!S::BWD) {
        if (q < nq) {
          p.rgb[3 * gq] = r0;
          p.rgb[3 * gq + 1] = r1;
          p.rgb[3 * gq + 2] = r2;
        }
      } else if (TRAIN) {  // radiances, turned into delta_L below
        dL[q] = r0;
        dL[LDA + q] = r1;
        dL[2 * LDA + q] = r2;
        dL[3 * LDA + q] = 0.f;
      } else {
        float d0 = 0.f, d1 = 0.f, d2 = 0.f;
        if (q < nq) {
          d0 = p.d_rgb[3 * gq];
          d1 = p.d_rgb[3 * gq + 1];
          d2 = p.d_rgb[3 * gq + 2];
        }
        dL[q] = d0 * r0;  // d exp(z) / dz = exp(z)
        dL[LDA + q] = d1 * r1;
        dL[2 * LDA + q] = d2 * r2;
        dL[3 * LDA + q] = 0.f;
      }
    }
    if (!S::BWD) continue;
    if (TRAIN) {
      // Eq. 14 with the one-sample target of Eq. 3, per pair and channel:
      // T = E + w L_s, r = (L_p - T) / (L_p + T + eps) (normaliser detached),
      // d/dL_p = S 2 r / (3 n den), d/dL_s = -w d/dL_p (rhs_grad); then
      // delta_L = d/dL * L (the derivative of exp is exp).
      __syncthreads();
      if (threadIdx.x < PR) {
        const int r = threadIdx.x;
        const int64_t gp = q0 + r;
        const float n3 = 3.f * static_cast<float>(sc.norm_pairs);
        float r2 = 0.f;  // the pair's three r^2 in binary32, one FP64 add
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float Lp = dL[c * LDA + r], Ls = dL[c * LDA + PR + r];
          float dp = 0.f, ds = 0.f;
          if (r < nq) {
            const float ww = p.w[3 * gp + c];
            const float T = p.E[3 * gp + c] + ww * Ls;
            const float den = Lp + T + p.eps;
            const float rr = (Lp - T) / den;
            r2 = fmaf(rr, rr, r2);
            dp = 2.f * lscale * rr / (n3 * den);
            ds = p.rhs_grad ? -dp * ww : 0.f;
          }
          dL[c * LDA + r] = dp * Lp;
          dL[c * LDA + PR + r] = ds * Ls;
        }
        loss_acc += double(r2);
      }
    }

    // ---- backward
    __syncthreads();
    if (threadIdx.x < 3 * H) {  // dW_L[m][k] += sum_q delta_L[m][q] a_NH[k][q]
      const int m = threadIdx.x / H, k = threadIdx.x % H;
      float sacc = g.wl;
#pragma unroll 4
      for (int q = 0; q < QT; q += 4) {
        const float4 d = *reinterpret_cast<const float4*>(dL + m * LDA + q);
        const float4 a = *reinterpret_cast<const float4*>(a_last + k * LDA + q);
        sacc = fmaf(d.x, a.x, sacc);
        sacc = fmaf(d.y, a.y, sacc);
        sacc = fmaf(d.z, a.z, sacc);
        sacc = fmaf(d.w, a.w, sacc);
      }
      g.wl = sacc;
    }
    __syncthreads();
    gemm_bwd_data<3, H, true, S::DUP>(Wl, dL, act_bwd(NH));  // delta_NH in place
    __syncthreads();
#pragma unroll
    for (int i = NH - 1; i >= 0; --i) {
      if (i == 0)
        g.w0.accumulate(act_bwd(1), act_bwd(0));
      else
        g.wh[i - 1].accumulate(act_bwd(i + 1), act_bwd(i));
      __syncthreads();
      if (i == 0)
        gemm_bwd_data<H, WP, false, S::DUP>(wsm, act_bwd(1), act_bwd(0));  // dh
      else
        gemm_bwd_data<H, H, true, S::DUP>(wsm + WD * (H * WP + (i - 1) * H * H), act_bwd(i + 1),
                                        act_bwd(i));
      __syncthreads();
    }
    scatter_tile<S::KMAX, S::F, TT, SHIFT>(p, sc, tree, node_sm, u_sm, act_bwd(0),
                                    want_dd ? dd_sm : nullptr);
    if (want_dd) {  // the shifted form's dL/dd of the tile's queries
      __syncthreads();
      if (threadIdx.x < QT && d_dsp && qrow < nq) d_dsp[q0 + qrow] = dd_sm[threadIdx.x];
    }
  }
  if (S::BWD && cur >= 0) g.flush(p.sc[cur]);
  if (TRAIN && cur >= 0) flush_loss_f64(loss_acc, p.loss + cur, p.sc[cur].norm_pairs);
}

}  // namespace f32
}  // namespace octa
