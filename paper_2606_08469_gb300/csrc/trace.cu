// Secondary hits of the training regime: x'(omega_i), the first intersection
// of the ray from x along omega_i with the synthetic scene (Eq. 2), for the
// M RHS samples of every LHS sample (Eq. 3).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "octa_internal.h"

namespace octa {
namespace {

constexpr int kTraceThreads = 256;
constexpr int kPlaneFloats = 13;
constexpr int kPlaneStride = 16;  // shared-memory row of a plane: four float4
constexpr int kSphereFloats = 4;

// ((a0 b0 + a1 b1) + a2 b2), one rounding per operation (no contraction).
__device__ __forceinline__ float dot3_rn(float a0, float a1, float a2, float b0, float b1,
                                         float b2) {
  return __fadd_rn(__fadd_rn(__fmul_rn(a0, b0), __fmul_rn(a1, b1)), __fmul_rn(a2, b2));
}

// One thread per ray; the scene is staged in shared memory.  Every value
// that decides the hit is formed with explicit round-to-nearest operations
// in the order the header states, so results are bit-reproducible.
__global__ void __launch_bounds__(kTraceThreads) trace_kernel(
    const float* __restrict__ planes_g, int n_planes, const float* __restrict__ spheres_g,
    int n_spheres, const float* __restrict__ origin, int rays_per_origin,
    const float* __restrict__ dir, int64_t n_rays, float t_min, float* __restrict__ hit,
    float* __restrict__ query_dir, int32_t* __restrict__ prim_out, float* __restrict__ t_out) {
  __shared__ float4 pl4[OCTA_MAX_PRIMS * kPlaneStride / 4];
  __shared__ float4 sp4[OCTA_MAX_PRIMS];
  float* pl = reinterpret_cast<float*>(pl4);
  float* sp = reinterpret_cast<float*>(sp4);
  for (int i = threadIdx.x; i < n_planes * kPlaneStride; i += blockDim.x) {
    const int k = i / kPlaneStride, e = i % kPlaneStride;
    pl[i] = e < kPlaneFloats ? planes_g[k * kPlaneFloats + e] : 0.f;
  }
  for (int i = threadIdx.x; i < n_spheres * kSphereFloats; i += blockDim.x) sp[i] = spheres_g[i];
  __syncthreads();
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n_rays; i += stride) {
    const int64_t oi = i / rays_per_origin;
    const float o0 = origin[3 * oi], o1 = origin[3 * oi + 1], o2 = origin[3 * oi + 2];
    const float d0 = __ldcs(dir + 3 * i), d1 = __ldcs(dir + 3 * i + 1), d2 = __ldcs(dir + 3 * i + 2);
    float best = INFINITY;
    int best_id = -1;
    // Only the decisions' values are fixed; work whose outcome cannot
    // change the hit is skipped (a patch test beyond t's range, an unbounded
    // plane's patch test, a square root of a negative discriminant).
    for (int k = 0; k < n_planes; ++k) {
      const float4 qa = pl4[k * 4], qb = pl4[k * 4 + 1];  // p, n.x | n.yz, t1.xy
      const float den = dot3_rn(d0, d1, d2, qa.w, qb.x, qb.y);
      if (den == 0.f) continue;
      const float num = dot3_rn(__fsub_rn(qa.x, o0), __fsub_rn(qa.y, o1), __fsub_rn(qa.z, o2),
                                qa.w, qb.x, qb.y);
      const float t = __fdiv_rn(num, den);
      if (!(t > t_min && t < best)) continue;
      const float4 qc = pl4[k * 4 + 2], qd = pl4[k * 4 + 3];  // t1.z, t2 | h
      if (qd.x != INFINITY) {  // a patch: the hit must lie on it
        const float r0 = __fsub_rn(__fadd_rn(o0, __fmul_rn(t, d0)), qa.x);
        const float r1 = __fsub_rn(__fadd_rn(o1, __fmul_rn(t, d1)), qa.y);
        const float r2 = __fsub_rn(__fadd_rn(o2, __fmul_rn(t, d2)), qa.z);
        const float a = dot3_rn(r0, r1, r2, qb.z, qb.w, qc.x);
        const float b = dot3_rn(r0, r1, r2, qc.y, qc.z, qc.w);
        if (!(fabsf(a) <= qd.x && fabsf(b) <= qd.x)) continue;
      }
      best = t;
      best_id = k;
    }
    for (int s = 0; s < n_spheres; ++s) {
      const float4 q = sp4[s];
      const float c0 = __fsub_rn(o0, q.x), c1 = __fsub_rn(o1, q.y), c2 = __fsub_rn(o2, q.z);
      const float bq = dot3_rn(c0, c1, c2, d0, d1, d2);
      const float cq = __fsub_rn(dot3_rn(c0, c1, c2, c0, c1, c2), __fmul_rn(q.w, q.w));
      const float disc = __fsub_rn(__fmul_rn(bq, bq), cq);
      if (!(disc >= 0.f)) continue;
      const float sq = __fsqrt_rn(disc);
      const float t0 = __fsub_rn(-bq, sq);
      const float t1 = __fadd_rn(-bq, sq);
      const float t = t0 > t_min ? t0 : t1;
      if (t > t_min && t < best) {
        best = t;
        best_id = n_planes + s;
      }
    }
    const float oa[3] = {o0, o1, o2}, da[3] = {d0, d1, d2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int wi = 0; wi < 2; ++wi) {
        const float t = __fdiv_rn(__fsub_rn(static_cast<float>(wi), oa[a]), da[a]);
        if (t > t_min && t < best) {
          best = t;
          best_id = n_planes + n_spheres + 2 * a + wi;
        }
      }
    }
    hit[3 * i] = __fadd_rn(o0, __fmul_rn(best, d0));
    hit[3 * i + 1] = __fadd_rn(o1, __fmul_rn(best, d1));
    hit[3 * i + 2] = __fadd_rn(o2, __fmul_rn(best, d2));
    if (query_dir) {
      query_dir[3 * i] = -d0;
      query_dir[3 * i + 1] = -d1;
      query_dir[3 * i + 2] = -d2;
    }
    if (prim_out) prim_out[i] = best_id;
    if (t_out) t_out[i] = best;
  }
}

int sm_count_of_device() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 148;
}

}  // namespace
}  // namespace octa

using namespace octa;

extern "C" int octa_trace_rays(const octa_prims* prims, const float* origin,
                               int32_t rays_per_origin, const float* dir, int64_t n_rays,
                               float t_min, float* hit, float* query_dir, int32_t* prim, float* t,
                               void* stream) {
  clear_error();
  if (!prims) return fail(OCTA_EINVAL, "prims must be non-NULL");
  if (n_rays < 0) return fail(OCTA_EINVAL, "negative ray count");
  if (rays_per_origin < 1) return fail(OCTA_EINVAL, "rays_per_origin must be >= 1");
  if (prims->n_planes < 0 || prims->n_planes > OCTA_MAX_PRIMS || prims->n_spheres < 0 ||
      prims->n_spheres > OCTA_MAX_PRIMS)
    return fail(OCTA_ERANGE, "primitive counts outside [0, %d]", OCTA_MAX_PRIMS);
  if ((prims->n_planes > 0 && !prims->planes) || (prims->n_spheres > 0 && !prims->spheres))
    return fail(OCTA_EINVAL, "NULL primitive array");
  if (!(t_min >= 0.f)) return fail(OCTA_EINVAL, "t_min must be >= 0");
  if (n_rays == 0) return OCTA_OK;
  if (!origin || !dir || !hit) return fail(OCTA_EINVAL, "origin, dir and hit must be non-NULL");
  const int64_t want = (n_rays + kTraceThreads - 1) / kTraceThreads;
  const int blocks = static_cast<int>(std::min<int64_t>(want, 8LL * sm_count_of_device()));
  trace_kernel<<<blocks, kTraceThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      prims->planes, prims->n_planes, prims->spheres, prims->n_spheres, origin, rays_per_origin,
      dir, n_rays, t_min, hit, query_dir, prim, t);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(OCTA_ECUDA, "octa_trace_rays: %s", cudaGetErrorString(e));
  return OCTA_OK;
}
