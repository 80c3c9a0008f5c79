// Launcher of the persistent tile kernels that take a QueryParams block.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>

#include "launch_util.h"
#include "octa_device.cuh"

namespace octa {

// Persistent grid: as many CTAs as fit on the device, never more than tiles.
// cap bounds the resident CTAs per SM (0: none); order is the work order of
// work_range (1: contiguous chunks, else interleaved, `run` consecutive
// tiles at a time); the shared-memory carveout follows the l1_carveout knob.
template <class Kern>
int launch_persistent(Kern kernel, size_t smem, const QueryParams& p0, cudaStream_t stream,
                      int threads, int cap, int order, int run = 1) {
  if (p0.n_tiles == 0) return OCTA_OK;
  int per_sm = 0;
  int rc = launch_cache().get(reinterpret_cast<const void*>(kernel), smem, threads, 0, &per_sm,
                              carve_mode(tuning_snapshot()), cap);
  if (rc) return rc;
  per_sm = apply_cap(per_sm, cap);
  QueryParams p = p0;
  p.order = order == 1 ? 1 : 0;
  p.run = run > 1 ? run : 1;
  const int64_t grid = std::min<int64_t>(p.n_tiles, int64_t(per_sm) * device_sm_count());
  kernel<<<static_cast<unsigned>(grid), threads, smem, stream>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(OCTA_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
  return OCTA_OK;
}

}  // namespace octa
