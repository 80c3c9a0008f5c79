// Tensor-core (tcgen05) path of the query: BF16 decoder weights, FP32
// accumulation in tensor memory.
#pragma once
#include <cuda_runtime.h>

#include "octa_device.cuh"

namespace octa {
namespace tc {

// Optimiser block of the persistent training step (one launch: fused pass,
// then Adam over every parameter group after grid-wide barriers).
struct AdamBlock {
  octa_param_group g[OCTA_MAX_GROUPS];
  int32_t vec4[OCTA_MAX_GROUPS];  // group may use 16-byte vector accesses
  int32_t n_groups;
  float beta1, beta2, eps;
  octa_scaler* scaler;
  unsigned* bar;            // [0] arrivals, [1] generation (workspace, zeroed once)
  double* partials;         // [gridDim.x] FP64 sums of squares
  uint64_t timeout_ns;      // bound of every barrier wait
  int32_t extra_arrivals;   // arrivals awaited beyond the grid (0; tests use > 0)
  int32_t skip_first_mma;   // test hook: no MMA for layer 0 of each CTA's first tile
};


int query_fwd(const octa_scene* scenes, int n_scenes, const QueryParams& p, cudaStream_t stream);
// The disparity predictor g_psi with its MLP on the tensor cores (BF16
// weights_bf16, FP32 accumulation); the caller has validated pred and q.
int predictor_fwd(const octa_predictor* pred, const octa_queries* q, float* disparity,
                  cudaStream_t stream);
int predictor_bwd(const octa_predictor* pred, const octa_queries* q, const float* d_disp,
                  float* d_table, float* d_weights, cudaStream_t stream);
int query_bwd(const octa_scene* scenes, int n_scenes, const QueryParams& p, cudaStream_t stream);
int train_fused(const octa_scene* scenes, int n_scenes, const QueryParams& p, cudaStream_t stream);
int train_step_persistent(const octa_scene* scenes, int n_scenes, const QueryParams& p,
                          const AdamBlock& adam, cudaStream_t stream);

}  // namespace tc
}  // namespace octa
