// Tensor-core (tcgen05) path of the query: BF16 decoder weights, FP32
// accumulation in tensor memory.
#pragma once
#include <cuda_runtime.h>

#include "octa_device.cuh"

namespace octa {
namespace tc {

int query_fwd(const octa_scene* scenes, int n_scenes, const QueryParams& p, cudaStream_t stream);
int query_bwd(const octa_scene* scenes, int n_scenes, const QueryParams& p, cudaStream_t stream);
int train_fused(const octa_scene* scenes, int n_scenes, const QueryParams& p, cudaStream_t stream);

}  // namespace tc
}  // namespace octa
