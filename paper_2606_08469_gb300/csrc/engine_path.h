// FP32 path of the query (CUDA cores): host entry of the engine kernels.
#pragma once
#include <cuda_runtime.h>

#include "octa_device.cuh"

namespace octa {
namespace f32 {

enum class Mode {
  kForward,   // RGB of every query
  kBackward,  // gradients of sum(d_rgb . L_hat), activations recomputed
  kTrain,     // fused training pass over pair tiles (QueryParams holds pairs)
};

// Picks the built shape for the scenes' widths and launches the engine.
int dispatch(const octa_scene* scenes, int n_scenes, const QueryParams& p, Mode mode,
             cudaStream_t stream);
// The same for scenes in the shifted form (its own instances).
int dispatch_shifted(const octa_scene* scenes, int n_scenes, const QueryParams& p, Mode mode,
                     cudaStream_t stream);

}  // namespace f32
}  // namespace octa
