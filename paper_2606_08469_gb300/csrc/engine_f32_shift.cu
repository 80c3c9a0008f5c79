// FP32 engine: the instances that evaluate the shifted form (Eq. 7-9).
#include "engine_dispatch.cuh"

namespace octa {
namespace f32 {

int dispatch_shifted(const octa_scene* scenes, int n_scenes, const QueryParams& p, Mode mode,
                     cudaStream_t stream) {
  return dispatch_shapes<true>(scenes, n_scenes, p, mode, stream);
}

}  // namespace f32
}  // namespace octa
