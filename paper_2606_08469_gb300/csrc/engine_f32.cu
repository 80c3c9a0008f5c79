// FP32 engine: the instances of the cell and trilinear vertex forms, and the
// entry that picks between them and the shifted form's (engine_f32_shift.cu).
#include "engine_dispatch.cuh"

namespace octa {
namespace f32 {

int dispatch(const octa_scene* scenes, int n_scenes, const QueryParams& p, Mode mode,
             cudaStream_t stream) {
  if (scenes[0].query_form == OCTA_FORM_SHIFTED)
    return dispatch_shifted(scenes, n_scenes, p, mode, stream);
  return dispatch_shapes<false>(scenes, n_scenes, p, mode, stream);
}

}  // namespace f32
}  // namespace octa
