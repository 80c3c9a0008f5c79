// Tensor-core (tcgen05) decoder path.  Placeholder until the kernels land.
#include "octa_internal.h"
#include "tc_path.h"

namespace octa {
namespace tc {

int query_fwd(const octa_scene*, int, const QueryParams&, cudaStream_t) {
  return fail(OCTA_EUNSUPPORTED, "BF16 tensor-core path not built yet");
}
int query_bwd(const octa_scene*, int, const QueryParams&, cudaStream_t) {
  return fail(OCTA_EUNSUPPORTED, "BF16 tensor-core path not built yet");
}

}  // namespace tc
}  // namespace octa
