// FP32 engine: the built shapes and their launches (forward, backward and
// the fused training pass).  Kept apart from query.cu so that the two
// translation units compile in parallel.
#include <cuda_runtime.h>

#include <algorithm>

#include "engine_f32.cuh"
#include "engine_path.h"
#include "launch_persistent.cuh"
#include "octa_internal.h"

namespace octa {
namespace f32 {
namespace {

template <int F, int WP, int H, int NH, typename TT>
int run_engine(const QueryParams& p, Mode mode, cudaStream_t stream) {
  const octa_tuning tu = tuning_snapshot();
  if (mode == Mode::kForward) {
    using S = Shape<F, WP, H, NH, false>;
    return launch_persistent(engine_kernel<S, TT>, S::SMEM, p, stream, NT, tu.engine_ctas_per_sm,
                             tu.fwd_order);
  }
  using S = Shape<F, WP, H, NH, true>;
  if (mode == Mode::kBackward)
    return launch_persistent(engine_kernel<S, TT>, S::SMEM, p, stream, NT, tu.engine_ctas_per_sm,
                             tu.train_order);
  return launch_persistent(engine_kernel<S, TT, true>, S::SMEM, p, stream, NT,
                           tu.engine_ctas_per_sm, tu.train_order);
}

}  // namespace

// Built shapes of the FP32 engine: (F, padded input width, hidden width,
// hidden layers) x table type.  A scene set uses the smallest padded width
// that holds every scene's K*F.
int dispatch(const octa_scene* scenes, int n_scenes, const QueryParams& p0, Mode mode,
             cudaStream_t stream) {
  const octa_scene& c0 = scenes[0];
  const int F = c0.F, L = c0.n_layers, H = c0.widths[1], tdt = c0.table_dtype;
  int need = 0;
  for (int s = 0; s < n_scenes; ++s) {
    const octa_scene& c = scenes[s];
    if (c.F != F || c.n_layers != L || c.table_dtype != tdt || c.weight_dtype != OCTA_F32)
      return fail(OCTA_EUNSUPPORTED, "scenes of one call must share F, depth of the MLP and dtypes");
    for (int i = 1; i < L; ++i)
      if (c.widths[i] != H)
        return fail(OCTA_EUNSUPPORTED, "FP32 path: hidden widths must all equal %d", H);
    need = std::max(need, c.widths[0]);
  }
  QueryParams p = p0;
  if (mode == Mode::kTrain) {  // tiles of QT / 2 pairs
    int64_t tiles = 0;
    for (int s = 0; s < p.n_scenes; ++s) {
      p.sc[s].tile_begin = tiles;
      tiles += (p.sc[s].q_end - p.sc[s].q_begin + QT / 2 - 1) / (QT / 2);
    }
    p.n_tiles = tiles;
  }
  const int NH = L - 1;
  const bool f16 = tdt == OCTA_F16;
#define OCTA_TRY(F_, WP_, H_, NH_)                                                   \
  if (F == F_ && H == H_ && NH == NH_ && need <= WP_)                                \
    return f16 ? run_engine<F_, WP_, H_, NH_, __half>(p, mode, stream)              \
               : run_engine<F_, WP_, H_, NH_, float>(p, mode, stream);
  OCTA_TRY(4, 24, 32, 2)
  OCTA_TRY(8, 56, 64, 2)
  OCTA_TRY(8, 72, 64, 2)
  OCTA_TRY(8, 80, 64, 2)
  OCTA_TRY(8, 72, 64, 3)
  OCTA_TRY(8, 80, 64, 3)
#undef OCTA_TRY
  return fail(OCTA_EUNSUPPORTED,
              "FP32 path: no built shape for F=%d, K*F=%d, hidden %d x %d", F, need, NH, H);
}

}  // namespace f32
}  // namespace octa
