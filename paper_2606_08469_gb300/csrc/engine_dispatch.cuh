// FP32 engine: the built shapes and their launches (forward, backward and
// the fused training pass), templated on whether the instances evaluate the
// shifted form; engine_f32.cu and engine_f32_shift.cu each instantiate one
// set, so the two compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>

#include "engine_f32.cuh"
#include "engine_path.h"
#include "launch_persistent.cuh"
#include "octa_internal.h"

namespace octa {
namespace f32 {

// SHIFT: the instance that also evaluates the shifted form (the cell and
// trilinear vertex forms run the instance without its code).
template <int F, int WP, int H, int NH, typename TT, bool SHIFT>
int run_engine_form(const QueryParams& p, Mode mode, cudaStream_t stream) {
  const octa_tuning tu = tuning_snapshot();
  if (mode == Mode::kForward) {
    using S = Shape<F, WP, H, NH, false>;
    return launch_persistent(engine_kernel<S, TT, false, SHIFT>, S::SMEM, p, stream, NT,
                             tu.engine_ctas_per_sm, tu.fwd_order, tu.fwd_run);
  }
  using S = Shape<F, WP, H, NH, true>;
  if (mode == Mode::kBackward)
    return launch_persistent(engine_kernel<S, TT, false, SHIFT>, S::SMEM, p, stream, NT,
                             tu.engine_ctas_per_sm, tu.train_order, tu.train_run);
  return launch_persistent(engine_kernel<S, TT, true, SHIFT>, S::SMEM, p, stream, NT,
                           tu.engine_ctas_per_sm, tu.train_order, tu.train_run);
}

// Built shapes of the FP32 engine: (F, padded input width, hidden width,
// hidden layers) x table type.  A scene set uses the smallest padded width
// that holds every scene's K*F.  The shifted form is built for F = 8.
template <bool SHIFT>
int dispatch_shapes(const octa_scene* scenes, int n_scenes, const QueryParams& p0, Mode mode,
                    cudaStream_t stream) {
  const octa_scene& c0 = scenes[0];
  const int F = c0.F, L = c0.n_layers, H = c0.widths[1], tdt = c0.table_dtype;
  int need = 0;
  for (int s = 0; s < n_scenes; ++s) {
    const octa_scene& c = scenes[s];
    if (c.F != F || c.n_layers != L || c.table_dtype != tdt || c.weight_dtype != OCTA_F32)
      return fail(OCTA_EUNSUPPORTED, "scenes of one call must share F, depth of the MLP and dtypes");
    if (c.query_form != c0.query_form)
      return fail(OCTA_EUNSUPPORTED, "scenes of one call must share the query form");
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
#define OCTA_TRY(F_, WP_, H_, NH_)                                                    \
  if (F == F_ && H == H_ && NH == NH_ && need <= WP_)                                 \
    return f16 ? run_engine_form<F_, WP_, H_, NH_, __half, SHIFT>(p, mode, stream)   \
               : run_engine_form<F_, WP_, H_, NH_, float, SHIFT>(p, mode, stream);
  if constexpr (!SHIFT) {
    OCTA_TRY(4, 24, 32, 2)
  }
  OCTA_TRY(8, 56, 64, 2)
  OCTA_TRY(8, 72, 64, 2)
  OCTA_TRY(8, 80, 64, 2)
  OCTA_TRY(8, 72, 64, 3)
  OCTA_TRY(8, 80, 64, 3)
#undef OCTA_TRY
  return fail(OCTA_EUNSUPPORTED,
              "FP32 path: no built shape for F=%d, K*F=%d, hidden %d x %d%s", F, need, NH, H,
              SHIFT ? " in the shifted form" : "");
}

}  // namespace f32
}  // namespace octa
