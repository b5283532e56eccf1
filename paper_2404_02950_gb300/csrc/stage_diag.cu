// Diagnostics stage 1 (fused winding tags and energy partials) instantiations
// of the fused stage kernel (stage_kernel.cuh), classic RK4 / SSPRK3 and
// Nystrom forms, in a translation unit of their own so that the build
// compiles them in parallel with the plain stages.
#include "stage_kernel.cuh"

namespace slh {

slh_status launch_stage_diag(slh_ctx* c, Level& L, const slh_eom_params& p, const StageLaunch& s, int* ctas_used,
                             bool rkn) {
  return rkn ? launch_tile<true, true>(c, L, p, s, ctas_used) : launch_tile<true, false>(c, L, p, s, ctas_used);
}

}  // namespace slh
