// Plain RKN4 / RKN5 (integrator types 21, 22) instantiations of the fused stage kernel
// (stage_kernel.cuh), in a translation unit of their own so that the build
// compiles them in parallel with the classic RK4 / SSPRK3 ones in stage.cu.
#include "stage_kernel.cuh"

namespace slh {

slh_status launch_stage_rkn(slh_ctx* c, Level& L, const slh_eom_params& p, const StageLaunch& s, int* ctas_used) {
  return launch_tile<false, true>(c, L, p, s, ctas_used);
}

}  // namespace slh
