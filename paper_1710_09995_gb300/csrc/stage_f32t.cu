// stage_f32t.cu -- stage-kernel instantiations: mixed path, Cartesian Euler blocks, the second
// tile height the group tuner may choose (TY_ALT_F32)
#include "stage_inst.cuh"

namespace gbcfd {
cudaError_t launch_stage_f32_alt(int stage, const GroupParams& P, int grid, cudaStream_t s) {
  return stage_dispatch_v<float, false, false, TY_ALT_F32>(stage, P, grid, s);
}
cudaError_t stage_prepare_f32_alt() { return stage_prepare_v<float, false, false, TY_ALT_F32>(); }
int stage_occupancy_f32_alt() { return stage_occupancy_v<float, false, false, TY_ALT_F32>(); }
}  // namespace gbcfd
