// stage_f32t.cu -- stage-kernel instantiations: mixed path, Cartesian Euler blocks, the second
// tile height the group tuner may choose, and stages 1 and 2 with the halo exchange folded in
// (both heights) (TY_ALT_F32)
#include "stage_inst.cuh"

namespace gbcfd {
cudaError_t launch_stage_f32_alt(int stage, const GroupParams& P, int grid, cudaStream_t s) {
  return stage_dispatch_v<float, false, false, TY_ALT_F32>(stage, P, grid, s);
}
cudaError_t stage_prepare_f32_alt() { return stage_prepare_v<float, false, false, TY_ALT_F32>(); }
int stage_occupancy_f32_alt() { return stage_occupancy_v<float, false, false, TY_ALT_F32>(); }
cudaError_t launch_stage_f32_push(int stage, int ty, const GroupParams& P, int grid, cudaStream_t s) {
  if (ty == TY_ALT_F32) return stage_dispatch_push<float, TY_ALT_F32>(stage, P, grid, s);
  if (ty == TY_DEFAULT) return stage_dispatch_push<float, TY_DEFAULT>(stage, P, grid, s);
  return cudaErrorInvalidValue;
}
cudaError_t stage_prepare_f32_push(int ty) {
  if (ty == TY_ALT_F32) return stage_prepare_push<float, TY_ALT_F32>();
  if (ty == TY_DEFAULT) return stage_prepare_push<float, TY_DEFAULT>();
  return cudaErrorInvalidValue;
}
}  // namespace gbcfd
