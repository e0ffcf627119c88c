// stage_f64t.cu -- stage-kernel instantiations: FP64 path, Cartesian Euler blocks, the second
// tile height the group tuner may choose, and stages 1 and 2 with the halo exchange folded in
// (both heights) (TY_ALT_F64)
#include "stage_inst.cuh"

namespace gbcfd {
cudaError_t launch_stage_f64_alt(int stage, const GroupParams& P, int grid, cudaStream_t s) {
  return stage_dispatch_v<double, false, false, TY_ALT_F64>(stage, P, grid, s);
}
cudaError_t stage_prepare_f64_alt() { return stage_prepare_v<double, false, false, TY_ALT_F64>(); }
int stage_occupancy_f64_alt() { return stage_occupancy_v<double, false, false, TY_ALT_F64>(); }
cudaError_t launch_stage_f64_push(int stage, int ty, const GroupParams& P, int grid, cudaStream_t s) {
  if (ty == TY_ALT_F64) return stage_dispatch_push<double, TY_ALT_F64>(stage, P, grid, s);
  if (ty == TY_DEFAULT) return stage_dispatch_push<double, TY_DEFAULT>(stage, P, grid, s);
  return cudaErrorInvalidValue;
}
cudaError_t stage_prepare_f64_push(int ty) {
  if (ty == TY_ALT_F64) return stage_prepare_push<double, TY_ALT_F64>();
  if (ty == TY_DEFAULT) return stage_prepare_push<double, TY_DEFAULT>();
  return cudaErrorInvalidValue;
}
}  // namespace gbcfd
