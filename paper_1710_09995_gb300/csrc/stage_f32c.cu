// stage_f32c.cu -- stage-kernel instantiations: mixed path (f32 fluxes), curvilinear grids
#include "stage_inst.cuh"

namespace gbcfd {
cudaError_t launch_stage_f32c(int viscous, int stage, const GroupParams& P, int grid,
                             cudaStream_t s) {
  return stage_dispatch<float, true>(viscous, stage, P, grid, s);
}
cudaError_t stage_prepare_f32c(int viscous) { return stage_prepare<float, true>(viscous); }
int stage_occupancy_f32c(int viscous) { return stage_occupancy<float, true>(viscous); }
}  // namespace gbcfd
