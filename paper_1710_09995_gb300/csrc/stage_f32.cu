// stage_f32.cu -- stage-kernel instantiations: mixed path (f32 fluxes), Cartesian grids
#include "stage_inst.cuh"

namespace gbcfd {
cudaError_t launch_stage_f32(int viscous, int stage, const GroupParams& P, int grid,
                             cudaStream_t s) {
  return stage_dispatch<float, false>(viscous, stage, P, grid, s);
}
cudaError_t stage_prepare_f32(int viscous) { return stage_prepare<float, false>(viscous); }
int stage_occupancy_f32(int viscous) { return stage_occupancy<float, false>(viscous); }
}  // namespace gbcfd
