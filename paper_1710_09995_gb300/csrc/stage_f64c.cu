// stage_f64c.cu -- stage-kernel instantiations: FP64 path, curvilinear grids
#include "stage_inst.cuh"

namespace gbcfd {
cudaError_t launch_stage_f64c(int viscous, int stage, const GroupParams& P, int grid,
                             cudaStream_t s) {
  return stage_dispatch<double, true>(viscous, stage, P, grid, s);
}
cudaError_t stage_prepare_f64c(int viscous) { return stage_prepare<double, true>(viscous); }
int stage_occupancy_f64c(int viscous) { return stage_occupancy<double, true>(viscous); }
}  // namespace gbcfd
