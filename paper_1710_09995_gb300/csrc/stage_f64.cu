// stage_f64.cu -- stage-kernel instantiations: FP64 path, Cartesian grids
#include "stage_inst.cuh"

namespace gbcfd {
cudaError_t launch_stage_f64(int viscous, int stage, const GroupParams& P, int grid,
                             cudaStream_t s) {
  return stage_dispatch<double, false>(viscous, stage, P, grid, s);
}
cudaError_t stage_prepare_f64(int viscous) { return stage_prepare<double, false>(viscous); }
int stage_occupancy_f64(int viscous) { return stage_occupancy<double, false>(viscous); }
}  // namespace gbcfd
