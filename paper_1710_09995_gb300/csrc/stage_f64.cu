// stage_f64.cu -- instantiations of the stage kernel for the FP64 path
#include "launch.h"
#include "stage.cuh"

namespace gbcfd {

template <bool VISC, int STAGE>
static cudaError_t go(const CUtensorMap& tmq, const CUtensorMap& tmd, const StageParams& P, int grid,
                      cudaStream_t s) {
  auto k = stage_kernel<double, VISC, STAGE>;
  const size_t bytes = Plan<double, VISC>::bytes;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  k<<<grid, NT, bytes, s>>>(tmq, tmd, P);
  return cudaGetLastError();
}

cudaError_t launch_stage_f64(int viscous, int stage, const CUtensorMap& tmq, const CUtensorMap& tmd,
                             const StageParams& P, int grid, cudaStream_t s) {
  if (viscous) {
    switch (stage) {
      case 0: return go<true, 0>(tmq, tmd, P, grid, s);
      case 1: return go<true, 1>(tmq, tmd, P, grid, s);
      case 2: return go<true, 2>(tmq, tmd, P, grid, s);
      case 3: return go<true, 3>(tmq, tmd, P, grid, s);
    }
  } else {
    switch (stage) {
      case 0: return go<false, 0>(tmq, tmd, P, grid, s);
      case 1: return go<false, 1>(tmq, tmd, P, grid, s);
      case 2: return go<false, 2>(tmq, tmd, P, grid, s);
      case 3: return go<false, 3>(tmq, tmd, P, grid, s);
    }
  }
  return cudaErrorInvalidValue;
}

size_t stage_smem_f64(int viscous) {
  return viscous ? Plan<double, true>::bytes : Plan<double, false>::bytes;
}

int stage_occupancy_f64(int viscous) {
  int n = 0;
  cudaError_t e;
  if (viscous) {
    auto k = stage_kernel<double, true, 1>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Plan<double, true>::bytes);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, NT, Plan<double, true>::bytes);
  } else {
    auto k = stage_kernel<double, false, 1>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Plan<double, false>::bytes);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, NT, Plan<double, false>::bytes);
  }
  return (e == cudaSuccess && n > 0) ? n : 1;
}

}  // namespace gbcfd
