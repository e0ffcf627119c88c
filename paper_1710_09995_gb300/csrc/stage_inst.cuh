// stage_inst.cuh -- launch helpers shared by the stage-kernel instantiation units
#pragma once
#include "launch.h"
#include "stage.cuh"

namespace gbcfd {

template <typename T, bool VISC, int STAGE, bool CURVI>
cudaError_t stage_go(const StageMaps& M, const StageParams& P, int grid, cudaStream_t s) {
  auto k = stage_kernel<T, VISC, STAGE, CURVI>;
  const size_t bytes = Plan<T, VISC, CURVI>::bytes;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  k<<<grid, NT, bytes, s>>>(*M.q, *M.d, *M.m, P);
  return cudaGetLastError();
}

template <typename T, bool CURVI>
cudaError_t stage_dispatch(int viscous, int stage, const StageMaps& M, const StageParams& P, int grid,
                           cudaStream_t s) {
  if (viscous) {
    switch (stage) {
      case 0: return stage_go<T, true, 0, CURVI>(M, P, grid, s);
      case 1: return stage_go<T, true, 1, CURVI>(M, P, grid, s);
      case 2: return stage_go<T, true, 2, CURVI>(M, P, grid, s);
      case 3: return stage_go<T, true, 3, CURVI>(M, P, grid, s);
    }
  } else {
    switch (stage) {
      case 0: return stage_go<T, false, 0, CURVI>(M, P, grid, s);
      case 1: return stage_go<T, false, 1, CURVI>(M, P, grid, s);
      case 2: return stage_go<T, false, 2, CURVI>(M, P, grid, s);
      case 3: return stage_go<T, false, 3, CURVI>(M, P, grid, s);
    }
  }
  return cudaErrorInvalidValue;
}

template <typename T, bool CURVI>
int stage_occupancy(int viscous) {
  int n = 0;
  cudaError_t e;
  if (viscous) {
    auto k = stage_kernel<T, true, 1, CURVI>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Plan<T, true, CURVI>::bytes);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, NT, Plan<T, true, CURVI>::bytes);
  } else {
    auto k = stage_kernel<T, false, 1, CURVI>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Plan<T, false, CURVI>::bytes);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, NT, Plan<T, false, CURVI>::bytes);
  }
  return (e == cudaSuccess && n > 0) ? n : 1;
}

}  // namespace gbcfd
