// stage_inst.cuh -- launch helpers shared by the stage-kernel instantiation units
#pragma once
#include <atomic>

#include "launch.h"
#include "stage.cuh"

namespace gbcfd {

// the kernel's dynamic shared-memory limit, set once per device (before any graph capture)
// (a per-device bit set atomically: host threads may set up blocks concurrently, and setting the
// attribute twice is harmless)
template <typename T, bool VISC, int STAGE, bool CURVI>
cudaError_t stage_attr() {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64 && ((done.load(std::memory_order_acquire) >> dev) & 1ull)) return cudaSuccess;
  e = cudaFuncSetAttribute(stage_kernel<T, VISC, STAGE, CURVI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)Plan<T, VISC, CURVI>::bytes);
  if (e == cudaSuccess && dev < 64) done.fetch_or(1ull << dev, std::memory_order_acq_rel);
  return e;
}

template <typename T, bool VISC, int STAGE, bool CURVI>
cudaError_t stage_go(const GroupParams& P, int grid, cudaStream_t s) {
  cudaError_t e = stage_attr<T, VISC, STAGE, CURVI>();
  if (e != cudaSuccess) return e;
  stage_kernel<T, VISC, STAGE, CURVI><<<grid, NT, Plan<T, VISC, CURVI>::bytes, s>>>(P);
  return cudaGetLastError();
}

template <typename T, bool CURVI>
cudaError_t stage_prepare(int viscous) {
  cudaError_t e = cudaSuccess;
  if (viscous) {
    if (e == cudaSuccess) e = stage_attr<T, true, 0, CURVI>();
    if (e == cudaSuccess) e = stage_attr<T, true, 1, CURVI>();
    if (e == cudaSuccess) e = stage_attr<T, true, 2, CURVI>();
    if (e == cudaSuccess) e = stage_attr<T, true, 3, CURVI>();
  } else {
    if (e == cudaSuccess) e = stage_attr<T, false, 0, CURVI>();
    if (e == cudaSuccess) e = stage_attr<T, false, 1, CURVI>();
    if (e == cudaSuccess) e = stage_attr<T, false, 2, CURVI>();
    if (e == cudaSuccess) e = stage_attr<T, false, 3, CURVI>();
  }
  return e;
}

template <typename T, bool CURVI>
cudaError_t stage_dispatch(int viscous, int stage, const GroupParams& P, int grid, cudaStream_t s) {
  if (viscous) {
    switch (stage) {
      case 0: return stage_go<T, true, 0, CURVI>(P, grid, s);
      case 1: return stage_go<T, true, 1, CURVI>(P, grid, s);
      case 2: return stage_go<T, true, 2, CURVI>(P, grid, s);
      case 3: return stage_go<T, true, 3, CURVI>(P, grid, s);
    }
  } else {
    switch (stage) {
      case 0: return stage_go<T, false, 0, CURVI>(P, grid, s);
      case 1: return stage_go<T, false, 1, CURVI>(P, grid, s);
      case 2: return stage_go<T, false, 2, CURVI>(P, grid, s);
      case 3: return stage_go<T, false, 3, CURVI>(P, grid, s);
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
