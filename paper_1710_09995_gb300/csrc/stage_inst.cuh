// stage_inst.cuh -- launch helpers shared by the stage-kernel instantiation units
#pragma once
#include <atomic>

#include "launch.h"
#include "stage.cuh"

namespace gbcfd {

// the kernel's dynamic shared-memory limit, set once per device (before any graph capture)
// (a per-device bit set atomically: host threads may set up blocks concurrently, and setting the
// attribute twice is harmless)
template <typename T, bool VISC, int STAGE, bool CURVI, int TYV, bool PUSH = false>
cudaError_t stage_attr() {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64 && ((done.load(std::memory_order_acquire) >> dev) & 1ull)) return cudaSuccess;
  e = cudaFuncSetAttribute(stage_kernel<T, VISC, STAGE, CURVI, TYV, PUSH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)Plan<T, VISC, CURVI, TYV>::bytes);
  if (e == cudaSuccess && dev < 64) done.fetch_or(1ull << dev, std::memory_order_acq_rel);
  return e;
}

template <typename T, bool VISC, int STAGE, bool CURVI, int TYV, bool PUSH = false>
cudaError_t stage_go(const GroupParams& P, int grid, cudaStream_t s) {
  cudaError_t e = stage_attr<T, VISC, STAGE, CURVI, TYV, PUSH>();
  if (e != cudaSuccess) return e;
  stage_kernel<T, VISC, STAGE, CURVI, TYV, PUSH><<<grid, tile_threads(TYV), Plan<T, VISC, CURVI, TYV>::bytes, s>>>(P);
  return cudaGetLastError();
}

// stages 1 and 2 with the halo exchange folded in (Cartesian Euler groups); stage 3 has none
template <typename T, int TYV>
cudaError_t stage_dispatch_push(int stage, const GroupParams& P, int grid, cudaStream_t s) {
  switch (stage) {
    case 1: return stage_go<T, false, 1, false, TYV, true>(P, grid, s);
    case 2: return stage_go<T, false, 2, false, TYV, true>(P, grid, s);
  }
  return cudaErrorInvalidValue;
}
template <typename T, int TYV>
cudaError_t stage_prepare_push() {
  cudaError_t e = stage_attr<T, false, 1, false, TYV, true>();
  if (e == cudaSuccess) e = stage_attr<T, false, 2, false, TYV, true>();
  return e;
}

template <typename T, bool VISC, bool CURVI, int TYV>
cudaError_t stage_prepare_v() {
  cudaError_t e = stage_attr<T, VISC, 0, CURVI, TYV>();
  if (e == cudaSuccess) e = stage_attr<T, VISC, 1, CURVI, TYV>();
  if (e == cudaSuccess) e = stage_attr<T, VISC, 2, CURVI, TYV>();
  if (e == cudaSuccess) e = stage_attr<T, VISC, 3, CURVI, TYV>();
  return e;
}

template <typename T, bool VISC, bool CURVI, int TYV>
cudaError_t stage_dispatch_v(int stage, const GroupParams& P, int grid, cudaStream_t s) {
  switch (stage) {
    case 0: return stage_go<T, VISC, 0, CURVI, TYV>(P, grid, s);
    case 1: return stage_go<T, VISC, 1, CURVI, TYV>(P, grid, s);
    case 2: return stage_go<T, VISC, 2, CURVI, TYV>(P, grid, s);
    case 3: return stage_go<T, VISC, 3, CURVI, TYV>(P, grid, s);
  }
  return cudaErrorInvalidValue;
}

template <typename T, bool VISC, bool CURVI, int TYV>
int stage_occupancy_v() {
  int n = 0;
  auto k = stage_kernel<T, VISC, 1, CURVI, TYV>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Plan<T, VISC, CURVI, TYV>::bytes);
  const cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, tile_threads(TYV), Plan<T, VISC, CURVI, TYV>::bytes);
  return (e == cudaSuccess && n > 0) ? n : 1;
}

// the default tile height, viscous or not
template <typename T, bool CURVI>
cudaError_t stage_prepare(int viscous) {
  return viscous ? stage_prepare_v<T, true, CURVI, TY_DEFAULT>() : stage_prepare_v<T, false, CURVI, TY_DEFAULT>();
}
template <typename T, bool CURVI>
cudaError_t stage_dispatch(int viscous, int stage, const GroupParams& P, int grid, cudaStream_t s) {
  return viscous ? stage_dispatch_v<T, true, CURVI, TY_DEFAULT>(stage, P, grid, s)
                 : stage_dispatch_v<T, false, CURVI, TY_DEFAULT>(stage, P, grid, s);
}
template <typename T, bool CURVI>
int stage_occupancy(int viscous) {
  return viscous ? stage_occupancy_v<T, true, CURVI, TY_DEFAULT>() : stage_occupancy_v<T, false, CURVI, TY_DEFAULT>();
}

}  // namespace gbcfd
