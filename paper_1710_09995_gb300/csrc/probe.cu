// probe.cu -- gbcfd_op_rate: the throughput of the arithmetic the stage kernels are built from
// (FP64 and FP32 fused multiply-adds, the FP64 reciprocal by IEEE division and by the Newton
// step the FP64 path uses, the FP64 reciprocal square root), measured on the current GPU.  The
// FP64 stage kernels are bound by the FP64 pipe, so its rate is their roofline's denominator
// (the unit count x clock gives 1.2586 TFLOP/s on this part) and the ratios of the other
// operations to it are the costs the FP64 path's arithmetic was chosen by.
//
// Each thread runs 8 independent dependent chains of the operation (enough in flight to fill
// the pipe), a grid of 8 CTAs of 256 threads per SM; a warm-up launch, then one launch timed with
// CUDA events on the caller's stream.
#include <string>

#include "gbcfd.h"
#include "launch.h"
#include "vmath.cuh"

namespace gbcfd {

constexpr int PROBE_THREADS = 256, PROBE_CHAINS = 8;

template <int OP>
__global__ void __launch_bounds__(PROBE_THREADS) op_rate_kernel(double* sink, int iters, double seed) {
  const double t = seed + 1e-7 * (threadIdx.x & 31);
  // the multiplier and addend formed at run time, so that they sit in registers as the stage
  // kernels' operands do (not in the constant bank)
  const double m = seed * 0.999999999, c = seed * 1e-9;
  if constexpr (OP == GBCFD_OP_FFMA) {
    float a[PROBE_CHAINS];
    const float mf = float(seed) * 0.9999999f, cf = float(seed) * 1e-7f;
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) a[i] = float(t) + 0.125f * i;
    for (int it = 0; it < iters; ++it)
#pragma unroll
      for (int i = 0; i < PROBE_CHAINS; ++i) a[i] = fmaf(a[i], mf, cf);  // stays near 1
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) s += a[i];
    if (s == -1.f) sink[blockIdx.x] = s;  // never true: keeps the chains
  } else {
    double a[PROBE_CHAINS];
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) a[i] = t + 0.125 * i;
    for (int it = 0; it < iters; ++it)
#pragma unroll
      for (int i = 0; i < PROBE_CHAINS; ++i) {
        if constexpr (OP == GBCFD_OP_DFMA) a[i] = fma(a[i], m, c);  // stays near 1
        if constexpr (OP == GBCFD_OP_DIV) a[i] = 1.0 / a[i];                     // x, 1/x, x, ...
        if constexpr (OP == GBCFD_OP_RCP_NEWTON) a[i] = VM<double>::rcp(a[i]);
        if constexpr (OP == GBCFD_OP_RSQRT) a[i] = rsqrt(a[i]);                  // tends to 1
        if constexpr (OP == GBCFD_OP_DADD) a[i] = a[i] + c;                      // register operands
        if constexpr (OP == GBCFD_OP_DMUL) a[i] = a[i] * m;
        if constexpr (OP == GBCFD_OP_DFMA_CONST) a[i] = fma(a[i], 0.999999999, 1e-9);  // constant-bank operands
      }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) s += a[i];
    if (s == -1.0) sink[blockIdx.x] = s;
  }
}

static int probe_err(cudaError_t e, const char* what) {
  return set_error(GBCFD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <int OP>
static cudaError_t op_rate_go(double* sink, int grid, int iters, cudaStream_t s) {
  op_rate_kernel<OP><<<grid, PROBE_THREADS, 0, s>>>(sink, iters, 1.0);
  return cudaGetLastError();
}

}  // namespace gbcfd

using namespace gbcfd;

extern "C" int gbcfd_op_rate(int op, void* scratch, double* ops_per_second, void* stream) {
  if (!scratch || !ops_per_second) return set_error(GBCFD_ERR_ARG, "NULL argument");
  if (op < GBCFD_OP_DFMA || op > GBCFD_OP_DFMA_CONST) return set_error(GBCFD_ERR_ARG, "unknown operation");
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return probe_err(e, "no CUDA device");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int grid = 8 * nsm;
  const int iters = op == GBCFD_OP_FFMA ? 65536
                    : ((op == GBCFD_OP_DIV || op == GBCFD_OP_RCP_NEWTON || op == GBCFD_OP_RSQRT) ? 1024 : 4096);
  double* sink = static_cast<double*>(scratch);
  auto go = [&]() -> cudaError_t {
    switch (op) {
      case GBCFD_OP_DFMA: return op_rate_go<GBCFD_OP_DFMA>(sink, grid, iters, s);
      case GBCFD_OP_FFMA: return op_rate_go<GBCFD_OP_FFMA>(sink, grid, iters, s);
      case GBCFD_OP_DIV: return op_rate_go<GBCFD_OP_DIV>(sink, grid, iters, s);
      case GBCFD_OP_RCP_NEWTON: return op_rate_go<GBCFD_OP_RCP_NEWTON>(sink, grid, iters, s);
      case GBCFD_OP_RSQRT: return op_rate_go<GBCFD_OP_RSQRT>(sink, grid, iters, s);
      case GBCFD_OP_DADD: return op_rate_go<GBCFD_OP_DADD>(sink, grid, iters, s);
      case GBCFD_OP_DMUL: return op_rate_go<GBCFD_OP_DMUL>(sink, grid, iters, s);
      default: return op_rate_go<GBCFD_OP_DFMA_CONST>(sink, grid, iters, s);
    }
  };
  cudaEvent_t e0, e1;
  e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return probe_err(e, "cudaEventCreate");
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return probe_err(e, "cudaEventCreate");
  }
  float ms = 0.f;
  e = go();  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) e = go();
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return probe_err(e, "op-rate probe");
  *ops_per_second = (double)grid * PROBE_THREADS * PROBE_CHAINS * iters / (ms * 1e-3);
  return GBCFD_OK;
}
