// noalloc.cu -- gbcfd_time_step_noalloc: the CFL time step of a caller-given state with no
// device allocation at all, for callers that cannot allocate device memory.
//
// The reduction scratch (one partial maximum per CTA, a CTA counter and the result slot) is a
// file-scope __device__ array of fixed size, so it exists on every GPU that loads this library
// from module load until process exit.  Host code cannot use the array's name as a device
// address (in host code it names a host-side stand-in), so the first call on each device asks
// the runtime for the device address with cudaGetSymbolAddress while that device is current,
// and passes the address to the kernel.
#include <mutex>
#include <string>

#include "gbcfd.h"
#include "launch.h"

namespace gbcfd {

constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_CELLS_PER_THREAD = 64;
constexpr int NOALLOC_MAX_CTAS = 8192;  // 8192 x 256 x 64 = 134,217,728 cells at most
constexpr long long NOALLOC_MAX_CELLS =
    (long long)NOALLOC_MAX_CTAS * NOALLOC_THREADS * NOALLOC_CELLS_PER_THREAD;

struct NoallocScratch {
  double partial[NOALLOC_MAX_CTAS];  // max rate of each CTA
  double result[2];                  // [0] = cfl / max rate, [1] = max rate
  unsigned int counter;              // CTAs finished; must be 0 when a call starts
  int flag;                          // non-physical state met
};

// 64 KB + 32 B, shared by every call on the device: calls that overlap on the GPU race on it
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

// Each thread reduces a fixed run of cells, each CTA its threads, and the last CTA to finish the
// per-CTA maxima in index order (deterministic; max is exact anyway).  The rate is the same as
// the block path's: sum over directions of (|u_d| + c) / h_d, plus 4 max(4/3, gamma/Pr) mu / rho
// / h_d^2 when viscous; the step is cfl / max rate.
template <typename T>
__global__ void __launch_bounds__(NOALLOC_THREADS)
    noalloc_rate_kernel(const double* __restrict__ q, long long n, Physics ph, NoallocScratch* S) {
  __shared__ double wmax[NOALLOC_THREADS / 32];
  __shared__ int last;
  const T f = T(fmax(4.0 / 3.0, ph.gamma / ph.Pr));
  const T s2 = T(ph.ihx * ph.ihx + ph.ihy * ph.ihy + ph.ihz * ph.ihz);
  const T gam = T(ph.gamma), gm1 = T(ph.gamma - 1.0), mu4 = T(4.0 * ph.mu);
  const T ihx = T(ph.ihx), ihy = T(ph.ihy), ihz = T(ph.ihz);
  double best = 0.0;
  bool bad = false;
  const long long first = (long long)blockIdx.x * NOALLOC_THREADS * NOALLOC_CELLS_PER_THREAD + threadIdx.x;
  for (int r = 0; r < NOALLOC_CELLS_PER_THREAD; ++r) {
    const long long c = first + (long long)r * NOALLOC_THREADS;  // coalesced across the CTA
    if (c >= n) break;
    const T rho = T(q[c]), ir = T(1) / rho;
    const T u = T(q[n + c]) * ir, v = T(q[2 * n + c]) * ir, w = T(q[3 * n + c]) * ir;
    const T p = gm1 * (T(q[4 * n + c]) - T(0.5) * rho * (u * u + v * v + w * w));
    const T a = sqrt(gam * p * ir);
    T rate = (fabs(u) + a) * ihx + (fabs(v) + a) * ihy + (fabs(w) + a) * ihz;
    if (ph.viscous) rate += f * mu4 * ir * s2;
    if (!(rho > T(0) && p > T(0))) bad = true;
    best = fmax(best, double(rate));
  }
  if (bad) atomicOr(&S->flag, 1);
  for (int off = 16; off > 0; off >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, off));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < NOALLOC_THREADS / 32; ++w) m = fmax(m, wmax[w]);
    S->partial[blockIdx.x] = m;
    __threadfence();
    last = (atomicAdd(&S->counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  double m = 0.0;
  for (unsigned b = 0; b < gridDim.x; ++b) m = fmax(m, __ldcg(&S->partial[b]));
  S->result[0] = ph.cfl / m;
  S->result[1] = m;
  S->counter = 0u;
}

__global__ void noalloc_publish_kernel(const NoallocScratch* S, double* dt_out) {
  if (threadIdx.x == 0) *dt_out = S->flag ? -1.0 : S->result[0];
}

}  // namespace gbcfd

using namespace gbcfd;

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
NoallocScratch* g_scratch_ptr[kMaxDevices] = {nullptr};
}  // namespace

extern "C" int gbcfd_time_step_noalloc(const double* q, int nx, int ny, int nz, const gbcfd_params* params,
                                       const double spacing[3], double* dt, void* stream) {
  if (!q || !dt || !params || !spacing) return set_error(GBCFD_ERR_ARG, "NULL argument");
  if (nx < 1 || ny < 1 || nz < 1) return set_error(GBCFD_ERR_ARG, "block sizes must be >= 1");
  if (!(spacing[0] > 0 && spacing[1] > 0 && spacing[2] > 0))
    return set_error(GBCFD_ERR_ARG, "spacing must be three positive cell sizes");
  if (!(params->gamma > 1.0) || !(params->cfl > 0.0) || (params->viscous && !(params->Pr > 0.0)) ||
      (params->precision != GBCFD_FP64 && params->precision != GBCFD_MIXED))
    return set_error(GBCFD_ERR_ARG, "bad params");
  const long long n = (long long)nx * ny * nz;
  if (n > NOALLOC_MAX_CELLS)
    return set_error(GBCFD_ERR_ARG, "gbcfd_time_step_noalloc handles at most 134217728 cells (its fixed "
                                    "scratch holds 8192 CTA partials); got " + std::to_string(n));
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(GBCFD_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_error(GBCFD_ERR_ARG, "device ordinal out of range");
  NoallocScratch* S = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {  // once per device, with that device current
      // the lookup may load the module, which a stream capture in progress would not survive:
      // refuse the first call on a device while its stream is being captured
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      e = cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cs);
      if (e != cudaSuccess)
        return set_error(GBCFD_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
      if (cs != cudaStreamCaptureStatusNone)
        return set_error(GBCFD_ERR_STATE, "the first gbcfd_time_step_noalloc call on a device must come before "
                                          "any stream capture (it looks up the scratch array's address)");
      void* addr = nullptr;
      e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
      if (e != cudaSuccess)
        return set_error(GBCFD_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_ptr[dev] = static_cast<NoallocScratch*>(addr);
    }
    S = g_scratch_ptr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the counter and the flag must start at zero (a failed earlier call may have left them set)
  e = cudaMemsetAsync(&S->counter, 0, sizeof(unsigned int) + sizeof(int), s);
  if (e != cudaSuccess) return set_error(GBCFD_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  Physics ph;
  ph.gamma = params->gamma;
  ph.mu = params->mu;
  ph.Pr = params->Pr;
  ph.cfl = params->cfl;
  ph.eps = params->entropy_eps;
  ph.ihx = 1.0 / spacing[0];
  ph.ihy = 1.0 / spacing[1];
  ph.ihz = 1.0 / spacing[2];
  ph.viscous = params->viscous;
  ph.limiter = params->limiter;
  const long long per_cta = (long long)NOALLOC_THREADS * NOALLOC_CELLS_PER_THREAD;
  const unsigned grid = (unsigned)((n + per_cta - 1) / per_cta);
  if (params->precision == GBCFD_MIXED)
    noalloc_rate_kernel<float><<<grid, NOALLOC_THREADS, 0, s>>>(q, n, ph, S);
  else
    noalloc_rate_kernel<double><<<grid, NOALLOC_THREADS, 0, s>>>(q, n, ph, S);
  noalloc_publish_kernel<<<1, 32, 0, s>>>(S, dt);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(GBCFD_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return GBCFD_OK;
}
