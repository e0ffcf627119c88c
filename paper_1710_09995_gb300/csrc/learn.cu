// learn.cu -- kernels of the learned convergence accelerator (see learn.cuh): the weight gradient
// of the convolutions, Adam, weight packing, the loss, and the kernels that connect the network
// to a block.  The convolutions themselves (tcgen05 implicit GEMM) are in learn_tc.cu.
#include <atomic>

#include "internal.cuh"
#include "learn.cuh"

namespace gbcfd {
namespace learn {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ float silu(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
  const float s = 1.0f / (1.0f + __expf(-z));
  return s * (1.0f + z * (1.0f - s));
}

// tile -> (x0, y0, z, b)
__device__ __forceinline__ void tile_coords(long long tile, int X, int Y, int Z, int& x0, int& y0, int& z, int& b) {
  const int tx = (X + TILE_X - 1) / TILE_X, ty = (Y + TILE_Y - 1) / TILE_Y;
  x0 = (int)(tile % tx) * TILE_X;
  tile /= tx;
  y0 = (int)(tile % ty) * TILE_Y;
  tile /= ty;
  z = (int)(tile % Z);
  b = (int)(tile / Z);
}

// the input cells a tile reads: box cell (bx, by, bz) is volume cell (x0 + bx - 1, y0 + by - 1,
// z + bz - 1); zero outside in x and y, periodic (or zero) in z
__device__ __forceinline__ long long box_source(int x0, int y0, int z, int b, int cellb, int X, int Y, int Z,
                                                int zper) {
  const int bx = cellb % BOX_X, r = cellb / BOX_X, by = r % BOX_Y, bz = r / BOX_Y;
  const int gx = x0 + bx - 1, gy = y0 + by - 1;
  int gz = z + bz - 1;
  if (gx < 0 || gx >= X || gy < 0 || gy >= Y) return -1;
  if (zper) gz = (gz + Z) % Z;
  else if (gz < 0 || gz >= Z) return -1;
  return (((long long)b * Z + gz) * Y + gy) * X + gx;
}

// a kernel's dynamic shared-memory limit, set once per device
template <typename F>
static cudaError_t smem_attr(F* kernel, size_t bytes, std::atomic<unsigned long long>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64 && ((done.load(std::memory_order_acquire) >> dev) & 1ull)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && dev < 64) done.fetch_or(1ull << dev, std::memory_order_acq_rel);
  return e;
}

// ---- weight gradient ---------------------------------------------------------------------------
// dW[o][c][t] = sum over cells of g[cell][o] a[cell + d_t][c], db[o] = sum of g[cell][o].  Each
// CTA loops over tiles (stride gridDim.x) with a chunk of the outputs (blockIdx.y, NJ per
// thread) in registers and writes them to its own partial row; launch_grad_reduce sums the rows
// in a fixed order (deterministic).
constexpr int WG_NJ = 16;
template <int CIP, int CI, int COPG, int CO>
__global__ void __launch_bounds__(NTHREADS) wgrad_kernel(const bf16* __restrict__ a, const bf16* __restrict__ g,
                                                          float* __restrict__ part, int off_w, int off_b, int X,
                                                          int Y, int Z, int B, int zper) {
  constexpr int NO = CO * CI * NTAP + CO;
  constexpr int NJ = WG_NJ;
  const int o0 = blockIdx.y * NTHREADS * NJ;
  extern __shared__ __align__(16) unsigned char smem[];
  float* a_s = reinterpret_cast<float*>(smem);            // [BOX][CI]
  float* g_s = a_s + BOX * CI;                            // [128][CO]
  const int tid = threadIdx.x;
  float acc[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) acc[j] = 0.f;
  const long long tiles = (long long)((X + TILE_X - 1) / TILE_X) * ((Y + TILE_Y - 1) / TILE_Y) * Z * B;
  for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    int x0, y0, z, b;
    tile_coords(tile, X, Y, Z, x0, y0, z, b);
    __syncthreads();
    for (int i = tid; i < BOX * CI; i += NTHREADS) {
      const int cellb = i / CI, c = i % CI;
      const long long src = box_source(x0, y0, z, b, cellb, X, Y, Z, zper);
      a_s[i] = src >= 0 ? __bfloat162float(a[src * CIP + c]) : 0.f;
    }
    for (int i = tid; i < TILE_X * TILE_Y * CO; i += NTHREADS) {
      const int c = i / CO, o = i % CO;
      const int gx = x0 + c % TILE_X, gy = y0 + c / TILE_X;
      const long long cell = (((long long)b * Z + z) * Y + gy) * X + gx;
      g_s[i] = (gx < X && gy < Y) ? __bfloat162float(g[cell * COPG + o]) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int o = o0 + tid + j * NTHREADS;
      if (o >= NO) break;
      float s = 0.f;
      if (o < CO * CI * NTAP) {
        const int co = o / (CI * NTAP), r = o % (CI * NTAP), ci = r / NTAP, t = r % NTAP;
        const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
        for (int c = 0; c < TILE_X * TILE_Y; ++c) {
          const int cb = (dz * BOX_Y + c / TILE_X + dy) * BOX_X + c % TILE_X + dx;
          s = fmaf(g_s[c * CO + co], a_s[cb * CI + ci], s);
        }
      } else {
        const int co = o - CO * CI * NTAP;
        for (int c = 0; c < TILE_X * TILE_Y; ++c) s += g_s[c * CO + co];
      }
      acc[j] += s;
    }
  }
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const int o = o0 + tid + j * NTHREADS;
    if (o >= NO) break;
    const int dst = o < CO * CI * NTAP ? off_w + o : off_b + (o - CO * CI * NTAP);
    part[(size_t)blockIdx.x * NPARAM + dst] = acc[j];
  }
}

template <int CIP, int CI, int COPG, int CO>
static cudaError_t wgrad_go(const bf16* a, const bf16* g, const Net& n, int off_w, int off_b, int X, int Y, int Z,
                            int B, int zper, cudaStream_t s) {
  const size_t bytes = (size_t)(BOX * CI + TILE_X * TILE_Y * CO) * sizeof(float);
  static std::atomic<unsigned long long> done{0};
  cudaError_t e = smem_attr(wgrad_kernel<CIP, CI, COPG, CO>, bytes, done);
  if (e != cudaSuccess) return e;
  constexpr int NO = CO * CI * NTAP + CO;
  const dim3 grid(n.wgrid, (NO + NTHREADS * WG_NJ - 1) / (NTHREADS * WG_NJ));
  wgrad_kernel<CIP, CI, COPG, CO><<<grid, NTHREADS, bytes, s>>>(a, g, n.wpart, off_w, off_b, X, Y, Z, B, zper);
  return cudaGetLastError();
}

// layer 1: a = input features (16 ch, 10 used), g = dZ1 (32); layer 2: a = a1, g = dZ2; layer 3:
// a = a2, g = dY (16 ch, 5 used)
cudaError_t launch_wgrad(int layer, const bf16* a, const bf16* g, const Net& n, int X, int Y, int Z, int B, int zper,
                         cudaStream_t s) {
  if (layer == 1) return wgrad_go<P0, C0, P1, C1>(a, g, n, OFF_W1, OFF_B1, X, Y, Z, B, zper, s);
  if (layer == 2) return wgrad_go<P1, C1, P2, C2>(a, g, n, OFF_W2, OFF_B2, X, Y, Z, B, zper, s);
  if (layer == 3) return wgrad_go<P2, C2, 16, C3>(a, g, n, OFF_W3, OFF_B3, X, Y, Z, B, zper, s);
  return cudaErrorInvalidValue;
}

__global__ void grad_reduce_kernel(const float* __restrict__ part, int rows, float* __restrict__ grad) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= NPARAM) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += part[(size_t)r * NPARAM + o];
  grad[o] = s;
}
cudaError_t launch_grad_reduce(const Net& n, cudaStream_t s) {
  grad_reduce_kernel<<<(NPARAM + 255) / 256, 256, 0, s>>>(n.wpart, n.wgrid, n.grad);
  return cudaGetLastError();
}

// ---- Adam and packing ----------------------------------------------------------------------------
__global__ void adam_kernel(float* w, float* m, float* v, const float* g, float lr, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAM) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}
cudaError_t launch_adam(const Net& n, float lr, int step, cudaStream_t s) {
  const float c1 = 1.0f - powf(0.9f, (float)step), c2 = 1.0f - powf(0.999f, (float)step);
  adam_kernel<<<(NPARAM + 255) / 256, 256, 0, s>>>(n.w, n.m, n.v, n.grad, lr, c1, c2);
  return cudaGetLastError();
}

// master weights -> bf16 GEMM layouts (forward [t][o][c], backward [t'][c][o] with t' = 26 - t)
// and padded biases; padding entries are zero
__global__ void pack_kernel(Net n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const float* w = n.w;
  if (i < NTAP * P1 * P0) {  // w1 [t][o<32][c<16]
    const int t = i / (P1 * P0), o = (i / P0) % P1, c = i % P0;
    n.w1[i] = __float2bfloat16(c < C0 ? w[OFF_W1 + (o * C0 + c) * NTAP + t] : 0.f);
  }
  if (i < NTAP * P2 * P1) {  // w2 [t][o][c], w2b [t'][c][o]
    const int t = i / (P2 * P1), o = (i / P1) % P2, c = i % P1;
    n.w2[i] = __float2bfloat16(w[OFF_W2 + (o * C1 + c) * NTAP + t]);
    const int tb = i / (P1 * P2), cb = (i / P2) % P1, ob = i % P2;  // w2b[tb][cb][ob] = W2[ob][cb][26 - tb]
    n.w2b[i] = __float2bfloat16(w[OFF_W2 + (ob * C1 + cb) * NTAP + (NTAP - 1 - tb)]);
  }
  if (i < NTAP * 16 * P2) {  // w3 [t][o<16][c<32] (the MMA is 16 wide; 5 used)
    const int t = i / (16 * P2), o = (i / P2) % 16, c = i % P2;
    n.w3[i] = __float2bfloat16(o < C3 ? w[OFF_W3 + (o * C2 + c) * NTAP + t] : 0.f);
  }
  if (i < NTAP * P2 * 16) {  // w3b [t'][c<32][o<16] = W3[o][c][26 - t']
    const int tb = i / (P2 * 16), cb = (i / 16) % P2, ob = i % 16;
    n.w3b[i] = __float2bfloat16(ob < C3 ? w[OFF_W3 + (ob * C2 + cb) * NTAP + (NTAP - 1 - tb)] : 0.f);
  }
  if (i < P1) n.b1[i] = w[OFF_B1 + i];
  if (i < P2) n.b2[i] = w[OFF_B2 + i];
  if (i < P3) n.b3[i] = i < C3 ? w[OFF_B3 + i] : 0.f;
}
cudaError_t launch_pack(const Net& n, cudaStream_t s) {
  pack_kernel<<<(NTAP * P2 * P1 + 255) / 256, 256, 0, s>>>(n);
  return cudaGetLastError();
}

// ---- loss: dY = 2 (y - t) / (5 cells) in bf16 (16 channels), per-CTA sums of (y - t)^2 ----------
__global__ void loss_kernel(const float* __restrict__ y, const float* __restrict__ t, bf16* __restrict__ dy,
                            double* __restrict__ partial, long long cells) {
  __shared__ double red[NTHREADS / 32];
  const double inv = 2.0 / (5.0 * (double)cells);
  double acc = 0.0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += (long long)gridDim.x * blockDim.x) {
    __align__(16) bf16 out[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) out[k] = __float2bfloat16(0.f);
#pragma unroll
    for (int k = 0; k < C3; ++k) {
      const float d = y[c * P3 + k] - t[c * P3 + k];
      acc += (double)d * d;
      out[k] = __float2bfloat16((float)(inv * d));
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) reinterpret_cast<uint4*>(dy + c * 16)[k] = reinterpret_cast<const uint4*>(out)[k];
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < NTHREADS / 32; ++w) s += red[w];
    partial[(size_t)blockIdx.x * NPART] = s;
  }
}
cudaError_t launch_loss(const float* y, const float* t, bf16* dy, double* partial, long long cells, int grid,
                        cudaStream_t s) {
  loss_kernel<<<grid, NTHREADS, 0, s>>>(y, t, dy, partial, cells);
  return cudaGetLastError();
}

// out[j] = sum over rows r < n of partial[r * NPART + j], j < nvals (fixed order)
__global__ void sum_kernel(const double* __restrict__ partial, int n, int nvals, double* __restrict__ out) {
  const int j = threadIdx.x;
  if (j >= nvals) return;
  double s = 0.0;
  for (int r = 0; r < n; ++r) s += partial[(size_t)r * NPART + j];
  out[j] = s;
}
cudaError_t launch_sum(const double* partial, int n, int nvals, double* out, cudaStream_t s) {
  sum_kernel<<<1, 32, 0, s>>>(partial, n, nvals, out);
  return cudaGetLastError();
}

// ---- block-facing kernels ----------------------------------------------------------------------
__device__ __forceinline__ long long vidx(const BlockView& v, int i, int j, int k) {
  return ((long long)(k + HALO) * (v.ny + 2 * HALO) + (j + HALO)) * v.px + (i + HALO);
}
__device__ __forceinline__ long long vidxf(const BlockView& v, int i, int j, int k) {
  return ((long long)(k + HALO) * (v.ny + 2 * HALO) + (j + HALO)) * v.pxf + (i + HALO);
}
__device__ __forceinline__ double cell_dt(const BlockView& v, int i, int j, int k) {
  if (!v.dtl) return *v.dt;
  return v.dtl_f32 ? (double)static_cast<const float*>(v.dtl)[vidxf(v, i, j, k)]
                   : static_cast<const double*>(v.dtl)[vidx(v, i, j, k)];
}

// per CTA: [0] sum over cells and variables of (dt R / ref)^2, [1] sum of R_rho^2
__global__ void feature_stats_kernel(BlockView v, const double* __restrict__ R, double* __restrict__ partial) {
  __shared__ double red[2][NTHREADS / 32];
  const long long n = (long long)v.nx * v.ny * v.nz;
  double s0 = 0.0, s1 = 0.0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % v.nx);
    const long long r = c / v.nx;
    const int j = (int)(r % v.ny), k = (int)(r / v.ny);
    const double dt = cell_dt(v, i, j, k);
    for (int m = 0; m < 5; ++m) {
      const double x = dt * R[m * n + c] / v.ref[m];
      s0 += x * x;
    }
    s1 += R[c] * R[c];
  }
  for (int off = 16; off > 0; off >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, off);
    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
  }
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = s0; red[1][threadIdx.x >> 5] = s1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < NTHREADS / 32; ++w) { a += red[0][w]; b += red[1][w]; }
    partial[(size_t)blockIdx.x * NPART] = a;
    partial[(size_t)blockIdx.x * NPART + 1] = b;
  }
}
cudaError_t launch_feature_stats(const BlockView& v, const double* R, double* partial, int grid, cudaStream_t s) {
  feature_stats_kernel<<<grid, NTHREADS, 0, s>>>(v, R, partial);
  return cudaGetLastError();
}

// x[cell] = (10 (Q - Q_inf) / ref, (-dt R / ref) / s, 0 x 6) in bf16; the compact state is saved
// (f64) for the prediction, the target and a revert.  s = sqrt(stats[0] / (5 cells)).
__global__ void features_kernel(BlockView v, const double* __restrict__ R, const double* __restrict__ stats,
                                bf16* __restrict__ x, double* __restrict__ qsave) {
  const long long n = (long long)v.nx * v.ny * v.nz;
  const double s = sqrt(stats[0] / (5.0 * (double)n));
  const double is = s > 0.0 ? 1.0 / s : 0.0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % v.nx);
    const long long r = c / v.nx;
    const int j = (int)(r % v.ny), k = (int)(r / v.ny);
    const long long o = vidx(v, i, j, k);
    const double dt = cell_dt(v, i, j, k);
    __align__(16) bf16 f[16];
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      const double q = v.q[m * v.field + o];
      qsave[m * n + c] = q;
      f[m] = __double2bfloat16((double)STATE_GAIN * (q - v.qinf[m]) / v.ref[m]);
      f[5 + m] = __double2bfloat16(-dt * R[m * n + c] / v.ref[m] * is);
    }
#pragma unroll
    for (int m = 10; m < 16; ++m) f[m] = __float2bfloat16(0.f);
    reinterpret_cast<uint4*>(x + c * 16)[0] = reinterpret_cast<const uint4*>(f)[0];
    reinterpret_cast<uint4*>(x + c * 16)[1] = reinterpret_cast<const uint4*>(f)[1];
  }
}
cudaError_t launch_features(const BlockView& v, const double* R, const double* stats, bf16* x, double* qsave,
                            cudaStream_t s) {
  const long long n = (long long)v.nx * v.ny * v.nz;
  long long grid = (n + 255) / 256;
  if (grid > 65535LL * 8) grid = 65535LL * 8;
  features_kernel<<<(unsigned)grid, 256, 0, s>>>(v, R, stats, x, qsave);
  return cudaGetLastError();
}

// Q = Q_saved + alpha K s ref y (or Q_saved when revert), into the padded state and its f32 shadow
__global__ void apply_kernel(BlockView v, const float* __restrict__ y, const double* __restrict__ qsave,
                             const double* __restrict__ stats, int revert, double alpha) {
  const long long n = (long long)v.nx * v.ny * v.nz;
  const double s = alpha * sqrt(stats[0] / (5.0 * (double)n));
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % v.nx);
    const long long r = c / v.nx;
    const int j = (int)(r % v.ny), k = (int)(r / v.ny);
    const long long o = vidx(v, i, j, k);
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      double q = qsave[m * n + c];
      if (!revert) q += (double)K_STEPS * s * v.ref[m] * (double)y[c * P3 + m];
      v.q[m * v.field + o] = q;
      if (v.sh) v.sh[m * v.fieldf + vidxf(v, i, j, k)] = (float)q;
    }
  }
}
cudaError_t launch_apply(const BlockView& v, const float* y, const double* qsave, const double* stats, int revert,
                         cudaStream_t s, double alpha) {
  const long long n = (long long)v.nx * v.ny * v.nz;
  long long grid = (n + 255) / 256;
  if (grid > 65535LL * 8) grid = 65535LL * 8;
  apply_kernel<<<(unsigned)grid, 256, 0, s>>>(v, y, qsave, stats, revert, alpha);
  return cudaGetLastError();
}

// t[cell][m] = (Q_now - Q_saved) / ref / (K s) (f32, 8 channels, 5 used)
__global__ void target_kernel(BlockView v, const double* __restrict__ qsave, const double* __restrict__ stats,
                              float* __restrict__ t) {
  const long long n = (long long)v.nx * v.ny * v.nz;
  const double s = sqrt(stats[0] / (5.0 * (double)n));
  const double is = s > 0.0 ? 1.0 / ((double)K_STEPS * s) : 0.0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % v.nx);
    const long long r = c / v.nx;
    const int j = (int)(r % v.ny), k = (int)(r / v.ny);
    const long long o = vidx(v, i, j, k);
#pragma unroll
    for (int m = 0; m < 5; ++m) t[c * P3 + m] = (float)((v.q[m * v.field + o] - qsave[m * n + c]) / v.ref[m] * is);
#pragma unroll
    for (int m = 5; m < P3; ++m) t[c * P3 + m] = 0.f;
  }
}
cudaError_t launch_target(const BlockView& v, const double* qsave, const double* stats, float* t, cudaStream_t s) {
  const long long n = (long long)v.nx * v.ny * v.nz;
  long long grid = (n + 255) / 256;
  if (grid > 65535LL * 8) grid = 65535LL * 8;
  target_kernel<<<(unsigned)grid, 256, 0, s>>>(v, qsave, stats, t);
  return cudaGetLastError();
}

}  // namespace learn
}  // namespace gbcfd
