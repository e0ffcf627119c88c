// aux_kernels.cu -- halo exchange, state scatter/gather and time-step kernels.
#include <algorithm>

#include "launch.h"
#include "vmath.cuh"

namespace gbcfd {

// ---- halo exchange -------------------------------------------------------------------------
// One thread per halo cell of every block in the group.  The source of a halo cell is found by
// walking face neighbours: first along x, then along y in the block reached, then along z, so
// that edge and corner cells come from the diagonal neighbour.  A direction without a neighbour
// (a physical boundary) is skipped and its index stays outside: an edge cell next to a boundary
// face then copies the neighbour's boundary ghost, and a cell of the boundary face slab itself
// (no move at all) is left to the boundary kernel.  Each block's halo is the union of the
// z-slabs (k < 0 or k >= nz, all i, j), the y-slabs (0 <= k < nz, j outside, all i) and the
// x-slabs (inside k and j, i outside).
__global__ void halo_kernel(const __grid_constant__ HaloGroup G) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < G.total; t += stride) {
    int lo = 0, hi = G.n - 1;
    while (lo < hi) {  // last block whose prefix start <= t
      const int mid = (lo + hi + 1) >> 1;
      if (G.b[mid].first <= t) lo = mid; else hi = mid - 1;
    }
    const HaloBlock& B = G.b[lo];
    long long h = t - B.first;
    const int nx = B.nx, ny = B.ny, nz = B.nz;
    const long long wx = nx + 2 * HALO, wy = ny + 2 * HALO;
    int i, j, k;
    const long long zc = 2LL * HALO * wx * wy, yc = (long long)nz * 2 * HALO * wx;
    if (h < zc) {
      const int kk = (int)(h / (wx * wy));
      const long long r = h - kk * wx * wy;
      k = kk < HALO ? kk - HALO : nz + kk - HALO;
      j = (int)(r / wx) - HALO;
      i = (int)(r % wx) - HALO;
    } else if ((h -= zc) < yc) {
      k = (int)(h / (2 * HALO * wx));
      const long long r = h - (long long)k * 2 * HALO * wx;
      const int jj = (int)(r / wx);
      j = jj < HALO ? jj - HALO : ny + jj - HALO;
      i = (int)(r % wx) - HALO;
    } else {
      h -= yc;
      k = (int)(h / ((long long)ny * 2 * HALO));
      const long long r = h - (long long)k * ny * 2 * HALO;
      j = (int)(r / (2 * HALO));
      const int ii = (int)(r % (2 * HALO));
      i = ii < HALO ? ii - HALO : nx + ii - HALO;
    }
    // walk to the source block (a missing neighbour leaves that index outside)
    int b = lo, si = i, sj = j, sk = k;
    bool moved = false;
    while (si < 0 && G.b[b].nbr[0] >= 0) { b = G.b[b].nbr[0]; si += G.b[b].nx; moved = true; }
    while (si >= G.b[b].nx && G.b[b].nbr[1] >= 0) { si -= G.b[b].nx; b = G.b[b].nbr[1]; moved = true; }
    while (sj < 0 && G.b[b].nbr[2] >= 0) { b = G.b[b].nbr[2]; sj += G.b[b].ny; moved = true; }
    while (sj >= G.b[b].ny && G.b[b].nbr[3] >= 0) { sj -= G.b[b].ny; b = G.b[b].nbr[3]; moved = true; }
    while (sk < 0 && G.b[b].nbr[4] >= 0) { b = G.b[b].nbr[4]; sk += G.b[b].nz; moved = true; }
    while (sk >= G.b[b].nz && G.b[b].nbr[5] >= 0) { sk -= G.b[b].nz; b = G.b[b].nbr[5]; moved = true; }
    // a source left outside a smaller neighbour's halo (only with blocks narrower than the halo)
    if (!moved || si < -HALO || si >= G.b[b].nx + HALO || sj < -HALO || sj >= G.b[b].ny + HALO ||
        sk < -HALO || sk >= G.b[b].nz + HALO)
      continue;
    const HaloBlock& S = G.b[b];
    const long long dplane = (long long)(ny + 2 * HALO) * B.pitch, dfield = dplane * (nz + 2 * HALO);
    const long long splane = (long long)(S.ny + 2 * HALO) * S.pitch, sfield = splane * (S.nz + 2 * HALO);
    const long long dof = (k + HALO) * dplane + (long long)(j + HALO) * B.pitch + (i + HALO);
    const long long sof = (sk + HALO) * splane + (long long)(sj + HALO) * S.pitch + (si + HALO);
    if (G.elem == 8) {
      double* d = reinterpret_cast<double*>(B.base[0]);
      const double* s = reinterpret_cast<const double*>(S.base[0]);
      for (int v = 0; v < G.nvar; ++v) d[v * dfield + dof] = s[v * sfield + sof];
    } else {
      float* d = reinterpret_cast<float*>(B.base[0]);
      const float* s = reinterpret_cast<const float*>(S.base[0]);
      for (int v = 0; v < G.nvar; ++v) d[v * dfield + dof] = s[v * sfield + sof];
    }
  }
}

cudaError_t launch_halo(const HaloGroup& G, cudaStream_t s) {
  if (G.total <= 0) return cudaSuccess;
  const int threads = 256;
  long long blocks = (G.total + threads - 1) / threads;
  if (blocks > 65535LL * 8) blocks = 65535LL * 8;
  halo_kernel<<<(unsigned)blocks, threads, 0, s>>>(G);
  return cudaGetLastError();
}

// ---- compact <-> padded state --------------------------------------------------------------
// shadow (may be null): the f32 rounding of the state, written alongside
// A CTA per row (v, k, j) of nx values: src is compact [5][nz][ny][nx] (device memory, or pinned
// host memory read over the host link), dst the padded f64 field; the mixed path's f32 shadow is
// rounded on the integer pipe (bitwise the hardware rounding, see vmath.cuh).
__global__ void scatter_kernel(Geometry g, const double* __restrict__ src, double* __restrict__ dst,
                               float* __restrict__ shadow) {
  const int rows = 5 * g.ny * g.nz;
  for (int row = blockIdx.x; row < rows; row += gridDim.x) {
    const int j = row % g.ny, r = row / g.ny, k = r % g.nz, v = r / g.nz;
    const double* s = src + (long long)row * g.nx;
    double* d = dst + v * g.field + gidx(g, 0, j, k);
    float* sh = shadow ? shadow + v * g.fieldf + gidxf(g, 0, j, k) : nullptr;
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
      const double x = s[i];
      d[i] = x;
      if (sh) sh[i] = f64_to_f32_bits(x);
    }
  }
}
// the reverse: padded f64 field -> compact [5][nz][ny][nx] (device memory or pinned host memory)
__global__ void gather_kernel(Geometry g, const double* __restrict__ src, double* __restrict__ dst) {
  const int rows = 5 * g.ny * g.nz;
  for (int row = blockIdx.x; row < rows; row += gridDim.x) {
    const int j = row % g.ny, r = row / g.ny, k = r % g.nz, v = r / g.nz;
    const double* s = src + v * g.field + gidx(g, 0, j, k);
    double* d = dst + (long long)row * g.nx;
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) d[i] = s[i];
  }
}
static unsigned grid_for(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  if (b > 65535LL * 16) b = 65535LL * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}
static unsigned row_grid(const Geometry& g) {
  const long long rows = 5LL * g.ny * g.nz;
  return (unsigned)std::min(rows, 65535LL * 16);
}
static int row_threads(const Geometry& g) { return g.nx >= 256 ? 256 : (g.nx >= 128 ? 128 : 64); }
cudaError_t launch_scatter(const Geometry& g, const double* src, double* dst, float* shadow, cudaStream_t s) {
  scatter_kernel<<<row_grid(g), row_threads(g), 0, s>>>(g, src, dst, shadow);
  return cudaGetLastError();
}
cudaError_t launch_gather(const Geometry& g, const double* src, double* dst, cudaStream_t s) {
  gather_kernel<<<row_grid(g), row_threads(g), 0, s>>>(g, src, dst);
  return cudaGetLastError();
}

// ---- time step -----------------------------------------------------------------------------
// rate = sum over directions of (|u_d| + c) / h_d (+ 4 max(4/3, gamma/Pr) mu / rho / h_d^2 when
// viscous); the CFL step is cfl / max(rate).  From the padded f64 state, in the path's flux
// precision T (the mixed path's time step is an f32 evaluation, like its fluxes).
template <typename T>
__global__ void init_rate_kernel(Geometry g, Physics ph, const double* __restrict__ q, DevCtrl* ctrl,
                                 double* partial, T* dtl) {
  __shared__ double wmax[32];
  __shared__ int last;
  const long long n = (long long)g.nx * g.ny * g.nz;
  double best = 0.0;
  const T f = T(fmax(4.0 / 3.0, ph.gamma / ph.Pr));
  const T s2 = T(ph.ihx * ph.ihx + ph.ihy * ph.ihy + ph.ihz * ph.ihz);
  const T gam = T(ph.gamma), gm1 = T(ph.gamma - 1.0), mu4 = T(4.0 * ph.mu);
  const T ihx = T(ph.ihx), ihy = T(ph.ihy), ihz = T(ph.ihz);
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.nx);
    const long long r = c / g.nx;
    const int j = (int)(r % g.ny), k = (int)(r / g.ny);
    const long long o = gidx(g, i, j, k);
    const T rho = T(q[o]), ir = T(1) / rho;
    const T u = T(q[g.field + o]) * ir, v = T(q[2 * g.field + o]) * ir, w = T(q[3 * g.field + o]) * ir;
    const T p = gm1 * (T(q[4 * g.field + o]) - T(0.5) * rho * (u * u + v * v + w * w));
    const T a = sqrt(gam * p * ir);
    T rate = (fabs(u) + a) * ihx + (fabs(v) + a) * ihy + (fabs(w) + a) * ihz;
    if (ph.viscous) rate += f * mu4 * ir * s2;
    if (dtl) dtl[sizeof(T) == 8 ? o : gidxf(g, i, j, k)] = T(ph.cfl) / rate;
    if (!(rho > T(0) && p > T(0))) atomicOr(&ctrl->flag, FLAG_NONPHYSICAL);
    best = fmax(best, double(rate));
  }
  for (int off = 16; off > 0; off >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, off));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, wmax[w]);
    partial[(size_t)blockIdx.x * NPART + 5] = m;
    __threadfence();
    last = (atomicAdd(&ctrl->counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  double m = 0.0;
  for (unsigned b = 0; b < gridDim.x; ++b) m = fmax(m, __ldcg(partial + (size_t)b * NPART + 5));
  ctrl->rate = m;
  ctrl->dt = ph.cfl / m;
  ctrl->counter = 0u;
}

cudaError_t launch_init_rate(const Geometry& g, const Physics& ph, const double* q, DevCtrl* ctrl,
                             double* partial, int grid, int mixed, void* dtl, cudaStream_t s) {
  if (mixed)
    init_rate_kernel<float><<<grid, 256, 0, s>>>(g, ph, q, ctrl, partial, static_cast<float*>(dtl));
  else
    init_rate_kernel<double><<<grid, 256, 0, s>>>(g, ph, q, ctrl, partial, static_cast<double*>(dtl));
  return cudaGetLastError();
}

// ---- curvilinear metrics -------------------------------------------------------------------
// Per interior cell: the area vectors of its lower xi, eta, zeta faces, S = 1/2 (d1 x d2) over
// the face diagonals, oriented towards +xi, +eta, +zeta, and the volume by the divergence
// theorem, V = 1/3 sum over the six faces of (face centroid - first corner) . outward S.
// nodes: x[3][nz+1][ny+1][nx+1] (f64).  M: 10 padded fields, f64 or f32 (elem bytes).
__device__ __forceinline__ void vsub(const double* a, const double* b, double* c) {
  c[0] = a[0] - b[0]; c[1] = a[1] - b[1]; c[2] = a[2] - b[2];
}
__device__ __forceinline__ void half_cross(const double* a, const double* b, double* c) {
  c[0] = 0.5 * (a[1] * b[2] - a[2] * b[1]);
  c[1] = 0.5 * (a[2] * b[0] - a[0] * b[2]);
  c[2] = 0.5 * (a[0] * b[1] - a[1] * b[0]);
}

// node (i, j, k); indices beyond the block's nodes are extended by reflection through the
// boundary node along the grid line, X(-m) = 2 X(0) - X(m), X(n + m) = 2 X(n) - X(n - m), the
// x index first, then y, then z
__device__ __forceinline__ void node_in(const Geometry& g, const double* X, long long nn, int i, int j, int k,
                                        double* x) {
  const long long o = ((long long)k * (g.ny + 1) + j) * (g.nx + 1) + i;
  x[0] = X[o]; x[1] = X[nn + o]; x[2] = X[2 * nn + o];
}
__device__ __forceinline__ void node_k(const Geometry& g, const double* X, long long nn, int i, int j, int k,
                                       double* x) {
  if (k < 0 || k > g.nz) {
    const int e = k < 0 ? 0 : g.nz;
    double a[3], b[3];
    node_in(g, X, nn, i, j, e, a);
    node_in(g, X, nn, i, j, min(max(2 * e - k, 0), g.nz), b);  // clamp: blocks thinner than 2 cells
    for (int c = 0; c < 3; ++c) x[c] = __dsub_rn(2.0 * a[c], b[c]);
  } else {
    node_in(g, X, nn, i, j, k, x);
  }
}
__device__ __forceinline__ void node_jk(const Geometry& g, const double* X, long long nn, int i, int j, int k,
                                        double* x) {
  if (j < 0 || j > g.ny) {
    const int e = j < 0 ? 0 : g.ny;
    double a[3], b[3];
    node_k(g, X, nn, i, e, k, a);
    node_k(g, X, nn, i, min(max(2 * e - j, 0), g.ny), k, b);
    for (int c = 0; c < 3; ++c) x[c] = __dsub_rn(2.0 * a[c], b[c]);
  } else {
    node_k(g, X, nn, i, j, k, x);
  }
}
__device__ __forceinline__ void node_ext(const Geometry& g, const double* X, long long nn, int i, int j, int k,
                                         double* x) {
  if (i < 0 || i > g.nx) {
    const int e = i < 0 ? 0 : g.nx;
    double a[3], b[3];
    node_jk(g, X, nn, e, j, k, a);
    node_jk(g, X, nn, min(max(2 * e - i, 0), g.nx), j, k, b);
    for (int c = 0; c < 3; ++c) x[c] = __dsub_rn(2.0 * a[c], b[c]);
  } else {
    node_jk(g, X, nn, i, j, k, x);
  }
}

// every padded cell, halo included (halo nodes by reflection; the halo exchange then replaces
// the halo cells of connected faces with the neighbour's)
__global__ void metrics_kernel(Geometry g, const double* __restrict__ X, void* M, int elem) {
  const long long wx = g.nx + 2 * HALO, wy = g.ny + 2 * HALO;
  const long long n = wx * wy * (g.nz + 2 * HALO);
  const long long nn = (long long)(g.nx + 1) * (g.ny + 1) * (g.nz + 1);
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % wx) - HALO;
    const long long r = c / wx;
    const int j = (int)(r % wy) - HALO, k = (int)(r / wy) - HALO;
    double p[8][3];  // corner (di, dj, dk) at index di + 2 dj + 4 dk
    for (int q = 0; q < 8; ++q) node_ext(g, X, nn, i + (q & 1), j + ((q >> 1) & 1), k + (q >> 2), p[q]);
    // quadrilateral a, b, c, d in counter-clockwise order seen from the side S points to:
    // S = 1/2 (c - a) x (d - b)
    auto face = [&](int a, int b, int cc, int d, double* S, double* cen) {
      double d1[3], d2[3];
      vsub(p[cc], p[a], d1);
      vsub(p[d], p[b], d2);
      half_cross(d1, d2, S);
      for (int x = 0; x < 3; ++x) cen[x] = 0.25 * (p[a][x] + p[b][x] + p[cc][x] + p[d][x]) - p[0][x];
    };
    double S[6][3], C[6][3];
    face(0, 2, 6, 4, S[0], C[0]);  // lower xi   (eta, zeta plane at di = 0)
    face(1, 3, 7, 5, S[1], C[1]);  // upper xi
    face(0, 4, 5, 1, S[2], C[2]);  // lower eta  (zeta, xi plane at dj = 0)
    face(2, 6, 7, 3, S[3], C[3]);  // upper eta
    face(0, 1, 3, 2, S[4], C[4]);  // lower zeta (xi, eta plane at dk = 0)
    face(4, 5, 7, 6, S[5], C[5]);  // upper zeta
    double vol = 0.0;
    for (int f = 0; f < 6; ++f) {
      const double sgn = (f & 1) ? 1.0 : -1.0;
      vol += sgn * (C[f][0] * S[f][0] + C[f][1] * S[f][1] + C[f][2] * S[f][2]);
    }
    vol *= 1.0 / 3.0;
    const double out[10] = {S[0][0], S[0][1], S[0][2], S[2][0], S[2][1], S[2][2],
                            S[4][0], S[4][1], S[4][2], vol};
    if (elem == 8) {
      double* m = static_cast<double*>(M);
      const long long o = gidx(g, i, j, k);
      for (int v = 0; v < 10; ++v) m[v * g.field + o] = out[v];
    } else {
      float* m = static_cast<float*>(M);
      const long long o = gidxf(g, i, j, k);
      for (int v = 0; v < 10; ++v) m[v * g.fieldf + o] = float(out[v]);
    }
  }
}

cudaError_t launch_metrics(const Geometry& g, const double* nodes, void* M, int elem, cudaStream_t s) {
  const long long n = (long long)(g.nx + 2 * HALO) * (g.ny + 2 * HALO) * (g.nz + 2 * HALO);
  metrics_kernel<<<grid_for(n, 128), 128, 0, s>>>(g, nodes, M, elem);
  return cudaGetLastError();
}

// spectral-radius rate on a curvilinear grid: sum over directions of |u.Sb| + c |Sb| (+ 4 max(4/3,
// gamma/Pr) mu/rho |Sb|^2 / V), divided by V, with Sb the mean of a cell's two faces in a direction
template <typename T>
__global__ void init_rate_curvi_kernel(Geometry g, Physics ph, const double* __restrict__ q,
                                       const T* __restrict__ M, DevCtrl* ctrl, double* partial, T* dtl) {
  __shared__ double wmax[32];
  __shared__ int last;
  const long long n = (long long)g.nx * g.ny * g.nz;
  const long long fm = sizeof(T) == 8 ? g.field : g.fieldf;
  const double f = fmax(4.0 / 3.0, ph.gamma / ph.Pr);
  double best = 0.0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.nx);
    const long long r = c / g.nx;
    const int j = (int)(r % g.ny), k = (int)(r / g.ny);
    const long long o = gidx(g, i, j, k);
    const long long om = sizeof(T) == 8 ? o : gidxf(g, i, j, k);
    const long long up[3] = {1, sizeof(T) == 8 ? g.px : g.pxf, sizeof(T) == 8 ? g.plane : g.planef};
    const T rho = T(q[o]), ir = T(1) / rho;
    const T u = T(q[g.field + o]) * ir, v = T(q[2 * g.field + o]) * ir, w = T(q[3 * g.field + o]) * ir;
    const T p = T(ph.gamma - 1.0) * (T(q[4 * g.field + o]) - T(0.5) * rho * (u * u + v * v + w * w));
    const T a = sqrt(T(ph.gamma) * p * ir);
    const T vol = M[9 * fm + om], iv = T(1) / vol;
    T rate = T(0);
    for (int d = 0; d < 3; ++d) {
      T sb[3];
      for (int x = 0; x < 3; ++x) sb[x] = T(0.5) * (M[(3 * d + x) * fm + om] + M[(3 * d + x) * fm + om + up[d]]);
      const T s2 = sb[0] * sb[0] + sb[1] * sb[1] + sb[2] * sb[2];
      T lam = fabs(u * sb[0] + v * sb[1] + w * sb[2]) + a * sqrt(s2);
      if (ph.viscous) lam += T(4.0 * f * ph.mu) * ir * s2 * iv;
      rate += lam;
    }
    rate *= iv;
    if (dtl) dtl[om] = T(ph.cfl) / rate;
    if (!(rho > T(0) && p > T(0))) atomicOr(&ctrl->flag, FLAG_NONPHYSICAL);
    best = fmax(best, double(rate));
  }
  for (int off = 16; off > 0; off >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, off));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, wmax[w]);
    partial[(size_t)blockIdx.x * NPART + 5] = m;
    __threadfence();
    last = (atomicAdd(&ctrl->counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  double m = 0.0;
  for (unsigned b = 0; b < gridDim.x; ++b) m = fmax(m, __ldcg(partial + (size_t)b * NPART + 5));
  ctrl->rate = m;
  ctrl->dt = ph.cfl / m;
  ctrl->counter = 0u;
}

cudaError_t launch_init_rate_curvi(const Geometry& g, const Physics& ph, const double* q, const void* M,
                                   DevCtrl* ctrl, double* partial, int grid, int mixed, void* dtl, cudaStream_t s) {
  if (mixed)
    init_rate_curvi_kernel<float><<<grid, 256, 0, s>>>(g, ph, q, static_cast<const float*>(M), ctrl, partial,
                                                       static_cast<float*>(dtl));
  else
    init_rate_curvi_kernel<double><<<grid, 256, 0, s>>>(g, ph, q, static_cast<const double*>(M), ctrl, partial,
                                                        static_cast<double*>(dtl));
  return cudaGetLastError();
}

// ---- boundary ghost cells ---------------------------------------------------------------------
// One thread per (side, ghost layer m, face-slab point) of the physical faces of direction
// B.dim, over the full padded extent of the other two directions so that edges and corners get
// physical values too (directions are filled one launch after the other: x, y, z).
//   slip wall: ghost m mirrors interior cell m about the wall face's unit normal n,
//              u_g = u - 2 (u.n) n, same density and pressure
//   far field: characteristic boundary state from the adjacent interior cell and the free
//              stream (outgoing invariant u.n + 2c/(gamma-1) from inside, incoming one from the
//              free stream; entropy and tangential velocity from the upwind side; supersonic
//              inflow takes the free stream, supersonic outflow the interior), both layers
// On the mixed path the state is f32; for stages 2 and 3 the field is the f32 increment D over
// the f32 state S^n (the stencil adds them): the ghost increment is f32(Q_ghost - S_ghost).
// The ghost-cell arithmetic runs in the precision of the field it fills: FP64 for the FP64 state,
// FP32 for the mixed path's f32 state and increments (the values the FP32 fluxes read; FP64 here
// would leave these small launches waiting on the FP64 pipe, 2 lanes per SM).
template <typename T> struct BcMath;
template <> struct BcMath<double> {
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double pow_(double x, double y) { return pow(x, y); }
};
template <> struct BcMath<float> {
  static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
  static __device__ __forceinline__ float pow_(float x, float y) { return powf(x, y); }
};

template <typename T>
__device__ __forceinline__ void bc_load(const BcBlock& B, long long o, long long of, T* q) {
  if (B.mode == BC_F64) {
    const double* f = static_cast<const double*>(B.field);
    for (int v = 0; v < 5; ++v) q[v] = T(f[v * B.g.field + o]);
  } else if (B.mode == BC_F32) {
    const float* f = static_cast<const float*>(B.field);
    for (int v = 0; v < 5; ++v) q[v] = T(f[v * B.g.fieldf + of]);
  } else {  // the stage input S + D, formed in f32 as the stage kernel forms it
    const float* f = static_cast<const float*>(B.field);
    for (int v = 0; v < 5; ++v) q[v] = T(B.shadow[v * B.g.fieldf + of] + f[v * B.g.fieldf + of]);
  }
}
template <typename T>
__device__ __forceinline__ void bc_store(const BcBlock& B, long long o, long long of, const T* w) {
  const T gm = T(B.gamma);
  T q[5];
  q[0] = w[0];
  q[1] = w[0] * w[1];
  q[2] = w[0] * w[2];
  q[3] = w[0] * w[3];
  q[4] = w[4] / (gm - T(1)) + T(0.5) * w[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
  if (B.mode == BC_F64) {
    double* f = static_cast<double*>(B.field);
    for (int v = 0; v < 5; ++v) f[v * B.g.field + o] = double(q[v]);
  } else if (B.mode == BC_F32) {
    float* f = static_cast<float*>(B.field);
    for (int v = 0; v < 5; ++v) f[v * B.g.fieldf + of] = float(q[v]);
  } else {
    float* f = static_cast<float*>(B.field);
    for (int v = 0; v < 5; ++v) f[v * B.g.fieldf + of] = float(q[v] - T(B.shadow[v * B.g.fieldf + of]));
  }
}
template <typename T>
__device__ __forceinline__ void bc_prim(T gm, const T* q, T* w) {
  w[0] = q[0];
  w[1] = q[1] / q[0];
  w[2] = q[2] / q[0];
  w[3] = q[3] / q[0];
  w[4] = (gm - T(1)) * (q[4] - T(0.5) * q[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]));
}

// one ghost cell: layer m (0 nearest the face) beyond face `hi` of direction d, at (a, b) along the
// other two directions
template <typename T>
__device__ __forceinline__ void bc_cell(const BcBlock& B, int d, int d1, int d2, const int* n, int a, int b, int m,
                                        int hi, int kind) {
  using M = BcMath<T>;
  const Geometry& g = B.g;
  int idx[3], gi[3], ii[3];
  idx[d1] = a; idx[d2] = b; idx[d] = hi ? n[d] : 0;  // the boundary face is this cell's lower face
  for (int x = 0; x < 3; ++x) { gi[x] = idx[x]; ii[x] = idx[x]; }
  gi[d] = hi ? n[d] + m : -1 - m;
  // unit normal (towards +d) of the boundary face
  T nrm[3] = {T(0), T(0), T(0)};
  if (B.metrics) {
    T S[3];
    if (B.mode == BC_F64) {
      const double* Mt = static_cast<const double*>(B.metrics);
      const long long oc = gidx(g, idx[0], idx[1], idx[2]);
      for (int x = 0; x < 3; ++x) S[x] = T(Mt[(3 * d + x) * g.field + oc]);
    } else {
      const float* Mt = static_cast<const float*>(B.metrics);
      const long long oc = gidxf(g, idx[0], idx[1], idx[2]);
      for (int x = 0; x < 3; ++x) S[x] = T(Mt[(3 * d + x) * g.fieldf + oc]);
    }
    const T len = M::sqrt_(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
    for (int x = 0; x < 3; ++x) nrm[x] = S[x] / len;
  } else {
    nrm[d] = T(1);
  }
  T q[5], wi[5], wb[5], inf[5];
  for (int v = 0; v < 5; ++v) inf[v] = T(B.inf[v]);
  const T gm = T(B.gamma);
  if (kind == BC_SLIP_WALL) {
    ii[d] = hi ? n[d] - 1 - m : m;  // the mirror image inside
    bc_load<T>(B, gidx(g, ii[0], ii[1], ii[2]), gidxf(g, ii[0], ii[1], ii[2]), q);
    bc_prim<T>(gm, q, wi);
    const T un = wi[1] * nrm[0] + wi[2] * nrm[1] + wi[3] * nrm[2];
    wb[0] = wi[0];
    for (int x = 0; x < 3; ++x) wb[1 + x] = wi[1 + x] - T(2) * un * nrm[x];
    wb[4] = wi[4];
  } else {
    ii[d] = hi ? n[d] - 1 : 0;  // the interior cell next to the face
    bc_load<T>(B, gidx(g, ii[0], ii[1], ii[2]), gidxf(g, ii[0], ii[1], ii[2]), q);
    bc_prim<T>(gm, q, wi);
    const T out[3] = {hi ? nrm[0] : -nrm[0], hi ? nrm[1] : -nrm[1], hi ? nrm[2] : -nrm[2]};
    const T ci = M::sqrt_(gm * wi[4] / wi[0]), cinf = M::sqrt_(gm * inf[4] / inf[0]);
    const T uni = wi[1] * out[0] + wi[2] * out[1] + wi[3] * out[2];
    const T uninf = inf[1] * out[0] + inf[2] * out[1] + inf[3] * out[2];
    if (uninf <= -cinf) {
      for (int v = 0; v < 5; ++v) wb[v] = inf[v];
    } else if (uni >= ci) {
      for (int v = 0; v < 5; ++v) wb[v] = wi[v];
    } else {
      const T rp = uni + T(2) * ci / (gm - T(1)), rm = uninf - T(2) * cinf / (gm - T(1));
      const T unb = T(0.5) * (rp + rm), cb = T(0.25) * (gm - T(1)) * (rp - rm);
      T src[5];  // the upwind side's state (selected by value: no local-memory array)
      for (int v = 0; v < 5; ++v) src[v] = unb < T(0) ? inf[v] : wi[v];
      const T un_src = src[1] * out[0] + src[2] * out[1] + src[3] * out[2];
      const T ent = src[4] / M::pow_(src[0], gm);
      const T rho = M::pow_(cb * cb / (gm * ent), T(1) / (gm - T(1)));
      wb[0] = rho;
      for (int x = 0; x < 3; ++x) wb[1 + x] = src[1 + x] + (unb - un_src) * out[x];
      wb[4] = rho * cb * cb / gm;
    }
  }
  bc_store<T>(B, gidx(g, gi[0], gi[1], gi[2]), gidxf(g, gi[0], gi[1], gi[2]), wb);
}

__global__ void bc_kernel(const BcBlock B) {
  const Geometry& g = B.g;
  const int d = B.dim, d1 = (d + 1) % 3, d2 = (d + 2) % 3;
  const int n[3] = {g.nx, g.ny, g.nz};
  const long long w1 = n[d1] + 2 * HALO, w2 = n[d2] + 2 * HALO;
  const long long total = 2LL * HALO * w1 * w2;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(t % w1) - HALO;
    long long r = t / w1;
    const int b = (int)(r % w2) - HALO;
    r /= w2;
    const int m = (int)(r % HALO), hi = (int)(r / HALO);
    const int kind = B.kind[2 * d + hi];
    if (kind == BC_NONE) continue;
    if (B.mode == BC_F64) bc_cell<double>(B, d, d1, d2, n, a, b, m, hi, kind);
    else bc_cell<float>(B, d, d1, d2, n, a, b, m, hi, kind);
  }
}

cudaError_t launch_bc(const BcBlock& B, cudaStream_t s) {
  const int n[3] = {B.g.nx, B.g.ny, B.g.nz};
  const long long total = 2LL * HALO * (n[(B.dim + 1) % 3] + 2 * HALO) * (n[(B.dim + 2) % 3] + 2 * HALO);
  bc_kernel<<<grid_for(total, 128), 128, 0, s>>>(B);
  return cudaGetLastError();
}

struct CtrlList {
  DevCtrl* c[MAX_GROUP];
};
// global time step of a group: cfl / max rate over the blocks, to every block (and to `extra`,
// the group's own control block, when given)
__global__ void group_dt_kernel(CtrlList L, int n, double cfl, DevCtrl* extra) {
  if (threadIdx.x != 0) return;
  double m = 0.0;
  for (int b = 0; b < n; ++b) m = fmax(m, L.c[b]->rate);
  for (int b = 0; b < n; ++b) L.c[b]->dt = cfl / m;
  if (extra) {
    extra->rate = m;
    extra->dt = cfl / m;
  }
}
cudaError_t launch_group_dt(DevCtrl* const* ctrls, int n, double cfl, cudaStream_t s, DevCtrl* extra) {
  CtrlList L;
  for (int b = 0; b < n && b < MAX_GROUP; ++b) L.c[b] = ctrls[b];
  group_dt_kernel<<<1, 32, 0, s>>>(L, n, cfl, extra);
  return cudaGetLastError();
}

}  // namespace gbcfd
