// wcns.cu -- the paper's own spatial scheme on periodic uniform Cartesian blocks: WCNS-E-5
// (arXiv 1710.09995 Sec. 2.2, Eq. 2) with fourth-order central viscous derivatives, advanced by
// the third-order Runge-Kutta stages of Eqs. 4-6 (lambda = -dt), and its C ABI (gbcfd_wcns_*).
//
// Per Runge-Kutta stage (all launches on the caller's stream):
//   prim_kernel  the stage input Q (compact, f64) -> primitives W = (rho, u, v, w, p, theta) of
//                every cell of a box padded by 5 cells (periodic images by index wrap: the halo
//                exchange of a self-connected block); stage 1 also reduces the CFL rate of Q^n to
//                the step's time step.
//   visc_kernel  (Navier-Stokes) the viscous flux vectors Fv, Gv, Hv of Eq. 1 at every cell of
//                the box padded by 2, from fourth-order central gradients (D4) of u, v, w, theta.
//   dir_kernel<D> for D = x, y, z: a tile of 16 lines x L cells along D; the tile's primitives
//                (L + 10 cells per line) go to shared memory, every edge flux of the tile
//                (L + 5 per line) is computed once (weighted interpolation of the left and right
//                states, Roe flux) into shared memory, and each cell takes Eq. 2 of its six edge
//                fluxes minus D4 of its viscous flux along D.  x writes R, y adds to it, z adds
//                and applies the stage update (or writes R out), with the residual norm of
//                stage 1 reduced per CTA and by the last CTA in a fixed order.
// The interpolation (the paper names it only "weighted nonlinear"): three three-point stencils,
// candidates u_i + g_k/2 + s_k/8 with g_k, s_k the stencil's first and second differences,
// smoothness beta_k = g_k^2 + s_k^2, weights C_k / (1e-6 + beta_k)^2 normalised, optimal
// C = (1/16, 10/16, 5/16); `limiter` = 1 takes C itself (linear fifth order).
#include <algorithm>
#include <cstring>
#include <string>

#include "gbcfd.h"
#include "launch.h"
#include "physics.cuh"

namespace gbcfd {
namespace wcns {

constexpr int H = 5;        // halo of the primitive box: Eq. 2 reaches 5 cells
constexpr int NL = 16;      // lines per tile
constexpr int NLP = NL + 1; // padded line stride in shared memory
constexpr int LMAX = 59;    // cells per line segment: <= 64 edge fluxes, <= 69 staged cells
constexpr int NTW = 256;    // threads per CTA
constexpr int NPW = 6;      // primitive fields: rho, u, v, w, p, theta

struct Box {                // the padded box of W (halo H) and of the viscous fluxes
  int nx, ny, nz, px;       // interior sizes, row pitch (elements)
  long long field;          // elements per field
};
__host__ __device__ __forceinline__ long long bidx(const Box& b, int i, int j, int k) {
  return ((long long)(k + H) * (b.ny + 2 * H) + (j + H)) * b.px + (i + H);
}
__device__ __forceinline__ int wrap(int i, int n) {
  const int r = i % n;
  return r < 0 ? r + n : r;
}

struct Args {
  Box b;
  long long n;              // interior cells
  double gamma, mu, Pr, cfl, eps;
  double ih[3];             // inverse cell sizes
  int viscous, linear;
  void* W;                  // NPW padded fields (T)
  void* Fv;                 // 12 padded fields (T): [d][mx, my, mz, energy]
  void* R;                  // compact [5][n] (T): the residual accumulated over the passes
  const double* qn;         // Q^n (compact f64)
  const double* qs;         // the stage input
  double* qout;             // the stage output (may be qn at stage 3)
  double* rout;             // residual mode: compact f64 R
  DevCtrl* ctrl;
  double* partial;          // per-CTA partials, NPART doubles each
  int stage;                // 1..3; 0 = residual mode (z pass writes rout)
  int Lseg[3];              // cells per line segment along x, y, z
};

// ---- primitives of the padded box (and the time step of Q^n) -------------------------------
template <typename T>
__global__ void __launch_bounds__(NTW) prim_kernel(Args a, int with_rate) {
  __shared__ double wmax[NTW / 32];
  __shared__ int last;
  const Box& b = a.b;
  const int wx = b.nx + 2 * H, wy = b.ny + 2 * H, wz = b.nz + 2 * H;
  const long long total = (long long)wx * wy * wz;
  T* W = static_cast<T*>(a.W);
  const double gm1 = a.gamma - 1.0;
  const double vf = 4.0 * fmax(4.0 / 3.0, a.gamma / a.Pr) * a.mu;
  double best = 0.0;
  bool bad = false;
  for (long long t = (long long)blockIdx.x * NTW + threadIdx.x; t < total; t += (long long)gridDim.x * NTW) {
    const int ii = (int)(t % wx);
    const long long r = t / wx;
    const int jj = (int)(r % wy), kk = (int)(r / wy);
    const int i = ii - H, j = jj - H, k = kk - H;
    const int si = wrap(i, b.nx), sj = wrap(j, b.ny), sk = wrap(k, b.nz);
    const long long c = ((long long)sk * b.ny + sj) * b.nx + si;
    const double rho = a.qs[c], ir = 1.0 / rho;
    const double u = a.qs[a.n + c] * ir, v = a.qs[2 * a.n + c] * ir, w = a.qs[3 * a.n + c] * ir;
    const double p = gm1 * (a.qs[4 * a.n + c] - 0.5 * rho * (u * u + v * v + w * w));
    const long long o = (long long)kk * wy * b.px + (long long)jj * b.px + ii;
    W[o] = T(rho);
    W[b.field + o] = T(u);
    W[2 * b.field + o] = T(v);
    W[3 * b.field + o] = T(w);
    W[4 * b.field + o] = T(p);
    W[5 * b.field + o] = T(p * ir);
    if (with_rate && i == si && j == sj && k == sk) {  // each interior cell once
      if (!(rho > 0.0 && p > 0.0)) bad = true;
      const double cs = sqrt(a.gamma * p * ir);
      double rate = (fabs(u) + cs) * a.ih[0] + (fabs(v) + cs) * a.ih[1] + (fabs(w) + cs) * a.ih[2];
      if (a.viscous) rate += vf * ir * (a.ih[0] * a.ih[0] + a.ih[1] * a.ih[1] + a.ih[2] * a.ih[2]);
      best = fmax(best, rate);
    }
  }
  if (!with_rate) return;
  if (bad) atomicOr(&a.ctrl->flag, FLAG_NONPHYSICAL);
  for (int off = 16; off > 0; off >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, off));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int q = 0; q < NTW / 32; ++q) m = fmax(m, wmax[q]);
    a.partial[(size_t)blockIdx.x * NPART + 5] = m;
    __threadfence();
    last = (atomicAdd(&a.ctrl->counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  double m = 0.0;
  for (unsigned q = 0; q < gridDim.x; ++q) m = fmax(m, __ldcg(a.partial + (size_t)q * NPART + 5));
  a.ctrl->rate = m;
  a.ctrl->dt = a.cfl / m;
  a.ctrl->counter = 0u;
}

// ---- viscous flux vectors at the cells of the box padded by 2 ------------------------------
template <typename T>
__device__ __forceinline__ T d4(const T* f, long long o, long long st, T ih) {
  // (f_{-2} - 8 f_{-1} + 8 f_{+1} - f_{+2}) / (12 h)
  return ((f[o - 2 * st] - f[o + 2 * st]) + T(8) * (f[o + st] - f[o - st])) * (ih * T(1.0 / 12.0));
}

template <typename T>
__global__ void __launch_bounds__(NTW) visc_kernel(Args a) {
  const Box& b = a.b;
  const int wx = b.nx + 4, wy = b.ny + 4, wz = b.nz + 4;
  const long long total = (long long)wx * wy * wz;
  const T* W = static_cast<const T*>(a.W);
  T* F = static_cast<T*>(a.Fv);
  const T mu = T(a.mu), kappa = T(a.mu * a.gamma / ((a.gamma - 1.0) * a.Pr));
  const T ih[3] = {T(a.ih[0]), T(a.ih[1]), T(a.ih[2])};
  const long long st[3] = {1, b.px, (long long)b.px * (b.ny + 2 * H)};
  for (long long t = (long long)blockIdx.x * NTW + threadIdx.x; t < total; t += (long long)gridDim.x * NTW) {
    const int i = (int)(t % wx) - 2;
    const long long r = t / wx;
    const int j = (int)(r % wy) - 2, k = (int)(r / wy) - 2;
    const long long o = bidx(b, i, j, k);
    T g[3][3], gt[3], vel[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      vel[q] = W[(1 + q) * b.field + o];
#pragma unroll
      for (int d = 0; d < 3; ++d) g[q][d] = d4(W + (1 + q) * b.field, o, st[d], ih[d]);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) gt[d] = d4(W + 5 * b.field, o, st[d], ih[d]);
    const T div = g[0][0] + g[1][1] + g[2][2];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      T tau[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) tau[q] = mu * (g[q][d] + g[d][q]);
      tau[d] = tau[d] - T(2.0 / 3.0) * mu * div;
#pragma unroll
      for (int q = 0; q < 3; ++q) F[(4 * d + q) * b.field + o] = tau[q];
      F[(4 * d + 3) * b.field + o] = vel[0] * tau[0] + vel[1] * tau[1] + vel[2] * tau[2] + kappa * gt[d];
    }
  }
}

// ---- the weighted interpolation (value at i + 1/2 from u_{i-2} .. u_{i+2}) --------------------
template <typename V>
__device__ __forceinline__ V edge(V u0, V u1, V u2, V u3, V u4, bool linear) {
  using O = VM<V>;
  const V half = O::c(0.5), eighth = O::c(0.125);
  const V g0 = half * (u0 - O::c(4) * u1 + O::c(3) * u2), s0 = u0 - O::c(2) * u1 + u2;
  const V g1 = half * (u3 - u1), s1 = u1 - O::c(2) * u2 + u3;
  const V g2 = half * (O::c(-3) * u2 + O::c(4) * u3 - u4), s2 = u2 - O::c(2) * u3 + u4;
  const V c0 = O::fma(half, g0, eighth * s0), c1 = O::fma(half, g1, eighth * s1), c2 = O::fma(half, g2, eighth * s2);
  if (linear) return u2 + (O::c(1.0 / 16.0) * c0 + O::c(10.0 / 16.0) * c1 + O::c(5.0 / 16.0) * c2);
  // alpha_k = C_k / d_k with d_k = (eps + beta_k)^2; the normalised combination takes one
  // reciprocal: sum_k C_k (prod_{m != k} d_m) c_k / sum_k C_k (prod_{m != k} d_m)
  const V e = O::c(1e-6);
  V d0 = e + O::fma(g0, g0, s0 * s0), d1 = e + O::fma(g1, g1, s1 * s1), d2 = e + O::fma(g2, g2, s2 * s2);
  d0 = d0 * d0; d1 = d1 * d1; d2 = d2 * d2;
  const V n0 = O::c(1.0 / 16.0) * (d1 * d2), n1 = O::c(10.0 / 16.0) * (d0 * d2), n2 = O::c(5.0 / 16.0) * (d0 * d1);
  const V num = O::fma(n0, c0, O::fma(n1, c1, n2 * c2));
  return u2 + num * O::rcp(n0 + n1 + n2);
}

template <int D> struct Fr;
template <> struct Fr<0> { static constexpr int N = 1, T1 = 2, T2 = 3; };
template <> struct Fr<1> { static constexpr int N = 2, T1 = 3, T2 = 1; };
template <> struct Fr<2> { static constexpr int N = 3, T1 = 1, T2 = 2; };

template <typename T>
struct Smem {
  static constexpr int WS = 5 * (LMAX + 10) * NLP;   // staged primitives [5][L+10][NLP]
  static constexpr int FS = 5 * (LMAX + 5) * NLP;    // edge fluxes [5][L+5][NLP]
  static constexpr size_t red = (sizeof(T) * (WS + FS) + 15) / 16 * 16;  // norm partials (double)
  static constexpr size_t bytes = red + sizeof(double) * (NTW / 32) * 5;
};

// MODE: 0 x pass (R =), 1 y pass (R +=), 2 z pass (stage update or residual output)
template <typename T, int D, int MODE>
__global__ void __launch_bounds__(NTW) dir_kernel(Args a) {
  using O = VM<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ws = reinterpret_cast<T*>(smem_raw);
  T* Fs = Ws + Smem<T>::WS;
  double* red = reinterpret_cast<double*>(smem_raw + Smem<T>::red);
  __shared__ int last;
  const Box& b = a.b;
  const int nd = D == 0 ? b.nx : (D == 1 ? b.ny : b.nz);   // along the lines
  const int na = D == 0 ? b.ny : b.nx;                      // across the lines (16 per tile)
  const int nb = D == 2 ? b.ny : b.nz;                      // the third direction
  const int L = a.Lseg[D];
  const int nseg = (nd + L - 1) / L, ngrp = (na + NL - 1) / NL;
  const long long tiles = (long long)nseg * ngrp * nb;
  const long long stD = D == 0 ? 1 : (D == 1 ? b.px : (long long)b.px * (b.ny + 2 * H));
  const T* W = static_cast<const T*>(a.W);
  const T* Fv = static_cast<const T*>(a.Fv);
  T* R = static_cast<T*>(a.R);
  const Consts<T> K = make_consts<T>(a.gamma, a.eps, a.mu, a.Pr, 0);
  const T ih = T(a.ih[D]);
  const bool linear = a.linear != 0;
  const double dt = (MODE == 2 && a.stage > 0) ? a.ctrl->dt : 0.0;
  double sq[5] = {0, 0, 0, 0, 0};
  constexpr int idx[5] = {0, Fr<D>::N, Fr<D>::T1, Fr<D>::T2, 4};
  for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int seg = (int)(tile % nseg);
    const long long r = tile / nseg;
    const int grp = (int)(r % ngrp), ob = (int)(r / ngrp);
    const int s0 = seg * L, Ls = min(L, nd - s0), a0 = grp * NL;
    // cell (line l, position s along D) -> (i, j, k)
    auto ijk = [&](int l, int s, int& i, int& j, int& k) {
      if (D == 0) { i = s; j = a0 + l; k = ob; }
      else if (D == 1) { i = a0 + l; j = s; k = ob; }
      else { i = a0 + l; j = ob; k = s; }
    };
    __syncthreads();  // the previous tile's readers are done with the shared arrays
    // 1. stage the primitives of cells s0 - 5 .. s0 + Ls + 4 of every line
    const int nst = Ls + 10, nfc = Ls + 5;
    for (int e = threadIdx.x; e < 5 * nst * NL; e += NTW) {
      const int v = e / (nst * NL), rr = e % (nst * NL);
      int l, s;
      if (D == 0) { l = rr / nst; s = rr % nst; } else { s = rr / NL; l = rr % NL; }
      T val;
      if (a0 + l < na) {
        int i, j, k;
        ijk(l, s0 - H + s, i, j, k);
        val = W[(long long)v * b.field + bidx(b, i, j, k)];
      } else {
        val = (v == 0 || v == 4) ? T(1) : T(0);  // lines past the block: any physical state
      }
      Ws[(v * (LMAX + 10) + s) * NLP + l] = val;
    }
    __syncthreads();
    // 2. every edge flux of the tile: face f lies between staged cells f + 2 and f + 3 (staged
    //    cell s is cell s0 - 5 + s), so cell c (staged c + 5) has faces c .. c + 5 around it
    for (int e = threadIdx.x; e < nfc * NL; e += NTW) {
      const int f = e / NL, l = e % NL;
      T Lq[5], Rq[5];
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const T* w = Ws + (idx[q] * (LMAX + 10) + f) * NLP + l;
        const T u0 = w[0], u1 = w[NLP], u2 = w[2 * NLP], u3 = w[3 * NLP], u4 = w[4 * NLP], u5 = w[5 * NLP];
        Lq[q] = edge<T>(u0, u1, u2, u3, u4, linear);
        Rq[q] = edge<T>(u5, u4, u3, u2, u1, linear);
      }
      T F[5];
      roe_frame<T>(Lq, Rq, K, F);
#pragma unroll
      for (int q = 0; q < 5; ++q) Fs[(idx[q] * (LMAX + 5) + f) * NLP + l] = F[q];
    }
    __syncthreads();
    // 3. Eq. 2 per cell, minus D4 of the viscous flux along D, then the pass's output
    for (int e = threadIdx.x; e < Ls * NL; e += NTW) {
      int l, c;
      if (D == 0) { l = e / Ls; c = e % Ls; } else { c = e / NL; l = e % NL; }
      if (a0 + l >= na) continue;
      int i, j, k;
      ijk(l, s0 + c, i, j, k);
      const long long cc = ((long long)k * b.ny + j) * b.nx + i;
      T add[5];
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const T* fq = Fs + (q * (LMAX + 5) + c) * NLP + l;
        const T f0 = fq[0], f1 = fq[NLP], f2 = fq[2 * NLP], f3 = fq[3 * NLP], f4 = fq[4 * NLP], f5 = fq[5 * NLP];
        add[q] = (O::c(75.0 / 64.0) * (f3 - f2) - O::c(25.0 / 384.0) * (f4 - f1) + O::c(3.0 / 640.0) * (f5 - f0)) * ih;
      }
      if (a.viscous) {
        const long long o = bidx(b, i, j, k);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const T* fv = Fv + (long long)(4 * D + q) * b.field;
          add[1 + q] = add[1 + q] - d4(fv, o, stD, ih);
        }
      }
      if (MODE == 0) {
#pragma unroll
        for (int q = 0; q < 5; ++q) R[q * a.n + cc] = add[q];
      } else if (MODE == 1) {
#pragma unroll
        for (int q = 0; q < 5; ++q) R[q * a.n + cc] = R[q * a.n + cc] + add[q];
      } else {
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          const double tot = double(R[q * a.n + cc]) + double(add[q]);
          if (a.stage == 0) {
            a.rout[q * a.n + cc] = tot;
            continue;
          }
          if (a.stage == 1) sq[q] += tot * tot;
          const double adv = a.qs[q * a.n + cc] - dt * tot;
          double out;
          if (a.stage == 1) out = adv;
          else if (a.stage == 2) out = 0.75 * a.qn[q * a.n + cc] + 0.25 * adv;
          else out = a.qn[q * a.n + cc] / 3.0 + 2.0 / 3.0 * adv;
          a.qout[q * a.n + cc] = out;
        }
      }
    }
  }
  if (MODE != 2 || a.stage != 1) return;
  // residual norm of R(Q^n): per-CTA sums of squares, the last CTA folds them in CTA order
#pragma unroll
  for (int q = 0; q < 5; ++q)
    for (int off = 16; off > 0; off >>= 1) sq[q] += __shfl_xor_sync(0xffffffffu, sq[q], off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int q = 0; q < 5; ++q) red[(threadIdx.x >> 5) * 5 + q] = sq[q];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < 5; ++q) {
      double s = 0.0;
      for (int w = 0; w < NTW / 32; ++w) s += red[w * 5 + q];
      a.partial[(size_t)blockIdx.x * NPART + q] = s;
    }
    __threadfence();
    last = (atomicAdd(&a.ctrl->counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  for (int q = 0; q < 5; ++q) {
    double s = 0.0;
    for (unsigned c = 0; c < gridDim.x; ++c) s += __ldcg(a.partial + (size_t)c * NPART + q);
    a.ctrl->norms[q] = sqrt(s / (double)a.n);
  }
  a.ctrl->counter = 0u;
}

template <typename T>
static cudaError_t set_smem() {
  const int bytes = (int)Smem<T>::bytes;
  cudaError_t e;
#define GB_SET(D, M)                                                                                    \
  e = cudaFuncSetAttribute(dir_kernel<T, D, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes); \
  if (e != cudaSuccess) return e;
  GB_SET(0, 0) GB_SET(1, 1) GB_SET(2, 2)
#undef GB_SET
  return cudaSuccess;
}

template <typename T>
static int dir_occupancy() {
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dir_kernel<T, 0, 0>, NTW, Smem<T>::bytes);
  return std::max(1, occ);
}

}  // namespace wcns
}  // namespace gbcfd

using namespace gbcfd;
using namespace gbcfd::wcns;

struct gbcfd_wcns_s {
  int nx, ny, nz;
  gbcfd_params p;
  double h[3];
  int device, nsm, mixed;
  Box box;
  double* q[3];      // Q^n, Q1, Q2 (compact f64)
  void* W;
  void* Fv;
  void* R;
  DevCtrl* ctrl;
  double* partial;
  int rows;          // partial rows (CTAs of the widest launch)
  int has_state;
  int dir_grid, occ;
  cudaEvent_t events[18];  // timing marks (gbcfd_wcns_set_timing), 6 per stage
  int timing;
};

namespace {

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct WLayout {
  size_t q, w, fv, r, ctrl, partial, total;
  Box box;
  int rows;
};

bool layout(int nx, int ny, int nz, const gbcfd_params* p, int nsm, WLayout* L) {
  const size_t elem = p->precision == GBCFD_MIXED ? 4 : 8;
  const long long n = (long long)nx * ny * nz;
  Box b;
  b.nx = nx; b.ny = ny; b.nz = nz;
  const int per = (int)(128 / elem);
  b.px = (nx + 2 * H + per - 1) / per * per;
  b.field = (long long)b.px * (ny + 2 * H) * (nz + 2 * H);
  L->box = b;
  L->rows = std::max(nsm * 8, 1024);
  size_t off = 0;
  L->q = off;       off += 3 * al256((size_t)n * 5 * 8);
  L->w = off;       off += al256((size_t)b.field * NPW * elem);
  L->fv = off;      off += p->viscous ? al256((size_t)b.field * 12 * elem) : 0;
  L->r = off;       off += al256((size_t)n * 5 * elem);
  L->ctrl = off;    off += al256(sizeof(DevCtrl));
  L->partial = off; off += al256((size_t)L->rows * NPART * sizeof(double));
  L->total = off;
  return true;
}

bool check_params(const gbcfd_params* p, std::string& why) {
  if (!p) { why = "params is NULL"; return false; }
  if (!(p->gamma > 1.0)) { why = "gamma must be > 1"; return false; }
  if (!(p->cfl > 0.0)) { why = "cfl must be > 0"; return false; }
  if (!(p->entropy_eps >= 0.0)) { why = "entropy_eps must be >= 0"; return false; }
  if (p->viscous && !(p->mu >= 0.0 && p->Pr > 0.0)) { why = "viscous needs mu >= 0 and Pr > 0"; return false; }
  if (p->limiter != 0 && p->limiter != 1) { why = "limiter must be 0 (nonlinear weights) or 1 (linear)"; return false; }
  if (p->precision != GBCFD_FP64 && p->precision != GBCFD_MIXED) { why = "bad precision"; return false; }
  if (p->local_dt != 0) { why = "WCNS blocks take one global time step (local_dt = 0)"; return false; }
  return true;
}

int cuda_err(cudaError_t e, const char* what) {
  return set_error(GBCFD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

Args make_args(gbcfd_wcns w) {
  Args a;
  std::memset(&a, 0, sizeof(a));
  a.b = w->box;
  a.n = (long long)w->nx * w->ny * w->nz;
  a.gamma = w->p.gamma;
  a.mu = w->p.viscous ? w->p.mu : 0.0;
  a.Pr = w->p.Pr > 0.0 ? w->p.Pr : 0.72;
  a.cfl = w->p.cfl;
  a.eps = w->p.entropy_eps;
  for (int d = 0; d < 3; ++d) a.ih[d] = 1.0 / w->h[d];
  a.viscous = w->p.viscous;
  a.linear = w->p.limiter;
  a.W = w->W;
  a.Fv = w->Fv;
  a.R = w->R;
  a.ctrl = w->ctrl;
  a.partial = w->partial;
  const int n3[3] = {w->nx, w->ny, w->nz};
  for (int d = 0; d < 3; ++d) {
    const int nseg = (n3[d] + LMAX - 1) / LMAX;
    a.Lseg[d] = (n3[d] + nseg - 1) / nseg;  // even segments of at most LMAX cells
  }
  return a;
}

template <typename T>
cudaError_t launch_pass(gbcfd_wcns w, Args a, int with_rate, const cudaEvent_t* ev, cudaStream_t s) {
  auto mark = [&](int m) {
    if (ev) cudaEventRecord(ev[m], s);
  };
  const int pgrid = std::min(w->rows, w->nsm * 8);
  mark(0);
  prim_kernel<T><<<pgrid, NTW, 0, s>>>(a, with_rate);
  mark(1);
  if (a.viscous) visc_kernel<T><<<w->nsm * 8, NTW, 0, s>>>(a);
  mark(2);
  const size_t sm = Smem<T>::bytes;
  const int g = w->dir_grid;
  dir_kernel<T, 0, 0><<<g, NTW, sm, s>>>(a);
  mark(3);
  dir_kernel<T, 1, 1><<<g, NTW, sm, s>>>(a);
  mark(4);
  dir_kernel<T, 2, 2><<<g, NTW, sm, s>>>(a);
  mark(5);
  return cudaGetLastError();
}

// one Runge-Kutta stage (1..3) or the residual (stage 0, written to rout)
int run_stage(gbcfd_wcns w, int stage, double* rout, cudaStream_t s) {
  Args a = make_args(w);
  a.stage = stage;
  a.rout = rout;
  a.qn = w->q[0];
  if (stage == 0) a.qs = w->q[0];
  else a.qs = w->q[stage - 1];
  a.qout = stage == 3 ? w->q[0] : (stage >= 1 ? w->q[stage] : nullptr);
  const cudaEvent_t* ev = (w->timing && stage >= 1) ? w->events + 6 * (stage - 1) : nullptr;
  const cudaError_t e = w->mixed ? launch_pass<float>(w, a, stage == 1, ev, s) : launch_pass<double>(w, a, stage == 1, ev, s);
  if (e != cudaSuccess) return cuda_err(e, "WCNS stage launch");
  return GBCFD_OK;
}

}  // namespace

extern "C" int gbcfd_wcns_required_bytes(int nx, int ny, int nz, const gbcfd_params* params, size_t* bytes) {
  std::string why;
  if (!bytes) return set_error(GBCFD_ERR_ARG, "bytes is NULL");
  if (nx < 1 || ny < 1 || nz < 1) return set_error(GBCFD_ERR_ARG, "block sizes must be >= 1");
  if (!check_params(params, why)) return set_error(GBCFD_ERR_ARG, why);
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return set_error(GBCFD_ERR_CUDA, "no CUDA device");
  WLayout L;
  layout(nx, ny, nz, params, nsm, &L);
  *bytes = L.total;
  return GBCFD_OK;
}

extern "C" int gbcfd_wcns_create(int nx, int ny, int nz, const gbcfd_params* params, const double spacing[3],
                                 void* dev_mem, size_t bytes, gbcfd_wcns* out) {
  std::string why;
  if (!out || !dev_mem || !spacing) return set_error(GBCFD_ERR_ARG, "NULL argument");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1) return set_error(GBCFD_ERR_ARG, "block sizes must be >= 1");
  if (!check_params(params, why)) return set_error(GBCFD_ERR_ARG, why);
  if (!(spacing[0] > 0 && spacing[1] > 0 && spacing[2] > 0))
    return set_error(GBCFD_ERR_ARG, "spacing must be three positive cell sizes");
  if (reinterpret_cast<uintptr_t>(dev_mem) % 256 != 0) return set_error(GBCFD_ERR_MEMORY, "dev_mem must be 256-byte aligned");
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_err(e, "cudaGetDevice");
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_err(e, "cudaDeviceGetAttribute");
  WLayout L;
  layout(nx, ny, nz, params, nsm, &L);
  if (bytes < L.total)
    return set_error(GBCFD_ERR_MEMORY, "caller memory too small: need " + std::to_string(L.total) + " bytes");
  const bool mixed = params->precision == GBCFD_MIXED;
  e = mixed ? set_smem<float>() : set_smem<double>();
  if (e != cudaSuccess) return cuda_err(e, "cudaFuncSetAttribute");
  gbcfd_wcns w = new gbcfd_wcns_s();
  w->nx = nx; w->ny = ny; w->nz = nz;
  w->p = *params;
  for (int d = 0; d < 3; ++d) w->h[d] = spacing[d];
  w->device = dev;
  w->nsm = nsm;
  w->mixed = mixed;
  w->box = L.box;
  char* base = static_cast<char*>(dev_mem);
  const size_t qbytes = al256((size_t)nx * ny * nz * 5 * 8);
  for (int s = 0; s < 3; ++s) w->q[s] = reinterpret_cast<double*>(base + L.q + s * qbytes);
  w->W = base + L.w;
  w->Fv = params->viscous ? base + L.fv : nullptr;
  w->R = base + L.r;
  w->ctrl = reinterpret_cast<DevCtrl*>(base + L.ctrl);
  w->partial = reinterpret_cast<double*>(base + L.partial);
  w->rows = L.rows;
  w->occ = mixed ? dir_occupancy<float>() : dir_occupancy<double>();
  w->dir_grid = std::min(w->rows, nsm * w->occ);
  e = cudaMemset(w->ctrl, 0, sizeof(DevCtrl));
  if (e != cudaSuccess) {
    delete w;
    return cuda_err(e, "cudaMemset");
  }
  *out = w;
  return GBCFD_OK;
}

extern "C" int gbcfd_wcns_destroy(gbcfd_wcns w) {
  if (!w) return set_error(GBCFD_ERR_ARG, "NULL block");
  cudaDeviceSynchronize();
  delete w;
  return GBCFD_OK;
}

extern "C" int gbcfd_wcns_set_state(gbcfd_wcns w, const double* q, void* stream) {
  if (!w || !q) return set_error(GBCFD_ERR_ARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t n = (size_t)w->nx * w->ny * w->nz;
  cudaError_t e = cudaMemcpyAsync(w->q[0], q, n * 5 * sizeof(double), cudaMemcpyDefault, s);
  if (e != cudaSuccess) return cuda_err(e, "cudaMemcpyAsync");
  e = cudaMemsetAsync(w->ctrl, 0, sizeof(DevCtrl), s);
  if (e != cudaSuccess) return cuda_err(e, "cudaMemsetAsync");
  w->has_state = 1;
  return GBCFD_OK;
}

extern "C" int gbcfd_wcns_get_state(gbcfd_wcns w, double* q, void* stream) {
  if (!w || !q) return set_error(GBCFD_ERR_ARG, "NULL argument");
  if (!w->has_state) return set_error(GBCFD_ERR_STATE, "no state set");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t n = (size_t)w->nx * w->ny * w->nz;
  cudaError_t e = cudaMemcpyAsync(q, w->q[0], n * 5 * sizeof(double), cudaMemcpyDefault, s);
  if (e != cudaSuccess) return cuda_err(e, "cudaMemcpyAsync");
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, q) == cudaSuccess && at.type != cudaMemoryTypeDevice &&
      at.type != cudaMemoryTypeManaged) {
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_err(e, "cudaStreamSynchronize");
  }
  return GBCFD_OK;
}

extern "C" int gbcfd_wcns_compute_residual(gbcfd_wcns w, double* r, void* stream) {
  if (!w || !r) return set_error(GBCFD_ERR_ARG, "NULL argument");
  if (!w->has_state) return set_error(GBCFD_ERR_STATE, "no state set");
  return run_stage(w, 0, r, static_cast<cudaStream_t>(stream));
}

extern "C" int gbcfd_wcns_step(gbcfd_wcns w, int nsteps, void* stream) {
  if (!w) return set_error(GBCFD_ERR_ARG, "NULL block");
  if (nsteps < 0) return set_error(GBCFD_ERR_ARG, "nsteps must be >= 0");
  if (!w->has_state) return set_error(GBCFD_ERR_STATE, "no state set");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int n = 0; n < nsteps; ++n)
    for (int st = 1; st <= 3; ++st) {
      const int rc = run_stage(w, st, nullptr, s);
      if (rc != GBCFD_OK) return rc;
    }
  return GBCFD_OK;
}

static int read_ctrl(gbcfd_wcns w, DevCtrl* h, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(h, w->ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_err(e, "reading the control block");
  return GBCFD_OK;
}

extern "C" int gbcfd_wcns_residual_norm(gbcfd_wcns w, double out[5], void* stream) {
  if (!w || !out) return set_error(GBCFD_ERR_ARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DevCtrl h;
  int rc = read_ctrl(w, &h, s);
  if (rc != GBCFD_OK) return rc;
  for (int q = 0; q < 5; ++q) out[q] = h.norms[q];
  if (h.flag) {
    const int zero = 0;
    cudaMemcpyAsync(&w->ctrl->flag, &zero, sizeof(int), cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
    if (h.flag & FLAG_NONPHYSICAL) return set_error(GBCFD_ERR_NONPHYSICAL, "rho <= 0 or p <= 0 met in a WCNS block");
  }
  return GBCFD_OK;
}

extern "C" int gbcfd_wcns_get_dt(gbcfd_wcns w, double* dt, void* stream) {
  if (!w || !dt) return set_error(GBCFD_ERR_ARG, "NULL argument");
  DevCtrl h;
  const int rc = read_ctrl(w, &h, static_cast<cudaStream_t>(stream));
  if (rc != GBCFD_OK) return rc;
  *dt = h.dt;
  return GBCFD_OK;
}

extern "C" int gbcfd_wcns_set_timing(gbcfd_wcns w, void* const* events, int n) {
  if (!w) return set_error(GBCFD_ERR_ARG, "NULL block");
  if (!events) {
    w->timing = 0;
    return GBCFD_OK;
  }
  if (n != 18) return set_error(GBCFD_ERR_ARG, "gbcfd_wcns_set_timing takes 18 events");
  for (int m = 0; m < 18; ++m) {
    if (!events[m]) return set_error(GBCFD_ERR_ARG, "NULL event");
    w->events[m] = static_cast<cudaEvent_t>(events[m]);
  }
  w->timing = 1;
  return GBCFD_OK;
}
