// wcns.cu -- the paper's own spatial scheme on uniform Cartesian blocks, periodic alone or
// connected into a periodic multi-block lattice: WCNS-E-5 (arXiv 1710.09995 Sec. 2.2, Eq. 2) with
// fourth-order central viscous derivatives, advanced by the third-order Runge-Kutta stages of
// Eqs. 4-6 (lambda = -dt), and its C ABI (gbcfd_wcns_*).
//
// Per Runge-Kutta stage (all launches on the caller's stream; blocks advanced together run on
// side streams forked from and joined into it):
//   prim_kernel  the stage input -> primitives W = (rho, u, v, w, p, theta) of every cell of a box
//                padded by 5 cells (periodic images by index wrap: the halo exchange of a
//                self-connected block); stage 1 also reduces the CFL rate of Q^n to the step's
//                time step.  prim_multi_kernel, for blocks advanced together, reads each halo
//                cell from the block that owns it (the members' table walked face to face) and
//                wcns_group_dt_kernel then gives every member the common time step.
//   viscres_kernel  (Navier-Stokes) the viscous residual Rv = -(D4_x Fv + D4_y Gv + D4_z Hv) at the
//                interior cells in one pass: tiles marching in z form the gradient tensor (D4 of
//                u, v, w, theta) once per cell of the tile's union box from a TMA-fed ring of
//                planes, keep the three viscous-flux families of Eq. 1 in shared rings and write
//                only Rv.
//   dir_kernel<D> for D = x, y, z: a tile of 16 lines x L cells along D.  The tile's primitives
//                (L + 10 cells per line) land in shared memory by cp.async one tile ahead; a lane
//                per cell evaluates both edge values of its cell (the two share the stencils'
//                smoothness indicators; on the mixed path two variables per packed f32x2
//                instruction), a shuffle pairs the left state of cell i with the right state of
//                cell i + 1, and the Roe flux of every edge of the tile (L + 5 per line) is
//                computed once; the fluxes replace the primitives in shared memory and each cell
//                takes Eq. 2 of its six edge fluxes (the x pass also adds Rv).  x writes R, y adds
//                to it, z adds and applies the stage update (or writes R out), with the residual
//                norm of stage 1 reduced per CTA and folded by a warp of the last CTA in a fixed
//                order.
// Precision: FP64 everywhere, or mixed: the stage inputs are the f32 shadow S^n of Q^n plus an
// f32 increment, D1 = -dt R(S^n), D2 = (D1 - dt R(S^n + D1)) / 4, and only the last stage touches
// FP64: Q^{n+1} = Q^n + 2/3 (D2 - dt R(S^n + D2)), S^{n+1} = f32(Q^{n+1}) (algebraically Eqs. 4-6);
// primitives, interpolation, fluxes and derivatives are f32.
// The interpolation (the paper names it only "weighted nonlinear"): three three-point stencils,
// candidates u_i + g_k/2 + s_k/8 with g_k, s_k the stencil's first and second differences,
// smoothness beta_k = g_k^2 + s_k^2, weights C_k / (1e-6 + beta_k)^2 normalised, optimal
// C = (1/16, 10/16, 5/16); `limiter` = 1 takes C itself (linear fifth order).
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "gbcfd.h"
#include "launch.h"
#include "stage.cuh"  // mbarrier / TMA helpers (and the shared physics)

namespace gbcfd {
namespace wcns {

constexpr int H = 5;        // halo of the primitive box: Eq. 2 reaches 5 cells
constexpr int NL = 16;      // lines per tile
constexpr int NLP = NL + 1; // padded line stride in shared memory
constexpr int FCH = 31;     // edges per warp chunk (lane 31 only lends its cell's right state)
constexpr int LMAX = 57;    // cells per line segment: <= 62 edges (two chunks), <= 67 staged cells
constexpr int NTW = 256;    // threads per CTA
constexpr int NPW = 6;      // primitive fields: rho, u, v, w, p, theta
constexpr int ITEMS = 2 * NL / (NTW / 32);  // (line, chunk) items per warp and tile

struct Box {                // the padded box of the primitives W (halo H)
  int nx, ny, nz, px;       // interior sizes, row pitch (elements)
  long long field;          // elements per field
};
__host__ __device__ __forceinline__ long long bidx(const Box& b, int i, int j, int k) {
  return ((long long)(k + H) * (b.ny + 2 * H) + (j + H)) * b.px + (i + H);
}
// periodic image of index i in [0, n): i lies within a few block lengths of the block
__device__ __forceinline__ int wrap(int i, int n) {
  while (i < 0) i += n;
  while (i >= n) i -= n;
  return i;
}

// the physical and grid coefficients every kernel needs, computed once on the host in the path's
// precision (no FP64 arithmetic in an FP32 kernel: it is slow on this part)
template <typename T>
struct Coef {
  T gm1, gam, half, vf;      // gamma - 1, gamma, 1/2, 4 max(4/3, gamma/Pr) mu (viscous rate)
  T mu, kappa;               // viscosity, heat conductivity mu gamma / ((gamma - 1) Pr)
  T ih[3], ih12[3], ihs;     // inverse cell sizes, the same / 12, sum of their squares
  Consts<T> K;               // the Roe / viscous flux constants
};

struct Args {
  Coef<float> cf;
  Coef<double> cd;
  CUtensorMap mwv;          // W: 6 padded fields, box 44 x 16 x 1 x 1 (one field's plane box)
  Box b;
  long long n;              // interior cells
  double gamma, mu, Pr, cfl, eps;
  double ih[3];             // inverse cell sizes
  int viscous, linear;
  void* W;                  // NPW padded fields (T)
  void* R;                  // compact [5][n] (T): the residual accumulated over the passes
  void* Rv;                 // compact [4][n] (T): the viscous part, -sum_d D4_d(F_v,d) (momentum, energy)
  // FP64 path
  const double* qn;         // Q^n (compact f64)
  const double* qs;         // the stage input
  double* qout;             // the stage output (qn at stage 3)
  // mixed path
  double* q;                // Q^n (f64), updated in place at stage 3
  float* sh;                // S^n = f32(Q^n), rewritten at stage 3
  const float* din;         // the stage input's increment over S^n (NULL at stage 1)
  float* d1;                // D1
  float* d2;                // D2
  double* rout;             // residual mode: compact f64 R
  DevCtrl* ctrl;
  double* partial;          // per-CTA partials, NPART doubles each
  int stage;                // 1..3; 0 = residual mode (z pass writes rout)
  int Lseg[3];              // cells per line segment along x, y, z
};

template <typename T> __device__ __forceinline__ const Coef<T>& coef(const Args& a);
template <> __device__ __forceinline__ const Coef<float>& coef<float>(const Args& a) { return a.cf; }
template <> __device__ __forceinline__ const Coef<double>& coef<double>(const Args& a) { return a.cd; }

// ---- primitives of the padded box (and the time step of Q^n) -------------------------------
template <typename T>
__device__ __forceinline__ void load_conserved(const Args& a, long long c, T* U);
template <>
__device__ __forceinline__ void load_conserved<double>(const Args& a, long long c, double* U) {
#pragma unroll
  for (int m = 0; m < 5; ++m) U[m] = a.qs[m * a.n + c];
}
template <>
__device__ __forceinline__ void load_conserved<float>(const Args& a, long long c, float* U) {
#pragma unroll
  for (int m = 0; m < 5; ++m) U[m] = a.din ? a.sh[m * a.n + c] + a.din[m * a.n + c] : a.sh[m * a.n + c];
}

// blocks advanced together (gbcfd_wcns_step_many): each member's stage-input arrays, sizes and
// face neighbours (indices into the table; the faces of a conforming periodic lattice, Sec. 2.2's
// multi-block interfaces), so that a member's halo cells are read from the block that owns them
constexpr int MAXW = 32;
struct WSrc {
  const double* q[3];       // FP64: Q^n, Q1, Q2.  mixed: q[0] = Q^n
  const float* sh;          // mixed: S^n
  const float* d[2];        // mixed: D1, D2
  DevCtrl* ctrl;
  int nx, ny, nz, pad;
  int nbr[6];               // -x, +x, -y, +y, -z, +z
};
struct WTab {
  WSrc e[MAXW];
  int n, self;              // members; the launching block's own index
};
static_assert(sizeof(Args) + sizeof(int) + sizeof(WTab) <= 4096, "prim_multi_kernel's parameters exceed 4 KB");

// the conserved state of cell c of member s of the table at a stage (as load_conserved)
template <typename T>
__device__ __forceinline__ void load_member(const WSrc& s, int stage, long long c, T* U);
template <>
__device__ __forceinline__ void load_member<double>(const WSrc& s, int stage, long long c, double* U) {
  const long long n = (long long)s.nx * s.ny * s.nz;
  const double* q = stage <= 1 ? s.q[0] : s.q[stage - 1];
#pragma unroll
  for (int m = 0; m < 5; ++m) U[m] = q[m * n + c];
}
template <>
__device__ __forceinline__ void load_member<float>(const WSrc& s, int stage, long long c, float* U) {
  const long long n = (long long)s.nx * s.ny * s.nz;
  const float* din = stage == 2 ? s.d[0] : (stage == 3 ? s.d[1] : nullptr);
#pragma unroll
  for (int m = 0; m < 5; ++m) U[m] = din ? s.sh[m * n + c] + din[m * n + c] : s.sh[m * n + c];
}

// primitives of the padded box (and, with_rate, the CFL rate of Q^n over the interior).  The
// source of padded cell (i, j, k): one block wraps its own indices (periodic); a member of a
// table walks face neighbours along z, then y, then x, so edge and corner halos come from the
// diagonal block (in a conforming lattice every order of the walk reaches the same block), and
// a neighbour thinner than the halo is crossed to the next one.
template <typename T, bool MULTI>
__device__ __forceinline__ void prim_body(const Args& a, int with_rate, const WTab* tab) {
  __shared__ double wmax[NTW / 32];
  __shared__ int last;
  const Box& b = a.b;
  const int wx = b.nx + 2 * H, wy = b.ny + 2 * H, wz = b.nz + 2 * H;
  T* W = static_cast<T*>(a.W);
  using O = VM<T>;
  const Coef<T>& C = coef<T>(a);
  const T gm1 = C.gm1, gam = C.gam, half = C.half, vf = C.vf;
  const T ih0 = C.ih[0], ih1 = C.ih[1], ih2 = C.ih[2], ihs = C.ihs;
  T best = T(0);
  bool bad = false;
  for (int row = blockIdx.x; row < wy * wz; row += gridDim.x) {  // rows (j, k) of the padded box
    const int jj = row % wy, kk = row / wy;
    const int j = jj - H, k = kk - H;
    int sj, sk, rb = 0;
    if constexpr (MULTI) {  // the row's block: walk z, then y
      rb = tab->self;
      sk = k;
      while (sk < 0) { rb = tab->e[rb].nbr[4]; sk += tab->e[rb].nz; }
      while (sk >= tab->e[rb].nz) { sk -= tab->e[rb].nz; rb = tab->e[rb].nbr[5]; }
      sj = j;
      while (sj < 0) { rb = tab->e[rb].nbr[2]; sj += tab->e[rb].ny; }
      while (sj >= tab->e[rb].ny) { sj -= tab->e[rb].ny; rb = tab->e[rb].nbr[3]; }
    } else {
      sj = wrap(j, b.ny);
      sk = wrap(k, b.nz);
    }
    T* dst = W + ((long long)kk * wy + jj) * b.px;
    const bool inner_row = j == sj && k == sk && (!MULTI || rb == tab->self);
    for (int ii = threadIdx.x; ii < wx; ii += NTW) {
      const int i = ii - H;
      T U[5];
      int si;
      if constexpr (MULTI) {
        int cb = rb;
        si = i;
        while (si < 0) { cb = tab->e[cb].nbr[0]; si += tab->e[cb].nx; }
        while (si >= tab->e[cb].nx) { si -= tab->e[cb].nx; cb = tab->e[cb].nbr[1]; }
        const WSrc& e = tab->e[cb];
        load_member<T>(e, a.stage, ((long long)sk * e.ny + sj) * e.nx + si, U);
      } else {
        si = wrap(i, b.nx);
        load_conserved<T>(a, ((long long)sk * b.ny + sj) * b.nx + si, U);
      }
      const T rho = U[0], ir = T(1) / rho;
      const T u = U[1] * ir, v = U[2] * ir, w = U[3] * ir;
      const T p = gm1 * (U[4] - half * rho * (u * u + v * v + w * w));
      dst[ii] = rho;
      dst[b.field + ii] = u;
      dst[2 * b.field + ii] = v;
      dst[3 * b.field + ii] = w;
      dst[4 * b.field + ii] = p;
      dst[5 * b.field + ii] = p * ir;
      if (with_rate && inner_row && i == si) {  // each interior cell once
        if (!(rho > T(0) && p > T(0))) bad = true;
        const T c2 = gam * p * ir;
        const T cs = c2 * O::rsqrt(c2);
        T rate = (O::ab(u) + cs) * ih0 + (O::ab(v) + cs) * ih1 + (O::ab(w) + cs) * ih2;
        if (a.viscous) rate += vf * ir * ihs;
        best = best > rate ? best : rate;
      }
    }
  }
  if (!with_rate) return;
  if (bad) atomicOr(&a.ctrl->flag, FLAG_NONPHYSICAL);
  for (int off = 16; off > 0; off >>= 1) {
    const T o = __shfl_xor_sync(0xffffffffu, best, off);
    best = best > o ? best : o;
  }
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = double(best);
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int q = 0; q < NTW / 32; ++q) m = fmax(m, wmax[q]);
    a.partial[(size_t)blockIdx.x * NPART + 5] = m;
    __threadfence();
    last = (atomicAdd(&a.ctrl->counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last || threadIdx.x >= 32) return;
  __threadfence();
  // the last CTA's first warp folds the per-CTA maxima: lane-strided, then a fixed shuffle tree
  double m = 0.0;
  for (unsigned q = threadIdx.x; q < gridDim.x; q += 32) m = fmax(m, __ldcg(a.partial + (size_t)q * NPART + 5));
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
  if (threadIdx.x == 0) {
    a.ctrl->rate = m;
    a.ctrl->dt = a.cfl / m;
    a.ctrl->counter = 0u;
  }
}

template <typename T>
__global__ void __launch_bounds__(NTW) prim_kernel(Args a, int with_rate) {
  prim_body<T, false>(a, with_rate, nullptr);
}
template <typename T>
__global__ void __launch_bounds__(NTW) prim_multi_kernel(Args a, int with_rate, const __grid_constant__ WTab tab) {
  prim_body<T, true>(a, with_rate, &tab);
}

// the common time step of blocks advanced together: cfl / the largest of their rates, written
// to every member (after each member's stage-1 primitive pass has reduced its own rate)
__global__ void wcns_group_dt_kernel(const __grid_constant__ WTab tab, double cfl) {
  if (threadIdx.x != 0) return;
  double m = 0.0;
  for (int b = 0; b < tab.n; ++b) m = fmax(m, tab.e[b].ctrl->rate);
  for (int b = 0; b < tab.n; ++b) {
    tab.e[b].ctrl->rate = m;
    tab.e[b].ctrl->dt = cfl / m;
  }
}

// S = f32(Q) of a compact state (mixed path, after the state is set)
__global__ void shadow_kernel(const double* __restrict__ q, float* __restrict__ sh, long long n) {
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
    sh[c] = f64_to_f32_bits(q[c]);
}

// ---- asynchronous global -> shared copies of single elements (cp.async, completed by group) ----
template <typename T>
__device__ __forceinline__ void cp_async(T* smem, const T* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// ---- the viscous residual Rv = -(D4_x Fv + D4_y Gv + D4_z Hv), in one pass ----------------------
// Tiles of 32 x 8 interior cells march in z over each CTA's contiguous share of tile-planes, with a
// lead plane p two planes ahead of the output plane k = p - 2.  Per lead plane the gradient
// tensor (D4 of u, v, w, theta along x, y, z) is formed once at every cell of the tile's union
// box (x0 - 2 .. x0 + 33, y0 - 2 .. y0 + 9), from a ring of u, v, w, theta planes p - 2 .. p + 2
// (each a TMA box of 44 x 16 cells starting at a 16-byte aligned column; plane p + 3 lands
// meanwhile); from it the x-fluxes of the tile's rows (+2 columns each side) and the y-fluxes of
// its columns (+2 rows each side) give the x- and y-parts of Rv at once (kept by each cell's
// thread for two planes), and the z-fluxes of the tile go to a 5-plane ring for the z-part.
// Only the 4-field residual reaches global memory.
constexpr int RX = 32, RY = 8;                 // tile
constexpr int GX = RX + 4, GY = RY + 4;        // union box of gradient cells (36 x 12)
constexpr int WX = 44, WY = RY + 8;            // primitive box (44 x 16): cells x0-5 .., y0-4 ..
constexpr int WRING = 6, ZRING = 5;            // 5 planes in use + 1 landing; z-fluxes k-2 .. k+2
template <typename T>
struct RSmem {
  static constexpr int WF = WY * WX;                 // one field's plane box
  static constexpr int WP = 4 * WF;                  // u, v, w, theta
  static constexpr int FXP = 4 * RY * GX;            // x-fluxes of the lead plane: 4 x 8 rows x 36
  static constexpr int GYP = 4 * GY * RX;            // y-fluxes: 4 x 12 rows x 32
  static constexpr int HZP = 4 * RY * RX;            // z-fluxes: 4 x 8 x 32
  static constexpr size_t w = 0;
  static constexpr size_t fx = w + sizeof(T) * WRING * WP;
  static constexpr size_t gy = fx + sizeof(T) * FXP;
  static constexpr size_t hz = gy + sizeof(T) * GYP;
  static constexpr size_t bar = (hz + sizeof(T) * ZRING * HZP + 15) / 16 * 16;
  static constexpr size_t bytes = bar + 8 * WRING + 16;
};

// drain the copies of a CTA that stops early (bounded), flag the timeout
__device__ __forceinline__ void tma_abort(uint64_t* bar, unsigned pending, unsigned parity, int nslot, DevCtrl* ctrl) {
  for (int q = 0; q < nslot; ++q)
    if (pending & (1u << q)) mbar_wait_bounded(&bar[q], (parity >> q) & 1u);
  atomicOr(&ctrl->flag, FLAG_TIMEOUT);
}

template <typename T>
__global__ void __launch_bounds__(NTW) viscres_kernel(const __grid_constant__ Args a) {
  extern __shared__ __align__(128) unsigned char rsm[];
  T* wr = reinterpret_cast<T*>(rsm + RSmem<T>::w);
  T* fxr = reinterpret_cast<T*>(rsm + RSmem<T>::fx);
  T* gyr = reinterpret_cast<T*>(rsm + RSmem<T>::gy);
  T* hzr = reinterpret_cast<T*>(rsm + RSmem<T>::hz);
  uint64_t* bar = reinterpret_cast<uint64_t*>(rsm + RSmem<T>::bar);
  int* sabort = reinterpret_cast<int*>(bar + WRING);
  const Box& b = a.b;
  T* Rv = static_cast<T*>(a.Rv);
  const Coef<T>& C = coef<T>(a);
  const T mu = C.mu, kappa = C.kappa, twothird = T(2.0 / 3.0);
  const T ih0 = C.ih12[0], ih1 = C.ih12[1], ih2 = C.ih12[2];
  const int ntx = (b.nx + RX - 1) / RX, nty = (b.ny + RY - 1) / RY;
  const long long units = (long long)ntx * nty * b.nz;
  const long long u0 = (long long)blockIdx.x * units / gridDim.x, u1 = (long long)(blockIdx.x + 1) * units / gridDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int q = 0; q < WRING; ++q) mbar_init(&bar[q], 1);
    fence_barrier_init();
    *sabort = 0;
  }
  __syncthreads();
  unsigned parity = 0, pending = 0;  // per W slot (parity uniform; pending in thread 0)
  auto ws = [](int kp) { return (kp + 4 * WRING) % WRING; };
  auto zs = [](int kp) { return (kp + 4 * ZRING) % ZRING; };
  T* fxp = fxr;
  T* gyp = gyr;
  for (long long u = u0; u < u1 && !*sabort;) {
    const long long tile = u / b.nz;
    const int k0 = (int)(u - tile * b.nz);
    const int k1 = (int)min((long long)b.nz, k0 + (u1 - u));
    u += k1 - k0;
    const int tx = (int)(tile % ntx), x0 = tx * RX, y0 = (int)(tile / ntx) * RY;
    auto issue = [&](int kp) {  // thread 0: u, v, w, theta of plane kp (fields 1, 2, 3, 5)
      const int q = ws(kp);
      T* dst = wr + q * RSmem<T>::WP;
      fence_proxy_async();
      mbar_expect_tx(&bar[q], (unsigned)(sizeof(T) * RSmem<T>::WP));
      const int fld[4] = {1, 2, 3, 5};
      for (int f = 0; f < 4; ++f)  // storage column x0 is cell x0 - 5; storage row y0 + 1 is cell y0 - 4
        tma_load_4d(dst + f * RSmem<T>::WF, &a.mwv, &bar[q], x0, y0 + 1, kp + H, fld[f]);
      pending |= 1u << q;
    };
    auto wait = [&](int kp) {  // all threads; a copy that never landed stays pending
      const int q = ws(kp);
      const bool ok = mbar_wait_bounded(&bar[q], (parity >> q) & 1u);
      if (!ok) atomicOr(sabort, 1);
      if (ok) parity ^= 1u << q;
      if (threadIdx.x == 0 && ok) pending &= ~(1u << q);
    };
    // each thread owns tile cell (lane, warp): its x- and y-parts of Rv for planes p-2, p-1, p stay
    // in registers until the z-part of plane p-2 is known
    T rv2[4] = {0, 0, 0, 0}, rv1[4] = {0, 0, 0, 0};
    __syncthreads();  // the previous segment is done with the rings
    if (threadIdx.x == 0)
      for (int kp = k0 - 4; kp <= k0; ++kp) issue(kp);
    for (int kp = k0 - 4; kp <= k0 - 1; ++kp) wait(kp);
    for (int p = k0 - 2; p <= k1 + 1; ++p) {  // lead plane p, output plane p - 2
      if (threadIdx.x == 0 && p <= k1 && !*sabort) issue(p + 3);  // into the slot of plane p - 3
      wait(p + 2);
      __syncthreads();
      if (*sabort) break;
      const T* pl[5];
#pragma unroll
      for (int m = 0; m < 5; ++m) pl[m] = wr + ws(p - 2 + m) * RSmem<T>::WP;
      T* hzp = hzr + zs(p) * RSmem<T>::HZP;
      // the union box: a warp per 32-cell row (rows 0..7, then 8..11), and warps 4, 5 of the second
      // pass take the 4 extra columns of all 12 rows (a row stride of 44 spreads them over distinct
      // banks); walking the 36-wide box row-major would split warps over two rows and conflict
      for (int pass = 0; pass < 2; ++pass) {
        int gx, gy;
        if (pass == 0) {
          gy = warp;
          gx = lane;
        } else if (warp < GY - RY) {
          gy = RY + warp;
          gx = lane;
        } else {
          const int sidx = (warp - (GY - RY)) * 32 + lane;  // 0 .. 63; 48 side cells
          if (sidx >= GY * (GX - RX)) continue;
          gy = sidx / (GX - RX);
          gx = RX + sidx % (GX - RX);
        }
        const int c = (gy + 2) * WX + gx + 3;  // the cell in the primitive box
        T gr[4][3], vel[3];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const T* p0 = pl[2] + f * RSmem<T>::WF;
          if (f < 3) vel[f] = p0[c];
          gr[f][0] = ((p0[c - 2] - p0[c + 2]) + T(8) * (p0[c + 1] - p0[c - 1])) * ih0;
          gr[f][1] = ((p0[c - 2 * WX] - p0[c + 2 * WX]) + T(8) * (p0[c + WX] - p0[c - WX])) * ih1;
          const int o = f * RSmem<T>::WF + c;
          gr[f][2] = ((pl[0][o] - pl[4][o]) + T(8) * (pl[3][o] - pl[1][o])) * ih2;
        }
        const T div = gr[0][0] + gr[1][1] + gr[2][2];
        const bool rows = gy >= 2 && gy < RY + 2, cols = gx >= 2 && gx < RX + 2;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          if ((d == 0 && !rows) || (d == 1 && !cols) || (d == 2 && !(rows && cols))) continue;
          T tau[3];
#pragma unroll
          for (int q = 0; q < 3; ++q) tau[q] = mu * (gr[q][d] + gr[d][q]);
          tau[d] = tau[d] - twothird * mu * div;
          const T e = vel[0] * tau[0] + vel[1] * tau[1] + vel[2] * tau[2] + kappa * gr[3][d];
          T* dst;
          int stride;
          if (d == 0) { dst = fxp + (gy - 2) * GX + gx; stride = RY * GX; }
          else if (d == 1) { dst = gyp + gy * RX + gx - 2; stride = GY * RX; }
          else { dst = hzp + (gy - 2) * RX + gx - 2; stride = RY * RX; }
          dst[0] = tau[0];
          dst[stride] = tau[1];
          dst[2 * stride] = tau[2];
          dst[3 * stride] = e;
        }
      }
      __syncthreads();
      // the x- and y-parts of the lead plane, then the output plane p - 2 with its z-part
      T rv0[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const T* f = fxp + (q * RY + warp) * GX + lane + 2;
        const T dx = (f[-2] - f[2]) + T(8) * (f[1] - f[-1]);
        const T* g = gyp + (q * GY + warp + 2) * RX + lane;
        const T dy = (g[-2 * RX] - g[2 * RX]) + T(8) * (g[RX] - g[-RX]);
        rv0[q] = dx * ih0 + dy * ih1;
      }
      const int k = p - 2;
      const int i = x0 + lane, j = y0 + warp;
      if (k >= k0 && i < b.nx && j < b.ny) {
        const long long cc = ((long long)k * b.ny + j) * b.nx + i;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int o = (q * RY + warp) * RX + lane;
          const T dz = (hzr[zs(k - 2) * RSmem<T>::HZP + o] - hzr[zs(k + 2) * RSmem<T>::HZP + o]) +
                       T(8) * (hzr[zs(k + 1) * RSmem<T>::HZP + o] - hzr[zs(k - 1) * RSmem<T>::HZP + o]);
          Rv[q * a.n + cc] = -(rv2[q] + dz * ih2);
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        rv2[q] = rv1[q];
        rv1[q] = rv0[q];
      }
      __syncthreads();  // the x-, y-flux buffers, the z-slot of plane p - 2 and W slots are reused
    }
  }
  if (*sabort && threadIdx.x == 0) tma_abort(bar, pending, parity, WRING, a.ctrl);
}

// ---- the weighted interpolation: both edge values of cell i from u_{i-2} .. u_{i+2} -----------
// The three stencils A = {i-2, i-1, i}, B = {i-1, i, i+1}, C = {i, i+1, i+2} give, with g and s
// their first and second differences at i, the candidates u_i +- g/2 + s/8 at i +- 1/2 and the
// smoothness g^2 + s^2; the optimal weights are (1, 10, 5)/16 on (A, B, C) at i + 1/2 and the
// mirrored (5, 10, 1)/16 at i - 1/2.  alpha = C_k / d_k with d_k = (1e-6 + smoothness)^2, and the
// normalised combination takes one reciprocal: sum C_k (prod_{m != k} d_m) c_k / sum C_k (...).
template <typename V>
__device__ __forceinline__ void edges(V u0, V u1, V u2, V u3, V u4, bool linear, V& up, V& um) {
  using O = VM<V>;
  const V half = O::c(0.5), eighth = O::c(0.125);
  const V gA = half * (u0 - O::c(4) * u1 + O::c(3) * u2), sA = u0 - O::c(2) * u1 + u2;
  const V gB = half * (u3 - u1), sB = u1 - O::c(2) * u2 + u3;
  const V gC = half * (O::c(-3) * u2 + O::c(4) * u3 - u4), sC = u2 - O::c(2) * u3 + u4;
  const V eA = eighth * sA, eB = eighth * sB, eC = eighth * sC;
  const V pA = O::fma(half, gA, eA), pB = O::fma(half, gB, eB), pC = O::fma(half, gC, eC);
  const V mA = O::fma(-half, gA, eA), mB = O::fma(-half, gB, eB), mC = O::fma(-half, gC, eC);
  if (linear) {
    up = u2 + (O::c(1.0 / 16.0) * pA + O::c(10.0 / 16.0) * pB + O::c(5.0 / 16.0) * pC);
    um = u2 + (O::c(5.0 / 16.0) * mA + O::c(10.0 / 16.0) * mB + O::c(1.0 / 16.0) * mC);
    return;
  }
  const V e = O::c(1e-6);
  V dA = e + O::fma(gA, gA, sA * sA), dB = e + O::fma(gB, gB, sB * sB), dC = e + O::fma(gC, gC, sC * sC);
  dA = dA * dA; dB = dB * dB; dC = dC * dC;
  const V bc = dB * dC, ac = dA * dC, ab = dA * dB;
  const V nA = O::c(1.0 / 16.0) * bc, nB = O::c(10.0 / 16.0) * ac, nC = O::c(5.0 / 16.0) * ab;
  const V kA = O::c(5.0 / 16.0) * bc, kC = O::c(1.0 / 16.0) * ab;
  const V dp = nA + nB + nC, dm = kA + nB + kC;
  V rp, rm;
  if constexpr (sizeof(V) == 8) {  // one FP64 division for both (dp, dm >= ~1e-25: no underflow)
    const V r = O::rcp(dp * dm);
    rp = dm * r;
    rm = dp * r;
  } else {
    rp = O::rcp(dp);
    rm = O::rcp(dm);
  }
  up = u2 + O::fma(nA, pA, O::fma(nB, pB, nC * pC)) * rp;
  um = u2 + O::fma(kA, mA, O::fma(nB, mB, kC * mC)) * rm;
}

// The same for two variables at once in packed f32x2 arithmetic (one instruction per pair of
// lanes' values: FFMA2 / FMUL2 / FADD2 of sm_100+); the reciprocals stay scalar.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ void edges2(float2 u0, float2 u1, float2 u2, float2 u3, float2 u4, bool linear,
                                       float2& up, float2& um) {
  const float2 half = f2(0.5f), eighth = f2(0.125f), mhalf = f2(-0.5f);
  const float2 gA = mul2(half, fma2(f2(3.f), u2, fma2(f2(-4.f), u1, u0)));
  const float2 sA = add2(fma2(f2(-2.f), u1, u0), u2);
  const float2 gB = fma2(half, u3, mul2(mhalf, u1));
  const float2 sB = add2(fma2(f2(-2.f), u2, u1), u3);
  const float2 gC = mul2(half, fma2(f2(-1.f), u4, fma2(f2(4.f), u3, mul2(f2(-3.f), u2))));
  const float2 sC = add2(fma2(f2(-2.f), u3, u2), u4);
  const float2 eA = mul2(eighth, sA), eB = mul2(eighth, sB), eC = mul2(eighth, sC);
  const float2 pA = fma2(half, gA, eA), pB = fma2(half, gB, eB), pC = fma2(half, gC, eC);
  const float2 mA = fma2(mhalf, gA, eA), mB = fma2(mhalf, gB, eB), mC = fma2(mhalf, gC, eC);
  if (linear) {
    up = add2(u2, fma2(f2(1.f / 16.f), pA, fma2(f2(10.f / 16.f), pB, mul2(f2(5.f / 16.f), pC))));
    um = add2(u2, fma2(f2(5.f / 16.f), mA, fma2(f2(10.f / 16.f), mB, mul2(f2(1.f / 16.f), mC))));
    return;
  }
  const float2 e = f2(1e-6f);
  float2 dA = add2(e, fma2(gA, gA, mul2(sA, sA)));
  float2 dB = add2(e, fma2(gB, gB, mul2(sB, sB)));
  float2 dC = add2(e, fma2(gC, gC, mul2(sC, sC)));
  dA = mul2(dA, dA); dB = mul2(dB, dB); dC = mul2(dC, dC);
  const float2 bc = mul2(dB, dC), ac = mul2(dA, dC), ab = mul2(dA, dB);
  const float2 nA = mul2(f2(1.f / 16.f), bc), nB = mul2(f2(10.f / 16.f), ac), nC = mul2(f2(5.f / 16.f), ab);
  const float2 kA = mul2(f2(5.f / 16.f), bc), kC = mul2(f2(1.f / 16.f), ab);
  const float2 np = fma2(nA, pA, fma2(nB, pB, mul2(nC, pC)));
  const float2 nm = fma2(kA, mA, fma2(nB, mB, mul2(kC, mC)));
  const float2 dp = add2(add2(nA, nB), nC), dm = add2(add2(kA, nB), kC);
  const float2 rp = make_float2(__fdividef(1.f, dp.x), __fdividef(1.f, dp.y));
  const float2 rm = make_float2(__fdividef(1.f, dm.x), __fdividef(1.f, dm.y));
  up = fma2(np, rp, u2);
  um = fma2(nm, rm, u2);
}

template <int D> struct Fr;
template <> struct Fr<0> { static constexpr int N = 1, T1 = 2, T2 = 3; };
template <> struct Fr<1> { static constexpr int N = 2, T1 = 3, T2 = 1; };
template <> struct Fr<2> { static constexpr int N = 3, T1 = 1, T2 = 2; };

template <typename T>
struct Smem {
  static constexpr int WS = 5 * (LMAX + 10) * NLP;   // staged primitives [5][L+10][NLP], then
                                                     // the edge fluxes [5][L+5][NLP] over them;
                                                     // two buffers (the next tile lands in one)
  static constexpr int RS = sizeof(T) == 4 ? 5 * LMAX * NLP : 0;  // the running residual of the tile's
                                                                   // cells (mixed path only)
  static constexpr size_t rs = (2 * sizeof(T) * WS + 15) / 16 * 16;
  static constexpr size_t red = (rs + sizeof(T) * RS + 15) / 16 * 16;  // norm partials (double)
  static constexpr size_t bytes = red + sizeof(double) * (NTW / 32) * 5;
};



// MODE: 0 x pass (R =), 1 y pass (R +=), 2 z pass (stage update or residual output)
template <typename T, int D, int MODE>
__global__ void __launch_bounds__(NTW, sizeof(T) == 4 ? 3 : 2) dir_kernel(Args a) {
  using O = VM<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* const Wbuf = reinterpret_cast<T*>(smem_raw);
  double* red = reinterpret_cast<double*>(smem_raw + Smem<T>::red);
  __shared__ int last;
  const Box& b = a.b;
  const int nd = D == 0 ? b.nx : (D == 1 ? b.ny : b.nz);   // along the lines
  const int na = D == 0 ? b.ny : b.nx;                      // across the lines (16 per tile)
  const int nb = D == 2 ? b.ny : b.nz;                      // the third direction
  const int L = a.Lseg[D];
  const int nseg = (nd + L - 1) / L, ngrp = (na + NL - 1) / NL;
  const long long tiles = (long long)nseg * ngrp * nb;
  const T* W = static_cast<const T*>(a.W);
  T* R = static_cast<T*>(a.R);
  const Consts<T> K = coef<T>(a).K;
  const T ih = coef<T>(a).ih[D];
  const bool linear = a.linear != 0;
  const double dt = (MODE == 2 && a.stage > 0) ? a.ctrl->dt : 0.0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double sq[5] = {0, 0, 0, 0, 0};  // FP64 sums of R^2 (an FP32 residual's square is exact in FP64)
  constexpr int idx[5] = {0, Fr<D>::N, Fr<D>::T1, Fr<D>::T2, 4};
  struct TileInfo { int s0, Ls, a0, ob; };
  auto decode = [&](long long tile) {
    TileInfo t;
    const int seg = (int)(tile % nseg);
    const long long r = tile / nseg;
    t.s0 = seg * L;
    t.Ls = min(L, nd - t.s0);
    t.a0 = (int)(r % ngrp) * NL;
    t.ob = (int)(r / ngrp);
    return t;
  };
  // cell (line l, position s along D) of tile t -> (i, j, k)
  auto ijk = [&](const TileInfo& t, int l, int s, int& i, int& j, int& k) {  // (the cell phase)
    if (D == 0) { i = s; j = t.a0 + l; k = t.ob; }
    else if (D == 1) { i = t.a0 + l; j = s; k = t.ob; }
    else { i = t.a0 + l; j = t.ob; k = s; }
  };
  // 1. stage the primitives of cells s0 - 5 .. s0 + Ls + 4 of every line into buffer Ws
  //    (staged cell s is cell s0 - 5 + s), asynchronously, as one commit group
  auto issue_stage = [&](const TileInfo& t, T* Ws) {
    const int nst = t.Ls + 10;
    // offset of cell (line l, position s along D) within a field (fits 32 bits)
    auto off = [&](int l, int s) {
      if (D == 0) return ((t.ob + H) * (b.ny + 2 * H) + t.a0 + l + H) * b.px + s + H;
      if (D == 1) return ((t.ob + H) * (b.ny + 2 * H) + s + H) * b.px + t.a0 + l + H;
      return ((s + H) * (b.ny + 2 * H) + t.ob + H) * b.px + t.a0 + l + H;
    };
    if (D == 0) {  // a warp per (variable, line), lanes along x
      for (int vl = warp; vl < 5 * NL; vl += NTW / 32) {
        const int v = vl / NL, l = vl % NL;
        T* drow = Ws + v * (LMAX + 10) * NLP + l;
        if (t.a0 + l < na) {
          const T* srow = W + (long long)v * b.field + off(l, t.s0 - H);
          for (int s = lane; s < nst; s += 32) cp_async(drow + s * NLP, srow + s);
        } else {
          for (int s = lane; s < nst; s += 32) drow[s * NLP] = (v == 0 || v == 4) ? T(1) : T(0);
        }
      }
    } else {       // 16 lines (x) per row s
      for (int v = 0; v < 5; ++v) {
        const T* src = W + (long long)v * b.field;
        T* dv = Ws + v * (LMAX + 10) * NLP;
        for (int e = threadIdx.x; e < nst * NL; e += NTW) {
          const int s = e / NL, l = e % NL;
          if (t.a0 + l < na) cp_async(dv + s * NLP + l, src + off(l, t.s0 - H + s));
          else dv[s * NLP + l] = (v == 0 || v == 4) ? T(1) : T(0);  // lines past the block
        }
      }
    }
    cp_async_commit();
  };
  // the y and z passes add to the residual R of the earlier passes: the tile's R lands in shared
  // memory (as its own commit group) while the edge fluxes are computed
  T* const Rs = reinterpret_cast<T*>(smem_raw + Smem<T>::rs);
  auto issue_r = [&](const TileInfo& t) {
    for (int q = 0; q < 5; ++q)
      for (int e = threadIdx.x; e < t.Ls * NL; e += NTW) {
        const int c = e / NL, l = e % NL;
        if (t.a0 + l >= na) continue;
        int i, j, k;
        ijk(t, l, t.s0 + c, i, j, k);
        cp_async(Rs + (q * LMAX + c) * NLP + l, R + q * a.n + ((long long)k * b.ny + j) * b.nx + i);
      }
    cp_async_commit();
  };
  int buf = 0;
  if ((long long)blockIdx.x < tiles) issue_stage(decode(blockIdx.x), Wbuf);
  for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x, buf ^= 1) {
    const TileInfo t = decode(tile);
    const int s0 = t.s0, Ls = t.Ls, a0 = t.a0;
    T* const Ws = Wbuf + buf * Smem<T>::WS;
    T* const Fs = Ws;  // the edge fluxes replace the primitives once every lane holds its fluxes
    const int nfc = Ls + 5;
    cp_async_wait_all();
    __syncthreads();  // the tile has landed; the previous tile's cells are done with the other buffer
    constexpr bool RSTAGE = MODE != 0 && sizeof(T) == 4;  // FP64: shared memory is kept for occupancy
    if (RSTAGE) issue_r(t);
    const bool more = tile + gridDim.x < tiles;
    if (more) issue_stage(decode(tile + gridDim.x), Wbuf + (buf ^ 1) * Smem<T>::WS);
    // 2. edge fluxes: edge f lies between staged cells f + 2 and f + 3, so cell c (staged c + 5)
    //    has edges c .. c + 5 around it.  Item (line, chunk): lane t takes staged cell
    //    m = 31 chunk + t + 2, evaluates its two edge states, and edge f = m - 2 pairs its
    //    left state with lane t + 1's right state.
    T F[ITEMS][5];
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
      const int item = warp * ITEMS + it, l = item >> 1, ch = item & 1;
      const int f = FCH * ch + lane;
      if (a0 + l >= na || FCH * ch >= nfc) continue;  // warp-uniform
      const int m = min(f + 2, nfc + 2);              // centres 2 .. nfc + 2 (stencil <= nst - 1)
      T Lq[5], Rq[5];
      if constexpr (sizeof(T) == 4) {  // mixed: frame variables (0, 1) and (2, 3) as packed pairs
#pragma unroll
        for (int q = 0; q < 4; q += 2) {
          const T* w0 = Ws + (idx[q] * (LMAX + 10) + m - 2) * NLP + l;
          const T* w1 = Ws + (idx[q + 1] * (LMAX + 10) + m - 2) * NLP + l;
          float2 up, um;
          edges2(make_float2(w0[0], w1[0]), make_float2(w0[NLP], w1[NLP]), make_float2(w0[2 * NLP], w1[2 * NLP]),
                 make_float2(w0[3 * NLP], w1[3 * NLP]), make_float2(w0[4 * NLP], w1[4 * NLP]), linear, up, um);
          Lq[q] = up.x;
          Lq[q + 1] = up.y;
          Rq[q] = __shfl_down_sync(0xffffffffu, um.x, 1);
          Rq[q + 1] = __shfl_down_sync(0xffffffffu, um.y, 1);
        }
        const T* w = Ws + (idx[4] * (LMAX + 10) + m - 2) * NLP + l;
        T up, um;
        edges<T>(w[0], w[NLP], w[2 * NLP], w[3 * NLP], w[4 * NLP], linear, up, um);
        Lq[4] = up;
        Rq[4] = __shfl_down_sync(0xffffffffu, um, 1);
      } else {
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          const T* w = Ws + (idx[q] * (LMAX + 10) + m - 2) * NLP + l;
          T up, um;
          edges<T>(w[0], w[NLP], w[2 * NLP], w[3 * NLP], w[4 * NLP], linear, up, um);
          Lq[q] = up;
          Rq[q] = __shfl_down_sync(0xffffffffu, um, 1);
        }
      }
      if (lane < FCH && f < nfc) roe_frame<T>(Lq, Rq, K, F[it]);
    }
    __syncthreads();  // every lane is done reading the primitives
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
      const int item = warp * ITEMS + it, l = item >> 1, ch = item & 1;
      const int f = FCH * ch + lane;
      if (a0 + l >= na || FCH * ch >= nfc || lane >= FCH || f >= nfc) continue;
#pragma unroll
      for (int q = 0; q < 5; ++q) Fs[(idx[q] * (LMAX + 5) + f) * NLP + l] = F[it][q];
    }
    if (RSTAGE) {  // the tile's R (the newest group, the next tile's primitives, may fly on)
      if (more) cp_async_wait_one();
      else cp_async_wait_all();
    }
    __syncthreads();
    // 3. Eq. 2 per cell (plus the viscous residual in the x pass), then the pass's output
    const int ncell = D == 0 ? NL * 64 : Ls * NL;  // D = 0: a warp per line, lanes along x
    for (int e = threadIdx.x; e < ncell; e += NTW) {
      int l, c;
      if (D == 0) {
        l = e >> 6;
        c = e & 63;
        if (c >= Ls) continue;
      } else {
        c = e / NL;
        l = e % NL;
      }
      if (a0 + l >= na) continue;
      int i, j, k;
      ijk(t, l, s0 + c, i, j, k);
      const long long cc = ((long long)k * b.ny + j) * b.nx + i;
      T add[5];
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const T* fq = Fs + (q * (LMAX + 5) + c) * NLP + l;
        const T f0 = fq[0], f1 = fq[NLP], f2 = fq[2 * NLP], f3 = fq[3 * NLP], f4 = fq[4 * NLP], f5 = fq[5 * NLP];
        add[q] = (O::c(75.0 / 64.0) * (f3 - f2) - O::c(25.0 / 384.0) * (f4 - f1) + O::c(3.0 / 640.0) * (f5 - f0)) * ih;
      }
      if (D == 0 && a.viscous) {  // the viscous residual, once (x pass)
        const T* rv = static_cast<const T*>(a.Rv);
#pragma unroll
        for (int q = 0; q < 4; ++q) add[1 + q] = add[1 + q] + rv[q * a.n + cc];
      }
      if (MODE == 0) {
#pragma unroll
        for (int q = 0; q < 5; ++q) R[q * a.n + cc] = add[q];
      } else if (MODE == 1) {
#pragma unroll
        for (int q = 0; q < 5; ++q) R[q * a.n + cc] = (RSTAGE ? Rs[(q * LMAX + c) * NLP + l] : R[q * a.n + cc]) + add[q];
      } else if (sizeof(T) == 8) {  // FP64: Eqs. 4-6 as written
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
      } else {  // mixed: f32 increments, FP64 only for Q^{n+1} = Q^n + 2/3 (D2 - dt R)
        const float dtf = float(dt);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          const float tot = float(Rs[(q * LMAX + c) * NLP + l]) + float(add[q]);
          const long long o = q * a.n + cc;
          if (a.stage == 0) {
            a.rout[o] = f32_to_f64_bits(tot);
          } else if (a.stage == 1) {
            sq[q] = fma(double(tot), double(tot), sq[q]);
            a.d1[o] = -dtf * tot;
          } else if (a.stage == 2) {
            a.d2[o] = 0.25f * (a.d1[o] - dtf * tot);
          } else {
            const double qn1 = a.q[o] + f32_to_f64_bits((2.0f / 3.0f) * (a.d2[o] - dtf * tot));
            a.q[o] = qn1;
            a.sh[o] = f64_to_f32_bits(qn1);
          }
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
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < 5; ++q) red[warp * 5 + q] = sq[q];
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
  if (!last || threadIdx.x >= 32) return;
  __threadfence();
  // the last CTA's first warp folds the per-CTA sums: lane-strided in CTA order, then a fixed
  // shuffle tree (the same order every run: deterministic)
  double tot[5] = {0, 0, 0, 0, 0};
  for (unsigned c = threadIdx.x; c < gridDim.x; c += 32)
#pragma unroll
    for (int q = 0; q < 5; ++q) tot[q] += __ldcg(a.partial + (size_t)c * NPART + q);
#pragma unroll
  for (int q = 0; q < 5; ++q)
    for (int off = 16; off > 0; off >>= 1) tot[q] += __shfl_xor_sync(0xffffffffu, tot[q], off);
  if (threadIdx.x == 0) {
    for (int q = 0; q < 5; ++q) a.ctrl->norms[q] = sqrt(tot[q] / (double)a.n);
    a.ctrl->counter = 0u;
  }
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
  e = cudaFuncSetAttribute(viscres_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RSmem<T>::bytes);
  if (e != cudaSuccess) return e;
  return cudaSuccess;
}

template <typename T>
static int viscres_occupancy() {
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, viscres_kernel<T>, NTW, RSmem<T>::bytes);
  return std::max(1, occ);
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
  CUtensorMap mwv;            // TMA map of the primitive box
  int nx, ny, nz;
  gbcfd_params p;
  double h[3];
  int device, nsm, mixed;
  Box box;
  double* q[3];      // FP64: Q^n, Q1, Q2.  mixed: Q^n only (compact f64)
  float* sh;         // mixed: S^n = f32(Q^n)
  float* d[2];       // mixed: D1, D2
  void* W;
  void* Rv;
  void* R;
  DevCtrl* ctrl;
  double* partial;
  int rows;          // partial rows (CTAs of the widest launch)
  int has_state;
  int dir_grid, occ, rocc;
  cudaEvent_t events[18];  // timing marks (gbcfd_wcns_set_timing), 6 per stage
  int timing;
  gbcfd_wcns nbr[6];       // face neighbours (gbcfd_wcns_connect); none: the block wraps periodically
};

namespace {

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct WLayout {
  size_t q, w, rv, r, ctrl, partial, total;
  Box box;
  int rows;
};

// FP64: Q^n, Q1, Q2 (f64).  mixed: Q^n (f64) and S^n, D1, D2 (f32) in the same three slots
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
  L->q = off;       off += elem == 8 ? 3 * al256((size_t)n * 5 * 8) : al256((size_t)n * 5 * 8) + 3 * al256((size_t)n * 5 * 4);
  L->w = off;       off += al256((size_t)b.field * NPW * elem);
  L->rv = off;      off += p->viscous ? al256((size_t)n * 4 * elem) : 0;
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

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}

// 4D map (x, y, z, field) over nfield padded fields of the box; boxes of bx x by x 1 x bf.  The x
// extent is the padded width nx + 10, so columns past it read zero.
int encode_box_map(CUtensorMap* m, void* base, const Box& b, int elem, int nfield, int bx, int by, int bf) {
  auto enc = tensor_map_encoder();
  if (!enc) return set_error(GBCFD_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  cuuint64_t dims[4] = {(cuuint64_t)(b.nx + 2 * H), (cuuint64_t)(b.ny + 2 * H), (cuuint64_t)(b.nz + 2 * H),
                        (cuuint64_t)nfield};
  cuuint64_t strides[3] = {(cuuint64_t)b.px * elem, (cuuint64_t)b.px * elem * (b.ny + 2 * H),
                           (cuuint64_t)b.field * elem};
  cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1, (cuuint32_t)bf};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = enc(m, elem == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims,
                   strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(GBCFD_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return GBCFD_OK;
}

template <typename T>
void fill_coef(const Args& a, Coef<T>& c) {
  const double kappa = a.Pr > 0.0 ? a.mu * a.gamma / ((a.gamma - 1.0) * a.Pr) : 0.0;
  c.gm1 = T(a.gamma - 1.0);
  c.gam = T(a.gamma);
  c.half = T(0.5);
  c.vf = T(4.0 * std::max(4.0 / 3.0, a.gamma / a.Pr) * a.mu);
  c.mu = T(a.mu);
  c.kappa = T(kappa);
  for (int d = 0; d < 3; ++d) {
    c.ih[d] = T(a.ih[d]);
    c.ih12[d] = T(a.ih[d] / 12.0);
  }
  c.ihs = T(a.ih[0] * a.ih[0] + a.ih[1] * a.ih[1] + a.ih[2] * a.ih[2]);
  c.K.gm1 = T(a.gamma - 1.0);
  c.K.ggm1 = T(a.gamma / (a.gamma - 1.0));
  c.K.eps = T(a.eps);
  c.K.mu = T(a.mu);
  c.K.kappa = T(kappa);
  c.K.lim = 0;
}

Args make_args(gbcfd_wcns w) {
  Args a;
  std::memset(&a, 0, sizeof(a));
  a.mwv = w->mwv;
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
  fill_coef(a, a.cf);
  fill_coef(a, a.cd);
  a.W = w->W;
  a.Rv = w->Rv;
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

// the passes after the primitives: viscous residual, then x, y and z (marks 1..5 of ev)
template <typename T>
cudaError_t launch_rest(gbcfd_wcns w, const Args& a, const cudaEvent_t* ev, cudaStream_t s) {
  auto mark = [&](int m) {
    if (ev) cudaEventRecord(ev[m], s);
  };
  if (a.viscous) viscres_kernel<T><<<w->nsm * w->rocc, NTW, RSmem<T>::bytes, s>>>(a);
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

template <typename T>
cudaError_t launch_pass(gbcfd_wcns w, Args a, int with_rate, const cudaEvent_t* ev, cudaStream_t s) {
  if (ev) cudaEventRecord(ev[0], s);
  const int pgrid = std::min(w->rows, w->nsm * 8);
  prim_kernel<T><<<pgrid, NTW, 0, s>>>(a, with_rate);
  if (ev) cudaEventRecord(ev[1], s);
  return launch_rest<T>(w, a, ev, s);
}

// the kernel arguments of one Runge-Kutta stage (1..3) or of the residual (stage 0, into rout)
Args stage_args(gbcfd_wcns w, int stage, double* rout) {
  Args a = make_args(w);
  a.stage = stage;
  a.rout = rout;
  if (w->mixed) {
    a.q = w->q[0];
    a.sh = w->sh;
    a.d1 = w->d[0];
    a.d2 = w->d[1];
    a.din = stage == 2 ? w->d[0] : (stage == 3 ? w->d[1] : nullptr);
  } else {
    a.qn = w->q[0];
    a.qs = stage <= 1 ? w->q[0] : w->q[stage - 1];
    a.qout = stage == 3 ? w->q[0] : (stage >= 1 ? w->q[stage] : nullptr);
  }
  return a;
}

// one Runge-Kutta stage (1..3) or the residual (stage 0, written to rout)
int run_stage(gbcfd_wcns w, int stage, double* rout, cudaStream_t s) {
  const Args a = stage_args(w, stage, rout);
  const cudaEvent_t* ev = (w->timing && stage >= 1) ? w->events + 6 * (stage - 1) : nullptr;
  const cudaError_t e = w->mixed ? launch_pass<float>(w, a, stage == 1, ev, s) : launch_pass<double>(w, a, stage == 1, ev, s);
  if (e != cudaSuccess) return cuda_err(e, "WCNS stage launch");
  return GBCFD_OK;
}

// side streams of the current device for blocks advanced together: the kernels of different
// blocks overlap (each block alone fills the GPU only partly, and its launches' tails leave SMs
// idle); created once per device, shared by all calls (events order the work of each call)
constexpr int NSIDE = 8;
struct SidePool {
  int device;
  cudaStream_t st[NSIDE];
  cudaEvent_t done[NSIDE], fork;
};
cudaError_t side_pool(SidePool** out) {
  static std::mutex mu;
  static std::vector<SidePool*> pools;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  for (SidePool* p : pools)
    if (p->device == dev) {
      *out = p;
      return cudaSuccess;
    }
  SidePool* p = new SidePool();
  p->device = dev;
  for (int k = 0; k < NSIDE && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&p->st[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->done[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming);
  if (e != cudaSuccess) return e;  // (a failed pool is not kept; its handles leak)
  pools.push_back(p);
  *out = p;
  return cudaSuccess;
}

// the side streams k < m wait for the work issued so far on s
cudaError_t fork(SidePool* p, int m, cudaStream_t s) {
  cudaError_t e = cudaEventRecord(p->fork, s);
  for (int k = 0; k < m && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(p->st[k], p->fork, 0);
  return e;
}
// s waits for the work issued so far on the side streams k < m
cudaError_t join(SidePool* p, int m, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < m && e == cudaSuccess; ++k) {
    e = cudaEventRecord(p->done[k], p->st[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->done[k], 0);
  }
  return e;
}

// one Runge-Kutta stage of blocks advanced together: every member's primitives first (a member's
// halo reads its neighbours' stage inputs, and on the mixed path stage 3 rewrites the shadow S^n
// its neighbours' halos read, so no member's passes start before all primitives are formed), the
// common time step after stage 1's, then each member's viscous and direction passes.  Members run
// on side streams (block i on stream i mod 8) between a fork from and a join into s.
template <typename T>
cudaError_t run_stage_many(const gbcfd_wcns* blocks, int n, WTab& tab, int stage, SidePool* pool, cudaStream_t s) {
  const int m = std::min(n, NSIDE);
  cudaError_t e = fork(pool, m, s);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    const gbcfd_wcns w = blocks[i];
    tab.self = i;
    const int pgrid = std::min(w->rows, w->nsm * 8);
    prim_multi_kernel<T><<<pgrid, NTW, 0, pool->st[i % NSIDE]>>>(stage_args(w, stage, nullptr), stage == 1, tab);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = join(pool, m, s);
  if (e == cudaSuccess && stage == 1) {
    wcns_group_dt_kernel<<<1, 32, 0, s>>>(tab, blocks[0]->p.cfl);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = fork(pool, m, s);
  for (int i = 0; i < n && e == cudaSuccess; ++i)
    e = launch_rest<T>(blocks[i], stage_args(blocks[i], stage, nullptr), nullptr, pool->st[i % NSIDE]);
  if (e == cudaSuccess) e = join(pool, m, s);
  return e;
}

bool connected_to_others(gbcfd_wcns w) {
  for (int f = 0; f < 6; ++f)
    if (w->nbr[f] && w->nbr[f] != w) return true;
  return false;
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
  if (L.box.field >= (1LL << 31))
    return set_error(GBCFD_ERR_ARG, "WCNS block too large: the padded box must hold fewer than 2^31 cells");
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
  const size_t qbytes = al256((size_t)nx * ny * nz * 5 * 8), fbytes = al256((size_t)nx * ny * nz * 5 * 4);
  if (mixed) {
    w->q[0] = reinterpret_cast<double*>(base + L.q);
    w->q[1] = w->q[2] = nullptr;
    w->sh = reinterpret_cast<float*>(base + L.q + qbytes);
    w->d[0] = reinterpret_cast<float*>(base + L.q + qbytes + fbytes);
    w->d[1] = reinterpret_cast<float*>(base + L.q + qbytes + 2 * fbytes);
  } else {
    for (int s = 0; s < 3; ++s) w->q[s] = reinterpret_cast<double*>(base + L.q + s * qbytes);
    w->sh = nullptr;
    w->d[0] = w->d[1] = nullptr;
  }
  w->W = base + L.w;
  w->Rv = params->viscous ? base + L.rv : nullptr;
  w->R = base + L.r;
  w->ctrl = reinterpret_cast<DevCtrl*>(base + L.ctrl);
  w->partial = reinterpret_cast<double*>(base + L.partial);
  w->rows = L.rows;
  {
    const int elem = mixed ? 4 : 8;
    const int rc = encode_box_map(&w->mwv, w->W, w->box, elem, NPW, WX, WY, 1);
    if (rc != GBCFD_OK) {
      delete w;
      return rc;
    }
  }
  w->occ = mixed ? dir_occupancy<float>() : dir_occupancy<double>();
  w->rocc = mixed ? viscres_occupancy<float>() : viscres_occupancy<double>();
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
  for (int f = 0; f < 6; ++f)  // the neighbours forget this block
    if (w->nbr[f] && w->nbr[f] != w && w->nbr[f]->nbr[f ^ 1] == w) w->nbr[f]->nbr[f ^ 1] = nullptr;
  delete w;
  return GBCFD_OK;
}

extern "C" int gbcfd_wcns_set_state(gbcfd_wcns w, const double* q, void* stream) {
  if (!w || !q) return set_error(GBCFD_ERR_ARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t n = (size_t)w->nx * w->ny * w->nz;
  cudaError_t e = cudaMemcpyAsync(w->q[0], q, n * 5 * sizeof(double), cudaMemcpyDefault, s);
  if (e != cudaSuccess) return cuda_err(e, "cudaMemcpyAsync");
  if (w->mixed) {
    shadow_kernel<<<w->nsm * 8, 256, 0, s>>>(w->q[0], w->sh, (long long)n * 5);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(e, "shadow kernel launch");
  }
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
  if (connected_to_others(w))
    return set_error(GBCFD_ERR_STATE, "the block is connected to other blocks: they advance with gbcfd_wcns_step_many");
  return run_stage(w, 0, r, static_cast<cudaStream_t>(stream));
}

extern "C" int gbcfd_wcns_step(gbcfd_wcns w, int nsteps, void* stream) {
  if (!w) return set_error(GBCFD_ERR_ARG, "NULL block");
  if (nsteps < 0) return set_error(GBCFD_ERR_ARG, "nsteps must be >= 0");
  if (!w->has_state) return set_error(GBCFD_ERR_STATE, "no state set");
  if (connected_to_others(w))
    return set_error(GBCFD_ERR_STATE, "the block is connected to other blocks: they advance with gbcfd_wcns_step_many");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int n = 0; n < nsteps; ++n)
    for (int st = 1; st <= 3; ++st) {
      const int rc = run_stage(w, st, nullptr, s);
      if (rc != GBCFD_OK) return rc;
    }
  return GBCFD_OK;
}

extern "C" int gbcfd_wcns_connect(gbcfd_wcns a, int face, gbcfd_wcns b) {
  if (!a || !b) return set_error(GBCFD_ERR_ARG, "NULL block");
  if (face < 0 || face > 5) return set_error(GBCFD_ERR_ARG, "face must be 0..5 (-x, +x, -y, +y, -z, +z)");
  const int ax = face >> 1;
  if ((ax != 0 && a->nx != b->nx) || (ax != 1 && a->ny != b->ny) || (ax != 2 && a->nz != b->nz))
    return set_error(GBCFD_ERR_ARG, "the two blocks' faces differ in size");
  if (a->mixed != b->mixed || memcmp(&a->p, &b->p, sizeof(gbcfd_params)) != 0 || memcmp(a->h, b->h, sizeof(a->h)) != 0)
    return set_error(GBCFD_ERR_ARG, "connected blocks must share parameters and cell sizes");
  a->nbr[face] = b;
  b->nbr[face ^ 1] = a;
  return GBCFD_OK;
}

extern "C" int gbcfd_wcns_step_many(const gbcfd_wcns* blocks, int n, int nsteps, void* stream) {
  if (!blocks) return set_error(GBCFD_ERR_ARG, "NULL block list");
  if (n < 1 || n > MAXW) return set_error(GBCFD_ERR_ARG, "gbcfd_wcns_step_many takes 1 to 32 blocks");
  if (nsteps < 0) return set_error(GBCFD_ERR_ARG, "nsteps must be >= 0");
  WTab tab;
  memset(&tab, 0, sizeof(tab));
  tab.n = n;
  for (int i = 0; i < n; ++i) {
    const gbcfd_wcns w = blocks[i];
    if (!w) return set_error(GBCFD_ERR_ARG, "NULL block");
    for (int k = 0; k < i; ++k)
      if (blocks[k] == w) return set_error(GBCFD_ERR_ARG, "a block is listed twice");
    if (!w->has_state) return set_error(GBCFD_ERR_STATE, "no state set");
    if (w->device != blocks[0]->device || w->mixed != blocks[0]->mixed ||
        memcmp(&w->p, &blocks[0]->p, sizeof(gbcfd_params)) != 0 || memcmp(w->h, blocks[0]->h, sizeof(w->h)) != 0)
      return set_error(GBCFD_ERR_ARG, "the blocks must share device, parameters and cell sizes");
    WSrc& e = tab.e[i];
    for (int q = 0; q < 3; ++q) e.q[q] = w->q[q];
    e.sh = w->sh;
    e.d[0] = w->d[0];
    e.d[1] = w->d[1];
    e.ctrl = w->ctrl;
    e.nx = w->nx; e.ny = w->ny; e.nz = w->nz;
  }
  // every face connected within the list, the two blocks of a face equal across it, and face
  // walks along two different axes reaching the same block in either order (a conforming periodic
  // lattice: every halo cell has one owner)
  for (int i = 0; i < n; ++i)
    for (int f = 0; f < 6; ++f) {
      const gbcfd_wcns nb = blocks[i]->nbr[f] ? blocks[i]->nbr[f] : (n == 1 ? blocks[i] : nullptr);
      int j = -1;
      for (int k = 0; k < n && nb; ++k)
        if (blocks[k] == nb) j = k;
      if (j < 0)
        return set_error(GBCFD_ERR_ARG, "face " + std::to_string(f) + " of block " + std::to_string(i) +
                                            " is not connected to a block of the list");
      tab.e[i].nbr[f] = j;
    }
  for (int i = 0; i < n; ++i)
    for (int f = 0; f < 6; ++f)  // links both ways (a face re-connected elsewhere leaves a stale one)
      if (tab.e[tab.e[i].nbr[f]].nbr[f ^ 1] != i)
        return set_error(GBCFD_ERR_ARG, "face " + std::to_string(f) + " of block " + std::to_string(i) +
                                            " is not connected back by its neighbour");
  for (int i = 0; i < n; ++i)
    for (int f1 = 0; f1 < 6; ++f1)
      for (int f2 = 0; f2 < 6; ++f2)
        if ((f1 >> 1) != (f2 >> 1) && tab.e[tab.e[i].nbr[f1]].nbr[f2] != tab.e[tab.e[i].nbr[f2]].nbr[f1])
          return set_error(GBCFD_ERR_ARG, "the blocks do not form a conforming lattice (face walks do not commute)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  SidePool* pool = nullptr;
  cudaError_t pe = side_pool(&pool);
  if (pe != cudaSuccess) return cuda_err(pe, "side streams");
  for (int step = 0; step < nsteps; ++step)
    for (int st = 1; st <= 3; ++st) {
      const cudaError_t e = blocks[0]->mixed ? run_stage_many<float>(blocks, n, tab, st, pool, s)
                                             : run_stage_many<double>(blocks, n, tab, st, pool, s);
      if (e != cudaSuccess) return cuda_err(e, "WCNS stage launch");
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

// ---- host-to-host pipeline members: the landing area is the compact state Q^n itself ----------
namespace {
int wp_upload(void* self, const double* q_in, cudaStream_t s) {
  gbcfd_wcns w = static_cast<gbcfd_wcns>(self);
  cudaError_t e = cudaMemcpyAsync(w->q[0], q_in, (size_t)w->nx * w->ny * w->nz * 5 * sizeof(double),
                                  cudaMemcpyHostToDevice, s);
  return e == cudaSuccess ? GBCFD_OK : cuda_err(e, "cudaMemcpyAsync");
}
int wp_run(void* self, int nsteps, cudaStream_t s) {
  gbcfd_wcns w = static_cast<gbcfd_wcns>(self);
  if (w->mixed) {  // as gbcfd_wcns_set_state; the control block keeps its flags until read
    shadow_kernel<<<w->nsm * 8, 256, 0, s>>>(w->q[0], w->sh, (long long)w->nx * w->ny * w->nz * 5);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(e, "shadow kernel launch");
  }
  w->has_state = 1;
  for (int n = 0; n < nsteps; ++n)
    for (int st = 1; st <= 3; ++st) {
      const int rc = run_stage(w, st, nullptr, s);
      if (rc != GBCFD_OK) return rc;
    }
  return GBCFD_OK;
}
int wp_download(void* self, double* q_out, double* norms, int nsteps, cudaStream_t s) {
  gbcfd_wcns w = static_cast<gbcfd_wcns>(self);
  cudaError_t e = cudaMemcpyAsync(q_out, w->q[0], (size_t)w->nx * w->ny * w->nz * 5 * sizeof(double),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && norms && nsteps > 0)
    e = cudaMemcpyAsync(norms, w->ctrl->norms, 5 * sizeof(double), cudaMemcpyDeviceToHost, s);
  return e == cudaSuccess ? GBCFD_OK : cuda_err(e, "cudaMemcpyAsync");
}
int wp_flags(void* self, cudaStream_t s, int* flags) {
  gbcfd_wcns w = static_cast<gbcfd_wcns>(self);
  DevCtrl h;
  int rc = read_ctrl(w, &h, s);
  if (rc != GBCFD_OK) return rc;
  *flags = h.flag;
  if (h.flag) {
    cudaError_t e = cudaMemsetAsync(&w->ctrl->flag, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_err(e, "clearing the device flag");
  }
  return GBCFD_OK;
}
}  // namespace

extern "C" int gbcfd_wcns_pipe_create(const gbcfd_wcns* blocks, int n, gbcfd_pipe* out) {
  if (!blocks || !out) return set_error(GBCFD_ERR_ARG, "NULL argument");
  *out = nullptr;
  if (n < 1 || n > 8) return set_error(GBCFD_ERR_ARG, "a pipeline takes 1 to 8 blocks");
  const gbcfd_wcns a = blocks[0];
  if (!a) return set_error(GBCFD_ERR_ARG, "NULL block");
  const size_t bytes = (size_t)a->nx * a->ny * a->nz * 5 * sizeof(double);
  std::vector<PipeMember> m(n);
  for (int i = 0; i < n; ++i) {
    const gbcfd_wcns w = blocks[i];
    if (!w) return set_error(GBCFD_ERR_ARG, "NULL block");
    for (int k = 0; k < i; ++k)
      if (blocks[k] == w) return set_error(GBCFD_ERR_ARG, "a block is listed twice");
    if (w->nx != a->nx || w->ny != a->ny || w->nz != a->nz) return set_error(GBCFD_ERR_ARG, "members differ in size");
    if (connected_to_others(w)) return set_error(GBCFD_ERR_ARG, "pipeline members are single periodic blocks");
    if (memcmp(&w->p, &a->p, sizeof(gbcfd_params)) != 0 || memcmp(w->h, a->h, sizeof(a->h)) != 0)
      return set_error(GBCFD_ERR_ARG, "members differ in parameters or cell sizes");
    m[i] = PipeMember{w, bytes, wp_upload, wp_run, wp_download, wp_flags, nullptr};
  }
  return pipe_create(m.data(), n, out);
}
