// stage.cuh -- the fused Runge-Kutta stage kernel (residual of Eq. 3 + update of Eqs. 4-6).
//
// Work decomposition: the block's (x, y) cross-section is cut into TX x TY tiles; a tile-plane
// (tile, k) is one work unit.  The grid is persistent (a multiple of the SM count) and CTA c
// owns the contiguous unit range [c W / G, (c+1) W / G) in tile-major order, so every CTA
// marches along z through one or two tiles.  Per plane k:
//   1. the TMA has already brought the conserved state of plane k+2 (tile + 2-cell halo) into a
//      shared staging slot; threads convert it to primitives into a 4-plane ring (k-1..k+2)
//      and the slot is refilled with plane k+4;
//   2. warps 0..TY-1 evaluate the lower x- and y-face of their cell and the upper z-face of
//      their column; warp TY evaluates the tile's upper x- and y-faces.  Every face flux is
//      computed once; the upper z-face becomes the next plane's lower z-face in registers;
//   3. each cell sums its six face fluxes (order -x +x -y +y -z +z per direction), applies the
//      stage update and writes its output.
// Stage 1 also accumulates sum R^2 (residual norm); stage 3 the maximum spectral-radius rate
// of the new state (next time step).  The last CTA to finish reduces the per-CTA partials in a
// fixed order (deterministic) and resets the counter.  No CTA ever waits on another.
#pragma once
#include "curvi.cuh"
#include "internal.cuh"
#include "physics.cuh"

namespace gbcfd {

// ---- mbarrier / TMA primitives (inline PTX) ------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y, int z, int v) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(v), "r"(smem_u32(bar))
      : "memory");
}
// the tensor maps live in global memory and the host rewrites them between launches (a group's
// table, possibly at an address an earlier group's maps occupied): make those writes visible to
// the tensor-map proxy before the first copy that uses a map
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* m) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(m))
               : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// bounded wait: true on completion, false after ~2 s
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer_ns() - t0 > 2000000000ull) return false;
  }
  return true;
}

// one destination of the halo push (push_table, push_halo below): direction (sx, sy, sz) in
// {-1,0,1}^3 from a block to the neighbour whose halo holds copies of its cells near those faces
struct PushDst {
  void* base;              // the neighbour's output field of this stage (element 0 of variable 0)
  long long field, plane;  // strides in elements
  int pitch, oi, oj, ok;   // row pitch; (i, j, k) shift into the neighbour's index space
};

// ---- shared-memory plan ----------------------------------------------------------------------
template <typename T, bool VISC, bool CURVI, int TYV>
struct Plan {
  static constexpr int TY = TYV, BY = box_rows(TYV), NWARP = tile_warps(TYV);
  static constexpr int NV = VISC ? 6 : 5;           // rho u v w p [theta]
  static constexpr int BOX = BY * BX;               // cells per staged plane
  static constexpr int RSLOT = NV * BOX;            // T per ring slot
  // staging slots are 128-byte aligned (TMA tensor-copy destinations); the state is staged in
  // f64 on the FP64 path and as its f32 shadow on the mixed path
  static constexpr size_t QSLOT = (sizeof(T) * 5 * BOX + 127) / 128 * 128;
  static constexpr size_t DSLOT = sizeof(T) == 4 ? (sizeof(float) * 5 * BOX + 127) / 128 * 128 : 0;
  static constexpr size_t stq = 0;                        // state staging
  static constexpr size_t std_ = stq + NSTAGE * QSLOT;    // f32 staging
  static constexpr size_t ring = std_ + NSTAGE * DSLOT;
  static constexpr size_t fx = ring + sizeof(T) * NRING * RSLOT;
  static constexpr size_t fy = fx + sizeof(T) * 5 * TY * (TX + 1);
  // curvilinear: a ring of metric planes (10 fields, k and k+1 in use, the next one landing)
  static constexpr int NMS = CURVI ? (sizeof(T) == 4 ? 3 : 2) : 0;
  static constexpr size_t MSLOT = (sizeof(T) * 10 * BOX + 127) / 128 * 128;
  static constexpr size_t mring = (fy + sizeof(T) * 5 * (TY + 1) * TX + 127) / 128 * 128;
  static constexpr size_t red = (mring + NMS * MSLOT + 15) / 16 * 16;
  static constexpr size_t bar = red + sizeof(double) * NWARP * NPART;
  static constexpr size_t misc = bar + 8 * (NSTAGE + NMS);
  static constexpr size_t push = (misc + 16 + 15) / 16 * 16;  // 27 PushDst (halo push of stages 1, 2)
  static constexpr size_t bytes = (push + 27 * sizeof(PushDst) + 127) / 128 * 128;
};

// stencil cell base index inside the ring: slot s, row cy, column cx (variable 0)
template <int NV, int BY>
__device__ __forceinline__ int rb(int s, int cy, int cx) {
  return (s * NV * BY + cy) * BX + cx;
}

// Ring indices of one face's stencil: b[0..3] the 4 cells along the normal (b[1] = L, b[2] = R);
// L and R neighbours +-1 along tangent 1 (lp1, lm1, rp1, rm1) and tangent 2 (lp2 ... rm2).
struct FaceIdx {
  int b[4];
  int lp1, lm1, rp1, rm1, lp2, lm2, rp2, rm2;
};

// face frames: primitive index of the normal velocity and of tangents 1 and 2 per direction
template <int D> struct Frame;
template <> struct Frame<0> { static constexpr int N = 1, T1 = 2, T2 = 3; };  // x: (u | v, w)
template <> struct Frame<1> { static constexpr int N = 2, T1 = 3, T2 = 1; };  // y: (v | w, u)
template <> struct Frame<2> { static constexpr int N = 3, T1 = 1, T2 = 2; };  // z: (w | u, v)

// x-face below box cell (cy, cx) in ring slot s; sm / sp = slots of planes k-1 / k+1
template <int NV, int BY>
__device__ __forceinline__ FaceIdx xface_idx(int s, int sm, int sp, int cy, int cx) {
  const int b = rb<NV, BY>(s, cy, cx);
  // tangent 1 = y (rows), tangent 2 = z (planes)
  return {{b - 2, b - 1, b, b + 1}, b - 1 + BX, b - 1 - BX, b + BX, b - BX,
          rb<NV, BY>(sp, cy, cx - 1), rb<NV, BY>(sm, cy, cx - 1), rb<NV, BY>(sp, cy, cx), rb<NV, BY>(sm, cy, cx)};
}
template <int NV, int BY>
__device__ __forceinline__ FaceIdx yface_idx(int s, int sm, int sp, int cy, int cx) {
  const int b = rb<NV, BY>(s, cy, cx);
  // tangent 1 = z (planes), tangent 2 = x (columns)
  return {{b - 2 * BX, b - BX, b, b + BX}, rb<NV, BY>(sp, cy - 1, cx), rb<NV, BY>(sm, cy - 1, cx),
          rb<NV, BY>(sp, cy, cx), rb<NV, BY>(sm, cy, cx), b - BX + 1, b - BX - 1, b + 1, b - 1};
}
// z-face between planes k (slot s1) and k+1 (slot s2); s0 = k-1, s3 = k+2
template <int NV, int BY>
__device__ __forceinline__ FaceIdx zface_idx(int s0, int s1, int s2, int s3, int cy, int cx) {
  const int b1 = rb<NV, BY>(s1, cy, cx), b2 = rb<NV, BY>(s2, cy, cx);
  // tangent 1 = x (columns), tangent 2 = y (rows)
  return {{rb<NV, BY>(s0, cy, cx), b1, b2, rb<NV, BY>(s3, cy, cx)}, b1 + 1, b1 - 1, b2 + 1, b2 - 1,
          b1 + BX, b1 - BX, b2 + BX, b2 - BX};
}

// the per-face arithmetic once the stencil is in registers: w[cell][frame variable].  Returns
// twice the face flux F - Fv (the assembly multiplies the differences by half the inverse cell
// sizes, which gives the same bits); K.mu = 2 mu and K.kappa = 4 kappa on this path, us = the
// sum of the two cells' velocities.
template <typename V, bool VISC>
__device__ __forceinline__ void flux_core(const V (&w)[4][5], const V* gn, V dnt1, V dnt2, V d11, V d22,
                                          const V* us, const Consts<V>& K, V* Fr) {
  V L[5], R[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) muscl(w[0][q], w[1][q], w[2][q], w[3][q], K.lim, L[q], R[q]);
  roe_frame<V, true>(L, R, K, Fr);
  if constexpr (VISC) viscous_sub_twice(gn, dnt1, dnt2, d11, d22, us, K, Fr);
}

// stencil gather of one face, then flux_core (twice the flux).  ih = inverse spacings along
// (normal, tangent 1, tangent 2), qih = a quarter of them (the tangential differences average
// two central differences of two cells: 1/4 x the sum of four differences).
template <typename T, bool VISC, int D, int BY>
__device__ __forceinline__ void face_flux(const T* __restrict__ ring, const FaceIdx& f, const T* ih, const T* qih,
                                          const Consts<T>& K, T* F) {
  constexpr int MS = BY * BX;
  using Fr_ = Frame<D>;
  constexpr int idx[5] = {0, Fr_::N, Fr_::T1, Fr_::T2, 4};
  T w[4][5];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int q = 0; q < 5; ++q) w[c][q] = ring[f.b[c] + idx[q] * MS];
  T gn[4], us[3], dnt1 = T(0), dnt2 = T(0), d11 = T(0), d22 = T(0);
  if constexpr (VISC) {
    const int L = f.b[1], R = f.b[2];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      gn[q] = (w[2][q + 1] - w[1][q + 1]) * ih[0];
      us[q] = w[1][q + 1] + w[2][q + 1];
    }
    constexpr int TH = 5 * MS, mn = Fr_::N * MS, m1 = Fr_::T1 * MS, m2 = Fr_::T2 * MS;
    gn[3] = (ring[R + TH] - ring[L + TH]) * ih[0];
    dnt1 = ((ring[f.lp1 + mn] - ring[f.lm1 + mn]) + (ring[f.rp1 + mn] - ring[f.rm1 + mn])) * qih[1];
    dnt2 = ((ring[f.lp2 + mn] - ring[f.lm2 + mn]) + (ring[f.rp2 + mn] - ring[f.rm2 + mn])) * qih[2];
    d11 = ((ring[f.lp1 + m1] - ring[f.lm1 + m1]) + (ring[f.rp1 + m1] - ring[f.rm1 + m1])) * qih[1];
    d22 = ((ring[f.lp2 + m2] - ring[f.lm2 + m2]) + (ring[f.rp2 + m2] - ring[f.rm2 + m2])) * qih[2];
  }
  T Fr[5];
  flux_core<T, VISC>(w, gn, dnt1, dnt2, d11, d22, us, K, Fr);
  F[0] = Fr[0];
  F[Fr_::N] = Fr[1];
  F[Fr_::T1] = Fr[2];
  F[Fr_::T2] = Fr[3];
  F[4] = Fr[4];
}

// tangential neighbour indices of a face as one array (lp1, lm1, rp1, rm1, lp2, lm2, rp2, rm2)
__device__ __forceinline__ const int (&tg_of(const FaceIdx& f))[8] {
  return *reinterpret_cast<const int(*)[8]>(&f.lp1);
}

// a cell's mean face vector per direction (lower and upper face), from the metric ring
template <typename T, int BY>
__device__ __forceinline__ void cell_face_means(const T* mring, int mk, int mk1, int cy, int cx, T* sb) {
  constexpr int MS = BY * BX;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    sb[x] = T(0.5) * (mring[mb<BY>(mk, cy, cx) + x * MS] + mring[mb<BY>(mk, cy, cx + 1) + x * MS]);
    sb[3 + x] = T(0.5) * (mring[mb<BY>(mk, cy, cx) + (3 + x) * MS] + mring[mb<BY>(mk, cy + 1, cx) + (3 + x) * MS]);
    sb[6 + x] = T(0.5) * (mring[mb<BY>(mk, cy, cx) + (6 + x) * MS] + mring[mb<BY>(mk1, cy, cx) + (6 + x) * MS]);
  }
}

// inverse spacings along (normal, tangent 1, tangent 2) of x-, y- and z-faces
template <typename T> struct Tri { T v[3]; };
template <typename T> __device__ __forceinline__ Tri<T> ihx3(T x, T y, T z) { return {{x, y, z}}; }
template <typename T> __device__ __forceinline__ Tri<T> ihy3(T x, T y, T z) { return {{y, z, x}}; }
template <typename T> __device__ __forceinline__ Tri<T> ihz3(T x, T y, T z) { return {{z, x, y}}; }

// spectral-radius rate of one cell: sum over directions of the convective radius (plus 4x the
// viscous one) divided by the volume, i.e. the inverse of the cell's stable step / CFL;
// s2 = ihx^2 + ihy^2 + ihz^2
template <typename T>
__device__ __forceinline__ T cell_rate(T r, T u, T v, T w, T p, const RateK<T>& RK, bool viscous, T ihx, T ihy,
                                       T ihz, T s2) {
  using O = VM<T>;
  const T ir = O::rcp(r);
  const T c2 = RK.gam * p * ir;
  const T c = c2 * O::rsqrt(c2);
  T rate = (O::ab(u) + c) * ihx + (O::ab(v) + c) * ihy + (O::ab(w) + c) * ihz;
  if (viscous) rate += RK.vf * ir * s2;
  return rate;
}

// The halo exchange folded into the stage (groups with GroupParams::push): the output of a cell
// within HALO cells of a block face is also written into the halo cells of the neighbouring
// blocks that hold its copy -- across the face, and across the edge and the corner for cells
// near two or three faces (the block diagonal reached by walking the face neighbours, in any
// order on a conforming lattice) -- the cells the halo kernel would fill from it.  No stage
// reads the halos of the field it writes, so the next launch finds them complete.
// One destination per direction (sx, sy, sz) in {-1,0,1}^3, built once per CTA for its block:
// the neighbour's output field and strides, and the index shift from this block's cell to the
// neighbour's halo cell.

template <typename T, int STAGE>
__device__ void push_table(const BlockDesc* tb, int b0, int t, PushDst* dst) {
  const int sx = t % 3 - 1, sy = (t / 3) % 3 - 1, sz = t / 9 - 1;
  int d = b0, oi = 0, oj = 0, ok = 0;
  if (sx > 0) { oi -= tb[d].g.nx; d = tb[d].nbr[1]; }
  if (sx < 0) { d = tb[d].nbr[0]; oi += tb[d].g.nx; }
  if (sy > 0) { oj -= tb[d].g.ny; d = tb[d].nbr[3]; }
  if (sy < 0) { d = tb[d].nbr[2]; oj += tb[d].g.ny; }
  if (sz > 0) { ok -= tb[d].g.nz; d = tb[d].nbr[5]; }
  if (sz < 0) { d = tb[d].nbr[4]; ok += tb[d].g.nz; }
  const BlockDesc& D = tb[d];
  PushDst e;
  if constexpr (sizeof(T) == 8) {
    e.base = D.q[STAGE % 3];
    e.field = D.g.field;
    e.plane = D.g.plane;
    e.pitch = D.g.px;
  } else {
    e.base = D.d[STAGE - 1];
    e.field = D.g.fieldf;
    e.plane = D.g.planef;
    e.pitch = D.g.pxf;
  }
  e.oi = oi; e.oj = oj; e.ok = ok;
  dst[t] = e;
}

// out of line: only cells next to a block face call it
template <typename T>
__device__ __noinline__ void push_halo(const PushDst* dst, int nx, int ny, int nz, int ci, int cj, int ck,
                                       T v0, T v1, T v2, T v3, T v4) {
  const T v[5] = {v0, v1, v2, v3, v4};
  const int lx = ci < HALO ? -1 : 0, hx = ci >= nx - HALO ? 1 : 0;
  const int ly = cj < HALO ? -1 : 0, hy = cj >= ny - HALO ? 1 : 0;
  const int lz = ck < HALO ? -1 : 0, hz = ck >= nz - HALO ? 1 : 0;
  for (int sz = lz; sz <= hz; ++sz)
    for (int sy = ly; sy <= hy; ++sy)
      for (int sx = lx; sx <= hx; ++sx) {
        const int t = (sx + 1) + 3 * (sy + 1) + 9 * (sz + 1);
        if (t == 13) continue;  // the cell itself
        const PushDst& e = dst[t];
        const long long o = (long long)(ck + e.ok + HALO) * e.plane + (long long)(cj + e.oj + HALO) * e.pitch +
                            (ci + e.oi + HALO);
        T* f = static_cast<T*>(e.base);
#pragma unroll
        for (int m = 0; m < 5; ++m) f[m * e.field + o] = v[m];
      }
}

// the path's constants from the launch parameters (formed on the host)
template <typename T> __device__ __forceinline__ const PathK<T>& path_k(const GroupParams& P);
template <> __device__ __forceinline__ const PathK<float>& path_k<float>(const GroupParams& P) { return P.pk.f; }
template <> __device__ __forceinline__ const PathK<double>& path_k<double>(const GroupParams& P) { return P.pk.d; }

// ---- the kernel ------------------------------------------------------------------------------
// One launch advances one Runge-Kutta stage of a group of blocks (a single block is a group of
// one).  STAGE 0: residual only (one block, R to P.rout); 1..3: the stages of Eqs. 4-6.
// registers: the register file is split over the SM's four sub-partitions (16K each) and warps
// are spread round-robin, so two 9-warp CTAs (5 warps on one sub-partition) allow 96 registers
// per thread on the mixed path, four 5-warp CTAs (TYV = 4) 102, one CTA of 9 or 12 warps (3 per
// sub-partition) 168 on the FP64 and curvilinear paths
// PUSH: stages 1 and 2 of a group with the halo exchange folded in (GroupParams::push); a separate
// instantiation, so kernels without it carry none of its code
template <typename T, bool VISC, int STAGE, bool CURVI, int TYV, bool PUSH = false>
__global__ void __launch_bounds__(tile_threads(TYV), (sizeof(T) == 4 && !CURVI) ? (TYV <= 4 ? 4 : 2) : 1)
    stage_kernel(const GroupParams P) {
  constexpr bool MIXED = sizeof(T) == 4;
  constexpr bool LOADD = MIXED && (STAGE == 2 || STAGE == 3);
  using PL = Plan<T, VISC, CURVI, TYV>;
  constexpr int TY = TYV, BY = PL::BY, NWARP = PL::NWARP, NT = tile_threads(TYV);
  constexpr int NMS = PL::NMS;
  constexpr int NV = PL::NV;
  constexpr int MS = BY * BX;
  using Fm = VM<T>;

  extern __shared__ __align__(128) unsigned char smem[];
  T* ring = reinterpret_cast<T*>(smem + PL::ring);
  T* fx = reinterpret_cast<T*>(smem + PL::fx);
  T* fy = reinterpret_cast<T*>(smem + PL::fy);
  T* mring = reinterpret_cast<T*>(smem + PL::mring);
  double* red = reinterpret_cast<double*>(smem + PL::red);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + PL::bar);
  int* sabort = reinterpret_cast<int*>(smem + PL::misc);
  int* slast = sabort + 1;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const Physics& ph = P.ph;
  const PathK<T>& PK = path_k<T>(P);
  Consts<T> K;
  K.gm1 = PK.gm1;
  K.ggm1 = PK.ggm1;
  K.eps = PK.eps;
  // the Cartesian face path returns twice the flux (flux_core): 2 mu, 4 kappa there
  K.mu = VISC ? (CURVI ? PK.mu : PK.mu + PK.mu) : T(0);
  K.kappa = VISC ? (CURVI ? PK.kappa : T(4) * PK.kappa) : T(0);
  K.lim = ph.limiter;
  const T gm1 = PK.gm1;
  const RateK<T> RK = {PK.gam, PK.vf};
  const T cflT = PK.cfl;

  if (tid == 0) {
    for (int s = 0; s < NSTAGE + NMS; ++s) mbar_init(&bar[s], 1);
    fence_barrier_init();
    *sabort = 0;
  }
  __syncthreads();

  const double dt = (STAGE == 0) ? 0.0 : P.gctrl->dt;
  const T dtT = T(dt);
  unsigned phase_bits = 0;   // parity of each staging slot (uniform across the CTA)
  unsigned pending = 0;      // slots with a copy in flight (meaningful in thread 0)
  unsigned mphase = 0;       // parity of each metric slot
  unsigned mpending = 0;     // metric slots with a copy in flight (thread 0)
  bool bad = false;          // non-physical value met by this thread
  // per-thread sums for the current block: R^2 (stage 1), max rate (stage 3)
  double nacc[5] = {0, 0, 0, 0, 0};  // FP64 sums of R^2 on both paths
  T rate_max = T(0);

  // the block of this CTA and the CTA's contiguous share of its tile-planes
  int bsel;
  {
    int lo = 0, hi = P.nblocks - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (P.table[mid].cta0 <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    bsel = lo;
  }
  const BlockDesc* D = P.table + bsel;
  PushDst* pushdst = reinterpret_cast<PushDst*>(smem + PL::push);
  if constexpr (PUSH && (STAGE == 1 || STAGE == 2)) {
    if (tid < 27) push_table<T, STAGE>(P.table, bsel, tid, pushdst);
    __syncthreads();
  }
  const int lcta = (int)blockIdx.x - D->cta0, nctas = D->ctas;
  const long long W = D->units;
  const long long u_begin = (long long)lcta * W / nctas;
  const long long u_end = (long long)(lcta + 1) * W / nctas;
  constexpr unsigned QBYTES = 5u * MS * sizeof(T);
  constexpr unsigned DBYTES = 5u * MS * sizeof(float);

  // this CTA's sums -> partial slot blockIdx.x; all threads call it together
  auto flush = [&]() {
    if constexpr (STAGE == 1 || STAGE == 3) {
      double part[6];
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        part[m] = nacc[m];
        nacc[m] = 0.0;
      }
      part[5] = double(rate_max);
      rate_max = T(0);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int m = 0; m < 5; ++m) part[m] += __shfl_xor_sync(0xffffffffu, part[m], off);
        part[5] = fmax(part[5], __shfl_xor_sync(0xffffffffu, part[5], off));
      }
      __syncthreads();
      if (lane == 0)
        for (int m = 0; m < 6; ++m) red[warp * NPART + m] = part[m];
      __syncthreads();
      if (tid == 0) {
        double sum[6] = {0, 0, 0, 0, 0, 0};
        for (int w = 0; w < NWARP; ++w) {
          for (int m = 0; m < 5; ++m) sum[m] += red[w * NPART + m];
          sum[5] = fmax(sum[5], red[w * NPART + 5]);
        }
        for (int m = 0; m < 6; ++m) P.partial[(size_t)blockIdx.x * NPART + m] = sum[m];
      }
    }
  };

  // ring slot of plane kp (kp >= -2)
  auto rslot = [](int kp) { return kp & 3; };
  const bool owner = warp < TY;  // warps 0..TY-1 own row `warp` of the tile; warp TY helps
  const Geometry g = D->g;

  for (long long u = u_begin; u < u_end;) {
    const int nz = g.nz;
    const long long tile = u / nz;
    const int k0 = (int)(u - tile * nz);
    const int k1 = (int)min((long long)nz, (long long)k0 + (u_end - u));
    u += k1 - k0;
    const int tix = (int)(tile % D->ntx), tiy = (int)(tile / D->ntx);
    const int x0 = tix * TX, y0 = tiy * TY;  // storage coordinates of the box origin
    const int last_plane = k1 + 1;
    // arrays of this stage
    const CUtensorMap* tmq;
    const CUtensorMap* tmd = &D->td[0];
    const double *qs = nullptr, *qn = nullptr;
    double* qout = nullptr;
    float *sout = nullptr, *dout = nullptr;
    const float* dprev = nullptr;
    if constexpr (!MIXED) {
      const int in = STAGE == 0 ? 0 : STAGE - 1;
      tmq = &D->tq[in];
      qs = D->q[in];
      qn = D->q[0];
      qout = D->q[STAGE % 3];
    } else {
      const int c = P.cur;
      tmq = &D->tq[c];
      qn = D->q[c];
      if (STAGE == 1) dout = D->d[0];
      if (STAGE == 2) { dprev = D->d[0]; dout = D->d[1]; tmd = &D->td[0]; }
      if (STAGE == 3) { dprev = D->d[1]; qout = D->q[1 - c]; sout = D->sh[1 - c]; tmd = &D->td[1]; }
    }
    const T hx = MIXED ? T(D->ihxf) : T(D->ihx), hy = MIXED ? T(D->ihyf) : T(D->ihy),
            hz = MIXED ? T(D->ihzf) : T(D->ihz);  // inverse cell sizes
    const T hs2 = hx * hx + hy * hy + hz * hz;
    // a quarter of the inverse cell sizes (tangential face derivatives) and half of them (the
    // assembly of the doubled Cartesian face fluxes); products by powers of two are exact
    const T qhx = T(0.25) * hx, qhy = T(0.25) * hy, qhz = T(0.25) * hz;
    const T hx2 = T(0.5) * hx, hy2 = T(0.5) * hy, hz2 = T(0.5) * hz;

    auto request = [&](int kp) {  // thread 0 only
      const int s = (kp + 2) & (NSTAGE - 1);
      fence_proxy_async();
      mbar_expect_tx(&bar[s], QBYTES + (LOADD ? DBYTES : 0u));
      tma_load_4d(smem + PL::stq + s * PL::QSLOT, tmq, &bar[s], x0, y0, kp + HALO, 0);
      if (LOADD) tma_load_4d(smem + PL::std_ + s * PL::DSLOT, tmd, &bar[s], x0, y0, kp + HALO, 0);
      pending |= 1u << s;
    };
    // wait for plane kp, convert it into ring slot kp & 3, then refill the staging slot
    auto consume = [&](int kp) -> bool {
      const int s = (kp + 2) & (NSTAGE - 1);
      const bool ok = mbar_wait_bounded(&bar[s], (phase_bits >> s) & 1u);
      if (!ok) atomicOr(sabort, 1);
      phase_bits ^= 1u << s;
      const T* sq = reinterpret_cast<const T*>(smem + PL::stq + s * PL::QSLOT);
      const float* sd = reinterpret_cast<const float*>(smem + PL::std_ + s * PL::DSLOT);
      T* rs = ring + (size_t)rslot(kp) * NV * MS;
      for (int c = tid; c < MS; c += NT) {
        const int cy = c / BX, cx = c - cy * BX;
        T q[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          if constexpr (LOADD) q[v] = sq[v * MS + c] + sd[v * MS + c];
          else q[v] = sq[v * MS + c];
        }
        const bool valid = (x0 - HALO + cx < g.nx + HALO) && (y0 - HALO + cy < g.ny + HALO);
        T r = q[0];
        const T ir = Fm::rcp(r);
        const T uu = q[1] * ir, vv = q[2] * ir, ww = q[3] * ir;
        T p = gm1 * (q[4] - T(0.5) * r * (uu * uu + vv * vv + ww * ww));
        if (valid && !(r > T(0) && p > T(0))) bad = true;
        const bool fill = !valid || !(r > T(0) && p > T(0));
        rs[0 * MS + c] = fill ? T(1) : r;
        rs[1 * MS + c] = fill ? T(0) : uu;
        rs[2 * MS + c] = fill ? T(0) : vv;
        rs[3 * MS + c] = fill ? T(0) : ww;
        rs[4 * MS + c] = fill ? T(1) : p;
        if (VISC) rs[5 * MS + c] = fill ? T(1) : p * ir;
      }
      __syncthreads();
      if (tid == 0) {
        pending &= ~(1u << s);
        if (kp + NSTAGE <= last_plane && *sabort == 0) request(kp + NSTAGE);
      }
      return *sabort == 0;
    };

    // metric planes (curvilinear): plane kp in slot (kp + 1) % NMS; iteration k reads k and k+1
    int m_req = k0 - 2, m_wait = k0 - 2;
    auto mslot = [](int kp) { return NMS ? (kp + 1) % (NMS ? NMS : 1) : 0; };
    auto mrequest_upto = [&](int upto) {  // thread 0 only
      if constexpr (CURVI) {
        upto = min(upto, k1);
        while (m_req < upto) {
          ++m_req;
          const int s = mslot(m_req);
          fence_proxy_async();
          mbar_expect_tx(&bar[NSTAGE + s], 10u * MS * sizeof(T));
          tma_load_4d(smem + PL::mring + s * PL::MSLOT, &D->tm, &bar[NSTAGE + s], x0, y0, m_req + HALO, 0);
          mpending |= 1u << s;
        }
      }
    };
    auto mwait_upto = [&](int upto) {  // all threads
      if constexpr (CURVI) {
        while (m_wait < upto) {
          ++m_wait;
          const int s = mslot(m_wait);
          if (!mbar_wait_bounded(&bar[NSTAGE + s], (mphase >> s) & 1u)) atomicOr(sabort, 1);
          mphase ^= 1u << s;
        }
      }
    };

    if (tid == 0) {
      tensormap_acquire(tmq);
      if (LOADD) tensormap_acquire(tmd);
      if (CURVI) tensormap_acquire(&D->tm);
      request(k0 - 2);
      request(k0 - 1);
      mrequest_upto(k0 - 2 + NMS);
    }
    bool ok = true;
    for (int kp = k0 - 2; kp <= k0 + 1 && ok; ++kp) ok = consume(kp);
    if (!ok) break;
    mwait_upto(k0);
    if (*sabort) break;

    // owning warps: cell (lane, warp) of the tile
    const int ci = x0 + lane, cj = y0 + warp;  // interior coordinates of the owned cell
    const bool live = owner && ci < g.nx && cj < g.ny;
    // rows of a ragged tile past the block's edge: the first one still computes its lower y-face
    // (the upper face of the block's last row), the others nothing (warp-uniform skips)
    const bool row_in = owner && cj < g.ny, row_edge = owner && cj == g.ny;
    // the helper's upper faces of the tile are read only where the tile does not end past the block
    const bool up_y = y0 + TY <= g.ny;
    const bool up_x = lane < TY && y0 + lane < g.ny && x0 + TX <= g.nx;
    const int ocy = warp + HALO, ocx = lane + HALO;
    T fzl[5], fzu[5];
    if (row_in) {
      const FaceIdx iz = zface_idx<NV, BY>(rslot(k0 - 2), rslot(k0 - 1), rslot(k0), rslot(k0 + 1), ocy, ocx);
      if constexpr (CURVI)
        face_flux_curvi<T, VISC, BY>(ring, mring, NV * MS, iz.b, tg_of(iz), zface_met<BY>(mslot(k0 - 1), mslot(k0), ocy, ocx),
                                 K, fzl);
      else
        face_flux<T, VISC, 2, BY>(ring, iz, ihz3(hx, hy, hz).v, ihz3(qhx, qhy, qhz).v, K, fzl);
    }
    __syncthreads();  // the first consume below overwrites plane k0-2, read by the z-face above

    for (int k = k0; k < k1; ++k) {
      if (!consume(k + 2)) { ok = false; break; }
      if (tid == 0) mrequest_upto(k - 1 + NMS);  // the slot of plane k-1 is free
      mwait_upto(k + 1);
      // per-cell inputs of the update (L2-resident planes), loaded before the face work
      double qs_[5], qn_[5];
      float dp_[5];
      T dtc = dtT;  // this cell's time step (its own one under local time stepping)
      if (live) {
        const long long o = gidx(g, ci, cj, k), of = gidxf(g, ci, cj, k);
        if constexpr (STAGE >= 1 && !VISC)  // local time steps: inviscid blocks only
          if (ph.local_dt) dtc = __ldg(static_cast<const T*>(D->dtl) + (MIXED ? of : o));
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          if constexpr (!MIXED && STAGE >= 1) qs_[v] = __ldg(qs + v * g.field + o);
          if constexpr (!MIXED && STAGE >= 2) qn_[v] = __ldg(qn + v * g.field + o);
          if constexpr (MIXED && STAGE == 3) qn_[v] = __ldg(qn + v * g.field + o);
          if constexpr (LOADD) dp_[v] = __ldg(dprev + v * g.fieldf + of);
        }
      }
      const int sk = rslot(k), sm = rslot(k - 1), sp = rslot(k + 1), s2 = rslot(k + 2);
      const int mk = mslot(k), mk1 = mslot(k + 1);
      if (owner) {
        T Fa[5], Fb[5];
        const FaceIdx ix = xface_idx<NV, BY>(sk, sm, sp, ocy, ocx), iy = yface_idx<NV, BY>(sk, sm, sp, ocy, ocx);
        if (row_in) {
          if constexpr (CURVI)
            face_flux_curvi<T, VISC, BY>(ring, mring, NV * MS, ix.b, tg_of(ix), xface_met<BY>(mk, mk1, ocy, ocx), K, Fa);
          else
            face_flux<T, VISC, 0, BY>(ring, ix, ihx3(hx, hy, hz).v, ihx3(qhx, qhy, qhz).v, K, Fa);
#pragma unroll
          for (int m = 0; m < 5; ++m) fx[(m * TY + warp) * (TX + 1) + lane] = Fa[m];
        }
        if (row_in || row_edge) {
          if constexpr (CURVI)
            face_flux_curvi<T, VISC, BY>(ring, mring, NV * MS, iy.b, tg_of(iy), yface_met<BY>(mk, mk1, ocy, ocx), K, Fb);
          else
            face_flux<T, VISC, 1, BY>(ring, iy, ihy3(hx, hy, hz).v, ihy3(qhx, qhy, qhz).v, K, Fb);
#pragma unroll
          for (int m = 0; m < 5; ++m) fy[(m * (TY + 1) + warp) * TX + lane] = Fb[m];
        }
        if (row_in) {
          const FaceIdx iz = zface_idx<NV, BY>(sm, sk, sp, s2, ocy, ocx);
          if constexpr (CURVI)
            face_flux_curvi<T, VISC, BY>(ring, mring, NV * MS, iz.b, tg_of(iz), zface_met<BY>(mk, mk1, ocy, ocx), K, fzu);
          else
            face_flux<T, VISC, 2, BY>(ring, iz, ihz3(hx, hy, hz).v, ihz3(qhx, qhy, qhz).v, K, fzu);
        }
      } else {
        // the tile's upper y-faces (all lanes) and upper x-faces (lanes < TY)
        T Fa[5], Fb[5];
        const FaceIdx iy = yface_idx<NV, BY>(sk, sm, sp, TY + HALO, lane + HALO);
        const FaceIdx ix = xface_idx<NV, BY>(sk, sm, sp, (lane % TY) + HALO, TX + HALO);
        if (up_y) {
          if constexpr (CURVI)
            face_flux_curvi<T, VISC, BY>(ring, mring, NV * MS, iy.b, tg_of(iy),
                                     yface_met<BY>(mk, mk1, TY + HALO, lane + HALO), K, Fa);
          else
            face_flux<T, VISC, 1, BY>(ring, iy, ihy3(hx, hy, hz).v, ihy3(qhx, qhy, qhz).v, K, Fa);
#pragma unroll
          for (int m = 0; m < 5; ++m) fy[(m * (TY + 1) + TY) * TX + lane] = Fa[m];
        }
        if (up_x) {
          if constexpr (CURVI)
            face_flux_curvi<T, VISC, BY>(ring, mring, NV * MS, ix.b, tg_of(ix),
                                     xface_met<BY>(mk, mk1, lane + HALO, TX + HALO), K, Fb);
          else
            face_flux<T, VISC, 0, BY>(ring, ix, ihx3(hx, hy, hz).v, ihx3(qhx, qhy, qhz).v, K, Fb);
#pragma unroll
          for (int m = 0; m < 5; ++m) fx[(m * TY + lane) * (TX + 1) + TX] = Fb[m];
        }
      }
      __syncthreads();
      if (live) {
        T R[5];
#pragma unroll
        for (int m = 0; m < 5; ++m) {
          const T ddx = fx[(m * TY + warp) * (TX + 1) + lane + 1] - fx[(m * TY + warp) * (TX + 1) + lane];
          const T ddy = fy[(m * (TY + 1) + warp + 1) * TX + lane] - fy[(m * (TY + 1) + warp) * TX + lane];
          if constexpr (CURVI)
            R[m] = (ddx + ddy) + (fzu[m] - fzl[m]);  // face fluxes carry |S|; divided by V below
          else
            R[m] = (ddx * hx2 + ddy * hy2) + (fzu[m] - fzl[m]) * hz2;  // doubled fluxes
        }
        if constexpr (CURVI) {
          const T iv = Fm::rcp(mring[mb<BY>(mk, ocy, ocx) + 9 * MS]);
#pragma unroll
          for (int m = 0; m < 5; ++m) R[m] = R[m] * iv;
        }
        const long long o = gidx(g, ci, cj, k), of = gidxf(g, ci, cj, k);
        if constexpr (STAGE == 0) {
          const long long oc = ((long long)k * g.ny + cj) * g.nx + ci;
          const long long n = (long long)g.nx * g.ny * g.nz;
#pragma unroll
          for (int m = 0; m < 5; ++m) P.rout[m * n + oc] = double(R[m]);
        } else if constexpr (!MIXED) {
          double out[5];
#pragma unroll
          for (int m = 0; m < 5; ++m) {
            const double adv = qs_[m] - double(dtc) * double(R[m]);
            if constexpr (STAGE == 1) out[m] = adv;
            else if constexpr (STAGE == 2) out[m] = 0.75 * qn_[m] + 0.25 * adv;
            else out[m] = fma(2.0 / 3.0, adv, (1.0 / 3.0) * qn_[m]);  // an FP64 division costs ~7 FMAs here
            qout[m * g.field + o] = out[m];
          }
          if constexpr (PUSH && (STAGE == 1 || STAGE == 2))
            if (ci < HALO || cj < HALO || k < HALO || ci >= g.nx - HALO || cj >= g.ny - HALO || k >= g.nz - HALO)
              push_halo<double>(pushdst, g.nx, g.ny, g.nz, ci, cj, k, out[0], out[1], out[2], out[3], out[4]);
          if constexpr (STAGE == 3) {
            const double ir = VM<double>::rcp(out[0]);
            const double uu = out[1] * ir, vv = out[2] * ir, ww = out[3] * ir;
            const double pp = double(gm1) * (out[4] - 0.5 * out[0] * (uu * uu + vv * vv + ww * ww));
            if (!(out[0] > 0.0 && pp > 0.0)) bad = true;
            double rate;
            if constexpr (CURVI) {
              T sb[9];
              cell_face_means<T, BY>(mring, mk, mk1, ocy, ocx, sb);
              rate = cell_rate_curvi<double>(out[0], uu, vv, ww, pp, sb, mring[mb<BY>(mk, ocy, ocx) + 9 * MS], RK,
                                             ph.viscous);
            } else {
              rate = cell_rate<double>(out[0], uu, vv, ww, pp, RK, ph.viscous, hx, hy, hz, hs2);
            }
            rate_max = fmax(rate_max, T(rate));
            if constexpr (!VISC)
              if (ph.local_dt) static_cast<double*>(D->dtl)[o] = ph.cfl * VM<double>::rcp(rate);
          }
        } else {
          float inc[5];
#pragma unroll
          for (int m = 0; m < 5; ++m) inc[m] = -float(dtc) * float(R[m]);
          if constexpr (STAGE == 1 || STAGE == 2) {
            float dv[5];
#pragma unroll
            for (int m = 0; m < 5; ++m) {
              dv[m] = STAGE == 1 ? inc[m] : 0.25f * (dp_[m] + inc[m]);
              dout[m * g.fieldf + of] = dv[m];
            }
            if (PUSH && (ci < HALO || cj < HALO || k < HALO || ci >= g.nx - HALO || cj >= g.ny - HALO ||
                         k >= g.nz - HALO))
              push_halo<float>(pushdst, g.nx, g.ny, g.nz, ci, cj, k, dv[0], dv[1], dv[2], dv[3], dv[4]);
          } else {
            float qf[5];
#pragma unroll
            for (int m = 0; m < 5; ++m) {
              const float d = (2.0f / 3.0f) * (dp_[m] + inc[m]);
              // hardware conversions (the FP64 pipe is otherwise idle here; same rounding as the
              // integer-pipe forms, measured 0.5% faster per launch on the 256^3 vortex)
              const double qnew = qn_[m] + double(d);
              qout[m * g.field + o] = qnew;
              qf[m] = float(qnew);
              sout[m * g.fieldf + of] = qf[m];
            }
            const float ir = VM<float>::rcp(qf[0]);
            const float uu = qf[1] * ir, vv = qf[2] * ir, ww = qf[3] * ir;
            const float pp = gm1 * (qf[4] - 0.5f * qf[0] * (uu * uu + vv * vv + ww * ww));
            if (!(qf[0] > 0.0f && pp > 0.0f)) bad = true;
            float rate;
            if constexpr (CURVI) {
              T sb[9];
              cell_face_means<T, BY>(mring, mk, mk1, ocy, ocx, sb);
              rate = cell_rate_curvi<float>(qf[0], uu, vv, ww, pp, sb, mring[mb<BY>(mk, ocy, ocx) + 9 * MS], RK,
                                            ph.viscous);
            } else {
              rate = cell_rate<float>(qf[0], uu, vv, ww, pp, RK, ph.viscous, hx, hy, hz, hs2);
            }
            rate_max = fmax(rate_max, T(rate));
            if constexpr (!VISC)
              if (ph.local_dt) static_cast<float*>(D->dtl)[of] = cflT / rate;
          }
        }
        if constexpr (STAGE == 1) {
          // the residual norm is reduced in FP64 on both paths: an FP32 residual's square is exact
          // in FP64 (24-bit significand), so the mixed path's sums round only in the FP64 additions;
          // it is widened on the integer pipe, leaving one FP64 operation per variable
#pragma unroll
          for (int m = 0; m < 5; ++m) {
            if constexpr (MIXED) {
              const double r = f32_to_f64_bits(float(R[m]));
              nacc[m] = fma(r, r, nacc[m]);
            } else {
              nacc[m] = fma(double(R[m]), double(R[m]), nacc[m]);
            }
          }
        }
      }
#pragma unroll
      for (int m = 0; m < 5; ++m) fzl[m] = fzu[m];
    }
    if (!ok) break;
  }

  // abort path: drain copies still in flight (bounded), flag the timeout
  if (*sabort) {
    if (tid == 0) {
      for (int s = 0; s < NSTAGE; ++s)
        if (pending & (1u << s)) mbar_wait_bounded(&bar[s], (phase_bits >> s) & 1u);
      for (int s = 0; s < NMS; ++s)
        if (mpending & (1u << s)) mbar_wait_bounded(&bar[NSTAGE + s], (mphase >> s) & 1u);
      atomicOr(&D->ctrl->flag, FLAG_TIMEOUT);
    }
  }
  if (bad) atomicOr(&D->ctrl->flag, FLAG_NONPHYSICAL);

  if constexpr (STAGE == 1 || STAGE == 3) {
    flush();
    // the last CTA to finish reduces, per block, the slots of the CTAs that worked on it (in CTA
    // order: deterministic), and for stage 3 takes the group's time step from the largest rate
    if (tid == 0) {
      __threadfence();
      const unsigned prev = atomicAdd(&P.gctrl->counter, 1u);
      *slast = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!*slast) return;
    __threadfence();
    // every warp of the last CTA folds blocks warp, warp + NWARP, ... (a group may hold many
    // blocks: one warp walking all of them serially left the SMs idle behind it)
    double wmax = 0.0;
    for (int b = warp; b < P.nblocks; b += NWARP) {
      const BlockDesc* Db = P.table + b;
      double s[6] = {0, 0, 0, 0, 0, 0};
      for (int c = lane; c < Db->ctas; c += 32) {
        const double* src = P.partial + (size_t)(Db->cta0 + c) * NPART;
        for (int m = 0; m < 5; ++m) s[m] += __ldcg(src + m);
        s[5] = fmax(s[5], __ldcg(src + 5));
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int m = 0; m < 5; ++m) s[m] += __shfl_xor_sync(0xffffffffu, s[m], off);
        s[5] = fmax(s[5], __shfl_xor_sync(0xffffffffu, s[5], off));
      }
      wmax = fmax(wmax, s[5]);
      if (lane == 0) {
        const double n = (double)Db->g.nx * Db->g.ny * Db->g.nz;
        if (STAGE == 1)
          for (int m = 0; m < 5; ++m) Db->ctrl->norms[m] = sqrt(s[m] / n);
        if (STAGE == 3) Db->ctrl->rate = s[5];
      }
    }
    if constexpr (STAGE == 3) {
      if (lane == 0) red[warp] = wmax;
      __syncthreads();
      double gmax = 0.0;
      for (int w = 0; w < NWARP; ++w) gmax = fmax(gmax, red[w]);
      const double dtn = ph.cfl / gmax;
      for (int b = tid; b < P.nblocks; b += NT) P.table[b].ctrl->dt = dtn;
      if (tid == 0) {
        P.gctrl->rate = gmax;
        P.gctrl->dt = dtn;
      }
    }
    if (tid == 0) {
      P.gctrl->counter = 0u;
    }
  }
}

}  // namespace gbcfd
