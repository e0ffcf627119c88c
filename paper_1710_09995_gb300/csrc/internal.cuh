// internal.cuh -- data layout, kernel parameter blocks and shared device helpers of the
// gbcfd library (not part of the C ABI).
//
// Layout in HBM (per block, carved from caller memory, every array 256-byte aligned):
//   fields are SoA with a 2-cell halo: a[v][k+2][j+2][x], x = i + 2, row pitch padded to
//   128 bytes (16 doubles / 32 floats), so a TMA box starting at interior column 32*t - 2
//   starts at storage column 32*t.
//   FP64 path:  Qn (f64) and stage states Q1, Q2 (f64).  Stage 3 writes Q^{n+1} over Qn (it
//               reads Qn only at its own cell).
//   mixed path: Q^n in a ping-pong pair QA/QB (f64), its f32 rounding S^n in a ping-pong pair
//               SA/SB (what the flux stencils read), and stage increments D1, D2 (f32):
//               Q1 = Sn + D1,  Q2 = Sn + D2,  D1 = -dt R(Sn),  D2 = (D1 - dt R(Q1)) / 4,
//               Q^{n+1} = Qn + 2/3 (D2 - dt R(Q2)) in f64, S^{n+1} = f32(Q^{n+1})
//               -- algebraically Eqs. 4-6.
//   metrics (curvilinear only): M[10][..] = S_xi(3), S_eta(3), S_zeta(3), V, f64 (f32 copy for
//               the mixed path), the lower-face area vectors of each cell.
//   control:    DevCtrl (time step, norms, flag, counter) + per-CTA partials.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gbcfd {

constexpr int HALO = 2;
constexpr int TX = 32;        // tile width (cells, x) = one warp
constexpr int BX = TX + 2 * HALO; // staged box width
// Tile height (cells, y) = the number of cell-owning warps; one more helper warp computes the
// tile's upper x and y faces.  The stage kernel is compiled for a few heights (the group tuner
// chooses among them); single blocks use TY_DEFAULT.
constexpr int TY_DEFAULT = 8;
constexpr int TY_ALT_F64 = 11;  // FP64 Euler: 12 warps = 3 per sub-partition, as many as 168 registers allow
constexpr int TY_ALT_F32 = 4;   // mixed Euler: 5 warps, four CTAs per SM
__host__ __device__ constexpr int tile_warps(int ty) { return ty + 1; }
__host__ __device__ constexpr int tile_threads(int ty) { return 32 * (ty + 1); }
__host__ __device__ constexpr int box_rows(int ty) { return ty + 2 * HALO; }  // staged box height
constexpr int NSTAGE = 2;     // TMA staging slots (prefetch distance 2 planes)
constexpr int NRING = 4;      // primitive planes kept: k-1, k, k+1, k+2
constexpr int MAX_GROUP = 128; // blocks per grouped launch (halo exchange, time-step minimum)

// device flags (DevCtrl::flag bits)
constexpr int FLAG_NONPHYSICAL = 1;
constexpr int FLAG_TIMEOUT = 2;

struct DevCtrl {
  double dt;          // time step of the next stage 1
  double norms[5];    // RMS of R(Q^n) from the last stage 1
  double rate;        // max over cells of sum of spectral radii / V (from the last stage 3)
  unsigned int counter; // CTAs finished in the current launch (last one reduces, resets to 0)
  int flag;           // FLAG_* bits, cleared by the host when read
  double pad[6];
};

// partial results per CTA: [0..4] sums of R^2 (stage 1), [5] max rate (stage 3)
constexpr int NPART = 8;

struct Geometry {
  int nx, ny, nz;
  int px, pxf;                 // row pitch in f64 / f32 elements
  long long plane, planef;     // elements per k-plane (f64 / f32)
  long long field, fieldf;     // elements per variable (f64 / f32)
};

__host__ __device__ inline long long gidx(const Geometry& g, int i, int j, int k) {
  return ((long long)(k + HALO) * (g.ny + 2 * HALO) + (j + HALO)) * g.px + (i + HALO);
}
__host__ __device__ inline long long gidxf(const Geometry& g, int i, int j, int k) {
  return ((long long)(k + HALO) * (g.ny + 2 * HALO) + (j + HALO)) * g.pxf + (i + HALO);
}

struct Physics {
  double gamma, mu, Pr, cfl, eps;
  double ihx, ihy, ihz;  // 1 / cell size (Cartesian grids)
  int viscous, limiter;
  int local_dt;          // 1: every cell advances with its own CFL step (BlockDesc::dtl)
};

// the constants the stage kernel uses, formed on the host in both precisions: the FP64 pipe is
// slow on this part, so an FP32 kernel must not convert or divide doubles when it re-forms a
// constant it could not keep in a register
template <typename T> struct PathK {
  T gm1, ggm1, eps, mu, kappa;  // gamma - 1, gamma/(gamma - 1), entropy fix, viscosity, mu gamma/((gamma-1) Pr)
  T gam, vf, cfl;               // gamma, 4 max(4/3, gamma/Pr) mu (viscous rate), CFL number
};
struct PathConsts {
  PathK<float> f;
  PathK<double> d;
};

// ---- one block as the stage kernel sees it (device-resident descriptor table) --------------
// The TMA descriptors live in global memory (written by the host before any launch that reads
// them); the kernel selects the arrays of a stage from `stage` and the mixed path's parity `cur`.
struct BlockDesc {
  CUtensorMap tq[3];   // FP64: Qn, Q1, Q2 (stage inputs).  mixed: shadows SA, SB ([2] unused)
  CUtensorMap td[2];   // mixed: D1, D2
  CUtensorMap tm;      // metric planes (curvilinear)
  Geometry g;
  double ihx, ihy, ihz;      // 1 / cell size (Cartesian)
  float ihxf, ihyf, ihzf;    // the same in FP32 (mixed path)
  double* q[3];              // FP64: Qn, Q1, Q2.  mixed: QA, QB
  float* sh[2];              // mixed: shadows
  float* d[2];               // mixed: increments
  DevCtrl* ctrl;
  int ntx, nty;              // tiles along x and y (tile height: the launch's kernel)
  long long units;           // work units (tile-planes) = ntx * nty * nz
  int cta0, ctas;            // the CTAs of a group launch that work on this block
  void* dtl;                 // local time steps, one padded field (f64 FP64 path, f32 mixed)
  int nbr[6];                // group index of the neighbour across each face (-x +x -y +y -z +z), -1 if none
  long long pad_;
};

// parameters of one stage launch over a group of blocks.  The grid is split between the blocks
// (block b owns CTAs cta0 .. cta0 + ctas - 1, about in proportion to its work), so each CTA works
// on one block and its partial sums go to slot blockIdx.x.
struct GroupParams {
  const BlockDesc* table;    // nblocks descriptors
  int nblocks;
  int cur;                   // mixed path: which of QA/QB, SA/SB holds Q^n
  Physics ph;                // shared physics (gamma, mu, Pr, cfl, eps, viscous, limiter)
  PathConsts pk;             // its constants in both precisions
  int push;                  // 1: stages 1 and 2 also write their output into the neighbours' halo
                             // cells (conforming periodic block lattices; no halo launch before
                             // stages 2 and 3)
  DevCtrl* gctrl;            // group control: counter, time step (read at stage start)
  double* partial;           // [gridDim.x * NPART]
  double* rout;              // residual mode (one block): compact R[5][nz][ny][nx]
};

// ---- boundary ghost cells of one block, one direction per launch ------------------------------
enum BcKind { BC_NONE = 0, BC_SLIP_WALL = 1, BC_FARFIELD = 2 };
enum BcMode { BC_F64 = 0, BC_F32 = 1, BC_F32_INC = 2 };
struct BcBlock {
  Geometry g;
  int kind[6];          // per face -x, +x, -y, +y, -z, +z
  double inf[5];        // free stream (rho, u, v, w, p)
  double gamma;
  int dim;              // the direction this launch fills
  int mode;             // BC_F64: f64 state; BC_F32: f32 state; BC_F32_INC: f32 increment over `shadow`
  void* field;
  const float* shadow;  // BC_F32_INC: the f32 state the increment is added to
  const void* metrics;  // curvilinear metrics (f64 on the FP64 path, f32 mixed) or null (Cartesian)
};

// ---- block group descriptors for halo exchange ----------------------------------------------
struct HaloBlock {
  char* base[1];       // field base pointer (the field being exchanged)
  int nx, ny, nz, pitch;
  int nbr[6];          // group index of the neighbour across each face, -1 if none
  long long first;     // prefix sum of halo cells before this block
};
struct HaloGroup {
  HaloBlock b[MAX_GROUP];
  int n;
  int nvar;
  int elem;            // element size in bytes (8 or 4)
  long long total;     // halo cells over all blocks
};

// ---- small device helpers ------------------------------------------------------------------
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

}  // namespace gbcfd
