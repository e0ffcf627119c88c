// launch.h -- host-side launchers of the gbcfd kernels (internal, not part of the C ABI)
#pragma once
#include <string>

#include "gbcfd.h"
#include "internal.cuh"

namespace gbcfd {

// record an error for gbcfd_last_error() on this host thread and return `code`
int set_error(int code, const std::string& msg);

// fused stage kernel over a group of blocks; precision GBCFD_FP64 / GBCFD_MIXED, stage 0 = residual;
// ty = the tile height the launch's descriptors were written for (TY_DEFAULT, or the path's
// second height on Cartesian Euler blocks)
cudaError_t launch_stage(int precision, int viscous, int curvi, int stage, const GroupParams& P, int grid,
                         cudaStream_t s, int ty = TY_DEFAULT);
// the tile heights the stage kernel is compiled for on a path (TY_DEFAULT first); returns the count
int stage_tiles(int precision, int viscous, int curvi, int* ty);
// CTAs per SM of the stage kernel for a tile height
int stage_occupancy_tile(int precision, int viscous, int curvi, int ty);
cudaError_t stage_prepare_tile(int precision, int viscous, int curvi, int ty);
cudaError_t launch_stage_f64_alt(int stage, const GroupParams& P, int grid, cudaStream_t s);
cudaError_t launch_stage_f32_alt(int stage, const GroupParams& P, int grid, cudaStream_t s);
cudaError_t stage_prepare_f64_alt();
cudaError_t stage_prepare_f32_alt();
int stage_occupancy_f64_alt();
int stage_occupancy_f32_alt();
// stages 1 and 2 with the halo exchange folded in (Cartesian Euler groups, both tile heights)
cudaError_t launch_stage_f64_push(int stage, int ty, const GroupParams& P, int grid, cudaStream_t s);
cudaError_t launch_stage_f32_push(int stage, int ty, const GroupParams& P, int grid, cudaStream_t s);
cudaError_t stage_prepare_f64_push(int ty);
cudaError_t stage_prepare_f32_push(int ty);
cudaError_t launch_stage_f64(int viscous, int stage, const GroupParams& P, int grid, cudaStream_t s);
cudaError_t launch_stage_f64c(int viscous, int stage, const GroupParams& P, int grid, cudaStream_t s);
cudaError_t launch_stage_f32(int viscous, int stage, const GroupParams& P, int grid, cudaStream_t s);
cudaError_t launch_stage_f32c(int viscous, int stage, const GroupParams& P, int grid, cudaStream_t s);
cudaError_t stage_prepare_f64(int viscous);
cudaError_t stage_prepare_f64c(int viscous);
cudaError_t stage_prepare_f32(int viscous);
cudaError_t stage_prepare_f32c(int viscous);
int stage_occupancy_f64(int viscous);
int stage_occupancy_f64c(int viscous);
int stage_occupancy_f32(int viscous);
int stage_occupancy_f32c(int viscous);

// halo exchange of one field over a group of blocks
cudaError_t launch_halo(const HaloGroup& G, cudaStream_t s);
// compact [5][nz][ny][nx] f64 <-> padded f64 field
cudaError_t launch_scatter(const Geometry& g, const double* src, double* dst, float* shadow, cudaStream_t s);
cudaError_t launch_gather(const Geometry& g, const double* src, double* dst, cudaStream_t s);
// ghost cells of a block's physical faces in one direction
cudaError_t launch_bc(const BcBlock& B, cudaStream_t s);
// spectral-radius rate and time step of a padded f64 state (per-CTA partials, last CTA reduces);
// dtl (may be null): every cell's own CFL step, f64 (FP64 path) or f32 (mixed) padded field
cudaError_t launch_init_rate(const Geometry& g, const Physics& ph, const double* q, DevCtrl* ctrl,
                             double* partial, int grid, int mixed, void* dtl, cudaStream_t s);
// curvilinear metrics of every padded cell from the block's nodes (10 padded fields)
cudaError_t launch_metrics(const Geometry& g, const double* nodes, void* M, int elem, cudaStream_t s);
cudaError_t launch_init_rate_curvi(const Geometry& g, const Physics& ph, const double* q, const void* M,
                                   DevCtrl* ctrl, double* partial, int grid, int mixed, void* dtl,
                                   cudaStream_t s);
// global time step of a group: dt = cfl / max rate, written to every block
cudaError_t launch_group_dt(DevCtrl* const* ctrls, int n, double cfl, cudaStream_t s, DevCtrl* extra = nullptr);

// one member of a host-to-host pipeline (gbcfd_pipe_*): its phases, each enqueued on the stream
// it is given; every one returns GBCFD_OK or an error code set by set_error
struct PipeMember {
  void* self;
  size_t bytes;  // one compact state, 5 nx ny nz doubles
  int (*upload)(void* self, const double* q_in, cudaStream_t s);    // host -> landing area (copy engine)
  int (*run)(void* self, int nsteps, cudaStream_t s);               // landing area -> state, steps, result -> landing area
  int (*download)(void* self, double* q_out, double* norms, int nsteps, cudaStream_t s);  // landing area -> host
  int (*flags)(void* self, cudaStream_t s, int* flags);             // read and clear the device flags (synchronises s)
  void (*release)(void* self);                                      // frees `self` with the pipeline (or null)
};
// a pipeline over n members (streams and events created here); waits for the device first and
// takes ownership of the members (their release functions run with the pipeline, or on failure)
int pipe_create(const PipeMember* members, int n, gbcfd_pipe* out);

}  // namespace gbcfd
