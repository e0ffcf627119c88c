/*
 * gbcfd.h -- C ABI of the GB300 (sm_103a) structured-grid finite-volume hot path.
 *
 * The operations are those of arXiv 1710.09995 Sec. 2.1-2.2 on 3D structured blocks:
 *   the residual R(Q) of the semi-discrete form dQ/dt = -R(Q) (Eq. 3) for the curvilinear
 *   Navier-Stokes equations (Eq. 1), with cell-edge left/right states combined by a flux
 *   function and central viscous fluxes (Sec. 2.2), the third-order Runge-Kutta time update
 *   (Eqs. 4-6, lambda read as -dt), the data exchange between neighbouring blocks after each
 *   update (Sec. 3.2.5 (2)) and the residual norm of the convergence check (Sec. 2.3).
 * The scheme where the paper leaves the choice open: cell-centred finite volume, MUSCL
 * reconstruction of primitive variables with the minmod limiter, Roe flux with Harten's entropy
 * fix, second-order central viscous fluxes, SSP-RK3, a 2-cell halo, a global CFL time step (or
 * every cell's own, for pseudo-time marching to a steady state).
 * Beyond the paper: inviscid boundary conditions of unconnected faces (slip wall,
 * characteristic far field), groups of blocks advanced by one launch per stage from a CUDA graph,
 * and a learned convergence accelerator (a conv3d network on the tensor cores whose predictions
 * are kept only when the residual drops).
 * The paper's own scheme, WCNS-E-5 (Eq. 2) with fourth-order central viscous terms, is the
 * gbcfd_wcns_* family, on periodic uniform Cartesian blocks.
 *
 * Conventions
 *  - Every function returns GBCFD_OK (0) or a negative GBCFD_ERR_* code; gbcfd_last_error()
 *    then returns a message for the calling host thread.  Nothing throws across the ABI.
 *  - Device memory is owned by the caller: gbcfd_required_bytes() tells how much one block
 *    needs, gbcfd_create_block() carves it.  The library allocates no device memory.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are asynchronous on it
 *    unless stated; a block must not be used from two streams at once.
 *  - State arrays passed in or out are compact SoA float64, q[5][nz][ny][nx] (x fastest), the
 *    conserved variables (rho, rho u, rho v, rho w, rho E) of Eq. 1.  Where a pointer may be
 *    host or device memory it says so; host memory should be pinned for speed.
 *  - Faces are numbered 0..5 = -x, +x, -y, +y, -z, +z.
 */
#ifndef GBCFD_H
#define GBCFD_H
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GBCFD_OK 0
#define GBCFD_ERR_ARG (-1)          /* bad argument: null pointer, size, range, mismatch */
#define GBCFD_ERR_CUDA (-2)         /* a CUDA runtime or driver call failed */
#define GBCFD_ERR_NONPHYSICAL (-3)  /* rho <= 0, p <= 0 or a non-finite value was met */
#define GBCFD_ERR_TIMEOUT (-4)      /* a bounded device wait ran out (a copy never landed) */
#define GBCFD_ERR_STATE (-5)        /* call out of order (e.g. step before set_state) */
#define GBCFD_ERR_MEMORY (-6)       /* caller memory too small or misaligned */

#define GBCFD_FP64 0   /* everything in FP64 */
#define GBCFD_MIXED 1  /* reconstruction, fluxes and stage increments in FP32; state, its
                          update and the residual-norm reduction in FP64 */

typedef struct gbcfd_block_s* gbcfd_block; /* opaque, host-side descriptor */

typedef struct {
  double gamma;       /* ratio of specific heats (1.4) */
  double mu;          /* constant dynamic viscosity; used when viscous != 0 */
  double Pr;          /* Prandtl number; heat conductivity = mu gamma / ((gamma - 1) Pr) */
  double cfl;         /* CFL number of the global time step */
  double entropy_eps; /* Harten entropy-fix fraction of (|u.n| + c); 0 disables the fix */
  int viscous;        /* 0: Euler, 1: Navier-Stokes (Eq. 1 with Fv, Gv, Hv) */
  int limiter;        /* 0: minmod, 1: unlimited central slope */
  int precision;      /* GBCFD_FP64 or GBCFD_MIXED */
  int local_dt;       /* 0: one global CFL time step; 1: every cell advances with its own CFL step
                         (pseudo-time marching to a steady state; the residual norm is unchanged);
                         inviscid blocks only (viscous = 0) */
} gbcfd_params;

/* Bytes of caller device memory one block of nx x ny x nz interior cells needs (state, stage
 * buffers, metrics, reduction scratch), for the given precision.  Sizes must be >= 1.
 * The halo is always 2 cells (the MUSCL stencil i-1..i+2 of Sec. 2.2's cell-edge states). */
int gbcfd_required_bytes(int nx, int ny, int nz, const gbcfd_params* params, size_t* bytes);

/* Create a block on the current CUDA device inside caller memory `dev_mem` of `bytes` bytes
 * (at least gbcfd_required_bytes, 256-byte aligned).  The memory must stay valid until
 * gbcfd_destroy_block.  The block starts unconnected, with uniform Cartesian metrics of unit
 * spacing and no state.  Returns the descriptor in *out. */
int gbcfd_create_block(int nx, int ny, int nz, const gbcfd_params* params, void* dev_mem,
                       size_t bytes, gbcfd_block* out);

/* Release the host descriptor (the caller frees the device memory).  Waits for the device. */
int gbcfd_destroy_block(gbcfd_block block);

/* Connect face `face` of `block` to the opposite face of `nbr` (conforming, same orientation:
 * equal cell counts along the two shared directions).  nbr == block makes the direction
 * periodic.  Multi-block interfaces share their grid points (Sec. 2.2); the halo then holds
 * the neighbour's first two cell layers.  A face with a boundary condition cannot be connected
 * (GBCFD_ERR_ARG).  Faces with neither keep whatever their halo holds. */
int gbcfd_connect(gbcfd_block block, int face, gbcfd_block nbr);

/* Boundary conditions of unconnected faces (the paper gives none; these are the usual inviscid
 * ones, for steady internal flows such as a channel).  Every halo fill of a stage input (the
 * stage's exchange) then also fills the face's two ghost layers:
 *   GBCFD_BC_SLIP_WALL  ghost layer m mirrors interior layer m about the face's unit normal n:
 *                       same density and pressure, velocity u - 2 (u.n) n
 *   GBCFD_BC_FARFIELD   characteristic subsonic inflow/outflow against the free stream
 *                       inf[5] = (rho, u, v, w, p): with n the outward unit normal, the
 *                       outgoing invariant u.n + 2c/(gamma-1) of the adjacent interior cell and
 *                       the incoming u.n - 2c/(gamma-1) of the free stream give the boundary
 *                       u.n and c; entropy p/rho^gamma and tangential velocity come from the
 *                       upwind side; supersonic inflow takes the free stream, supersonic
 *                       outflow the interior cell.  Both ghost layers get that state.
 *   GBCFD_BC_NONE       removes the condition.
 * Face slabs are filled over the padded extent of the other two directions (x faces, then y,
 * then z), so edges and corners hold physical states.  Halo metrics of such faces come from
 * the block's nodes reflected through the boundary node along each grid line (computed by
 * gbcfd_set_metrics for every halo cell; connected faces take the neighbour's).
 * Errors: GBCFD_ERR_ARG for a connected face, a viscous block, fewer than 2 cells across the
 * face's direction, an unknown kind, or a far-field free stream without rho > 0, p > 0. */
#define GBCFD_BC_NONE 0
#define GBCFD_BC_SLIP_WALL 1
#define GBCFD_BC_FARFIELD 2
int gbcfd_set_boundary(gbcfd_block block, int face, int kind, const double inf[5]);

/* Set the grid (Eq. 1's curvilinear coordinates).  nodes == NULL: uniform Cartesian grid with
 * cell sizes spacing[0..2].  Otherwise `nodes` is a device pointer to float64
 * x[3][nz+1][ny+1][nx+1], the block's grid points; face area vectors (half the cross product
 * of the face diagonals) and cell volumes are computed on the device, and the halo cells take
 * their neighbours' metrics at the next exchange, so that a uniform flow is preserved exactly
 * across block interfaces (the geometric conservation of Sec. 2.2). */
int gbcfd_set_metrics(gbcfd_block block, const double* nodes, const double spacing[3],
                      void* stream);

/* Load the conserved state q[5][nz][ny][nx] (host or device pointer), exchange nothing, and
 * evaluate the CFL time step of the first step.  Halos are filled by the next
 * gbcfd_exchange_halos or gbcfd_step. */
int gbcfd_set_state(gbcfd_block block, const double* q, void* stream);

/* Copy the conserved state out to q[5][nz][ny][nx] (host or device pointer).  A host
 * destination synchronises the stream before returning. */
int gbcfd_get_state(gbcfd_block block, double* q, void* stream);

/* Fill the 2-cell halos of the array the next Runge-Kutta stage reads (the state Q^n between
 * steps, the stage-1 / stage-2 result between stages) of n blocks from their connected
 * neighbours: the data exchange among blocks after each update (Sec. 3.2.5 (2)).  One launch
 * for all blocks; edge and corner cells come from the diagonal neighbour reached through the
 * face neighbours.  All n blocks must be at the same stage. */
int gbcfd_exchange_halos(const gbcfd_block* blocks, int n, void* stream);

/* R(Q) of Eq. 3 for the current state, written to r[5][nz][ny][nx] float64 (device pointer):
 * the sum over the six faces of (inviscid - viscous) flux through the face area vector,
 * divided by the cell volume; dQ/dt = -R.  Exchanges the block's halo first. */
int gbcfd_compute_residual(gbcfd_block block, double* r, void* stream);

/* One Runge-Kutta stage (1, 2 or 3; Eqs. 4-6 with lambda = -dt) of n blocks, halos assumed
 * exchanged.  Stages must come in order 1, 2, 3 (GBCFD_ERR_STATE otherwise); set_state restarts
 * at 1.  Stage 1 also records the residual norm of R(Q^n) and, for n > 1, takes the global time
 * step as the minimum over the blocks; stage 3 also evaluates the next CFL time step.
 * gbcfd_step is gbcfd_exchange_halos + gbcfd_stage, three times. */
int gbcfd_stage(const gbcfd_block* blocks, int n, int stage, void* stream);

/* nsteps full SSP-RK3 steps of n blocks (halo exchange before each stage, the global time
 * step the minimum over all blocks).  Asynchronous: errors met on the device are reported by
 * the next gbcfd_residual_norm. */
int gbcfd_step(const gbcfd_block* blocks, int n, int nsteps, void* stream);

/* RMS over the block's interior cells of each component of R(Q^n) from the last stage 1 (the
 * convergence criterion of Sec. 2.3), copied to out[5] on the host.  Synchronises the stream
 * and reports GBCFD_ERR_NONPHYSICAL / GBCFD_ERR_TIMEOUT if a kernel flagged one since the
 * last call (the flag is then cleared). */
int gbcfd_residual_norm(gbcfd_block block, double out[5], void* stream);

/* The time step the next stage 1 will use, copied to *dt on the host (synchronises). */
int gbcfd_get_dt(gbcfd_block block, double* dt, void* stream);

/* ---- host-to-host pipeline ------------------------------------------------------------------
 * Advances many states that live in host memory (independent problems: an ensemble, the
 * trajectories a learned model is trained on, states streamed in by a service) through a set
 * of identical blocks, so that the host-link transfers overlap the computation.  Not in the
 * paper.  Item i runs on member i mod n: its state q_in[5][nz][ny][nx] (float64, host) is
 * uploaded by a copy engine into the member's staging area, set as by gbcfd_set_state (time step
 * included), advanced nsteps SSP-RK3 steps as by gbcfd_step, and copied back to q_out[5][nz][ny][nx]
 * on the host; results are bitwise those of gbcfd_set_state / gbcfd_step / gbcfd_get_state on
 * one block.  Uploads, device work and downloads run on three streams of the pipeline, so with
 * 3 members item i+1's upload and item i-1's download (the two directions of the link) run while
 * item i steps. */
typedef struct gbcfd_pipe_s* gbcfd_pipe;

/* Create a pipeline over n (1..8) blocks of equal sizes, parameters, grid and boundary
 * conditions, none connected to another block (periodic self-connections and boundary faces
 * only).  The blocks must outlive the pipeline and are used by nothing else while items are in
 * flight.  Waits for the device (the members' earlier work) before returning.  GBCFD_ERR_ARG for
 * a mismatch, GBCFD_ERR_MEMORY if a member's staging area cannot hold a state. */
int gbcfd_pipe_create(const gbcfd_block* blocks, int n, gbcfd_pipe* out);

/* Wait for the pipeline's work and release its streams and events (not the blocks). */
int gbcfd_pipe_destroy(gbcfd_pipe pipe);

/* Enqueue one item and return.  q_in, q_out and norms (5 doubles: the RMS residual of the item's
 * last step, as gbcfd_residual_norm reports it; NULL for none; not written when nsteps is 0) must
 * be page-locked host memory (cudaHostAlloc, or a pinned torch tensor), else GBCFD_ERR_ARG;
 * q_in must not change and q_out / norms must not be read until gbcfd_pipe_sync returns.  After
 * an item fails (error code returned), further submits return GBCFD_ERR_STATE until a sync. */
int gbcfd_pipe_submit(gbcfd_pipe pipe, const double* q_in, double* q_out, int nsteps, double* norms);

/* Wait until every submitted item is in host memory.  Reports GBCFD_ERR_NONPHYSICAL /
 * GBCFD_ERR_TIMEOUT if a kernel of any item flagged one (the flags are then cleared). */
int gbcfd_pipe_sync(gbcfd_pipe pipe);

/* The CFL time step of a state, with no device memory allocated by anyone: for callers that
 * cannot call cudaMalloc -- code running where the device allocator is off limits (inside a
 * pre-sized memory pool or a fixed-footprint service) or that holds no block.  The paper has no
 * counterpart; it is the same time step gbcfd_set_state evaluates (cfl / max over cells of the
 * summed spectral-radius rate, in the precision params->precision selects), on a uniform
 * Cartesian grid with cell sizes spacing[0..2].
 *   q:  device pointer, compact q[5][nz][ny][nx] float64 (caller-owned, read only)
 *   dt: device pointer to one float64 (caller-owned), written asynchronously on `stream`; a
 *       negative value means a cell had rho <= 0 or p <= 0.
 * Scratch: a fixed 64 KB array in the library's device image (one per GPU that loads the
 * library, kept until exit), so at most 134,217,728 cells (GBCFD_ERR_ARG beyond).  The first call
 * on each device looks up that array's device address (cudaGetSymbolAddress), so make it before
 * any stream capture.  Every call shares the array and the previous call's contents remain there:
 * two calls that overlap on the GPU (different streams, or devices sharing nothing else) race. */
int gbcfd_time_step_noalloc(const double* q, int nx, int ny, int nz, const gbcfd_params* params,
                            const double spacing[3], double* dt, void* stream);

/* ---- batched groups of blocks --------------------------------------------------------------
 * A group advances many blocks with one kernel launch per Runge-Kutta stage (the multi-zone
 * parallelism of Sec. 3.1.1 (1) on one GPU): the persistent grid is split between the blocks in
 * proportion to their cells, every stage of every block is one launch, the halos of all blocks
 * one launch, and a whole step is replayed from a CUDA graph captured on the first step.  The
 * blocks must share precision, physics and grid kind (Cartesian or curvilinear); every block a
 * member connects to must be a member.  Results equal gbcfd_step on the same blocks bitwise. */
typedef struct gbcfd_group_s* gbcfd_group;

/* Device bytes a group of n blocks needs (descriptor table, control block, partial sums). */
int gbcfd_group_required_bytes(int n, size_t* bytes);

/* Create a group of n blocks in caller memory dev_mem (256-byte aligned, at least
 * gbcfd_group_required_bytes).  The blocks must outlive the group; their connections and grids
 * must not change while it exists (the captured graphs hold their halo tables). */
int gbcfd_group_create(const gbcfd_block* blocks, int n, void* dev_mem, size_t bytes, gbcfd_group* out);

/* Release the group's host objects (graphs, capture stream).  Waits for the device. */
int gbcfd_group_destroy(gbcfd_group group);

/* nsteps SSP-RK3 steps of all member blocks (global time step over the group).  Members must
 * hold a state and be between steps.  Asynchronous on `stream`; errors met on the device are
 * reported per block by gbcfd_residual_norm. */
int gbcfd_group_step(gbcfd_group group, int nsteps, void* stream);

/* Autotuner (Sec. 3.1.1 distributes uneven zones over the hardware; here the schedule of one
 * GPU): times pairs of stage-1 and stage-2 launches (which write only the stage scratch and the
 * norms; stage 1's output gets its halos between them) for every tile shape the
 * stage kernel is compiled for on this path -- 32 x 8 cells, and on Cartesian Euler blocks a
 * second height (32 x 11 on the FP64 path, 32 x 4 on the mixed path) -- and for each of them
 * several grid splits (1x .. 16x the resident CTAs per SM, at most 16 per SM, shared between
 * the blocks in proportion to their tile-planes), keeps the fastest, and then for it times the
 * halo exchange of the stage outputs as launches against its fold into the stages (where the
 * group allows the fold, see gbcfd_group_set_schedule) and keeps the faster.  Synchronises the
 * stream; drops the captured graphs.  The chosen CTAs per SM and tile height (cells along y)
 * are returned in *ctas_per_sm and *tile_rows when not NULL; gbcfd_group_tune is the same
 * without the tile height. */
int gbcfd_group_tune(gbcfd_group group, void* stream, int* ctas_per_sm);
int gbcfd_group_tune_tile(gbcfd_group group, void* stream, int* ctas_per_sm, int* tile_rows);

/* Set the schedule the tuner would choose: tile height tile_rows (8, or the path's second height
 * on Cartesian Euler blocks: 11 FP64, 4 mixed; GBCFD_ERR_ARG otherwise), ctas_per_sm CTAs per
 * SM (1..16, split between the blocks as by the tuner), and halo_push: 0 runs the halo exchange
 * of the stage-1 and stage-2 outputs as launches between the stages, 1 folds it into those
 * stages (each cell near a block face also writes its output into the neighbours' halo cells
 * that copy it, faces, edges and corners; Sec. 3.2.5 merges such small kernels), which needs
 * Cartesian Euler blocks forming a conforming periodic lattice: every face connected to a member, the blocks of a face equal in
 * the face's two directions, at least 2 cells per direction, face-neighbour walks that commute
 * (GBCFD_ERR_ARG otherwise).  Results do not depend on the schedule (every face flux and every
 * cell's update is the same arithmetic); the residual norms' rounding does (their partial sums
 * follow the grid).  Synchronises the stream; drops the captured graphs. */
int gbcfd_group_set_schedule(gbcfd_group group, int ctas_per_sm, int tile_rows, int halo_push, void* stream);

/* The group's current schedule (from the tuner or gbcfd_group_set_schedule); NULL pointers are
 * skipped. */
int gbcfd_group_get_schedule(gbcfd_group group, int* ctas_per_sm, int* tile_rows, int* halo_push);

/* Timing marks inside each step of the group: events[0..6] are CUDA events (cudaEvent_t) the
 * caller created with timing enabled and owns.  Each step records events[0] before the time-step
 * kernel, events[2s-1] after the halo exchange of stage s and events[2s] after its stage kernel,
 * so elapsed(events[2s-1], events[2s]) is the stage-s kernel's duration.  events NULL removes
 * them.  Drops the captured graphs; the events of one step are overwritten by the next. */
int gbcfd_group_set_timing(gbcfd_group group, void* const* events, int n);

/* A host-to-host pipeline (gbcfd_pipe_submit / _sync / _destroy) over n (1..8) groups built
 * alike: the same number of blocks, block k of every group with the same sizes, parameters,
 * grid, boundary conditions and connections (to the same member indices).  An item's state is
 * the concatenation, in the group's block order, of the blocks' compact states
 * q[5][nz][ny][nx] (float64); norms, when not NULL, receives 5 doubles per block in that order.
 * Each item is set block by block as by gbcfd_set_state and advanced as by gbcfd_group_step;
 * the results are bitwise those calls'.  No block may belong to two member groups. */
int gbcfd_group_pipe_create(const gbcfd_group* groups, int n, gbcfd_pipe* out);

/* ---- learned convergence accelerator (not in the paper: the project's addition) --------------
 * A 3-layer 3D convolutional network (channels 10 -> 32 -> 32 -> 5, 3x3x3 taps, SiLU, zero
 * padding in x and y, periodic in z) predicts the change of a block's state over K = 20
 * pseudo-time steps from the state and its residual; a prediction is kept only if the RMS of
 * the density residual then drops (the plain iteration decides).  Features per cell:
 * 10 (Q - Q_inf) / ref and (-dt_cell R) / ref / s, with ref = (rho, rho c, rho c, rho c, rho c^2)
 * of the free stream and s the RMS of (-dt_cell R) / ref over the block; prediction
 * Q + 20 s ref y.  The free stream is the block's far-field one (gbcfd_set_boundary).
 * Tensors are channels-last: features bfloat16 [cell][16] (10 used), outputs and targets float
 * [cell][8] (5 used); cell = ((b nz + k) ny + j) nx + i.  Weights are bfloat16 with FP32
 * accumulation on the tensor cores; FP32 master weights and Adam moments.
 * Parameters (host float, GBCFD_ACCEL_NPARAM): per layer W[out][in][tap] then b[out], tap
 * t = 9 (dz+1) + 3 (dy+1) + (dx+1). */
#define GBCFD_ACCEL_NPARAM 40677
typedef struct gbcfd_accel_s* gbcfd_accel;

/* Device bytes of an accelerator over `batch` volumes of nx x ny x nz cells. */
int gbcfd_accel_required_bytes(int nx, int ny, int nz, int batch, size_t* bytes);

/* Create it in caller memory (256-byte aligned).  zperiodic: the volume wraps in z. */
int gbcfd_accel_create(int nx, int ny, int nz, int batch, int zperiodic, void* dev_mem, size_t bytes,
                       gbcfd_accel* out);
int gbcfd_accel_destroy(gbcfd_accel accel);

/* Load / read the parameters (host, GBCFD_ACCEL_NPARAM floats).  Loading resets Adam. */
int gbcfd_accel_set_params(gbcfd_accel accel, const float* params, void* stream);
int gbcfd_accel_get_params(gbcfd_accel accel, float* params, void* stream);

/* Network output y (device float [batch cells][8]) for features x (device bf16 [batch cells][16]). */
int gbcfd_accel_forward(gbcfd_accel accel, const void* x, float* y, void* stream);

/* One Adam step (learning rate lr, step counts from 1) on the mean squared error between the
 * network's output for x and target t (device float [batch cells][8]); *loss (host) gets the
 * loss before the step.  Synchronises the stream. */
int gbcfd_accel_train_step(gbcfd_accel accel, const void* x, const float* t, float lr, int step, double* loss,
                           void* stream);

/* The training state after the last gbcfd_accel_train_step, copied to host arrays of
 * GBCFD_ACCEL_NPARAM floats (any pointer may be NULL to skip it), in the parameter layout of
 * gbcfd_accel_set_params: grad = the gradient of that step's mean squared error at the
 * parameters it started from (before the Adam move), m and v = Adam's first and second moments
 * after the move (Kingma & Ba's m_t, v_t, not bias-corrected).  Zeros before any step.
 * Synchronises the stream. */
int gbcfd_accel_get_train_state(gbcfd_accel accel, float* grad, float* m, float* v, void* stream);

/* Features of a block (its size must be the accelerator's volume) into x (device bf16
 * [cells][16], NULL: the accelerator's own buffer); remembers the state and s for
 * gbcfd_accel_target.  The block must hold a state, be between steps and have a far-field face. */
int gbcfd_accel_features(gbcfd_accel accel, gbcfd_block block, void* x, void* stream);

/* Training target of the block's state now against the one remembered by the last
 * gbcfd_accel_features: (Q_now - Q_then) / ref / (20 s), into t (device float [cells][8]). */
int gbcfd_accel_target(gbcfd_accel accel, gbcfd_block block, float* t, void* stream);

/* One accelerated update: residual and features at Q, prediction Q' = Q + 20 s ref y, residual at
 * Q'; Q' is kept when RMS(R_rho(Q')) < RMS(R_rho(Q)) (the time steps are then re-evaluated from
 * it), else Q is restored and the block is left bit for bit as it was.  *accepted (host) tells
 * which; norms[0], norms[1] (host, may be NULL) get the two RMS values.  Synchronises. */
int gbcfd_accel_try(gbcfd_accel accel, gbcfd_block block, void* stream, int* accepted, double norms[2]);

/* One accelerated update with smoothing: the prediction scaled by alpha (0 < alpha <= 4) is applied
 * (Q' = Q + alpha 20 s ref y), the time steps re-evaluated, and nsteps (0..1000) plain steps run
 * from Q' (gbcfd_step); the result is kept when RMS(R_rho) then lies below min(ratio, 1) x RMS(R_rho(Q))
 * -- the caller passes the factor the plain iteration achieved over nsteps steps lately, so a
 * prediction is kept only if the residual drops and it beat the plain steps -- else the state, the
 * local time steps and the control block (time step, norms, flags) are restored bit for bit, and
 * the steps count for nothing.  The plain steps damp the small-scale error of the prediction that
 * the bare test of gbcfd_accel_try sees first.  *accepted, norms as gbcfd_accel_try (norms[1]: after
 * the steps).  Synchronises. */
int gbcfd_accel_try_smooth(gbcfd_accel accel, gbcfd_block block, double alpha, int nsteps, double ratio,
                           void* stream, int* accepted, double norms[2]);

/* ---- the paper's own scheme: WCNS-E-5 on periodic uniform Cartesian blocks -------------------
 * Sec. 2.2: the inviscid derivative at a cell centre is Eq. 2, the sixth-order combination of the
 * flux differences at the cell edges i +- 1/2, i +- 3/2, i +- 5/2, each edge flux the Roe flux
 * (Harten's fix) of left and right cell-edge states from a fifth-order weighted nonlinear
 * interpolation of the primitive variables; the viscous derivatives are fourth-order central
 * (gradients of u, v, w, p/rho by (f_{i-2} - 8 f_{i-1} + 8 f_{i+1} - f_{i+2}) / 12h at the cell
 * centres, the viscous flux vectors of Eq. 1 there, and the same difference of those).  The
 * interpolation, which the paper does not spell out: per variable, three three-point stencils
 * with candidates u_i + g_k/2 + s_k/8 (g_k, s_k the stencil's first and second differences),
 * smoothness g_k^2 + s_k^2, weights C_k / (1e-6 + smoothness)^2 normalised, C = (1/16, 10/16,
 * 5/16); the right state at i + 1/2 from the mirrored stencil.  Time stepping as gbcfd_step
 * (Eqs. 4-6, lambda = -dt, the global CFL step of Q^n).  A block on its own is periodic in every
 * direction (its own neighbour; its 5-cell halo is filled by index wrap); blocks connected face
 * to face (gbcfd_wcns_connect) form a periodic multi-block lattice advanced together by
 * gbcfd_wcns_step_many (Sec. 2.2's multi-block interfaces, uniform Cartesian grids).
 * params: as for blocks; `limiter` 0 takes the nonlinear weights, 1 the optimal linear ones
 * (linear fifth-order interpolation); `precision` GBCFD_MIXED evaluates the interpolation, the
 * fluxes and the derivatives in FP32 (state and update in FP64); `local_dt` must be 0. */
typedef struct gbcfd_wcns_s* gbcfd_wcns;

/* Bytes of caller device memory a WCNS block of nx x ny x nz cells needs (the states Q^n, Q1, Q2,
 * the padded primitive box, the viscous flux vectors when viscous, the residual, the control
 * block and reduction partials).  Sizes must be >= 1.  Needs a current CUDA device. */
int gbcfd_wcns_required_bytes(int nx, int ny, int nz, const gbcfd_params* params, size_t* bytes);

/* Create a WCNS block with cell sizes spacing[0..2] on the current device inside caller memory
 * dev_mem (256-byte aligned, at least gbcfd_wcns_required_bytes), which must stay valid until
 * gbcfd_wcns_destroy.  GBCFD_ERR_ARG for bad sizes or params, GBCFD_ERR_MEMORY for short or
 * misaligned memory. */
int gbcfd_wcns_create(int nx, int ny, int nz, const gbcfd_params* params, const double spacing[3],
                      void* dev_mem, size_t bytes, gbcfd_wcns* out);

/* Release the host descriptor (the caller frees the device memory).  Waits for the device. */
int gbcfd_wcns_destroy(gbcfd_wcns block);

/* Load the conserved state q[5][nz][ny][nx] (host or device pointer). */
int gbcfd_wcns_set_state(gbcfd_wcns block, const double* q, void* stream);

/* Copy the state out to q[5][nz][ny][nx] (host or device pointer; a host one synchronises). */
int gbcfd_wcns_get_state(gbcfd_wcns block, double* q, void* stream);

/* R(Q) of Eq. 3 for the current state into r[5][nz][ny][nx] float64 (device pointer). */
int gbcfd_wcns_compute_residual(gbcfd_wcns block, double* r, void* stream);

/* nsteps SSP-RK3 steps; asynchronous, device errors reported by gbcfd_wcns_residual_norm.
 * GBCFD_ERR_STATE for a block connected to other blocks (they advance with
 * gbcfd_wcns_step_many; gbcfd_wcns_compute_residual refuses such a block too). */
int gbcfd_wcns_step(gbcfd_wcns block, int nsteps, void* stream);

/* Connect face `face` of block a (0..5 = -x, +x, -y, +y, -z, +z) to block b: a's cells beyond
 * that face are b's first cells across b's opposite face, and the link is recorded both ways
 * (a == b makes that direction periodic).  The two blocks must match in the face's two
 * directions and share parameters and cell sizes (GBCFD_ERR_ARG otherwise).  Destroying a block
 * removes the links to it. */
int gbcfd_wcns_connect(gbcfd_wcns a, int face, gbcfd_wcns b);

/* nsteps SSP-RK3 steps of the n (1..32) blocks blocks[0..n-1] together, on one stream: every
 * stage first forms each block's primitives over its 5-cell halo from the stage inputs of the
 * blocks that own the halo cells (face neighbours walked along z, y and x, so edges and corners
 * come from the diagonal blocks and neighbours thinner than the halo are crossed), then each
 * block's viscous and direction passes; the time step is cfl / the largest CFL rate of Q^n over
 * all the blocks, the same in every block.  Results equal one periodic block holding the whole
 * lattice (the same arithmetic on the same values).  Requirements (GBCFD_ERR_ARG otherwise):
 * every face of every block connected to a block of the list and connected back by it (a lone
 * unconnected block counts as periodic), the blocks form a conforming lattice (face walks along two different axes reach
 * the same block in either order), and share device, parameters and cell sizes; every block has
 * a state (GBCFD_ERR_STATE).  Asynchronous with respect to the host: the blocks' kernels run on
 * up to 8 internal streams of the device that fork from and join into `stream` at every stage
 * (so the blocks overlap on the GPU; `stream` sees the whole step in order, also when captured
 * into a graph).  Each block's norms and time step are read with gbcfd_wcns_residual_norm /
 * gbcfd_wcns_get_dt. */
int gbcfd_wcns_step_many(const gbcfd_wcns* blocks, int n, int nsteps, void* stream);

/* RMS per component of R(Q^n) of the last step's stage 1, to out[5] on the host (synchronises;
 * GBCFD_ERR_NONPHYSICAL if rho <= 0 or p <= 0 was met since the last call). */
int gbcfd_wcns_residual_norm(gbcfd_wcns block, double out[5], void* stream);

/* The time step of the last step (0 before the first), to *dt on the host (synchronises). */
int gbcfd_wcns_get_dt(gbcfd_wcns block, double* dt, void* stream);

/* Timing marks inside every step: events[0..17] are CUDA events (cudaEvent_t) the caller created
 * with timing enabled and owns.  Stage s (1..3) records events[6(s-1) + m] before its primitive
 * kernel (m = 0) and after its primitive, viscous (also when inviscid: no launch), x, y and z
 * kernels (m = 1..5); the next step overwrites them.  events NULL removes them; n must be 18. */
int gbcfd_wcns_set_timing(gbcfd_wcns block, void* const* events, int n);

/* A host-to-host pipeline (gbcfd_pipe_submit / _sync / _destroy) over n (1..8) WCNS blocks of
 * equal sizes, parameters and cell sizes: each item's state is uploaded into a member's Q^n,
 * set as by gbcfd_wcns_set_state, advanced nsteps steps as by gbcfd_wcns_step and copied back;
 * bitwise the results of those calls on one block.  Waits for the device before returning. */
int gbcfd_wcns_pipe_create(const gbcfd_wcns* blocks, int n, gbcfd_pipe* out);

/* Throughput of one arithmetic operation on the current GPU, in operations per second, to
 * *ops_per_second: op GBCFD_OP_DFMA (FP64 fused multiply-add; x 2 = FP64 flop/s, the FP64 stage
 * kernels' bound), GBCFD_OP_FFMA (FP32 fused multiply-add), GBCFD_OP_DIV (FP64 1/x by IEEE
 * division), GBCFD_OP_RCP_NEWTON (the FP64 path's reciprocal: hardware estimate and one
 * third-order Newton step), GBCFD_OP_RSQRT (FP64 1/sqrt(x)), GBCFD_OP_DADD and GBCFD_OP_DMUL (FP64
 * add and multiply of registers), GBCFD_OP_DFMA_CONST (FP64 FMA whose multiplier and addend are
 * literal constants).  8 independent chains per thread,
 * 8 CTAs of 256 threads per SM; a warm-up launch, then one launch timed with CUDA events on
 * `stream` (synchronises; tens of milliseconds).  scratch: caller device memory of at least
 * 8 x (SMs x 8) bytes the kernel may write.  GBCFD_ERR_ARG for an unknown op or NULL pointers. */
#define GBCFD_OP_DFMA 0
#define GBCFD_OP_FFMA 1
#define GBCFD_OP_DIV 2
#define GBCFD_OP_RCP_NEWTON 3
#define GBCFD_OP_RSQRT 4
#define GBCFD_OP_DADD 5
#define GBCFD_OP_DMUL 6
#define GBCFD_OP_DFMA_CONST 7
int gbcfd_op_rate(int op, void* scratch, double* ops_per_second, void* stream);

/* Message of the last error on the calling host thread ("" if none). */
const char* gbcfd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
