/*
 * oracle.h -- plain FP64 CPU oracle of the structured-grid finite-volume hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load this library.  It shares no code, header, table or helper with the CUDA
 * library; the two are checked against each other on the same seeded inputs.
 *
 * What it computes (arXiv 1710.09995, Sec. 2.1-2.2):
 *   Eq. 1  compressible Navier-Stokes in curvilinear coordinates, Q = (rho, rho u, rho v, rho w, rho E);
 *   Eq. 3  semi-discrete form dQ/dt = -R(Q);
 *   Eqs. 4-6  third-order Runge-Kutta in Shu-Osher form with lambda read as -dt;
 *   Sec. 2.2  cell-edge left/right states combined by a flux function, central viscous fluxes,
 *             multi-block interfaces that preserve a uniform flow (geometric conservation).
 * Two spatial schemes.  oracle.c: cell-centred finite volume with MUSCL reconstruction of
 * primitive variables and the minmod limiter, the Roe flux with Harten's entropy fix,
 * second-order central viscous fluxes (the scheme taken where the paper leaves the choice
 * open).  wcns.c: the paper's own WCNS-E-5 (Eq. 2) with a fifth-order weighted nonlinear
 * interpolation and fourth-order central viscous derivatives, on periodic Cartesian blocks.
 * Both advance with SSP-RK3.
 *
 * Layout (the oracle's own): every field is stored with a 2-cell halo on all sides,
 *   a[v][k+2][j+2][i+2], i in [-2, nx+1], dims (nx+4) x (ny+4) x (nz+4), no padding.
 * Metrics: M[10][cells] = S_xi(3), S_eta(3), S_zeta(3), V; S_d of cell c is the area vector of
 * the cell's lower face in direction d (pointing towards +d).
 * Nodes: X[3][nz+1][ny+1][nx+1] (interior block only); halo metrics are periodic copies, or on
 * non-periodic faces (oracle_metrics_bc) come from nodes reflected through the boundary node.
 *
 * Every function returns 0 on success and a negative number on bad arguments or allocation
 * failure.  Nothing is kept between calls.
 */
#ifndef CFD_ORACLE_H
#define CFD_ORACLE_H
#include <stddef.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double gamma;    /* ratio of specific heats */
  double mu;       /* constant dynamic viscosity (0 with viscous=0) */
  double Pr;       /* Prandtl number */
  double cfl;      /* CFL number of the global time step */
  double eps;      /* Harten entropy-fix fraction of (|u.n| + c); 0 disables the fix */
  int viscous;     /* 1: add the viscous fluxes of Eq. 1 */
  int limiter;     /* 0: minmod slopes; 1: unlimited central slope (Fromm) */
} oracle_params;

/* Boundary conditions of the six block faces (-x, +x, -y, +y, -z, +z).  Not in the paper,
 * which gives no boundary treatment: these are the usual inviscid ones.
 *   PERIODIC  the opposite face's interior (both faces of a direction must be periodic)
 *   SLIP_WALL ghost cell m (m = 0, 1 away from the face) mirrors interior cell m: same density
 *             and pressure, velocity reflected about the face's unit normal, u - 2 (u.n) n
 *   FARFIELD  characteristic (Riemann-invariant) subsonic inflow/outflow against the free
 *             stream inf[]: with n the outward unit normal, R+ = u.n + 2c/(gamma-1) from the
 *             adjacent interior cell and R- = u_inf.n - 2c_inf/(gamma-1) give u_b.n and c_b;
 *             entropy p/rho^gamma and tangential velocity come from the free stream where
 *             u_b.n < 0 (inflow), else from the interior cell; supersonic inflow takes the free
 *             stream, supersonic outflow the interior cell.  Both ghost layers get that state.
 * Ghost cells are filled on the face slabs only (the other two indices interior); the inviscid
 * stencil reads nothing else there.  Metrics of halo cells on non-periodic faces come from the
 * block's nodes reflected through the boundary node along each grid line. */
#define ORACLE_BC_PERIODIC 0
#define ORACLE_BC_SLIP_WALL 1
#define ORACLE_BC_FARFIELD 2
typedef struct {
  int kind[6];     /* per face -x, +x, -y, +y, -z, +z */
  double inf[5];   /* free-stream primitive state rho, u, v, w, p (FARFIELD faces) */
} oracle_bc;

/* number of cells of one halo-padded field */
size_t oracle_cells(int nx, int ny, int nz);

/* primitive (rho,u,v,w,p) from conserved (Eq. 1 definitions, ideal gas) */
void oracle_primitive(double gamma, const double U[5], double W[5]);

/* MUSCL states at the face between w1 and w2 of the stencil w0,w1,w2,w3 (primitives) */
void oracle_muscl(int limiter, const double w0[5], const double w1[5], const double w2[5],
                  const double w3[5], double wl[5], double wr[5]);

/* Roe flux through the area vector S (not normalised) from primitive states wl, wr */
void oracle_roe_flux(double gamma, double eps, const double wl[5], const double wr[5],
                     const double S[3], double F[5]);

/* face area vectors and volumes of interior cells from nodes, halo cells by periodic copy
 * (oracle_metrics_bc with bc NULL) */
int oracle_metrics(int nx, int ny, int nz, const double* X, double* M);

/* metrics as oracle_metrics; halo cells of non-periodic directions from reflected nodes
 * (bc NULL: all periodic) */
int oracle_metrics_bc(int nx, int ny, int nz, const double* X, const oracle_bc* bc, double* M);

/* fill the halo of the state Q: periodic images in periodic directions, then the ghost cells
 * of the SLIP_WALL and FARFIELD faces (x faces, then y, then z) */
int oracle_fill_halo_bc(double gamma, int nx, int ny, int nz, const double* M, const oracle_bc* bc,
                        double* Q);

/* local CFL time step of every interior cell, compact [nz][ny][nx] (Q's halo filled) */
int oracle_dt_local(const oracle_params* p, int nx, int ny, int nz, const double* M, const double* Q,
                    double* dt);

/* nsteps SSP-RK3 steps with boundary conditions bc (NULL: periodic); local_dt != 0 advances
 * every cell with its own CFL time step (pseudo-time marching to a steady state), evaluated
 * from Q^n at the start of each step; fixed_dt > 0 (with local_dt 0) takes that step instead of
 * the CFL one.  dts[s] gets the smallest time step of step s. */
int oracle_step_ex(const oracle_params* p, int nx, int ny, int nz, const double* M, const oracle_bc* bc,
                   int local_dt, double fixed_dt, double* Q, int nsteps, double* dts, double* norms);

/* copy periodic images into the 2-cell halo of nvar fields */
int oracle_fill_halo_periodic(int nx, int ny, int nz, int nvar, double* a);

/* R(Q) of Eq. 3 at interior cells; Q's halo must be filled. R is [5][nz][ny][nx] compact. */
int oracle_residual(const oracle_params* p, int nx, int ny, int nz, const double* M,
                    const double* Q, double* R);

/* global CFL time step from Q (halo filled) */
int oracle_dt(const oracle_params* p, int nx, int ny, int nz, const double* M, const double* Q,
              double* dt);

/* RMS over interior cells of each component of a compact residual R[5][n] */
int oracle_norms(size_t n, const double* R, double out[5]);

/* one stage of Eqs. 4-6 (lambda = -dt) on flat arrays of n values */
int oracle_rk3_stage(int stage, size_t n, const double* Qn, const double* Qs, const double* R,
                     double dt, double* Qout);

/* nsteps SSP-RK3 steps on a periodic block. Q is halo-padded, updated in place.
 * dts[nsteps] and norms[nsteps][5] (RMS of the stage-1 residual) are written when not NULL. */
int oracle_step(const oracle_params* p, int nx, int ny, int nz, const double* M, double* Q,
                int nsteps, double* dts, double* norms);

/* same as oracle_step with the time step fixed to dt (no CFL evaluation) */
int oracle_step_fixed_dt(const oracle_params* p, int nx, int ny, int nz, const double* M,
                         double* Q, int nsteps, double dt, double* norms);

/* ---- the paper's own scheme: WCNS-E-5 (Sec. 2.2, Eq. 2), periodic uniform Cartesian blocks ----
 * (wcns.c).  Arrays are compact q[5][nz][ny][nx]; h[3] the cell sizes.  `limiter` selects the
 * interpolation weights: 0 the nonlinear ones, 1 the optimal linear ones. */

/* value at i + 1/2 interpolated from the left, u[0..4] = u_{i-2} .. u_{i+2} */
double oracle_wcns_edge(int linear, const double u[5]);

/* R(Q) of Eq. 3: Eq. 2 in each direction with Roe edge fluxes of the interpolated primitives,
 * minus the fourth-order central viscous derivatives (viscous != 0) */
int oracle_wcns_residual(const oracle_params* p, int nx, int ny, int nz, const double h[3], const double* Q,
                         double* R);

/* global CFL time step of Q */
int oracle_wcns_dt(const oracle_params* p, int nx, int ny, int nz, const double h[3], const double* Q,
                   double* dt);

/* nsteps SSP-RK3 steps (Eqs. 4-6, lambda = -dt) in place; fixed_dt > 0 replaces the CFL step.
 * dts[nsteps] and norms[nsteps][5] (RMS of the stage-1 residual) when not NULL. */
int oracle_wcns_step(const oracle_params* p, int nx, int ny, int nz, const double h[3], double* Q, int nsteps,
                     double fixed_dt, double* dts, double* norms);

/* threads the oracle's OpenMP loops use (1 when built without OpenMP) */
int oracle_threads(void);

/* set that number (n >= 1) and return the one now in force */
int oracle_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
