/*
 * oracle.c -- plain FP64 CPU oracle of the structured-grid finite-volume hot path.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the benchmark's CPU
 * baseline, never by the CUDA library or its Python binding.  It is written for a reader who
 * checks it against arXiv 1710.09995 Sec. 2.1-2.2 (Eqs. 1, 3, 4-6) by eye: straight loops over
 * faces into face-flux arrays, then over cells; nothing tiled, fused or reordered.
 * Compiled with -ffp-contract=off so that x86 and Arm hosts round identically.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define HALO 2

/* ------------------------------------------------------------------------------------------ */
/* indexing of halo-padded fields                                                              */

size_t oracle_cells(int nx, int ny, int nz) {
  return (size_t)(nx + 2 * HALO) * (size_t)(ny + 2 * HALO) * (size_t)(nz + 2 * HALO);
}

typedef struct {
  int nx, ny, nz;
  size_t sx, sy, sz; /* strides of i, j, k */
  size_t ncell;
} grid_t;

static grid_t make_grid(int nx, int ny, int nz) {
  grid_t g;
  g.nx = nx; g.ny = ny; g.nz = nz;
  g.sx = 1;
  g.sy = (size_t)(nx + 2 * HALO);
  g.sz = g.sy * (size_t)(ny + 2 * HALO);
  g.ncell = oracle_cells(nx, ny, nz);
  return g;
}

/* i, j, k are interior coordinates: 0..n-1 inside, -2..-1 and n..n+1 in the halo */
static size_t cell(const grid_t* g, int i, int j, int k) {
  return (size_t)(k + HALO) * g->sz + (size_t)(j + HALO) * g->sy + (size_t)(i + HALO);
}

static int bad_dims(int nx, int ny, int nz) {
  return nx < 1 || ny < 1 || nz < 1;
}

int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ------------------------------------------------------------------------------------------ */
/* Eq. 1 state definitions                                                                     */

void oracle_primitive(double gamma, const double U[5], double W[5]) {
  double rho = U[0];
  double u = U[1] / rho;
  double v = U[2] / rho;
  double w = U[3] / rho;
  double kinetic = 0.5 * rho * (u * u + v * v + w * w);
  W[0] = rho;
  W[1] = u;
  W[2] = v;
  W[3] = w;
  W[4] = (gamma - 1.0) * (U[4] - kinetic);
}

/* ------------------------------------------------------------------------------------------ */
/* MUSCL reconstruction in index space, minmod limiter                                        */

static double minmod(double a, double b) {
  if (a > 0.0 && b > 0.0) return a < b ? a : b;
  if (a < 0.0 && b < 0.0) return a > b ? a : b;
  return 0.0;
}

static double limited_slope(int limiter, double backward, double forward) {
  if (limiter == 0) return minmod(backward, forward);
  return 0.5 * (backward + forward);
}

void oracle_muscl(int limiter, const double w0[5], const double w1[5], const double w2[5],
                  const double w3[5], double wl[5], double wr[5]) {
  for (int m = 0; m < 5; ++m) {
    double slope_left = limited_slope(limiter, w1[m] - w0[m], w2[m] - w1[m]);
    double slope_right = limited_slope(limiter, w2[m] - w1[m], w3[m] - w2[m]);
    wl[m] = w1[m] + 0.5 * slope_left;
    wr[m] = w2[m] - 0.5 * slope_right;
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Roe flux with Harten's entropy fix                                                          */

static double harten(double lambda, double delta) {
  double a = fabs(lambda);
  if (a < delta) return (lambda * lambda + delta * delta) / (2.0 * delta);
  return a;
}

void oracle_roe_flux(double gamma, double eps, const double wl[5], const double wr[5],
                     const double S[3], double F[5]) {
  double area = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
  double n[3] = {S[0] / area, S[1] / area, S[2] / area};

  /* left state */
  double rl = wl[0], ul = wl[1], vl = wl[2], xl = wl[3], pl = wl[4];
  double unl = ul * n[0] + vl * n[1] + xl * n[2];
  double hl = gamma / (gamma - 1.0) * pl / rl + 0.5 * (ul * ul + vl * vl + xl * xl);
  /* right state */
  double rr = wr[0], ur = wr[1], vr = wr[2], xr = wr[3], pr = wr[4];
  double unr = ur * n[0] + vr * n[1] + xr * n[2];
  double hr = gamma / (gamma - 1.0) * pr / rr + 0.5 * (ur * ur + vr * vr + xr * xr);

  /* physical fluxes per unit area (Eq. 1 inviscid flux in the face-normal direction) */
  double fl[5] = {rl * unl, rl * ul * unl + pl * n[0], rl * vl * unl + pl * n[1],
                  rl * xl * unl + pl * n[2], rl * hl * unl};
  double fr[5] = {rr * unr, rr * ur * unr + pr * n[0], rr * vr * unr + pr * n[1],
                  rr * xr * unr + pr * n[2], rr * hr * unr};

  /* Roe-averaged state */
  double sl = sqrt(rl), sr = sqrt(rr);
  double rho_t = sl * sr;
  double u_t = (sl * ul + sr * ur) / (sl + sr);
  double v_t = (sl * vl + sr * vr) / (sl + sr);
  double w_t = (sl * xl + sr * xr) / (sl + sr);
  double h_t = (sl * hl + sr * hr) / (sl + sr);
  double q2_t = u_t * u_t + v_t * v_t + w_t * w_t;
  double c2_t = (gamma - 1.0) * (h_t - 0.5 * q2_t);
  double c_t = sqrt(c2_t);
  double un_t = u_t * n[0] + v_t * n[1] + w_t * n[2];

  /* jumps */
  double drho = rr - rl, dp = pr - pl;
  double du = ur - ul, dv = vr - vl, dw = xr - xl;
  double dun = unr - unl;

  /* wave strengths: acoustic (u-c), (u+c); entropy; shear (vector) */
  double a1 = (dp - rho_t * c_t * dun) / (2.0 * c2_t);
  double a5 = (dp + rho_t * c_t * dun) / (2.0 * c2_t);
  double a2 = drho - dp / c2_t;
  double shear[3] = {rho_t * (du - dun * n[0]), rho_t * (dv - dun * n[1]),
                     rho_t * (dw - dun * n[2])};

  /* eigenvalue moduli */
  double delta = eps * (fabs(un_t) + c_t);
  double l1 = harten(un_t - c_t, delta);
  double l2 = harten(un_t, delta);
  double l5 = harten(un_t + c_t, delta);

  /* right eigenvectors of the Roe matrix */
  double r1[5] = {1.0, u_t - c_t * n[0], v_t - c_t * n[1], w_t - c_t * n[2], h_t - c_t * un_t};
  double r5[5] = {1.0, u_t + c_t * n[0], v_t + c_t * n[1], w_t + c_t * n[2], h_t + c_t * un_t};
  double r2[5] = {1.0, u_t, v_t, w_t, 0.5 * q2_t};
  double rs[5] = {0.0, shear[0], shear[1], shear[2],
                  u_t * shear[0] + v_t * shear[1] + w_t * shear[2]};

  for (int m = 0; m < 5; ++m) {
    double dissipation = l1 * a1 * r1[m] + l2 * (a2 * r2[m] + rs[m]) + l5 * a5 * r5[m];
    F[m] = area * (0.5 * (fl[m] + fr[m]) - 0.5 * dissipation);
  }
}

/* ------------------------------------------------------------------------------------------ */
/* metrics: face area vectors from the face diagonals, volumes by the divergence theorem      */

static void node_at(const double* X, int nx, int ny, int nz, int i, int j, int k, double x[3]) {
  size_t nn = (size_t)(nx + 1) * (size_t)(ny + 1) * (size_t)(nz + 1);
  size_t o = ((size_t)k * (size_t)(ny + 1) + (size_t)j) * (size_t)(nx + 1) + (size_t)i;
  x[0] = X[o];
  x[1] = X[nn + o];
  x[2] = X[2 * nn + o];
}

static void cross(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

/* area vector 0.5 * d1 x d2 of the quadrilateral p00,p10,p11,p01 (counter-clockwise seen from
 * the side it points to): d1 = p11 - p00, d2 = p01 - p10 */
static void quad_area(const double p00[3], const double p10[3], const double p11[3],
                      const double p01[3], double S[3]) {
  double d1[3] = {p11[0] - p00[0], p11[1] - p00[1], p11[2] - p00[2]};
  double d2[3] = {p01[0] - p10[0], p01[1] - p10[1], p01[2] - p10[2]};
  double c[3];
  cross(d1, d2, c);
  S[0] = 0.5 * c[0];
  S[1] = 0.5 * c[1];
  S[2] = 0.5 * c[2];
}

/* node (i, j, k) of the block, for indices beyond the block's nodes extended by reflecting
 * through the boundary node along the grid line: X(-m) = 2 X(0) - X(m), X(n + m) = 2 X(n) - X(n - m),
 * one dimension after the other */
static void node_ext(const double* X, int nx, int ny, int nz, int i, int j, int k, double x[3]) {
  double a[3], b[3];
  if (i < 0 || i > nx) {
    int e = i < 0 ? 0 : nx;
    node_ext(X, nx, ny, nz, e, j, k, a);
    node_ext(X, nx, ny, nz, 2 * e - i, j, k, b);
  } else if (j < 0 || j > ny) {
    int e = j < 0 ? 0 : ny;
    node_ext(X, nx, ny, nz, i, e, k, a);
    node_ext(X, nx, ny, nz, i, 2 * e - j, k, b);
  } else if (k < 0 || k > nz) {
    int e = k < 0 ? 0 : nz;
    node_ext(X, nx, ny, nz, i, j, e, a);
    node_ext(X, nx, ny, nz, i, j, 2 * e - k, b);
  } else {
    node_at(X, nx, ny, nz, i, j, k, x);
    return;
  }
  for (int c = 0; c < 3; ++c) x[c] = 2.0 * a[c] - b[c];
}

/* metrics of cell (i, j, k): lower-face area vectors S_xi, S_eta, S_zeta and the volume */
static void cell_metrics(const double* X, int nx, int ny, int nz, int i, int j, int k, double out[10]) {
  double c[2][2][2][3]; /* corner nodes c[dk][dj][di] */
  for (int dk = 0; dk < 2; ++dk)
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) node_ext(X, nx, ny, nz, i + di, j + dj, k + dk, c[dk][dj][di]);
  /* lower faces (towards +d) and upper faces (towards +d) of this cell */
  double sxl[3], sxu[3], syl[3], syu[3], szl[3], szu[3];
  /* xi faces: corners in the (eta, zeta) plane; eta x zeta = +xi */
  quad_area(c[0][0][0], c[0][1][0], c[1][1][0], c[1][0][0], sxl);
  quad_area(c[0][0][1], c[0][1][1], c[1][1][1], c[1][0][1], sxu);
  /* eta faces: corners in the (zeta, xi) plane; zeta x xi = +eta */
  quad_area(c[0][0][0], c[1][0][0], c[1][0][1], c[0][0][1], syl);
  quad_area(c[0][1][0], c[1][1][0], c[1][1][1], c[0][1][1], syu);
  /* zeta faces: corners in the (xi, eta) plane; xi x eta = +zeta */
  quad_area(c[0][0][0], c[0][0][1], c[0][1][1], c[0][1][0], szl);
  quad_area(c[1][0][0], c[1][0][1], c[1][1][1], c[1][1][0], szu);

  /* V = (1/3) sum over faces of (face centroid - corner 000) . outward area vector */
  double o[3] = {c[0][0][0][0], c[0][0][0][1], c[0][0][0][2]};
  double cen[6][3];
  const double* faces[6][4] = {
      {c[0][0][0], c[0][1][0], c[1][1][0], c[1][0][0]},
      {c[0][0][1], c[0][1][1], c[1][1][1], c[1][0][1]},
      {c[0][0][0], c[1][0][0], c[1][0][1], c[0][0][1]},
      {c[0][1][0], c[1][1][0], c[1][1][1], c[0][1][1]},
      {c[0][0][0], c[0][0][1], c[0][1][1], c[0][1][0]},
      {c[1][0][0], c[1][0][1], c[1][1][1], c[1][1][0]}};
  for (int f = 0; f < 6; ++f)
    for (int a = 0; a < 3; ++a)
      cen[f][a] = 0.25 * (faces[f][0][a] + faces[f][1][a] + faces[f][2][a] + faces[f][3][a]) - o[a];
  const double* outward[6] = {sxl, sxu, syl, syu, szl, szu};
  double sign[6] = {-1.0, 1.0, -1.0, 1.0, -1.0, 1.0};
  double vol = 0.0;
  for (int f = 0; f < 6; ++f)
    vol += sign[f] * (cen[f][0] * outward[f][0] + cen[f][1] * outward[f][1] + cen[f][2] * outward[f][2]);
  vol /= 3.0;
  for (int a = 0; a < 3; ++a) {
    out[0 + a] = sxl[a];
    out[3 + a] = syl[a];
    out[6 + a] = szl[a];
  }
  out[9] = vol;
}

int oracle_metrics(int nx, int ny, int nz, const double* X, double* M) {
  return oracle_metrics_bc(nx, ny, nz, X, NULL, M);
}

static int periodic_dim(const oracle_bc* bc, int d) {
  return !bc || (bc->kind[2 * d] == ORACLE_BC_PERIODIC && bc->kind[2 * d + 1] == ORACLE_BC_PERIODIC);
}

static int bad_bc(const oracle_bc* bc) {
  if (!bc) return 0;
  for (int d = 0; d < 3; ++d) {
    int a = bc->kind[2 * d], b = bc->kind[2 * d + 1];
    if (a < 0 || a > 2 || b < 0 || b > 2) return 1;
    if ((a == ORACLE_BC_PERIODIC) != (b == ORACLE_BC_PERIODIC)) return 1; /* periodic pairs only */
  }
  return 0;
}

static int wrap(int i, int n);

int oracle_metrics_bc(int nx, int ny, int nz, const double* X, const oracle_bc* bc, double* M) {
  if (bad_dims(nx, ny, nz) || !X || !M || bad_bc(bc)) return -1;
  if (bc && ((!periodic_dim(bc, 0) && nx < 2) || (!periodic_dim(bc, 1) && ny < 2) ||
             (!periodic_dim(bc, 2) && nz < 2)))
    return -1; /* the reflected halo nodes need two cells */
  grid_t g = make_grid(nx, ny, nz);
  memset(M, 0, 10 * g.ncell * sizeof(double));
  for (int k = -HALO; k < nz + HALO; ++k)
    for (int j = -HALO; j < ny + HALO; ++j)
      for (int i = -HALO; i < nx + HALO; ++i) {
        /* periodic dimensions: the periodic image (metrics are translation invariant) */
        int ii = periodic_dim(bc, 0) ? wrap(i, nx) : i;
        int jj = periodic_dim(bc, 1) ? wrap(j, ny) : j;
        int kk = periodic_dim(bc, 2) ? wrap(k, nz) : k;
        double out[10];
        cell_metrics(X, nx, ny, nz, ii, jj, kk, out);
        size_t ci = cell(&g, i, j, k);
        for (int a = 0; a < 10; ++a) M[(size_t)a * g.ncell + ci] = out[a];
      }
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* periodic halo                                                                               */

static int wrap(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

int oracle_fill_halo_periodic(int nx, int ny, int nz, int nvar, double* a) {
  if (bad_dims(nx, ny, nz) || nvar < 1 || !a) return -1;
  grid_t g = make_grid(nx, ny, nz);
  for (int v = 0; v < nvar; ++v) {
    double* f = a + (size_t)v * g.ncell;
    for (int k = -HALO; k < nz + HALO; ++k)
      for (int j = -HALO; j < ny + HALO; ++j)
        for (int i = -HALO; i < nx + HALO; ++i) {
          int inside = i >= 0 && i < nx && j >= 0 && j < ny && k >= 0 && k < nz;
          if (inside) continue;
          f[cell(&g, i, j, k)] = f[cell(&g, wrap(i, nx), wrap(j, ny), wrap(k, nz))];
        }
  }
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* boundary ghost cells (not in the paper: the usual inviscid slip wall and characteristic     */
/* far field)                                                                                  */

/* unit normal of the boundary face of direction d at the face slab point (a, b), pointing
 * towards +d; hi selects the upper face of the block */
static void face_normal(const grid_t* g, const double* M, int d, int hi, int i, int j, int k, double n[3]) {
  int idx[3] = {i, j, k};
  int nd = d == 0 ? g->nx : (d == 1 ? g->ny : g->nz);
  idx[d] = hi ? nd : 0; /* the face is the lower face of this cell */
  size_t c = cell(g, idx[0], idx[1], idx[2]);
  double S[3];
  for (int a = 0; a < 3; ++a) S[a] = M[(size_t)(3 * d + a) * g->ncell + c];
  double len = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
  for (int a = 0; a < 3; ++a) n[a] = S[a] / len;
}

/* boundary state of a FARFIELD face from the interior primitive state wi, the free stream winf
 * and the outward unit normal n */
static void farfield_state(double gamma, const double wi[5], const double winf[5], const double n[3],
                           double wb[5]) {
  double ci = sqrt(gamma * wi[4] / wi[0]), cinf = sqrt(gamma * winf[4] / winf[0]);
  double uni = wi[1] * n[0] + wi[2] * n[1] + wi[3] * n[2];
  double uninf = winf[1] * n[0] + winf[2] * n[1] + winf[3] * n[2];
  if (uninf <= -cinf) { /* supersonic inflow */
    for (int m = 0; m < 5; ++m) wb[m] = winf[m];
    return;
  }
  if (uni >= ci) { /* supersonic outflow */
    for (int m = 0; m < 5; ++m) wb[m] = wi[m];
    return;
  }
  double rplus = uni + 2.0 * ci / (gamma - 1.0);
  double rminus = uninf - 2.0 * cinf / (gamma - 1.0);
  double unb = 0.5 * (rplus + rminus);
  double cb = 0.25 * (gamma - 1.0) * (rplus - rminus);
  const double* src = unb < 0.0 ? winf : wi; /* upwind side: entropy and tangential velocity */
  double un_src = src[1] * n[0] + src[2] * n[1] + src[3] * n[2];
  double entropy = src[4] / pow(src[0], gamma);
  double rho = pow(cb * cb / (gamma * entropy), 1.0 / (gamma - 1.0));
  wb[0] = rho;
  for (int a = 0; a < 3; ++a) wb[1 + a] = src[1 + a] + (unb - un_src) * n[a];
  wb[4] = rho * cb * cb / gamma;
}

static void prim_at(double gamma, const grid_t* g, const double* Q, size_t c, double w[5]) {
  double U[5];
  for (int m = 0; m < 5; ++m) U[m] = Q[(size_t)m * g->ncell + c];
  oracle_primitive(gamma, U, w);
}

static void store_prim(double gamma, const grid_t* g, double* Q, size_t c, const double w[5]) {
  Q[c] = w[0];
  Q[g->ncell + c] = w[0] * w[1];
  Q[2 * g->ncell + c] = w[0] * w[2];
  Q[3 * g->ncell + c] = w[0] * w[3];
  Q[4 * g->ncell + c] = w[4] / (gamma - 1.0) + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
}

int oracle_fill_halo_bc(double gamma, int nx, int ny, int nz, const double* M, const oracle_bc* bc,
                        double* Q) {
  if (bad_dims(nx, ny, nz) || !Q || bad_bc(bc) || (bc && !M)) return -1;
  int rc = oracle_fill_halo_periodic(nx, ny, nz, 5, Q);
  if (rc || !bc) return rc;
  grid_t g = make_grid(nx, ny, nz);
  int n[3] = {nx, ny, nz};
  for (int d = 0; d < 3; ++d) {
    if (periodic_dim(bc, d)) continue;
    int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
    for (int hi = 0; hi < 2; ++hi) {
      int kind = bc->kind[2 * d + hi];
      for (int b = 0; b < n[d2]; ++b)
        for (int a = 0; a < n[d1]; ++a) {
          int idx[3];
          idx[d1] = a;
          idx[d2] = b;
          idx[d] = 0;
          double nrm[3];
          face_normal(&g, M, d, hi, idx[0], idx[1], idx[2], nrm);
          for (int m = 0; m < HALO; ++m) {
            int gi[3] = {idx[0], idx[1], idx[2]}, ii[3] = {idx[0], idx[1], idx[2]};
            gi[d] = hi ? n[d] + m : -1 - m;  /* ghost cell */
            ii[d] = hi ? n[d] - 1 - m : m;   /* its mirror image inside */
            double wi[5], wb[5];
            if (kind == ORACLE_BC_SLIP_WALL) {
              prim_at(gamma, &g, Q, cell(&g, ii[0], ii[1], ii[2]), wi);
              double un = wi[1] * nrm[0] + wi[2] * nrm[1] + wi[3] * nrm[2];
              wb[0] = wi[0];
              for (int x = 0; x < 3; ++x) wb[1 + x] = wi[1 + x] - 2.0 * un * nrm[x];
              wb[4] = wi[4];
            } else {
              double out[3] = {hi ? nrm[0] : -nrm[0], hi ? nrm[1] : -nrm[1], hi ? nrm[2] : -nrm[2]};
              int adj[3] = {idx[0], idx[1], idx[2]};
              adj[d] = hi ? n[d] - 1 : 0;  /* the interior cell next to the face */
              prim_at(gamma, &g, Q, cell(&g, adj[0], adj[1], adj[2]), wi);
              farfield_state(gamma, wi, bc->inf, out, wb);
            }
            store_prim(gamma, &g, Q, cell(&g, gi[0], gi[1], gi[2]), wb);
          }
        }
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* residual R(Q) of Eq. 3                                                                      */

typedef struct {
  const oracle_params* p;
  grid_t g;
  const double* M;
  const double* W; /* primitives, halo-padded, [5][ncell] */
} field_t;

static void load_w(const field_t* f, size_t c, double w[5]) {
  for (int m = 0; m < 5; ++m) w[m] = f->W[(size_t)m * f->g.ncell + c];
}

static void load_s(const field_t* f, int d, size_t c, double s[3]) {
  for (int a = 0; a < 3; ++a) s[a] = f->M[(size_t)(3 * d + a) * f->g.ncell + c];
}

static size_t stride(const grid_t* g, int d) {
  return d == 0 ? g->sx : (d == 1 ? g->sy : g->sz);
}

/* viscous flux (the Fv, Gv, Hv of Eq. 1) through the lower face of cell c in direction d.
 * Face gradients by the chain rule through the metrics: the face-normal index difference, and
 * the mean of the two cells' central index differences in the two other directions. */
static void viscous_flux(const field_t* f, int d, size_t c, double Fv[5]) {
  const grid_t* g = &f->g;
  double gamma = f->p->gamma, mu = f->p->mu, Pr = f->p->Pr;
  size_t sd = stride(g, d);
  int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  size_t s1 = stride(g, t1), s2 = stride(g, t2);
  size_t L = c - sd, R = c;
  size_t n = g->ncell;
  const double* W = f->W;

  /* the four scalar fields u, v, w, theta = p / rho */
#define PHI(q, x) ((q) < 3 ? W[(size_t)((q) + 1) * n + (x)] : W[4 * n + (x)] / W[(x)])
  double dn[4], dt1[4], dt2[4];
  for (int q = 0; q < 4; ++q) {
    dn[q] = PHI(q, R) - PHI(q, L);
    dt1[q] = 0.25 * ((PHI(q, L + s1) - PHI(q, L - s1)) + (PHI(q, R + s1) - PHI(q, R - s1)));
    dt2[q] = 0.25 * ((PHI(q, L + s2) - PHI(q, L - s2)) + (PHI(q, R + s2) - PHI(q, R - s2)));
  }
#undef PHI

  double Sf[3], a[3], b[3], cc[3], e[3], Sb1[3], Sb2[3];
  load_s(f, d, R, Sf);
  load_s(f, t1, L, a);
  load_s(f, t1, L + s1, b);
  load_s(f, t1, R, cc);
  load_s(f, t1, R + s1, e);
  for (int x = 0; x < 3; ++x) Sb1[x] = 0.25 * (a[x] + b[x] + cc[x] + e[x]);
  load_s(f, t2, L, a);
  load_s(f, t2, L + s2, b);
  load_s(f, t2, R, cc);
  load_s(f, t2, R + s2, e);
  for (int x = 0; x < 3; ++x) Sb2[x] = 0.25 * (a[x] + b[x] + cc[x] + e[x]);
  double Vf = 0.5 * (f->M[9 * n + L] + f->M[9 * n + R]);

  double grad[4][3]; /* grad[q][x] = d phi_q / d x_x */
  for (int q = 0; q < 4; ++q)
    for (int x = 0; x < 3; ++x) grad[q][x] = (dn[q] * Sf[x] + dt1[q] * Sb1[x] + dt2[q] * Sb2[x]) / Vf;

  double divu = grad[0][0] + grad[1][1] + grad[2][2];
  double tau[3][3];
  for (int r = 0; r < 3; ++r)
    for (int s = 0; s < 3; ++s) {
      tau[r][s] = mu * (grad[r][s] + grad[s][r]);
      if (r == s) tau[r][s] -= 2.0 / 3.0 * mu * divu;
    }
  double kappa = mu * gamma / ((gamma - 1.0) * Pr);
  double ubar[3];
  for (int x = 0; x < 3; ++x) ubar[x] = 0.5 * (W[(size_t)(x + 1) * n + L] + W[(size_t)(x + 1) * n + R]);

  double tS[3];
  for (int r = 0; r < 3; ++r) tS[r] = tau[r][0] * Sf[0] + tau[r][1] * Sf[1] + tau[r][2] * Sf[2];
  Fv[0] = 0.0;
  Fv[1] = tS[0];
  Fv[2] = tS[1];
  Fv[3] = tS[2];
  Fv[4] = ubar[0] * tS[0] + ubar[1] * tS[1] + ubar[2] * tS[2] +
          kappa * (grad[3][0] * Sf[0] + grad[3][1] * Sf[1] + grad[3][2] * Sf[2]);
}

/* total flux F - Fv through the lower face of cell c in direction d */
static void face_flux(const field_t* f, int d, size_t c, double F[5]) {
  size_t sd = stride(&f->g, d);
  double w0[5], w1[5], w2[5], w3[5], wl[5], wr[5], S[3];
  load_w(f, c - 2 * sd, w0);
  load_w(f, c - sd, w1);
  load_w(f, c, w2);
  load_w(f, c + sd, w3);
  oracle_muscl(f->p->limiter, w0, w1, w2, w3, wl, wr);
  load_s(f, d, c, S);
  oracle_roe_flux(f->p->gamma, f->p->eps, wl, wr, S, F);
  if (f->p->viscous) {
    double Fv[5];
    viscous_flux(f, d, c, Fv);
    for (int m = 0; m < 5; ++m) F[m] -= Fv[m];
  }
}

static double* primitives(const oracle_params* p, const grid_t* g, const double* Q) {
  double* W = (double*)malloc(5 * g->ncell * sizeof(double));
  if (!W) return NULL;
  long long nc = (long long)g->ncell;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (long long c = 0; c < nc; ++c) {
    double U[5], w[5];
    for (int m = 0; m < 5; ++m) U[m] = Q[(size_t)m * g->ncell + (size_t)c];
    oracle_primitive(p->gamma, U, w);
    for (int m = 0; m < 5; ++m) W[(size_t)m * g->ncell + (size_t)c] = w[m];
  }
  return W;
}

int oracle_residual(const oracle_params* p, int nx, int ny, int nz, const double* M,
                    const double* Q, double* R) {
  if (!p || bad_dims(nx, ny, nz) || !M || !Q || !R) return -1;
  grid_t g = make_grid(nx, ny, nz);
  double* W = primitives(p, &g, Q);
  if (!W) return -2;
  field_t f = {p, g, M, W};

  /* face-flux arrays: direction d has n_d + 1 faces along d */
  int ext[3][3] = {{nx + 1, ny, nz}, {nx, ny + 1, nz}, {nx, ny, nz + 1}};
  double* Fd[3];
  for (int d = 0; d < 3; ++d) {
    size_t nf = (size_t)ext[d][0] * ext[d][1] * ext[d][2];
    Fd[d] = (double*)malloc(5 * nf * sizeof(double));
    if (!Fd[d]) {
      for (int e = 0; e < d; ++e) free(Fd[e]);
      free(W);
      return -2;
    }
    /* face (i,j,k) of direction d is the lower face of cell (i,j,k) */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int k = 0; k < ext[d][2]; ++k)
      for (int j = 0; j < ext[d][1]; ++j)
        for (int i = 0; i < ext[d][0]; ++i) {
          double F[5];
          face_flux(&f, d, cell(&g, i, j, k), F);
          size_t o = ((size_t)k * ext[d][1] + (size_t)j) * ext[d][0] + (size_t)i;
          for (int m = 0; m < 5; ++m) Fd[d][(size_t)m * nf + o] = F[m];
        }
  }

  /* cell residual: fixed order -x, +x, -y, +y, -z, +z, divided by the volume */
  size_t nint = (size_t)nx * ny * nz;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t nfx = (size_t)(nx + 1) * ny * nz, nfy = (size_t)nx * (ny + 1) * nz,
               nfz = (size_t)nx * ny * (nz + 1);
        size_t xm = ((size_t)k * ny + j) * (nx + 1) + i, xp = xm + 1;
        size_t ym = ((size_t)k * (ny + 1) + j) * nx + i, yp = ym + nx;
        size_t zm = ((size_t)k * ny + j) * nx + i, zp = zm + (size_t)nx * ny;
        double vol = M[9 * g.ncell + cell(&g, i, j, k)];
        size_t o = ((size_t)k * ny + j) * nx + i;
        for (int m = 0; m < 5; ++m) {
          double acc = -Fd[0][m * nfx + xm];
          acc += Fd[0][m * nfx + xp];
          acc -= Fd[1][m * nfy + ym];
          acc += Fd[1][m * nfy + yp];
          acc -= Fd[2][m * nfz + zm];
          acc += Fd[2][m * nfz + zp];
          R[(size_t)m * nint + o] = acc / vol;
        }
      }
  for (int d = 0; d < 3; ++d) free(Fd[d]);
  free(W);
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* time step: dt = CFL * min over cells of V / sum_d (convective + 4 * viscous spectral radius) */

/* the CFL time step of one cell: CFL V / sum over directions of the spectral radius with the
 * cell-averaged area vector (mean of its lower and upper faces) */
static double cell_dt(const oracle_params* p, const grid_t* g, const double* M, const double* Q, size_t c) {
  double visc_factor = 4.0 / 3.0 > p->gamma / p->Pr ? 4.0 / 3.0 : p->gamma / p->Pr;
  double U[5], w[5];
  for (int m = 0; m < 5; ++m) U[m] = Q[(size_t)m * g->ncell + c];
  oracle_primitive(p->gamma, U, w);
  double a = sqrt(p->gamma * w[4] / w[0]);
  double vol = M[9 * g->ncell + c];
  double sum = 0.0;
  for (int d = 0; d < 3; ++d) {
    size_t up = c + stride(g, d);
    double Sb[3];
    for (int x = 0; x < 3; ++x)
      Sb[x] = 0.5 * (M[(size_t)(3 * d + x) * g->ncell + c] + M[(size_t)(3 * d + x) * g->ncell + up]);
    double s2 = Sb[0] * Sb[0] + Sb[1] * Sb[1] + Sb[2] * Sb[2];
    double lam = fabs(w[1] * Sb[0] + w[2] * Sb[1] + w[3] * Sb[2]) + a * sqrt(s2);
    if (p->viscous) lam += 4.0 * visc_factor * (p->mu / w[0]) * s2 / vol;
    sum += lam;
  }
  return p->cfl * vol / sum;
}

int oracle_dt(const oracle_params* p, int nx, int ny, int nz, const double* M, const double* Q,
              double* dt) {
  if (!p || bad_dims(nx, ny, nz) || !M || !Q || !dt) return -1;
  grid_t g = make_grid(nx, ny, nz);
  double best = INFINITY;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double local = cell_dt(p, &g, M, Q, cell(&g, i, j, k));
        if (local < best) best = local;
      }
  *dt = best;
  return 0;
}

int oracle_dt_local(const oracle_params* p, int nx, int ny, int nz, const double* M, const double* Q,
                    double* dt) {
  if (!p || bad_dims(nx, ny, nz) || !M || !Q || !dt) return -1;
  grid_t g = make_grid(nx, ny, nz);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) dt[((size_t)k * ny + j) * nx + i] = cell_dt(p, &g, M, Q, cell(&g, i, j, k));
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* residual norms and the Runge-Kutta stages                                                   */

int oracle_norms(size_t n, const double* R, double out[5]) {
  if (!R || !out || n == 0) return -1;
  for (int m = 0; m < 5; ++m) {
    double s = 0.0;
    for (size_t c = 0; c < n; ++c) s += R[(size_t)m * n + c] * R[(size_t)m * n + c];
    out[m] = sqrt(s / (double)n);
  }
  return 0;
}

/* Eqs. 4-6 with lambda = -dt:
 *   stage 1: Q1 = Qn - dt R(Qn)
 *   stage 2: Q2 = 3/4 Qn + 1/4 (Q1 - dt R(Q1))
 *   stage 3: Q  = 1/3 Qn + 2/3 (Q2 - dt R(Q2)) */
/* one stage with the time step dtc[c % ncell] of every cell when dtc is not NULL, else dt */
static int rk3_stage_impl(int stage, size_t n, const double* Qn, const double* Qs, const double* R,
                          double dt, const double* dtc, size_t ncell, double* Qout) {
  if (stage < 1 || stage > 3 || !Qn || !Qs || !R || !Qout) return -1;
  for (size_t c = 0; c < n; ++c) {
    double h = dtc ? dtc[c % ncell] : dt;
    double advanced = Qs[c] - h * R[c];
    if (stage == 1) Qout[c] = advanced;
    else if (stage == 2) Qout[c] = 0.75 * Qn[c] + 0.25 * advanced;
    else Qout[c] = Qn[c] / 3.0 + 2.0 / 3.0 * advanced;
  }
  return 0;
}

int oracle_rk3_stage(int stage, size_t n, const double* Qn, const double* Qs, const double* R,
                     double dt, double* Qout) {
  return rk3_stage_impl(stage, n, Qn, Qs, R, dt, NULL, 1, Qout);
}

/* scatter a compact interior residual into a halo-padded array (halo entries zero) */
static void pad_residual(const grid_t* g, const double* R, double* Rp) {
  memset(Rp, 0, 5 * g->ncell * sizeof(double));
  size_t nint = (size_t)g->nx * g->ny * g->nz;
  for (int m = 0; m < 5; ++m)
    for (int k = 0; k < g->nz; ++k)
      for (int j = 0; j < g->ny; ++j)
        for (int i = 0; i < g->nx; ++i)
          Rp[(size_t)m * g->ncell + cell(g, i, j, k)] =
              R[(size_t)m * nint + ((size_t)k * g->ny + j) * g->nx + i];
}

static int step_impl(const oracle_params* p, int nx, int ny, int nz, const double* M, const oracle_bc* bc,
                     int local_dt, double* Q, int nsteps, int cfl_dt, double fixed_dt, double* dts,
                     double* norms) {
  if (!p || bad_dims(nx, ny, nz) || !M || !Q || nsteps < 0 || bad_bc(bc)) return -1;
  grid_t g = make_grid(nx, ny, nz);
  size_t nint = (size_t)nx * ny * nz;
  size_t nall = 5 * g.ncell;
  double* R = (double*)malloc(5 * nint * sizeof(double));
  double* Rp = (double*)malloc(nall * sizeof(double));
  double* Q1 = (double*)malloc(nall * sizeof(double));
  double* Q2 = (double*)malloc(nall * sizeof(double));
  double* dl = local_dt ? (double*)malloc(nint * sizeof(double)) : NULL;
  double* dlp = local_dt ? (double*)calloc(g.ncell, sizeof(double)) : NULL;  /* halo entries 0 */
  int rc = 0;
  if (!R || !Rp || !Q1 || !Q2 || (local_dt && (!dl || !dlp))) { rc = -2; goto done; }
  for (int s = 0; s < nsteps; ++s) {
    double dt = fixed_dt;
    oracle_fill_halo_bc(p->gamma, nx, ny, nz, M, bc, Q);
    if (local_dt) {
      oracle_dt_local(p, nx, ny, nz, M, Q, dl);
      dt = INFINITY;
      for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
          for (int i = 0; i < nx; ++i) {
            double v = dl[((size_t)k * ny + j) * nx + i];
            dlp[cell(&g, i, j, k)] = v;
            if (v < dt) dt = v;
          }
    } else if (cfl_dt) {
      oracle_dt(p, nx, ny, nz, M, Q, &dt);
    }
    if (dts) dts[s] = dt;

    oracle_residual(p, nx, ny, nz, M, Q, R);
    if (norms) oracle_norms(nint, R, norms + 5 * (size_t)s);
    pad_residual(&g, R, Rp);
    rk3_stage_impl(1, nall, Q, Q, Rp, dt, dlp, g.ncell, Q1);

    oracle_fill_halo_bc(p->gamma, nx, ny, nz, M, bc, Q1);
    oracle_residual(p, nx, ny, nz, M, Q1, R);
    pad_residual(&g, R, Rp);
    rk3_stage_impl(2, nall, Q, Q1, Rp, dt, dlp, g.ncell, Q2);

    oracle_fill_halo_bc(p->gamma, nx, ny, nz, M, bc, Q2);
    oracle_residual(p, nx, ny, nz, M, Q2, R);
    pad_residual(&g, R, Rp);
    rk3_stage_impl(3, nall, Q, Q2, Rp, dt, dlp, g.ncell, Q);
  }
  oracle_fill_halo_bc(p->gamma, nx, ny, nz, M, bc, Q);
done:
  free(R);
  free(Rp);
  free(Q1);
  free(Q2);
  free(dl);
  free(dlp);
  return rc;
}

int oracle_step(const oracle_params* p, int nx, int ny, int nz, const double* M, double* Q,
                int nsteps, double* dts, double* norms) {
  return step_impl(p, nx, ny, nz, M, NULL, 0, Q, nsteps, 1, 0.0, dts, norms);
}

int oracle_step_fixed_dt(const oracle_params* p, int nx, int ny, int nz, const double* M,
                         double* Q, int nsteps, double dt, double* norms) {
  return step_impl(p, nx, ny, nz, M, NULL, 0, Q, nsteps, 0, dt, NULL, norms);
}

int oracle_step_ex(const oracle_params* p, int nx, int ny, int nz, const double* M, const oracle_bc* bc,
                   int local_dt, double fixed_dt, double* Q, int nsteps, double* dts, double* norms) {
  if (local_dt && fixed_dt > 0.0) return -1;
  return step_impl(p, nx, ny, nz, M, bc, local_dt, Q, nsteps, fixed_dt > 0.0 ? 0 : 1, fixed_dt, dts, norms);
}
