/*
 * wcns.c -- plain FP64 CPU oracle of the paper's own spatial scheme: the fifth-order explicit
 * weighted compact nonlinear scheme WCNS-E-5 of arXiv 1710.09995 Sec. 2.2 (Eq. 2), with
 * fourth-order central viscous derivatives, on periodic uniform Cartesian blocks.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the benchmark's CPU
 * baseline, never by the CUDA library or its Python binding.  Written to be checked by eye
 * against the paper; straight loops over lines, faces and cells.
 *
 * What the paper fixes (Sec. 2.2): the inviscid derivative at a cell centre i is Eq. 2, a
 * combination of flux differences at the cell edges i +- 1/2, i +- 3/2, i +- 5/2, where each edge
 * flux comes from a flux function of the left-hand and right-hand cell-edge flow variables, and
 * those come from a fifth-order weighted nonlinear interpolation; viscous derivatives are
 * fourth-order central differences.  Where it is silent this oracle takes (its readings):
 *   - interpolated variables: the primitive ones (rho, u, v, w, p), component by component;
 *   - interpolation: three three-point candidate stencils S0 = {i-2, i-1, i}, S1 = {i-1, i, i+1},
 *     S2 = {i, i+1, i+2}; on each, the first and second differences g_k, s_k (h u', h^2 u'') give
 *     the candidate edge value u_i + g_k / 2 + s_k / 8 and the smoothness indicator
 *     beta_k = g_k^2 + s_k^2; weights alpha_k = C_k / (EPS + beta_k)^2 with the optimal weights
 *     C = (1/16, 10/16, 5/16) (which make the combination the unique fifth-order interpolation)
 *     and EPS = 1e-6, normalised to sum 1.  `limiter` = 1 uses the optimal weights themselves
 *     (linear fifth-order interpolation; for order tests).  The right-hand value at i + 1/2 is
 *     the same interpolation on the mirrored stencil i+3, i+2, i+1, i, i-1;
 *   - flux function: the Roe flux with Harten's entropy fix of the finite-volume oracle, per
 *     unit area, normal along the axis;
 *   - viscous terms: at every cell centre the gradients of u, v, w and theta = p / rho by the
 *     fourth-order central difference D4 f_i = (f_{i-2} - 8 f_{i-1} + 8 f_{i+1} - f_{i+2}) / (12 h),
 *     the Stokes stress with constant mu and the heat flux -kappa grad theta give the viscous
 *     flux vectors Fv, Gv, Hv of Eq. 1 at the cell centres, whose derivatives are D4 again;
 *   - R = dF/dx + dG/dy + dH/dz - (dFv/dx + dGv/dy + dHv/dz), so that dQ/dt = -R (Eq. 3).
 * Arrays are compact q[5][nz][ny][nx] (x fastest); periodic neighbours by index wrap.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define WCNS_EPS 1e-6

static int wrap(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

double oracle_wcns_edge(int linear, const double u[5]) {
  /* u[0..4] = u_{i-2} .. u_{i+2}; the value at i + 1/2 interpolated from the left */
  const double C[3] = {1.0 / 16.0, 10.0 / 16.0, 5.0 / 16.0};
  double g[3], s[3];
  g[0] = 0.5 * (u[0] - 4.0 * u[1] + 3.0 * u[2]);
  s[0] = u[0] - 2.0 * u[1] + u[2];
  g[1] = 0.5 * (u[3] - u[1]);
  s[1] = u[1] - 2.0 * u[2] + u[3];
  g[2] = 0.5 * (-3.0 * u[2] + 4.0 * u[3] - u[4]);
  s[2] = u[2] - 2.0 * u[3] + u[4];
  double w[3];
  if (linear) {
    for (int k = 0; k < 3; ++k) w[k] = C[k];
  } else {
    double alpha[3], total = 0.0;
    for (int k = 0; k < 3; ++k) {
      double beta = g[k] * g[k] + s[k] * s[k];
      alpha[k] = C[k] / ((WCNS_EPS + beta) * (WCNS_EPS + beta));
      total += alpha[k];
    }
    for (int k = 0; k < 3; ++k) w[k] = alpha[k] / total;
  }
  double value = 0.0;
  for (int k = 0; k < 3; ++k) value += w[k] * (u[2] + 0.5 * g[k] + 0.125 * s[k]);
  return value;
}

/* index of cell (i, j, k) of a compact field */
static size_t at(int nx, int ny, int i, int j, int k) {
  return ((size_t)k * ny + j) * nx + i;
}

/* primitive state of every cell, W[5][cells] */
static void primitives(double gamma, size_t n, const double* Q, double* W) {
  for (size_t c = 0; c < n; ++c) {
    double U[5], P[5];
    for (int m = 0; m < 5; ++m) U[m] = Q[(size_t)m * n + c];
    oracle_primitive(gamma, U, P);
    for (int m = 0; m < 5; ++m) W[(size_t)m * n + c] = P[m];
  }
}

/* the cell of line position s: direction d, line through (i, j, k) */
static size_t line_cell(int nx, int ny, int nz, int d, int i, int j, int k, int s) {
  if (d == 0) return at(nx, ny, wrap(s, nx), j, k);
  if (d == 1) return at(nx, ny, i, wrap(s, ny), k);
  return at(nx, ny, i, j, wrap(s, nz));
}

/* Eq. 2: add dF/dx_d to R along every line of direction d */
static void inviscid_direction(const oracle_params* p, int nx, int ny, int nz, int d, double h,
                               const double* W, double* R) {
  size_t n = (size_t)nx * ny * nz;
  int len = d == 0 ? nx : (d == 1 ? ny : nz);
  int na = d == 0 ? ny : nx;  /* the two transverse extents */
  int nb = d == 2 ? ny : nz;
  double S[3] = {0.0, 0.0, 0.0};
  S[d] = 1.0;
#pragma omp parallel for collapse(2) schedule(static)
  for (int b = 0; b < nb; ++b)
    for (int a = 0; a < na; ++a) {
      int i = d == 0 ? 0 : a, j = d == 1 ? 0 : (d == 0 ? a : b), k = d == 2 ? 0 : b;
      double* F = (double*)malloc((size_t)len * 5 * sizeof(double));
      if (!F) continue;
      /* face f lies between cells f and f+1 (index f + 1/2) */
      for (int f = 0; f < len; ++f) {
        double wl[5], wr[5];
        for (int m = 0; m < 5; ++m) {
          double left[5], right[5];
          for (int t = 0; t < 5; ++t) {
            left[t] = W[(size_t)m * n + line_cell(nx, ny, nz, d, i, j, k, f - 2 + t)];
            right[t] = W[(size_t)m * n + line_cell(nx, ny, nz, d, i, j, k, f + 3 - t)];
          }
          wl[m] = oracle_wcns_edge(p->limiter, left);
          wr[m] = oracle_wcns_edge(p->limiter, right);
        }
        oracle_roe_flux(p->gamma, p->eps, wl, wr, S, F + 5 * (size_t)f);
      }
      /* Eq. 2 at cell c: F_{c+1/2} is face c, F_{c-1/2} face c-1, and so on */
      for (int c = 0; c < len; ++c) {
        size_t cc = line_cell(nx, ny, nz, d, i, j, k, c);
        for (int m = 0; m < 5; ++m) {
          double fp1 = F[5 * (size_t)wrap(c, len) + m], fm1 = F[5 * (size_t)wrap(c - 1, len) + m];
          double fp3 = F[5 * (size_t)wrap(c + 1, len) + m], fm3 = F[5 * (size_t)wrap(c - 2, len) + m];
          double fp5 = F[5 * (size_t)wrap(c + 2, len) + m], fm5 = F[5 * (size_t)wrap(c - 3, len) + m];
          double deriv = 75.0 / 64.0 * (fp1 - fm1) - 25.0 / 384.0 * (fp3 - fm3) + 3.0 / 640.0 * (fp5 - fm5);
          R[(size_t)m * n + cc] += deriv / h;
        }
      }
      free(F);
    }
}

/* fourth-order central first derivative along d of field f at (i, j, k) */
static double d4(int nx, int ny, int nz, int d, const double* f, int i, int j, int k, double h) {
  int s = d == 0 ? i : (d == 1 ? j : k);
  double fm2 = f[line_cell(nx, ny, nz, d, i, j, k, s - 2)];
  double fm1 = f[line_cell(nx, ny, nz, d, i, j, k, s - 1)];
  double fp1 = f[line_cell(nx, ny, nz, d, i, j, k, s + 1)];
  double fp2 = f[line_cell(nx, ny, nz, d, i, j, k, s + 2)];
  return (fm2 - 8.0 * fm1 + 8.0 * fp1 - fp2) / (12.0 * h);
}

/* subtract dFv/dx + dGv/dy + dHv/dz from R */
static int viscous_terms(const oracle_params* p, int nx, int ny, int nz, const double h[3],
                         const double* W, double* R) {
  size_t n = (size_t)nx * ny * nz;
  double kappa = p->mu * p->gamma / ((p->gamma - 1.0) * p->Pr);
  double* theta = (double*)malloc(n * sizeof(double));
  double* Fv = (double*)malloc(3 * 4 * n * sizeof(double)); /* [d][momentum x, y, z, energy][cells] */
  if (!theta || !Fv) {
    free(theta);
    free(Fv);
    return -2;
  }
  for (size_t c = 0; c < n; ++c) theta[c] = W[4 * n + c] / W[c];
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t c = at(nx, ny, i, j, k);
        double grad[3][3], gtheta[3], vel[3];
        for (int a = 0; a < 3; ++a) {
          vel[a] = W[(size_t)(1 + a) * n + c];
          for (int b = 0; b < 3; ++b) grad[a][b] = d4(nx, ny, nz, b, W + (size_t)(1 + a) * n, i, j, k, h[b]);
        }
        for (int b = 0; b < 3; ++b) gtheta[b] = d4(nx, ny, nz, b, theta, i, j, k, h[b]);
        double div = grad[0][0] + grad[1][1] + grad[2][2];
        for (int d = 0; d < 3; ++d) {
          double tau[3];
          for (int a = 0; a < 3; ++a) {
            tau[a] = p->mu * (grad[a][d] + grad[d][a]);
            if (a == d) tau[a] -= 2.0 / 3.0 * p->mu * div;
          }
          for (int a = 0; a < 3; ++a) Fv[((size_t)d * 4 + a) * n + c] = tau[a];
          Fv[((size_t)d * 4 + 3) * n + c] = vel[0] * tau[0] + vel[1] * tau[1] + vel[2] * tau[2] + kappa * gtheta[d];
        }
      }
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t c = at(nx, ny, i, j, k);
        for (int a = 0; a < 4; ++a) {
          double total = 0.0;
          for (int d = 0; d < 3; ++d) total += d4(nx, ny, nz, d, Fv + ((size_t)d * 4 + a) * n, i, j, k, h[d]);
          R[(size_t)(1 + a) * n + c] -= total;
        }
      }
  free(theta);
  free(Fv);
  return 0;
}

int oracle_wcns_residual(const oracle_params* p, int nx, int ny, int nz, const double h[3], const double* Q,
                         double* R) {
  if (!p || nx < 1 || ny < 1 || nz < 1 || !h || !Q || !R) return -1;
  size_t n = (size_t)nx * ny * nz;
  double* W = (double*)malloc(5 * n * sizeof(double));
  if (!W) return -2;
  primitives(p->gamma, n, Q, W);
  memset(R, 0, 5 * n * sizeof(double));
  for (int d = 0; d < 3; ++d) inviscid_direction(p, nx, ny, nz, d, h[d], W, R);
  int rc = 0;
  if (p->viscous) rc = viscous_terms(p, nx, ny, nz, h, W, R);
  free(W);
  return rc;
}

/* the global CFL time step: cfl / max over cells of sum_d [(|u_d| + c) / h_d + viscous term],
 * the viscous term 4 max(4/3, gamma/Pr) (mu/rho) / h_d^2 (the finite-volume oracle's rate on a
 * uniform Cartesian grid) */
int oracle_wcns_dt(const oracle_params* p, int nx, int ny, int nz, const double h[3], const double* Q,
                   double* dt) {
  if (!p || nx < 1 || ny < 1 || nz < 1 || !h || !Q || !dt) return -1;
  size_t n = (size_t)nx * ny * nz;
  double visc_factor = fmax(4.0 / 3.0, p->gamma / p->Pr);
  double worst = 0.0;
  for (size_t c = 0; c < n; ++c) {
    double U[5], w[5];
    for (int m = 0; m < 5; ++m) U[m] = Q[(size_t)m * n + c];
    oracle_primitive(p->gamma, U, w);
    double a = sqrt(p->gamma * w[4] / w[0]);
    double rate = 0.0;
    for (int d = 0; d < 3; ++d) {
      rate += (fabs(w[1 + d]) + a) / h[d];
      if (p->viscous) rate += 4.0 * visc_factor * (p->mu / w[0]) / (h[d] * h[d]);
    }
    if (rate > worst) worst = rate;
  }
  *dt = p->cfl / worst;
  return 0;
}

int oracle_wcns_step(const oracle_params* p, int nx, int ny, int nz, const double h[3], double* Q, int nsteps,
                     double fixed_dt, double* dts, double* norms) {
  if (!p || nx < 1 || ny < 1 || nz < 1 || !h || !Q || nsteps < 0) return -1;
  size_t n = (size_t)nx * ny * nz;
  double* R = (double*)malloc(5 * n * sizeof(double));
  double* Q1 = (double*)malloc(5 * n * sizeof(double));
  double* Q2 = (double*)malloc(5 * n * sizeof(double));
  int rc = 0;
  if (!R || !Q1 || !Q2) {
    rc = -2;
    goto done;
  }
  for (int s = 0; s < nsteps && rc == 0; ++s) {
    double dt = fixed_dt;
    if (fixed_dt <= 0.0) oracle_wcns_dt(p, nx, ny, nz, h, Q, &dt);
    if (dts) dts[s] = dt;
    rc |= oracle_wcns_residual(p, nx, ny, nz, h, Q, R);
    if (norms) oracle_norms(n, R, norms + 5 * (size_t)s);
    oracle_rk3_stage(1, 5 * n, Q, Q, R, dt, Q1);
    rc |= oracle_wcns_residual(p, nx, ny, nz, h, Q1, R);
    oracle_rk3_stage(2, 5 * n, Q, Q1, R, dt, Q2);
    rc |= oracle_wcns_residual(p, nx, ny, nz, h, Q2, R);
    oracle_rk3_stage(3, 5 * n, Q, Q2, R, dt, Q);
  }
done:
  free(R);
  free(Q1);
  free(Q2);
  return rc;
}
