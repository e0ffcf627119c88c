// physics.cuh -- per-face arithmetic of the finite-volume residual (arXiv 1710.09995 Sec. 2.2):
// MUSCL cell-edge states with the minmod limiter, Roe flux with Harten's entropy fix, central
// viscous flux (Eq. 1's Fv, Gv, Hv).  Templated on the flux precision T (double for the FP64
// path, float for the mixed path).  Faces of a Cartesian block are axis-aligned, so the flux is
// evaluated in the face frame (normal, tangent 1, tangent 2) and mapped back to x, y, z.
#pragma once
#include <cuda_runtime.h>

namespace gbcfd {

template <typename T> struct Fast;
template <> struct Fast<double> {
  static __device__ __forceinline__ double rsqrt(double x) { return ::rsqrt(x); }
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
  static __device__ __forceinline__ double sqrt_(double x) { return ::sqrt(x); }
  static __device__ __forceinline__ double mn(double a, double b) { return fmin(a, b); }
  static __device__ __forceinline__ double mx(double a, double b) { return fmax(a, b); }
  static __device__ __forceinline__ double ab(double a) { return fabs(a); }
};
template <> struct Fast<float> {
  static __device__ __forceinline__ float rsqrt(float x) { return rsqrtf(x); }
  static __device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
  static __device__ __forceinline__ float sqrt_(float x) { return x * rsqrtf(x); }
  static __device__ __forceinline__ float mn(float a, float b) { return fminf(a, b); }
  static __device__ __forceinline__ float mx(float a, float b) { return fmaxf(a, b); }
  static __device__ __forceinline__ float ab(float a) { return fabsf(a); }
};

template <typename T> struct Consts {
  T gm1;     // gamma - 1
  T ggm1;    // gamma / (gamma - 1)
  T eps;     // entropy-fix fraction
  T mu;      // viscosity
  T kappa;   // mu gamma / ((gamma - 1) Pr)
  int lim;   // 0 minmod, 1 central slope
};

// half the limited slope from the backward and forward differences.  minmod without compares:
// (copysign(1/4, a) + copysign(1/4, b)) * min(|a|, |b|) is 0.5 min(a,b) when both are positive,
// 0.5 max(a,b) when both are negative and 0 otherwise -- exactly 0.5 * minmod(a, b) (the sum is
// 0, +-1/2 and the product by a power of two is exact).
template <typename T>
__device__ __forceinline__ T half_slope(T dm, T dp, int lim) {
  using F = Fast<T>;
  if (lim) return T(0.25) * (dm + dp);
  return (copysign(T(0.25), dm) + copysign(T(0.25), dp)) * F::mn(F::ab(dm), F::ab(dp));
}

// Roe flux per unit area in the face frame.  L, R: (rho, u_n, u_t1, u_t2, p).
// F: (mass, normal momentum, t1 momentum, t2 momentum, energy).
template <typename T>
__device__ __forceinline__ void roe_frame(const T* L, const T* R, const Consts<T>& K, T* F) {
  using Fm = Fast<T>;
  const T rl = L[0], ul = L[1], vl = L[2], wl = L[3], pl = L[4];
  const T rr = R[0], ur = R[1], vr = R[2], wr = R[3], pr = R[4];
  const T isl = Fm::rsqrt(rl), isr = Fm::rsqrt(rr);
  const T sl = rl * isl, sr = rr * isr;          // sqrt(rho)
  const T hl = K.ggm1 * pl * (isl * isl) + T(0.5) * (ul * ul + vl * vl + wl * wl);
  const T hr = K.ggm1 * pr * (isr * isr) + T(0.5) * (ur * ur + vr * vr + wr * wr);
  const T ml = rl * ul, mr = rr * ur;            // mass fluxes
  // Roe averages
  const T iw = Fm::rcp(sl + sr);
  const T al = sl * iw, ar = sr * iw;
  const T ut = al * ul + ar * ur, vt = al * vl + ar * vr, wt = al * wl + ar * wr;
  const T ht = al * hl + ar * hr;
  const T q2 = ut * ut + vt * vt + wt * wt;
  const T c2 = K.gm1 * (ht - T(0.5) * q2);
  const T ic = Fm::rsqrt(c2);
  const T c = c2 * ic, ic2 = ic * ic;
  const T rt = sl * sr;
  // jumps and wave strengths
  const T drho = rr - rl, dp = pr - pl, dun = ur - ul, dt1 = vr - vl, dt2 = wr - wl;
  const T rcd = rt * c * dun;
  const T a1 = T(0.5) * (dp - rcd) * ic2;
  const T a5 = T(0.5) * (dp + rcd) * ic2;
  const T a2 = drho - dp * ic2;
  const T s1 = rt * dt1, s2 = rt * dt2;          // shear strengths (normal part is zero)
  // eigenvalue moduli with Harten's fix
  const T delta = K.eps * (Fm::ab(ut) + c);
  const T hid = delta > T(0) ? T(0.5) * Fm::rcp(delta) : T(0);
  T l1 = ut - c, l2 = ut, l5 = ut + c;
  l1 = Fm::ab(l1) < delta ? (l1 * l1 + delta * delta) * hid : Fm::ab(l1);
  l2 = Fm::ab(l2) < delta ? (l2 * l2 + delta * delta) * hid : Fm::ab(l2);
  l5 = Fm::ab(l5) < delta ? (l5 * l5 + delta * delta) * hid : Fm::ab(l5);
  const T w1 = l1 * a1, w5 = l5 * a5, w2 = l2 * a2;
  const T d0 = w1 + w2 + w5;
  const T dn = w1 * (ut - c) + w2 * ut + w5 * (ut + c);
  const T dv = (w1 + w2 + w5) * vt + l2 * s1;
  const T dw = (w1 + w2 + w5) * wt + l2 * s2;
  const T de = w1 * (ht - c * ut) + l2 * (a2 * T(0.5) * q2 + vt * s1 + wt * s2) + w5 * (ht + c * ut);
  F[0] = T(0.5) * ((ml + mr) - d0);
  F[1] = T(0.5) * ((ml * ul + pl + mr * ur + pr) - dn);
  F[2] = T(0.5) * ((ml * vl + mr * vr) - dv);
  F[3] = T(0.5) * ((ml * wl + mr * wr) - dw);
  F[4] = T(0.5) * ((ml * hl + mr * hr) - de);
}

// Viscous flux per unit area in the face frame from index-space differences:
//   gn[q]  = d(phi_q)/dn at the face,  q = u_n, u_t1, u_t2, theta
//   dnt1   = d(u_n)/dt1,  dnt2 = d(u_n)/dt2,  dt1t1 = d(u_t1)/dt1,  dt2t2 = d(u_t2)/dt2
//   ub     = face-average (u_n, u_t1, u_t2)
template <typename T>
__device__ __forceinline__ void viscous_frame(const T* gn, T dnt1, T dnt2, T dt1t1, T dt2t2,
                                              const T* ub, const Consts<T>& K, T* Fv) {
  const T div = gn[0] + dt1t1 + dt2t2;
  const T tnn = K.mu * (T(2) * gn[0] - T(2.0 / 3.0) * div);
  const T tt1 = K.mu * (gn[1] + dnt1);
  const T tt2 = K.mu * (gn[2] + dnt2);
  Fv[0] = T(0);
  Fv[1] = tnn;
  Fv[2] = tt1;
  Fv[3] = tt2;
  Fv[4] = ub[0] * tnn + ub[1] * tt1 + ub[2] * tt2 + K.kappa * gn[3];
}

}  // namespace gbcfd
