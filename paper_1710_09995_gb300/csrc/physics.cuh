// physics.cuh -- per-face arithmetic of the finite-volume residual (arXiv 1710.09995 Sec. 2.2):
// MUSCL cell-edge states with the minmod limiter, Roe flux with Harten's entropy fix, central
// viscous flux (Eq. 1's Fv, Gv, Hv).  Written once over the value type V (vmath.cuh): double for
// the FP64 path, float for the mixed path.  Faces of
// a Cartesian block are axis-aligned, so the flux is evaluated in the face frame (normal,
// tangent 1, tangent 2) and mapped back to x, y, z by the caller.
#pragma once
#include "vmath.cuh"

namespace gbcfd {

template <typename V> struct Consts {
  V gm1;     // gamma - 1
  V ggm1;    // gamma / (gamma - 1)
  V eps;     // entropy-fix fraction
  V mu;      // viscosity
  V kappa;   // mu gamma / ((gamma - 1) Pr)
  int lim;   // 0 minmod, 1 central slope
};

// constants of the spectral-radius rate (time step): gamma and 4 max(4/3, gamma/Pr) mu
template <typename V> struct RateK { V gam, vf; };

template <typename V>
__device__ __forceinline__ Consts<V> make_consts(double gamma, double eps, double mu, double Pr, int lim) {
  using O = VM<V>;
  using S = typename O::S;
  Consts<V> K;
  K.gm1 = O::c(S(gamma - 1.0));
  K.ggm1 = O::c(S(gamma / (gamma - 1.0)));
  K.eps = O::c(S(eps));
  K.mu = O::c(S(mu));
  K.kappa = O::c(S(Pr > 0.0 ? mu * gamma / ((gamma - 1.0) * Pr) : 0.0));
  K.lim = lim;
  return K;
}

// MUSCL states at the face between w1 and w2 of the stencil w0..w3 (one variable).  minmod
// without compares: (copysign(1/4, a) + copysign(1/4, b)) * min(|a|, |b|) is exactly half the
// minmod slope (0.5 min(a,b) when both are positive, 0.5 max(a,b) when both are negative, 0
// otherwise: the sum is 0 or +-1/2 and a product by a power of two is exact).  In FP64 the same
// halved slope comes from integer operations on the bit patterns (half_minmod_f64), so the
// states are the same bits without any FP64-pipe comparison.
template <typename V>
__device__ __forceinline__ void muscl(V w0, V w1, V w2, V w3, int lim, V& L, V& R) {
  using O = VM<V>;
  const V d01 = w1 - w0, d12 = w2 - w1, d23 = w3 - w2;
  if (lim) {
    const V q = O::c(0.25);
    L = O::fma(q, d01 + d12, w1);
    R = w2 - q * (d12 + d23);
  } else if constexpr (sizeof(V) == 8) {  // FP64: the halved slopes on the integer pipe (same bits)
    L = w1 + half_minmod_f64(d01, d12);
    R = w2 - half_minmod_f64(d12, d23);
  } else {
    const V q = O::c(0.25);
    const V sl = O::csign(q, d01) + O::csign(q, d12);
    const V sr = O::csign(q, d12) + O::csign(q, d23);
    L = O::fma(sl, O::mn(O::ab(d01), O::ab(d12)), w1);
    R = w2 - sr * O::mn(O::ab(d12), O::ab(d23));
  }
}

// Roe flux per unit area in the face frame.  L, R: (rho, u_n, u_t1, u_t2, p).
// F: (mass, normal momentum, t1 momentum, t2 momentum, energy); TWICE: 2F, the factor 1/2 left
// to the caller (exact: a product by a power of two only moves the exponent).
template <typename V, bool TWICE = false>
__device__ __forceinline__ void roe_frame(const V* L, const V* R, const Consts<V>& K, V* F) {
  using O = VM<V>;
  const V half = O::c(0.5);
  const V rl = L[0], ul = L[1], vl = L[2], wl = L[3], pl = L[4];
  const V rr = R[0], ur = R[1], vr = R[2], wr = R[3], pr = R[4];
  const V isl = O::rsqrt(rl), isr = O::rsqrt(rr);
  const V sl = rl * isl, sr = rr * isr;  // sqrt(rho)
  const V hl = O::fma(K.ggm1 * pl, isl * isl, half * O::fma(ul, ul, O::fma(vl, vl, wl * wl)));
  const V hr = O::fma(K.ggm1 * pr, isr * isr, half * O::fma(ur, ur, O::fma(vr, vr, wr * wr)));
  const V ml = rl * ul, mr = rr * ur;  // mass fluxes
  // Roe averages
  const V iw = O::rcp(sl + sr);
  const V al = sl * iw, ar = sr * iw;
  const V ut = O::fma(al, ul, ar * ur), vt = O::fma(al, vl, ar * vr), wt = O::fma(al, wl, ar * wr);
  const V ht = O::fma(al, hl, ar * hr);
  const V q2 = O::fma(ut, ut, O::fma(vt, vt, wt * wt));
  const V c2 = K.gm1 * O::fma(O::c(-0.5), q2, ht);
  const V ic = O::rsqrt(c2);
  const V c = c2 * ic, ic2 = ic * ic;
  const V rt = sl * sr;
  // jumps and wave strengths: acoustic (u-c), (u+c), entropy, shear (normal part zero)
  const V drho = rr - rl, dp = pr - pl, dun = ur - ul, dt1 = vr - vl, dt2 = wr - wl;
  const V rcd = rt * c * dun;
  const V hic2 = half * ic2;
  const V a1 = (dp - rcd) * hic2;
  const V a5 = (dp + rcd) * hic2;
  const V a2 = drho - dp * ic2;
  const V s1 = rt * dt1, s2 = rt * dt2;
  // eigenvalue moduli with Harten's fix: |l| -> (l^2 + d^2) / (2 d) where |l| < d
  const V delta = K.eps * (O::ab(ut) + c);
  const V hid = O::pos(delta, half * O::rcp(delta), O::c(0));
  const V dd = delta * delta;
  const V e1 = ut - c, e5 = ut + c;
  const V l1 = O::lt(O::ab(e1), delta, O::fma(e1, e1, dd) * hid, O::ab(e1));
  const V l2 = O::lt(O::ab(ut), delta, O::fma(ut, ut, dd) * hid, O::ab(ut));
  const V l5 = O::lt(O::ab(e5), delta, O::fma(e5, e5, dd) * hid, O::ab(e5));
  // dissipation |A| dU = l1 a1 r1 + l2 (a2 r2 + shear) + l5 a5 r5
  const V w1 = l1 * a1, w5 = l5 * a5, w2 = l2 * a2;
  const V ws = w1 + w2 + w5;
  const V dn = O::fma(w1, e1, O::fma(w2, ut, w5 * e5));
  const V dv = O::fma(ws, vt, l2 * s1);
  const V dw = O::fma(ws, wt, l2 * s2);
  const V cu = c * ut;
  const V sh = O::fma(a2 * half, q2, O::fma(vt, s1, wt * s2));
  const V de = O::fma(w1, ht - cu, O::fma(l2, sh, w5 * (ht + cu)));
  F[0] = (ml + mr) - ws;
  F[1] = (O::fma(ml, ul, pl) + O::fma(mr, ur, pr)) - dn;
  F[2] = O::fma(ml, vl, mr * vr) - dv;
  F[3] = O::fma(ml, wl, mr * wr) - dw;
  F[4] = O::fma(ml, hl, mr * hr) - de;
  if constexpr (!TWICE) {
#pragma unroll
    for (int q = 0; q < 5; ++q) F[q] = half * F[q];
  }
}

// Viscous flux of Eq. 1 (Fv, Gv, Hv) per unit area in the face frame from index-space
// differences, subtracted from a doubled Roe flux F2 = 2F in place:
//   gn[q]  = d(phi_q)/dn at the face,  q = u_n, u_t1, u_t2, theta
//   dnt1   = d(u_n)/dt1,  dnt2 = d(u_n)/dt2,  dt1t1 = d(u_t1)/dt1,  dt2t2 = d(u_t2)/dt2
//   us     = u_L + u_R of (u_n, u_t1, u_t2) (twice the face average)
// tau_nn = mu (2 du_n/dn - 2/3 div u), tau_nt = mu (du_t/dn + du_n/dt), energy flux
// u_face . tau + kappa dtheta/dn.  The caller passes K.mu = 2 mu and K.kappa = 4 kappa, so the
// result is F2 - 2 Fv, bit for bit twice F - Fv (products by powers of two are exact), with the
// face average and the final halving folded into one fused multiply-add.
template <typename V>
__device__ __forceinline__ void viscous_sub_twice(const V* gn, V dnt1, V dnt2, V dt1t1, V dt2t2, const V* us,
                                                  const Consts<V>& K, V* F2) {
  using O = VM<V>;
  const V div = gn[0] + dt1t1 + dt2t2;
  const V tnn = K.mu * O::fma(O::c(-2.0 / 3.0), div, gn[0] + gn[0]);
  const V tt1 = K.mu * (gn[1] + dnt1);
  const V tt2 = K.mu * (gn[2] + dnt2);
  F2[1] = F2[1] - tnn;
  F2[2] = F2[2] - tt1;
  F2[3] = F2[3] - tt2;
  // 4 (u_face . tau + kappa dtheta/dn) accumulated, then halved inside the subtraction
  F2[4] = O::fma(O::c(-0.5), O::fma(us[0], tnn, O::fma(us[1], tt1, O::fma(us[2], tt2, K.kappa * gn[3]))), F2[4]);
}

}  // namespace gbcfd
