// curvi.cuh -- face fluxes on curvilinear blocks (Eq. 1 in curvilinear coordinates, Sec. 2.2).
//
// A face carries its area vector S (from the metric ring, see stage.cuh).  MUSCL reconstructs the
// primitives (rho, u, v, w, p) in index space with x, y, z velocity components; the left and right
// states are then rotated into the face frame (n = S/|S|, t1 built from the axis least aligned
// with n, t2 = n x t1), the Roe flux is evaluated there (roe_frame, rotation invariant) and rotated
// back, times |S|.  Viscous fluxes use face gradients by the chain rule through the metrics:
//   grad phi = [ (phi_R - phi_L) S_f + dt1 Sb_t1 + dt2 Sb_t2 ] / Vb,
// dt the mean of the two cells' central index differences along a tangent direction, Sb_t the
// mean of the two cells' cell-averaged face vectors in that direction, Vb the mean volume.
#pragma once
#include "physics.cuh"

namespace gbcfd {

// metric-ring indices of one face: S_f (x component), the four face vectors averaged for each
// tangent direction (x components) and the two cell volumes
struct MetIdx {
  int sf;
  int t1[4];
  int t2[4];
  int vl, vr;
};

template <typename T, bool VISC, int BY>
__device__ __forceinline__ void face_flux_curvi(const T* __restrict__ ring, const T* __restrict__ mring,
                                                int nv_ms, const int (&b)[4], const int (&tg)[8],
                                                const MetIdx& mi, const Consts<T>& K, T* F) {
  using O = VM<T>;
  constexpr int MS = BY * BX;
  (void)nv_ms;
  T L[5], R[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const int m = q * MS;
    muscl(ring[b[0] + m], ring[b[1] + m], ring[b[2] + m], ring[b[3] + m], K.lim, L[q], R[q]);
  }
  const T S[3] = {mring[mi.sf], mring[mi.sf + MS], mring[mi.sf + 2 * MS]};
  const T s2 = O::fma(S[0], S[0], O::fma(S[1], S[1], S[2] * S[2]));
  const T ia = O::rsqrt(s2);
  const T area = s2 * ia;
  const T n[3] = {S[0] * ia, S[1] * ia, S[2] * ia};
  // t1 = (e_a - n_a n) / sqrt(1 - n_a^2) for the axis a with the smallest |n_a|
  const T ax = O::ab(n[0]), ay = O::ab(n[1]), az = O::ab(n[2]);
  const int a = (ax <= ay && ax <= az) ? 0 : (ay <= az ? 1 : 2);
  const T na = a == 0 ? n[0] : (a == 1 ? n[1] : n[2]);
  const T it = O::rsqrt(O::fma(-na, na, T(1)));
  T t1[3];
#pragma unroll
  for (int x = 0; x < 3; ++x) t1[x] = ((x == a ? T(1) : T(0)) - na * n[x]) * it;
  const T t2[3] = {n[1] * t1[2] - n[2] * t1[1], n[2] * t1[0] - n[0] * t1[2], n[0] * t1[1] - n[1] * t1[0]};
  T Lf[5], Rf[5];
  Lf[0] = L[0];
  Lf[4] = L[4];
  Rf[0] = R[0];
  Rf[4] = R[4];
  Lf[1] = O::fma(L[1], n[0], O::fma(L[2], n[1], L[3] * n[2]));
  Lf[2] = O::fma(L[1], t1[0], O::fma(L[2], t1[1], L[3] * t1[2]));
  Lf[3] = O::fma(L[1], t2[0], O::fma(L[2], t2[1], L[3] * t2[2]));
  Rf[1] = O::fma(R[1], n[0], O::fma(R[2], n[1], R[3] * n[2]));
  Rf[2] = O::fma(R[1], t1[0], O::fma(R[2], t1[1], R[3] * t1[2]));
  Rf[3] = O::fma(R[1], t2[0], O::fma(R[2], t2[1], R[3] * t2[2]));
  T Fr[5];
  roe_frame<T, true>(Lf, Rf, K, Fr);  // twice the flux: the 1/2 rides on the area (exact)
  const T ha = T(0.5) * area;
  F[0] = ha * Fr[0];
#pragma unroll
  for (int x = 0; x < 3; ++x) F[1 + x] = ha * O::fma(Fr[1], n[x], O::fma(Fr[2], t1[x], Fr[3] * t2[x]));
  F[4] = ha * Fr[4];

  if constexpr (VISC) {
    constexpr int TH = 5 * MS;
    const int lp1 = tg[0], lm1 = tg[1], rp1 = tg[2], rm1 = tg[3];
    const int lp2 = tg[4], lm2 = tg[5], rp2 = tg[6], rm2 = tg[7];
    // the tangential means (1/4 of four face vectors, 1/4 of two central differences) are kept
    // as sums: their product carries 1/16, folded into 16 x the normal difference and 1/16 x the
    // inverse volume (products by powers of two are exact: the same gradients bit for bit)
    T sb1[3], sb2[3];
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      const int m = x * MS;
      sb1[x] = (mring[mi.t1[0] + m] + mring[mi.t1[1] + m]) + (mring[mi.t1[2] + m] + mring[mi.t1[3] + m]);
      sb2[x] = (mring[mi.t2[0] + m] + mring[mi.t2[1] + m]) + (mring[mi.t2[2] + m] + mring[mi.t2[3] + m]);
    }
    const T iv16 = T(0.0625) * O::rcp(T(0.5) * (mring[mi.vl] + mring[mi.vr]));
    // gradients of u, v, w (primitives 1..3) and theta (slot 5)
    T g[4][3];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const int m = (f < 3 ? f + 1 : 5) * MS;
      const T dn16 = T(16) * (ring[b[2] + m] - ring[b[1] + m]);
      const T d1 = (ring[lp1 + m] - ring[lm1 + m]) + (ring[rp1 + m] - ring[rm1 + m]);
      const T d2 = (ring[lp2 + m] - ring[lm2 + m]) + (ring[rp2 + m] - ring[rm2 + m]);
#pragma unroll
      for (int x = 0; x < 3; ++x) g[f][x] = O::fma(dn16, S[x], O::fma(d1, sb1[x], d2 * sb2[x])) * iv16;
    }
    (void)TH;
    const T div = g[0][0] + g[1][1] + g[2][2];
    T tS[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      T acc = T(0);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T tau = K.mu * (g[r][c] + g[c][r]);
        if (r == c) tau = O::fma(T(-2.0 / 3.0) * K.mu, div, tau);
        acc = O::fma(tau, S[c], acc);
      }
      tS[r] = acc;
    }
    const T ub[3] = {T(0.5) * (ring[b[1] + MS] + ring[b[2] + MS]), T(0.5) * (ring[b[1] + 2 * MS] + ring[b[2] + 2 * MS]),
                     T(0.5) * (ring[b[1] + 3 * MS] + ring[b[2] + 3 * MS])};
    const T gth = O::fma(g[3][0], S[0], O::fma(g[3][1], S[1], g[3][2] * S[2]));
    F[1] = F[1] - tS[0];
    F[2] = F[2] - tS[1];
    F[3] = F[3] - tS[2];
    F[4] = F[4] - O::fma(ub[0], tS[0], O::fma(ub[1], tS[1], O::fma(ub[2], tS[2], K.kappa * gth)));
  }
}

// metric-ring base of slot s, box row cy, column cx (field 0)
template <int BY>
__device__ __forceinline__ int mb(int s, int cy, int cx) { return (s * 10 * BY + cy) * BX + cx; }

// faces below box cell (cy, cx) of plane k (metric slots mk = k, mk1 = k+1); fields 0-2 S_xi,
// 3-5 S_eta, 6-8 S_zeta, 9 V
template <int BY>
__device__ __forceinline__ MetIdx xface_met(int mk, int mk1, int cy, int cx) {
  constexpr int MS = BY * BX;
  MetIdx m;
  m.sf = mb<BY>(mk, cy, cx) + 0 * MS;
  // tangent 1 = y: S_eta of L=(cy,cx-1), L+y, R=(cy,cx), R+y ; tangent 2 = z: S_zeta of L, L+z, R, R+z
  m.t1[0] = mb<BY>(mk, cy, cx - 1) + 3 * MS; m.t1[1] = mb<BY>(mk, cy + 1, cx - 1) + 3 * MS;
  m.t1[2] = mb<BY>(mk, cy, cx) + 3 * MS;     m.t1[3] = mb<BY>(mk, cy + 1, cx) + 3 * MS;
  m.t2[0] = mb<BY>(mk, cy, cx - 1) + 6 * MS; m.t2[1] = mb<BY>(mk1, cy, cx - 1) + 6 * MS;
  m.t2[2] = mb<BY>(mk, cy, cx) + 6 * MS;     m.t2[3] = mb<BY>(mk1, cy, cx) + 6 * MS;
  m.vl = mb<BY>(mk, cy, cx - 1) + 9 * MS;
  m.vr = mb<BY>(mk, cy, cx) + 9 * MS;
  return m;
}
template <int BY>
__device__ __forceinline__ MetIdx yface_met(int mk, int mk1, int cy, int cx) {
  constexpr int MS = BY * BX;
  MetIdx m;
  m.sf = mb<BY>(mk, cy, cx) + 3 * MS;
  // tangent 1 = z: S_zeta of L=(cy-1,cx), L+z, R, R+z ; tangent 2 = x: S_xi of L, L+x, R, R+x
  m.t1[0] = mb<BY>(mk, cy - 1, cx) + 6 * MS; m.t1[1] = mb<BY>(mk1, cy - 1, cx) + 6 * MS;
  m.t1[2] = mb<BY>(mk, cy, cx) + 6 * MS;     m.t1[3] = mb<BY>(mk1, cy, cx) + 6 * MS;
  m.t2[0] = mb<BY>(mk, cy - 1, cx) + 0 * MS; m.t2[1] = mb<BY>(mk, cy - 1, cx + 1) + 0 * MS;
  m.t2[2] = mb<BY>(mk, cy, cx) + 0 * MS;     m.t2[3] = mb<BY>(mk, cy, cx + 1) + 0 * MS;
  m.vl = mb<BY>(mk, cy - 1, cx) + 9 * MS;
  m.vr = mb<BY>(mk, cy, cx) + 9 * MS;
  return m;
}
// z-face between plane k (slot mk, cell L) and k+1 (slot mk1, cell R) at column (cy, cx)
template <int BY>
__device__ __forceinline__ MetIdx zface_met(int mk, int mk1, int cy, int cx) {
  constexpr int MS = BY * BX;
  MetIdx m;
  m.sf = mb<BY>(mk1, cy, cx) + 6 * MS;
  // tangent 1 = x: S_xi of L, L+x, R, R+x ; tangent 2 = y: S_eta of L, L+y, R, R+y
  m.t1[0] = mb<BY>(mk, cy, cx) + 0 * MS;  m.t1[1] = mb<BY>(mk, cy, cx + 1) + 0 * MS;
  m.t1[2] = mb<BY>(mk1, cy, cx) + 0 * MS; m.t1[3] = mb<BY>(mk1, cy, cx + 1) + 0 * MS;
  m.t2[0] = mb<BY>(mk, cy, cx) + 3 * MS;  m.t2[1] = mb<BY>(mk, cy + 1, cx) + 3 * MS;
  m.t2[2] = mb<BY>(mk1, cy, cx) + 3 * MS; m.t2[3] = mb<BY>(mk1, cy + 1, cx) + 3 * MS;
  m.vl = mb<BY>(mk, cy, cx) + 9 * MS;
  m.vr = mb<BY>(mk1, cy, cx) + 9 * MS;
  return m;
}

// spectral-radius rate of one cell on a curvilinear grid: sum over directions of
// |u.Sb| + c |Sb| (+ 4 max(4/3, gamma/Pr) mu/rho |Sb|^2 / V), divided by V
template <typename T>
__device__ __forceinline__ T cell_rate_curvi(T r, T u, T v, T w, T p, const T* sb /*[9]*/, T vol,
                                             const RateK<T>& RK, bool viscous) {
  using O = VM<T>;
  const T ir = O::rcp(r), iv = O::rcp(vol);
  const T c2 = RK.gam * p * ir;
  const T c = c2 * O::rsqrt(c2);
  const T fv = RK.vf * ir * iv;
  T rate = T(0);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const T* s = sb + 3 * d;
    const T s2 = O::fma(s[0], s[0], O::fma(s[1], s[1], s[2] * s[2]));
    T lam = O::ab(O::fma(u, s[0], O::fma(v, s[1], w * s[2]))) + c * (s2 * O::rsqrt(s2));
    if (viscous) lam = O::fma(fv, s2, lam);
    rate = rate + lam;
  }
  return rate * iv;
}

}  // namespace gbcfd
