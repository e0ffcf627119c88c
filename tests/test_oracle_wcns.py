"""Pins of the WCNS-E-5 oracle (the paper's own scheme, Sec. 2.2, Eq. 2) against closed forms,
invariants and convergence to the continuous operators of Eq. 1.  None of these recomputes the
oracle's formulas: they test what the scheme must satisfy."""
import math

import numpy as np
import pytest

import oracle
from paper_1710_09995_gb300 import cases

from test_oracle_fields import _analytic_fields, _inviscid_divergence, _order, _sample, _viscous_operator

G = 1.4


# ---- the interpolation ---------------------------------------------------------------------------

def _midpoint(poly, h):
    """exact value at x = h/2 of a polynomial sampled at x = -2h .. 2h"""
    xs = np.arange(-2, 3) * h
    return np.polyval(poly, xs), np.polyval(poly, 0.5 * h)


@pytest.mark.parametrize("deg", [0, 1, 2, 3, 4])
def test_linear_weights_reproduce_quartics(deg):
    """With the optimal weights the interpolation is the unique fifth-order (degree-4 exact)
    midpoint interpolation from five points."""
    rng = np.random.default_rng(deg)
    poly = rng.standard_normal(deg + 1)
    for h in (0.3, 1.0, 1.7):
        u, exact = _midpoint(poly, h)
        assert abs(oracle.wcns_edge(u, linear=True) - exact) < 1e-13 * (1 + abs(exact))


def test_linear_weights_not_exact_for_quintic():
    u, exact = _midpoint([1, 0, 0, 0, 0, 0], 1.0)
    assert abs(oracle.wcns_edge(u, linear=True) - exact) > 1e-3


def test_constant_is_preserved_bitwise():
    for c in (1.0, 0.7142857142857143, -3.25):
        assert oracle.wcns_edge(np.full(5, c)) == c


def test_nonlinear_interpolation_converges_fifth_order():
    """On smooth data without critical points the nonlinear weights approach the optimal ones
    fast enough to keep fifth order (error ratio 32 per halving)."""
    errs = []
    x0 = 0.37
    f = lambda x: np.exp(0.8 * x) + 0.3 * x
    for h in (0.2, 0.1, 0.05, 0.025):
        u = f(x0 + np.arange(-2, 3) * h)
        errs.append(abs(oracle.wcns_edge(u) - f(x0 + 0.5 * h)))
    order = _order(errs)
    assert order[-1] > 4.6, (errs, order)


def test_nonlinear_weights_pick_the_smooth_stencil():
    """A jump between i and i+1: only S0 = {i-2, i-1, i} is smooth, so the left value at i+1/2
    is the smooth extrapolation (here u_i on constant data) up to a tiny weight on the others;
    the mirrored right value likewise takes u_{i+1}."""
    u = np.array([0.0, 0.0, 0.0, 1.0, 1.0])            # u_{i-2} .. u_{i+2}
    assert abs(oracle.wcns_edge(u) - 0.0) < 1e-9
    right = np.array([1.0, 1.0, 1.0, 0.0, 0.0])        # u_{i+3}, u_{i+2}, u_{i+1}, u_i, u_{i-1}
    assert abs(oracle.wcns_edge(right) - 1.0) < 1e-9
    # the linear interpolation overshoots there
    assert oracle.wcns_edge(u, linear=True) > 0.3


def test_nonlinear_interpolation_bounded_on_steps():
    """Monotone data with one jump anywhere in the stencil: the interpolated value stays within
    the local data range (to the tiny weight of the non-smooth stencils), where the linear
    interpolation overshoots."""
    for pos in range(1, 5):
        u = np.where(np.arange(5) >= pos, 1.0, 0.0)
        v = oracle.wcns_edge(u)
        assert -1e-6 < v < 1 + 1e-6
        v = oracle.wcns_edge(1.0 - u)
        assert -1e-6 < v < 1 + 1e-6


# ---- residual invariants ---------------------------------------------------------------------------

@pytest.mark.parametrize("viscous", [False, True])
def test_uniform_flow_residual_is_zero(viscous):
    """Constant data: every edge state equals the cell state, F(q, q) = F(q) on all faces and
    the differences of Eq. 2 vanish exactly; the central differences vanish to rounding (the
    sum f - 8 f + 8 f - f of equal values is not exactly zero in floating point)."""
    nx, ny, nz = 11, 9, 8
    Q = cases.conserved(np.full((nz, ny, nx), 1.1), 0.3, -0.2, 0.1, 0.8)
    p = oracle.params(mu=1e-2 if viscous else 0.0, viscous=viscous)
    R = oracle.wcns_residual(p, Q, (0.1, 0.12, 0.13))
    if viscous:
        assert np.max(np.abs(R)) < 1e-25
    else:
        assert np.all(R == 0.0)


@pytest.mark.parametrize("viscous", [False, True])
def test_discrete_conservation(viscous):
    """Periodic block: Eq. 2 and the central differences are telescoping sums, so sum R = 0."""
    nx, ny, nz = 12, 10, 9
    c = cases.smooth_random(nx, ny, nz, seed=4, amp=0.1)
    p = oracle.params(mu=5e-3 if viscous else 0.0, viscous=viscous)
    R = oracle.wcns_residual(p, c.state, c.spacing)
    for m in range(5):
        assert abs(np.sum(R[m])) < 1e-13 * np.sum(np.abs(R[m]))


def test_planar_data_gives_planar_residual():
    nx, ny, nz = 16, 6, 5
    x = (np.arange(nx) + 0.5) / nx
    rho = 1 + 0.1 * np.sin(2 * np.pi * x)
    pr = (1 + 0.2 * np.cos(2 * np.pi * x)) / G
    Q = cases.conserved(np.broadcast_to(rho, (nz, ny, nx)), 0.4, 0.1, -0.2, np.broadcast_to(pr, (nz, ny, nx)))
    R = oracle.wcns_residual(oracle.params(mu=1e-2, viscous=True), Q, (1 / nx, 0.25, 0.125))
    assert np.all(R == R[:, :1, :1, :])


def _cyclic(Q):
    out = np.transpose(Q, (0, 2, 3, 1)).copy()
    out[[1, 2, 3]] = out[[3, 1, 2]]
    return out


@pytest.mark.parametrize("viscous", [False, True])
def test_axis_permutation_symmetry(viscous):
    nx, ny, nz = 9, 8, 7
    h = (0.11, 0.13, 0.17)
    c = cases.smooth_random(nx, ny, nz, seed=6, amp=0.1, h=h)
    p = oracle.params(mu=1e-2, viscous=viscous)
    R = oracle.wcns_residual(p, c.state, h)
    R2 = oracle.wcns_residual(p, _cyclic(c.state), (h[2], h[0], h[1]))
    assert np.max(np.abs(R2 - _cyclic(R))) < 1e-12 * np.max(np.abs(R))


def test_mirror_symmetry():
    """Reflecting x (i -> n-1-i, u -> -u) reflects the residual (R_rho u changes sign): the
    right-hand interpolation is the left-hand one on the mirrored stencil."""
    nx, ny, nz = 10, 6, 5
    c = cases.smooth_random(nx, ny, nz, seed=8, amp=0.2)
    p = oracle.params()
    R = oracle.wcns_residual(p, c.state, c.spacing)
    Qm = c.state[:, :, :, ::-1].copy()
    Qm[1] *= -1
    Rm = oracle.wcns_residual(p, Qm, c.spacing)[:, :, :, ::-1].copy()
    Rm[1] *= -1
    assert np.max(np.abs(Rm - R)) < 1e-12 * np.max(np.abs(R))


# ---- convergence to Eq. 1's continuous operators -------------------------------------------------

def _cart(n):
    nx, ny, nz = n, n + n // 4, n + n // 2
    X, Y, Z = cases.cell_centres(nx, ny, nz, 1 / nx, 1 / ny, 1 / nz)
    return (1 / nx, 1 / ny, 1 / nz), X, Y, Z


@pytest.mark.parametrize("linear,min_order", [(True, 4.6), (False, 4.3)])
def test_inviscid_residual_converges_fifth_order(linear, min_order):
    """Point values at cell centres of smooth periodic fields: R -> div F at fifth order (the
    interpolation's order; Eq. 2 itself is sixth order), with the linear and the nonlinear
    weights."""
    syms, prim, div = _inviscid_divergence()
    errs = []
    for n in (16, 32, 64):
        h, X, Y, Z = _cart(n)
        rho, u, v, w, p = _sample(prim, syms, X, Y, Z)
        R = oracle.wcns_residual(oracle.params(limiter=int(linear), eps=0.1), cases.conserved(rho, u, v, w, p), h)
        exact = _sample(div, syms, X, Y, Z)
        errs.append(max(np.sqrt(np.mean((R[m] - exact[m]) ** 2)) for m in range(5)))
    order = _order(errs)
    assert order[-1] > min_order, (errs, order)


def test_viscous_residual_converges_fourth_order():
    """R(Q; mu) - R(Q; 0) -> -[0, div tau, div(tau u) + kappa lap(p/rho)] at fourth order."""
    mu, Pr = 0.05, 0.72
    syms, prim, op = _viscous_operator(mu, Pr)
    errs = []
    for n in (8, 16, 32):
        h, X, Y, Z = _cart(n)
        rho, u, v, w, p = _sample(prim, syms, X, Y, Z)
        Q = cases.conserved(rho, u, v, w, p)
        Rv = (oracle.wcns_residual(oracle.params(mu=mu, Pr=Pr, viscous=True), Q, h)
              - oracle.wcns_residual(oracle.params(), Q, h))
        exact = _sample(op, syms, X, Y, Z)
        errs.append(max(np.sqrt(np.mean((Rv[m] - exact[m]) ** 2)) for m in range(1, 5)))
    order = _order(errs)
    assert order[-1] > 3.7, (errs, order)


# ---- time stepping -------------------------------------------------------------------------------

def test_step_wiring_matches_shu_osher():
    c = cases.smooth_random(10, 9, 8, seed=11, amp=0.05)
    h = c.spacing
    prm = oracle.params(mu=2e-3, viscous=True, cfl=0.6)
    Q0 = c.state
    Qs, dts, norms = oracle.wcns_step(prm, Q0, h, 1)
    dt = oracle.wcns_dt(prm, Q0, h)
    assert dts[0] == dt
    R0 = oracle.wcns_residual(prm, Q0, h)
    Q1 = Q0 - dt * R0
    Q2 = 0.75 * Q0 + 0.25 * (Q1 - dt * oracle.wcns_residual(prm, Q1, h))
    Q3 = Q0 / 3.0 + 2.0 / 3.0 * (Q2 - dt * oracle.wcns_residual(prm, Q2, h))
    assert np.max(np.abs(Qs - Q3)) < 1e-15
    assert np.allclose(norms[0], np.sqrt(np.mean(R0.reshape(5, -1) ** 2, axis=1)), rtol=1e-14, atol=0)


def test_dt_uniform_flow_closed_form():
    nx, ny, nz = 6, 5, 4
    h = (0.1, 0.2, 0.25)
    vel = (0.3, -0.2, 0.1)
    Q = cases.conserved(np.ones((nz, ny, nx)), *vel, 1.0 / G)
    inv = sum((abs(vel[d]) + 1.0) / h[d] for d in range(3))
    assert abs(oracle.wcns_dt(oracle.params(cfl=0.7), Q, h) - 0.7 / inv) < 1e-15
    mu, Pr = 0.02, 0.72
    visc = sum(4.0 * max(4.0 / 3.0, G / Pr) * mu / h[d] ** 2 for d in range(3))
    assert abs(oracle.wcns_dt(oracle.params(cfl=0.7, mu=mu, Pr=Pr, viscous=True), Q, h) - 0.7 / (inv + visc)) < 1e-15


def test_step_conserves_totals():
    c = cases.smooth_random(10, 9, 8, seed=12, amp=0.1)
    prm = oracle.params(mu=5e-3, viscous=True, cfl=0.5)
    Q, _, _ = oracle.wcns_step(prm, c.state, c.spacing, 4)
    for m in range(5):
        t0, t1 = np.sum(c.state[m]), np.sum(Q[m])
        assert abs(t1 - t0) < 1e-13 * np.sum(np.abs(c.state[m]))


def test_isentropic_vortex_beats_muscl():
    """Euler vortex (closed form) after t = 1 on the same 32x32 grid and time step: WCNS-E-5's
    density error is far below the second-order MUSCL scheme's, and falls faster than second order
    (the time step shrinks with h, so RK3's third order caps the observed rate)."""
    L, t_end = 10.0, 1.0
    errs_w = []
    for n in (32, 64):
        c = cases.isentropic_vortex(n=n, L=L, nz=1, viscous=False, limiter=0, eps=0.1)
        h = L / n
        nsteps = int(math.ceil(t_end / (0.25 * h)))
        dt = t_end / nsteps
        Q, _, _ = oracle.wcns_step(oracle.params(eps=0.1), c.state, (h, h, h), nsteps, dt_fixed=dt)
        X, Y, _ = cases.cell_centres(n, n, 1, h, h, h)
        rho_exact, _, _, _ = cases.vortex_fields(X, Y, t_end, L)
        errs_w.append(np.sqrt(np.mean((Q[0] - rho_exact) ** 2)))
        if n == 32:
            Qm, _, _ = oracle.step(oracle.params(limiter=1, eps=0.1), oracle.pad(c.state),
                                   oracle.metrics(cases.cartesian_nodes(n, n, 1, h, h, h)), nsteps, dt_fixed=dt)
            err_muscl = np.sqrt(np.mean((oracle.interior(Qm)[0] - rho_exact) ** 2))
    assert errs_w[0] < 0.2 * err_muscl, (errs_w, err_muscl)
    assert math.log2(errs_w[0] / errs_w[1]) > 2.7, errs_w
