"""Pins of the oracle's field functions (metrics, residual, time step, RK3 step) against closed
forms, invariants and convergence to the continuous operators of Eq. 1."""
import math

import numpy as np
import pytest

import oracle
from paper_1710_09995_gb300 import cases

G = 1.4


def affine_nodes(nx, ny, nz, A, origin=(0.0, 0.0, 0.0)):
    """x = origin + A @ (i, j, k): every cell is the same parallelepiped"""
    k, j, i = np.meshgrid(np.arange(nz + 1.0), np.arange(ny + 1.0), np.arange(nx + 1.0), indexing="ij")
    idx = np.stack([i, j, k])
    X = np.einsum("ab,bkji->akji", A, idx)
    for a in range(3):
        X[a] += origin[a]
    return np.ascontiguousarray(X)


def interior_m(M):
    return M[:, 2:-2, 2:-2, 2:-2]


# ---- metrics ---------------------------------------------------------------------------------

def test_metrics_cartesian():
    hx, hy, hz = 0.5, 0.25, 0.125
    M = interior_m(oracle.metrics(cases.cartesian_nodes(5, 4, 3, hx, hy, hz)))
    expect = [hy * hz, 0, 0, 0, hx * hz, 0, 0, 0, hx * hy, hx * hy * hz]
    for a in range(10):
        assert np.all(np.abs(M[a] - expect[a]) <= 1e-16)


def test_metrics_affine_closed_form():
    """Parallelepiped cells spanned by a, b, c: S_xi = b x c, S_eta = c x a, S_zeta = a x b,
    V = a . (b x c)."""
    A = np.array([[0.9, 0.2, -0.1], [0.15, 1.1, 0.3], [-0.2, 0.05, 0.8]])
    a, b, c = A[:, 0], A[:, 1], A[:, 2]
    M = interior_m(oracle.metrics(affine_nodes(4, 3, 5, A, origin=(3.0, -2.0, 7.0))))
    expect = np.concatenate([np.cross(b, c), np.cross(c, a), np.cross(a, b), [a @ np.cross(b, c)]])
    for q in range(10):
        assert np.max(np.abs(M[q] - expect[q])) < 1e-14


def test_metrics_closure_and_periodic_halo():
    """Outward area vectors of every cell sum to zero (the discrete geometric conservation law),
    and halo cells carry the periodic images."""
    nx, ny, nz = 8, 7, 6
    M = oracle.metrics(cases.warped_nodes(nx, ny, nz, 0.05))
    closure = np.zeros((3, nz, ny, nx))
    for d in range(3):
        lower = M[3 * d:3 * d + 3, 2:-2, 2:-2, 2:-2]
        if d == 0:
            upper = M[0:3, 2:-2, 2:-2, 3:-1]
        elif d == 1:
            upper = M[3:6, 2:-2, 3:-1, 2:-2]
        else:
            upper = M[6:9, 3:-1, 2:-2, 2:-2]
        closure += upper - lower
    assert np.max(np.abs(closure)) < 1e-14 * np.max(np.abs(M[0:9]))
    assert np.all(M[:, 0:2] == M[:, nz:nz + 2])
    assert np.all(M[:, :, :, nx + 2:] == M[:, :, :, 2:4])
    assert np.all(interior_m(M)[9] > 0)


# ---- residual invariants -----------------------------------------------------------------------

def uniform_state(nx, ny, nz, vel=(0.3, -0.2, 0.1), rho=1.0, p=1.0 / G):
    return cases.conserved(np.full((nz, ny, nx), rho), *vel, p)


@pytest.mark.parametrize("viscous", [False, True])
def test_freestream_preserved_on_warped_grid(viscous):
    nx, ny, nz = 12, 10, 8
    M = oracle.metrics(cases.warped_nodes(nx, ny, nz, 0.05))
    Q = oracle.pad(uniform_state(nx, ny, nz))
    p = oracle.params(mu=1e-2 if viscous else 0.0, viscous=viscous)
    R = oracle.residual(p, Q, M)
    h = 1.0 / nx
    assert np.max(np.abs(R)) * h < 1e-13


def test_discrete_conservation_warped():
    nx, ny, nz = 12, 10, 8
    c = cases.smooth_random(nx, ny, nz, seed=3, amp=0.1)
    M = oracle.metrics(cases.warped_nodes(nx, ny, nz, 0.05))
    p = oracle.params(mu=5e-3, viscous=True)
    R = oracle.residual(p, oracle.pad(c.state), M)
    V = interior_m(M)[9]
    for m in range(5):
        tot = np.sum(V * R[m])
        assert abs(tot) < 1e-13 * np.sum(np.abs(V * R[m]))


def cyclic(Q):
    """relabel axes x->y->z->x: the new field at (i,j,k) is the old one at (k,i,j)... expressed
    on arrays [v][z][y][x]: new[z,y,x] = old[y,x,z]; velocity (u,v,w) -> (w,u,v)"""
    out = np.transpose(Q, (0, 2, 3, 1)).copy()
    out[[1, 2, 3]] = out[[3, 1, 2]]
    return out


@pytest.mark.parametrize("viscous", [False, True])
def test_axis_permutation_symmetry(viscous):
    """Relabelling the axes cyclically (with the velocity components and the grid spacings)
    relabels the residual the same way: pins the y and z code paths against the x one."""
    nx, ny, nz = 9, 7, 6
    h = (0.11, 0.13, 0.17)
    c = cases.smooth_random(nx, ny, nz, seed=5, amp=0.1, h=h)
    p = oracle.params(mu=1e-2, viscous=viscous)
    M = oracle.metrics(cases.cartesian_nodes(nx, ny, nz, *h))
    R = oracle.residual(p, oracle.pad(c.state), M)
    Qc = cyclic(c.state)
    nz2, ny2, nx2 = Qc.shape[1:]
    h2 = (h[2], h[0], h[1])
    M2 = oracle.metrics(cases.cartesian_nodes(nx2, ny2, nz2, *h2))
    R2 = oracle.residual(p, oracle.pad(Qc), M2)
    assert np.max(np.abs(R2 - cyclic(R))) < 1e-12 * np.max(np.abs(R))


def test_planar_data_gives_planar_residual():
    """Data that varies along x only: y and z fluxes cancel exactly, so R is independent of
    (j, k) bitwise."""
    nx, ny, nz = 16, 5, 4
    x = (np.arange(nx) + 0.5) / nx
    rho = 1 + 0.1 * np.sin(2 * np.pi * x)
    p = (1 + 0.2 * np.cos(2 * np.pi * x)) / G
    Q = cases.conserved(np.broadcast_to(rho, (nz, ny, nx)), 0.4, 0.1, -0.2, np.broadcast_to(p, (nz, ny, nx)))
    prm = oracle.params(mu=1e-2, viscous=True)
    R = oracle.residual(prm, oracle.pad(Q), oracle.metrics(cases.cartesian_nodes(nx, ny, nz, 1 / nx, 0.25, 0.125)))
    assert np.all(R == R[:, :1, :1, :])


# ---- closed forms ------------------------------------------------------------------------------

def test_viscous_shear_wave_discrete_closed_form():
    """u = A sin(2 pi y) with rho, p uniform and v = w = 0, no entropy fix: the inviscid fluxes
    cancel and the x-momentum residual is the 3-point second difference, whose action on a sine
    is exact: R = -mu A sin(2 pi y_j) (2 cos(2 pi h) - 2) / h^2."""
    n, A, mu = 24, 1e-2, 0.03
    h = 1.0 / n
    y = (np.arange(n) + 0.5) * h
    u = A * np.sin(2 * np.pi * y)[None, :, None] * np.ones((4, n, 3))
    Q = cases.conserved(np.ones((4, n, 3)), u, 0.0, 0.0, 1.0 / G)
    prm = oracle.params(mu=mu, viscous=True, eps=0.0)
    R = oracle.residual(prm, oracle.pad(Q), oracle.metrics(cases.cartesian_nodes(3, n, 4, 0.7, h, 0.9)))
    expect = -mu * A * np.sin(2 * np.pi * y) * (2 * np.cos(2 * np.pi * h) - 2) / h ** 2
    assert np.max(np.abs(R[1] - expect[None, :, None])) < 1e-12 * np.max(np.abs(expect))
    assert np.max(np.abs(R[0])) < 1e-13 and np.max(np.abs(R[2])) < 1e-13 and np.max(np.abs(R[3])) < 1e-13


def test_dt_uniform_flow_closed_form():
    nx, ny, nz = 6, 5, 4
    h = (0.1, 0.2, 0.25)
    vel = (0.3, -0.2, 0.1)
    Q = oracle.pad(uniform_state(nx, ny, nz, vel))
    M = oracle.metrics(cases.cartesian_nodes(nx, ny, nz, *h))
    c = 1.0
    inv = sum((abs(vel[d]) + c) / h[d] for d in range(3))
    prm = oracle.params(cfl=0.7)
    assert abs(oracle.dt(prm, Q, M) - 0.7 / inv) < 1e-15
    mu, Pr = 0.02, 0.72
    prm = oracle.params(cfl=0.7, mu=mu, Pr=Pr, viscous=True)
    visc = sum(4.0 * max(4.0 / 3.0, G / Pr) * mu / h[d] ** 2 for d in range(3))
    assert abs(oracle.dt(prm, Q, M) - 0.7 / (inv + visc)) < 1e-15


# ---- convergence to the continuous operators of Eq. 1 ------------------------------------------

def _analytic_fields():
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    tp = 2 * sp.pi
    rho = 1 + sp.Rational(1, 10) * sp.sin(tp * x + 1) * sp.cos(tp * y) + sp.Rational(1, 10) * sp.sin(2 * tp * z + sp.Rational(1, 2))
    u = sp.Rational(3, 10) + sp.Rational(1, 10) * sp.cos(tp * y + sp.Rational(3, 10)) * sp.sin(tp * z)
    v = -sp.Rational(1, 5) + sp.Rational(1, 10) * sp.sin(tp * z + sp.Rational(7, 10)) * sp.cos(tp * x)
    w = sp.Rational(1, 10) + sp.Rational(1, 10) * sp.cos(tp * x + sp.Rational(1, 5)) * sp.sin(tp * y + sp.Rational(2, 5))
    g = sp.Rational(7, 5)
    p = 1 / g + sp.Rational(1, 20) * sp.sin(tp * (x - y) + sp.Rational(1, 10)) + sp.Rational(1, 20) * sp.cos(tp * z)
    return sp, (x, y, z), (rho, u, v, w, p), g


def _sample(exprs, syms, X, Y, Z):
    sp = __import__("sympy")
    return [np.broadcast_to(sp.lambdify(syms, e, "numpy")(X, Y, Z), X.shape).astype(np.float64) for e in exprs]


def _inviscid_divergence():
    sp, (x, y, z), (rho, u, v, w, p), g = _analytic_fields()
    E = p / (g - 1) + rho * (u * u + v * v + w * w) / 2
    vel = (u, v, w)
    div = [0] * 5
    for d, s in enumerate((x, y, z)):
        un = vel[d]
        flux = [rho * un, rho * u * un + (p if d == 0 else 0), rho * v * un + (p if d == 1 else 0),
                rho * w * un + (p if d == 2 else 0), (E + p) * un]
        for m in range(5):
            div[m] = div[m] + sp.diff(flux[m], s)
    return (x, y, z), (rho, u, v, w, p), div


def _viscous_operator(mu, Pr):
    sp, (x, y, z), (rho, u, v, w, p), g = _analytic_fields()
    X = (x, y, z)
    vel = (u, v, w)
    grad = [[sp.diff(vel[a], X[b]) for b in range(3)] for a in range(3)]
    divu = grad[0][0] + grad[1][1] + grad[2][2]
    tau = [[mu * (grad[a][b] + grad[b][a]) - (sp.Rational(2, 3) * mu * divu if a == b else 0) for b in range(3)] for a in range(3)]
    theta = p / rho
    kappa = mu * g / ((g - 1) * Pr)
    mom = [sum(sp.diff(tau[a][b], X[b]) for b in range(3)) for a in range(3)]
    work = sum(sp.diff(sum(tau[a][b] * vel[a] for a in range(3)), X[b]) for b in range(3))
    heat = kappa * sum(sp.diff(theta, X[b], 2) for b in range(3))
    # the oracle's R carries -(F_v): R_visc = -[0, div tau, div(tau u) + kappa lap theta]
    return X, (rho, u, v, w, p), [0 * x, -mom[0], -mom[1], -mom[2], -(work + heat)]


def _grid(n, warped):
    nx, ny, nz = n, n + n // 4, n + n // 2
    if warped:
        nodes = cases.warped_nodes(nx, ny, nz, 0.04)
        c = 0.125 * sum(nodes[:, a:a + nz, b:b + ny, e:e + nx] for a in (0, 1) for b in (0, 1) for e in (0, 1))
        return nodes, c[0], c[1], c[2]
    nodes = cases.cartesian_nodes(nx, ny, nz, 1 / nx, 1 / ny, 1 / nz)
    X, Y, Z = cases.cell_centres(nx, ny, nz, 1 / nx, 1 / ny, 1 / nz)
    return nodes, X, Y, Z


def _order(errs):
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


@pytest.mark.parametrize("warped", [False, True])
def test_inviscid_residual_converges_second_order(warped):
    """With unlimited slopes R(Q) -> div F(Q) at second order (cell values sampled from smooth
    periodic fields; the continuous divergence is differentiated symbolically)."""
    syms, prim, div = _inviscid_divergence()
    errs = []
    for n in (8, 16, 32):
        nodes, X, Y, Z = _grid(n, warped)
        rho, u, v, w, p = _sample(prim, syms, X, Y, Z)
        Q = cases.conserved(rho, u, v, w, p)
        R = oracle.residual(oracle.params(limiter=1, eps=0.1), oracle.pad(Q), oracle.metrics(nodes))
        exact = _sample(div, syms, X, Y, Z)
        errs.append(max(np.sqrt(np.mean((R[m] - exact[m]) ** 2)) for m in range(5)))
    order = _order(errs)
    assert order[-1] > 1.8, (errs, order)


@pytest.mark.parametrize("warped", [False, True])
def test_viscous_residual_converges_second_order(warped):
    """R(Q; mu) - R(Q; 0) -> -[0, div tau, div(tau u) + kappa lap(p/rho)] at second order."""
    mu, Pr = 0.05, 0.72
    syms, prim, op = _viscous_operator(mu, Pr)
    errs = []
    for n in (8, 16, 32):
        nodes, X, Y, Z = _grid(n, warped)
        rho, u, v, w, p = _sample(prim, syms, X, Y, Z)
        Q = oracle.pad(cases.conserved(rho, u, v, w, p))
        M = oracle.metrics(nodes)
        Rv = (oracle.residual(oracle.params(mu=mu, Pr=Pr, viscous=True), Q, M)
              - oracle.residual(oracle.params(), Q, M))
        exact = _sample(op, syms, X, Y, Z)
        errs.append(max(np.sqrt(np.mean((Rv[m] - exact[m]) ** 2)) for m in range(1, 5)))
    order = _order(errs)
    assert order[-1] > 1.8, (errs, order)


# ---- time stepping ---------------------------------------------------------------------------

def test_step_wiring_matches_shu_osher():
    """oracle_step equals residual evaluations combined by the Shu-Osher formulas of Eqs. 4-6
    written out here (lambda = -dt), with the CFL time step taken from Q^n."""
    c = cases.smooth_random(10, 9, 8, seed=11, amp=0.05)
    M = oracle.metrics(cases.cartesian_nodes(10, 9, 8, 0.1, 0.11, 0.125))
    prm = oracle.params(mu=2e-3, viscous=True, cfl=0.6)
    Q0 = oracle.pad(c.state)
    Qs, dts, norms = oracle.step(prm, Q0, M, 1)
    dt = oracle.dt(prm, Q0, M)
    assert dts[0] == dt
    inner = lambda a: oracle.interior(a)
    R0 = oracle.residual(prm, Q0, M)
    Q1 = inner(Q0) - dt * R0
    R1 = oracle.residual(prm, oracle.pad(Q1), M)
    Q2 = 0.75 * inner(Q0) + 0.25 * (Q1 - dt * R1)
    R2 = oracle.residual(prm, oracle.pad(Q2), M)
    Q3 = inner(Q0) / 3.0 + 2.0 / 3.0 * (Q2 - dt * R2)
    assert np.max(np.abs(inner(Qs) - Q3)) < 1e-15
    assert np.allclose(norms[0], np.sqrt(np.mean(R0.reshape(5, -1) ** 2, axis=1)), rtol=1e-14, atol=0)


def test_step_conserves_totals_on_warped_grid():
    nx, ny, nz = 10, 9, 8
    c = cases.smooth_random(nx, ny, nz, seed=12, amp=0.1)
    M = oracle.metrics(cases.warped_nodes(nx, ny, nz, 0.05))
    prm = oracle.params(mu=5e-3, viscous=True, cfl=0.5)
    Q0 = oracle.pad(c.state)
    Q, _, _ = oracle.step(prm, Q0, M, 5)
    V = interior_m(M)[9]
    for m in range(5):
        t0 = np.sum(V * oracle.interior(Q0)[m])
        t1 = np.sum(V * oracle.interior(Q)[m])
        scale = np.sum(np.abs(V * oracle.interior(Q0)[m])) + 1e-300
        assert abs(t1 - t0) < 1e-14 * scale


@pytest.mark.parametrize("limiter,min_order", [(1, 1.8), (0, 1.3)])
def test_isentropic_vortex_convergence(limiter, min_order):
    """Euler isentropic vortex (closed form): L2 density error at t = 1 falls at second order
    without a limiter; minmod clips the smooth extremum and lowers the observed order."""
    L, t_end = 10.0, 1.0
    errs = []
    for n in (32, 64, 128):
        c = cases.isentropic_vortex(n=n, L=L, nz=1, viscous=False, limiter=limiter, eps=0.1)
        M = oracle.metrics(cases.cartesian_nodes(n, n, 1, L / n, L / n, L / n))
        prm = oracle.params(limiter=limiter, eps=0.1)
        h = L / n
        nsteps = int(math.ceil(t_end / (0.25 * h)))
        dt = t_end / nsteps
        Q, _, _ = oracle.step(prm, oracle.pad(c.state), M, nsteps, dt_fixed=dt)
        X, Y, _ = cases.cell_centres(n, n, 1, h, h, h)
        rho_exact, _, _, _ = cases.vortex_fields(X, Y, t_end, L)
        errs.append(np.sqrt(np.mean((oracle.interior(Q)[0] - rho_exact) ** 2)))
    order = _order(errs)
    assert order[-1] > min_order, (errs, order)
