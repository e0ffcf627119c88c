"""Pins of the oracle's point functions (primitive recovery, MUSCL, Roe flux, RK3 stages)
against what the mathematics fixes, independently of the oracle's own formulas."""
import math

import numpy as np
import pytest

import oracle

G = 1.4


def euler_flux(w, S, gamma=G):
    """Textbook inviscid flux of Eq. 1 through the area vector S (not the oracle's code)."""
    rho, u, v, x, p = w
    vel = np.array([u, v, x])
    un = vel @ np.asarray(S)
    E = p / (gamma - 1.0) + 0.5 * rho * vel @ vel
    return np.array([rho * un, rho * u * un + p * S[0], rho * v * un + p * S[1],
                     rho * x * un + p * S[2], (E + p) * un])


def random_state(rng, mach=0.5):
    rho = 0.5 + rng.random()
    p = 0.4 + rng.random()
    c = math.sqrt(G * p / rho)
    vel = rng.standard_normal(3)
    vel *= mach * c / np.linalg.norm(vel)
    return np.array([rho, *vel, p])


def rotation(rng):
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def test_primitive_roundtrip():
    rng = np.random.default_rng(1)
    for _ in range(50):
        w = random_state(rng, mach=2.0)
        rho, u, v, x, p = w
        U = np.array([rho, rho * u, rho * v, rho * x, p / (G - 1) + 0.5 * rho * (u * u + v * v + x * x)])
        assert rel(oracle.primitive(U), w) < 1e-14


@pytest.mark.parametrize("eps", [0.0, 0.1])
def test_roe_consistency(eps):
    """F(q, q, S) equals the physical flux: the dissipation multiplies a zero jump."""
    rng = np.random.default_rng(2)
    for _ in range(200):
        w = random_state(rng, mach=3.0 * rng.random())
        S = rng.standard_normal(3)
        F = oracle.roe_flux(w, w, S, eps=eps)
        assert rel(F, euler_flux(w, S)) < 1e-14


@pytest.mark.parametrize("direction", [1.0, -1.0])
def test_roe_supersonic_is_upwind(direction):
    """All Roe eigenvalues of one sign (and outside the entropy-fix band) -> pure upwinding:
    F = F(q_L) for flow along +n and F(q_R) along -n.  This holds only if the wave decomposition
    reproduces the flux jump exactly (the Roe property), so it pins every wave term."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        S = rng.standard_normal(3)
        n = S / np.linalg.norm(S)
        wl, wr = random_state(rng, 0.3), random_state(rng, 0.3)
        for w in (wl, wr):  # add a Mach >= 2.5 stream along +-n
            c = math.sqrt(G * w[4] / w[0])
            w[1:4] += direction * (2.5 + rng.random()) * c * n
        F = oracle.roe_flux(wl, wr, S, eps=0.1)
        ref = euler_flux(wl if direction > 0 else wr, S)
        assert rel(F, ref) < 1e-12


def test_roe_antisymmetry():
    """Swapping the states and reversing S reverses the flux (conservation across a face)."""
    rng = np.random.default_rng(4)
    for _ in range(200):
        wl, wr = random_state(rng, 1.5), random_state(rng, 1.5)
        S = rng.standard_normal(3)
        assert rel(oracle.roe_flux(wr, wl, -S), -oracle.roe_flux(wl, wr, S)) < 1e-13


def test_roe_rotation_invariance():
    """Rotating velocities and S rotates the momentum flux and keeps mass and energy fluxes."""
    rng = np.random.default_rng(5)
    for _ in range(200):
        wl, wr = random_state(rng, 1.2), random_state(rng, 1.2)
        S = rng.standard_normal(3)
        Rm = rotation(rng)
        F = oracle.roe_flux(wl, wr, S)
        wl2, wr2 = wl.copy(), wr.copy()
        wl2[1:4], wr2[1:4] = Rm @ wl[1:4], Rm @ wr[1:4]
        F2 = oracle.roe_flux(wl2, wr2, Rm @ S)
        expect = np.concatenate([[F[0]], Rm @ F[1:4], [F[4]]])
        assert rel(F2, expect) < 1e-13


def test_roe_area_scaling():
    rng = np.random.default_rng(6)
    for _ in range(50):
        wl, wr = random_state(rng), random_state(rng)
        S = rng.standard_normal(3)
        assert rel(oracle.roe_flux(wl, wr, 2.0 * S), 2.0 * oracle.roe_flux(wl, wr, S)) < 1e-15


def test_roe_stationary_contact_without_fix():
    """A contact at rest (pressure and velocity continuous, density jumps) is exact for Roe
    without the entropy fix: mass and energy fluxes vanish, momentum flux is p S."""
    S = np.array([0.3, -0.2, 0.7])
    wl = np.array([1.0, 0.0, 0.0, 0.0, 0.7])
    wr = np.array([0.25, 0.0, 0.0, 0.0, 0.7])
    F = oracle.roe_flux(wl, wr, S, eps=0.0)
    assert np.allclose(F, [0.0, 0.7 * S[0], 0.7 * S[1], 0.7 * S[2], 0.0], atol=1e-15, rtol=0)


def test_roe_sod_mass_flux_value():
    """1D Riemann problem (Sod, gamma 1.4): the Roe flux without entropy fix equals the upwind
    flux of the wave decomposition; check it against a direct 1D Roe evaluation written from
    Roe's averages in a different (characteristic-matrix) form."""
    wl = np.array([1.0, 0.0, 0.0, 0.0, 1.0])
    wr = np.array([0.125, 0.0, 0.0, 0.0, 0.1])
    S = np.array([1.0, 0.0, 0.0])
    F = oracle.roe_flux(wl, wr, S, eps=0.0)
    # 1D Roe with the full eigen-decomposition |A| = R |L| R^-1 computed numerically
    def cons(w):
        r, u, p = w[0], w[1], w[4]
        return np.array([r, r * u, p / (G - 1) + 0.5 * r * u * u])
    def flux1(w):
        r, u, p = w[0], w[1], w[4]
        E = p / (G - 1) + 0.5 * r * u * u
        return np.array([r * u, r * u * u + p, (E + p) * u])
    sl, sr = math.sqrt(wl[0]), math.sqrt(wr[0])
    hl = G / (G - 1) * wl[4] / wl[0] + 0.5 * wl[1] ** 2
    hr = G / (G - 1) * wr[4] / wr[0] + 0.5 * wr[1] ** 2
    u = (sl * wl[1] + sr * wr[1]) / (sl + sr)
    H = (sl * hl + sr * hr) / (sl + sr)
    A = np.array([[0, 1, 0],
                  [0.5 * (G - 3) * u * u, (3 - G) * u, G - 1],
                  [u * (0.5 * (G - 1) * u * u - H), H - (G - 1) * u * u, G * u]])
    lam, Rv = np.linalg.eig(A)
    absA = (Rv @ np.diag(np.abs(lam)) @ np.linalg.inv(Rv)).real
    ref = 0.5 * (flux1(wl) + flux1(wr)) - 0.5 * absA @ (cons(wr) - cons(wl))
    assert rel(F[[0, 1, 4]], ref) < 1e-12
    assert abs(F[2]) < 1e-15 and abs(F[3]) < 1e-15


def test_muscl_linear_data_exact():
    """On linear data both slopes agree, so left and right states equal the face value."""
    rng = np.random.default_rng(7)
    for lim in (0, 1):
        for _ in range(50):
            a, b = rng.standard_normal(5), rng.standard_normal(5)
            w = [a + b * i for i in range(4)]
            wl, wr = oracle.muscl(*w, limiter=lim)
            mid = a + 1.5 * b
            assert np.max(np.abs(wl - mid)) < 1e-14 and np.max(np.abs(wr - mid)) < 1e-14


def test_muscl_minmod_properties():
    rng = np.random.default_rng(8)
    for _ in range(500):
        w = [rng.standard_normal(5) for _ in range(4)]
        wl, wr = oracle.muscl(*w, limiter=0)
        for m in range(5):
            w0, w1, w2, w3 = (x[m] for x in w)
            # left state stays between w1 and its neighbours' range (TVD bound)
            lo, hi = min(w1, 0.5 * (w1 + w2), 0.5 * (w0 + w1)), max(w1, 0.5 * (w1 + w2), 0.5 * (w0 + w1))
            assert lo - 1e-15 <= wl[m] <= hi + 1e-15
            if (w1 - w0) * (w2 - w1) <= 0:      # extremum: first order
                assert wl[m] == w1
            if (w2 - w1) * (w3 - w2) <= 0:
                assert wr[m] == w2
            if (w1 - w0) * (w2 - w1) > 0:      # monotone: the smaller one-sided slope
                s = min(abs(w1 - w0), abs(w2 - w1)) * math.copysign(1.0, w2 - w1)
                assert wl[m] == w1 + 0.5 * s


def test_muscl_fromm_slope():
    w = [np.full(5, v) for v in (0.0, 1.0, 4.0, 9.0)]
    wl, wr = oracle.muscl(*w, limiter=1)
    assert np.all(wl == 1.0 + 0.25 * (4.0 - 0.0))
    assert np.all(wr == 4.0 - 0.25 * (9.0 - 1.0))


def test_rk3_stability_polynomial():
    """Stages of Eqs. 4-6 (lambda = -dt) on dQ/dt = z Q reproduce 1 + x + x^2/2 + x^3/6, x = z dt:
    the third-order SSP Runge-Kutta amplification factor."""
    rng = np.random.default_rng(9)
    Q0 = rng.standard_normal(64)
    z = -rng.random(64) * 3.0
    dt = 0.7
    Q1 = oracle.rk3_stage(1, Q0, Q0, -z * Q0, dt)
    Q2 = oracle.rk3_stage(2, Q0, Q1, -z * Q1, dt)
    Q3 = oracle.rk3_stage(3, Q0, Q2, -z * Q2, dt)
    x = z * dt
    assert rel(Q3, (1 + x + x * x / 2 + x ** 3 / 6) * Q0) < 1e-14
    assert rel(Q1, (1 + x) * Q0) < 1e-15


def test_norms_bruteforce():
    rng = np.random.default_rng(10)
    R = rng.standard_normal((5, 3, 4, 5))
    out = oracle.norms(R)
    for m in range(5):
        s = sum(float(v) ** 2 for v in R[m].ravel())
        assert abs(out[m] - math.sqrt(s / R[m].size)) <= 1e-15 * out[m]


# ---- Harten's entropy fix where it is active ---------------------------------------------------
def _jacobian_fn():
    """d F_n / d U of Eq. 1's inviscid flux through a unit normal, differentiated symbolically
    (sympy) from the conserved variables: independent of every formula of the oracle's flux"""
    sp = pytest.importorskip("sympy")
    U = sp.symbols("U0:5")
    n = sp.symbols("n0:3")
    g = sp.Symbol("gamma")
    rho, mx, my, mz, E = U
    u, v, w = mx / rho, my / rho, mz / rho
    p = (g - 1) * (E - (mx * mx + my * my + mz * mz) / (2 * rho))
    un = u * n[0] + v * n[1] + w * n[2]
    F = [rho * un, mx * un + p * n[0], my * un + p * n[1], mz * un + p * n[2], (E + p) * un]
    J = sp.Matrix(F).jacobian(sp.Matrix(U))
    return sp.lambdify((U, n, g), J, "numpy")


def _conserved(w, gamma=G):
    rho, u, v, x, p = w
    return np.array([rho, rho * u, rho * v, rho * x, p / (gamma - 1) + 0.5 * rho * (u * u + v * v + x * x)])


def _roe_harten_by_eig(jac, wl, wr, S, eps, gamma=G):
    """(F_L + F_R)/2 - |A|_H (U_R - U_L)/2 with A the flux Jacobian at Roe's average (sqrt(rho)-weighted
    velocity and total enthalpy) and |A|_H = sum_k h(l_k) P_k over its three distinct eigenvalues
    (numpy's eigvals), P_k the spectral projectors prod_{j != k} (A - l_j) / (l_k - l_j) (Sylvester's
    formula; A is diagonalisable with minimal polynomial (A - l_1)(A - l_2)(A - l_5)), and Harten's
    modulus h(l) = (l^2 + d^2) / (2 d) below d = eps (|u.n| + c) of that average, |l| above"""
    area = np.linalg.norm(S)
    n = np.asarray(S) / area
    sl, sr = math.sqrt(wl[0]), math.sqrt(wr[0])
    H = lambda w: gamma / (gamma - 1) * w[4] / w[0] + 0.5 * (w[1] ** 2 + w[2] ** 2 + w[3] ** 2)
    vel = (sl * np.asarray(wl[1:4]) + sr * np.asarray(wr[1:4])) / (sl + sr)
    Ht = (sl * H(wl) + sr * H(wr)) / (sl + sr)
    rho_t = sl * sr
    c2 = (gamma - 1) * (Ht - 0.5 * vel @ vel)
    p_t = rho_t * c2 / gamma
    Ut = _conserved(np.array([rho_t, *vel, p_t]), gamma)
    A = np.array(jac(tuple(Ut), tuple(n), gamma), dtype=np.float64)
    # the Roe property A dU = dF holds for this average (pins the average itself)
    dU = _conserved(wr, gamma) - _conserved(wl, gamma)
    dF = euler_flux(wr, n, gamma) - euler_flux(wl, n, gamma)
    assert np.max(np.abs(A @ dU - dF)) <= 1e-13 * max(1.0, np.max(np.abs(dF)))
    ev = np.sort(np.linalg.eigvals(A).real)
    assert np.ptp(ev[1:4]) < 1e-10 * (1 + np.max(np.abs(ev)))  # the triple eigenvalue
    lam = np.array([ev[0], np.mean(ev[1:4]), ev[4]])
    delta = eps * (abs(vel @ n) + math.sqrt(c2))
    mod = np.where(np.abs(lam) < delta, (lam * lam + delta * delta) / (2 * delta), np.abs(lam))
    I5 = np.eye(5)
    absA = np.zeros((5, 5))
    for k in range(3):
        P = I5.copy()
        for j in range(3):
            if j != k:
                P = P @ (A - lam[j] * I5) / (lam[k] - lam[j])
        absA += mod[k] * P
    return area * (0.5 * (euler_flux(wl, n, gamma) + euler_flux(wr, n, gamma)) - 0.5 * absA @ dU), lam, delta


@pytest.mark.parametrize("kind", ["contact", "transonic_left", "transonic_right", "random"])
def test_roe_harten_active_matches_eigendecomposition(kind):
    """States whose Roe average puts one or more eigenvalues inside Harten's band (|l| < d): a
    near-stationary contact (u.n ~ 0: the entropy and shear waves), a sonic point of the u - c or
    the u + c wave (transonic rarefaction), and random low-Mach pairs with a wide band.  The
    oracle must equal the flux assembled from a numerical eigen-decomposition."""
    jac = _jacobian_fn()
    rng = np.random.default_rng(11)
    eps = {"contact": 0.1, "transonic_left": 0.1, "transonic_right": 0.1, "random": 0.6}[kind]
    active = 0
    for _ in range(40):
        S = rng.standard_normal(3)
        n = S / np.linalg.norm(S)
        wl, wr = random_state(rng, 0.05), random_state(rng, 0.05)
        if kind == "contact":      # small normal velocity, pressure nearly continuous
            wr[4] = wl[4] * (1 + 0.02 * rng.standard_normal())
        elif kind.startswith("transonic"):  # u.n close to -c / +c on the two sides
            sgn = -1.0 if kind == "transonic_left" else 1.0
            for w, f in ((wl, 0.97), (wr, 1.03)):
                c = math.sqrt(G * w[4] / w[0])
                w[1:4] += sgn * f * c * n
        F = oracle.roe_flux(wl, wr, S, eps=eps)
        ref, lam, delta = _roe_harten_by_eig(jac, wl, wr, S, eps)
        active += int(np.any(np.abs(lam) < delta))
        assert rel(F, ref) < 1e-12, (kind, F, ref)
    assert active >= 30, active  # the fix really is exercised


def test_roe_harten_stationary_contact_closed_form():
    """A contact at rest (u = 0 on both sides, equal p, density jump) has only the entropy wave,
    with Roe speed 0 < d = eps c~, so Harten's modulus is d / 2.  With c~^2 = gamma p / sqrt(rho_L rho_R)
    (Roe's enthalpy average at equal p) the flux is exactly
        F = |S| (-(eps c~ / 4) (rho_R - rho_L), p n, 0):
    the fix adds mass diffusion eps c~ / 4 and nothing else."""
    S = np.array([0.3, -0.2, 0.7])
    area = np.linalg.norm(S)
    for rl, rr, p, eps in ((1.0, 0.25, 0.7, 0.1), (0.8, 1.9, 1.3, 0.3), (2.0, 0.5, 0.2, 0.05)):
        wl = np.array([rl, 0.0, 0.0, 0.0, p])
        wr = np.array([rr, 0.0, 0.0, 0.0, p])
        ct = math.sqrt(G * p / math.sqrt(rl * rr))
        F = oracle.roe_flux(wl, wr, S, eps=eps)
        want = np.array([-area * eps * ct / 4.0 * (rr - rl), p * S[0], p * S[1], p * S[2], 0.0])
        assert np.allclose(F, want, rtol=1e-13, atol=1e-15), (F, want)
