"""Pins of the learned accelerator's plain definitions (oracle/learn.py) against library routines,
adjoint identities, finite differences and closed forms."""
import numpy as np
import pytest

from oracle import learn as L

scipy_signal = pytest.importorskip("scipy.signal")


def rng(seed=0):
    return np.random.Generator(np.random.PCG64(seed))


def test_bf16_rounding():
    """bfloat16 keeps 8 significant bits (unit roundoff 2^-8): ties go to even, 1 + 2^-8 rounds
    to 1, 1 + 3 * 2^-8 up to 1 + 2^-6"""
    assert L.bf16(1.0 + 2 ** -8) == 1.0
    assert L.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6
    assert L.bf16(1.0 + 2 ** -7) == 1.0 + 2 ** -7
    x = rng().standard_normal(1000)
    assert np.all(np.abs(L.bf16(x) - x) <= 2 ** -8 * np.abs(x) * (1 + 1e-12))


@pytest.mark.parametrize("zper", [True, False])
def test_conv3d_is_a_sum_of_scipy_correlations(zper):
    """every (out, in) channel pair is scipy's 3D cross-correlation of the padded input"""
    r = rng(1)
    x = r.standard_normal((3, 5, 6, 7))
    W = r.standard_normal((4, 3, 27))
    b = r.standard_normal(4)
    got = L.conv3d(x, W, b, zper)
    mode_z = "wrap" if zper else "constant"
    for o in range(4):
        want = np.full(x.shape[1:], b[o])
        for c in range(3):
            xp = np.pad(x[c], ((1, 1), (0, 0), (0, 0)), mode=mode_z)
            xp = np.pad(xp, ((0, 0), (1, 1), (1, 1)))
            want = want + scipy_signal.correlate(xp, W[o, c].reshape(3, 3, 3), mode="valid")
        assert np.allclose(got[o], want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("zper", [True, False])
def test_conv3d_transpose_is_the_adjoint(zper):
    r = rng(2)
    x = r.standard_normal((3, 4, 5, 6))
    g = r.standard_normal((4, 4, 5, 6))
    W = r.standard_normal((4, 3, 27))
    lhs = np.sum(L.conv3d(x, W, np.zeros(4), zper) * g)
    rhs = np.sum(x * L.conv3d_transpose(g, W, zper))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_silu_derivative():
    z = np.linspace(-6, 6, 41)
    h = 1e-6
    assert np.allclose(L.dsilu(z), (L.silu(z + h) - L.silu(z - h)) / (2 * h), rtol=1e-7, atol=1e-9)


def test_gradient_matches_finite_differences():
    """the analytic gradient of the FP64 network (no rounding) against central differences"""
    r = rng(3)
    p = 0.1 * r.standard_normal(L.n_params())
    x = r.standard_normal((10, 3, 4, 5))
    y = r.standard_normal((5, 3, 4, 5))
    loss, g = L.loss_and_grad(p, x, y, bf16_storage=False)
    idx = r.choice(L.n_params(), 12, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        lp, _ = L.loss_and_grad(p + e, x, y, bf16_storage=False)
        lm, _ = L.loss_and_grad(p - e, x, y, bf16_storage=False)
        assert abs((lp - lm) / (2 * h) - g[i]) <= 1e-6 * max(1.0, abs(g[i])), i


def test_adam_first_step_moves_by_lr_sign():
    """from zero moments the bias-corrected first step is lr g / (|g| + eps) ~ lr sign(g)"""
    r = rng(4)
    w = r.standard_normal(50)
    g = r.standard_normal(50)
    w1, m, v = L.adam(w, g, np.zeros(50), np.zeros(50), 1, 1e-3)
    assert np.allclose(w - w1, 1e-3 * np.sign(g), rtol=1e-6)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_features_of_free_stream_and_uniform_residual():
    """the free stream gives zero state channels; a uniform residual gives residual channels of
    unit RMS with the residual's direction"""
    inf = (1.0, 0.6, 0.0, 0.0, 1.0 / 1.4)
    Q = np.broadcast_to(L.conserved_inf(inf)[:, None, None, None], (5, 2, 3, 4)).copy()
    Rv = np.array([1.0, -2.0, 0.5, 0.0, 3.0])
    R = np.broadcast_to(Rv[:, None, None, None], (5, 2, 3, 4)).copy()
    dtl = np.full((2, 3, 4), 0.01)
    x, s = L.features(Q, R, dtl, inf)
    assert np.array_equal(x[:5], np.zeros((5, 2, 3, 4)))
    inc = -0.01 * Rv / L.reference_scales(inf)
    assert np.isclose(s, np.sqrt(np.mean(inc * inc)), rtol=1e-14)
    assert np.allclose(x[5:, 0, 0, 0], inc / s, rtol=1e-14)
    assert np.isclose(np.sqrt(np.mean(x[5:] ** 2)), 1.0, rtol=1e-14)


def test_target_and_prediction_are_inverse():
    r = rng(5)
    inf = (1.1, 0.5, 0.1, 0.0, 0.9)
    Q0 = L.conserved_inf(inf)[:, None, None, None] + 0.01 * r.standard_normal((5, 2, 2, 3))
    Q1 = Q0 + 1e-4 * r.standard_normal(Q0.shape)
    y = L.target(Q0, Q1, 3e-3, inf)
    assert np.allclose(L.apply_prediction(Q0, y, 3e-3, inf), Q1, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("b1,b2", [(0.9, 0.999), (0.5, 0.9)])
def test_adam_constant_gradient_closed_form(b1, b2):
    """From zero moments under a constant gradient g, m_t = (1 - b1^t) g and v_t = (1 - b2^t) g^2
    (geometric sums), so both bias corrections give back g and g^2 exactly and every step moves
    by lr g / (|g| + eps): after T steps w_T = w_0 - T lr g / (|g| + eps).  A missing or wrong
    correction (t-independent, or b1 and b2 swapped) breaks this from t = 2 on."""
    r = rng(6)
    w0 = r.standard_normal(40)
    g = r.standard_normal(40)
    lr, eps = 2e-3, 1e-8
    w, m, v = w0.copy(), np.zeros(40), np.zeros(40)
    for t in range(1, 8):
        w, m, v = L.adam(w, g, m, v, t, lr, b1=b1, b2=b2, eps=eps)
        assert np.allclose(m, (1 - b1 ** t) * g, rtol=1e-14, atol=0)
        assert np.allclose(v, (1 - b2 ** t) * g * g, rtol=1e-13, atol=0)
        assert np.allclose(w, w0 - t * lr * g / (np.abs(g) + eps), rtol=1e-13, atol=1e-15)


def test_adam_alternating_gradient_closed_form():
    """Gradients g, -g, g, ... from zero moments: m_t = (1 - b1) g (-1)^(t+1) (1 - (-b1)^t) / (1 + b1)
    and v_t = (1 - b2^t) g^2, so step t moves by
        -lr (1 - b1) (-1)^(t+1) (1 - (-b1)^t) / ((1 + b1)(1 - b1^t)) g / (|g| + eps).
    This fixes the first-moment bias correction independently of the second."""
    b1, b2, lr, eps = 0.9, 0.999, 1e-3, 1e-8
    r = rng(7)
    g = r.standard_normal(30)
    w = r.standard_normal(30)
    m, v = np.zeros(30), np.zeros(30)
    for t in range(1, 10):
        gt = g if t % 2 else -g
        w1, m, v = L.adam(w, gt, m, v, t, lr, b1=b1, b2=b2, eps=eps)
        sgn = 1.0 if t % 2 else -1.0
        coef = (1 - b1) * sgn * (1 - (-b1) ** t) / (1 + b1)
        assert np.allclose(m, coef * g, rtol=1e-13, atol=0)
        step = -lr * coef / (1 - b1 ** t) * g / (np.abs(g) + eps)
        assert np.allclose(w1 - w, step, rtol=1e-10, atol=1e-18)
        w = w1
