"""The learned convergence accelerator's kernels against the plain definitions in oracle/learn.py:
the tensor-core convolutions (forward), the training step (loss, the gradient of every weight and
bias tensor element by element, Adam's moments and moves over several steps), the block features
and training targets, and the accept-or-restore update."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import learn as L  # noqa: E402
from paper_1710_09995_gb300 import cases  # noqa: E402


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09995_gb300 import gbcfd
    gbcfd.lib()
    return gbcfd


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def random_params(seed, scale=0.15):
    r = rng(seed)
    p = np.zeros(L.n_params())
    o = 0
    for ci, co in zip(L.CH[:-1], L.CH[1:]):
        n = co * ci * 27
        p[o:o + n] = r.standard_normal(n) * scale / np.sqrt(ci * 27 / 10)
        o += n
        p[o:o + co] = 0.05 * r.standard_normal(co)
        o += co
    return p.astype(np.float32).astype(np.float64)


def to_gpu_features(x):
    """x [B][10][Z][Y][X] -> bf16 [B Z Y X][16]"""
    B, C, Z, Y, X = x.shape
    t = np.zeros((B, Z, Y, X, 16), dtype=np.float32)
    t[..., :C] = np.transpose(x, (0, 2, 3, 4, 1))
    return torch.from_numpy(t.reshape(-1, 16)).to(torch.bfloat16).cuda()


def from_gpu(y, B, Z, Y, X, C=5):
    return np.transpose(y.float().cpu().numpy().reshape(B, Z, Y, X, -1)[..., :C], (0, 4, 1, 2, 3)).astype(np.float64)


@pytest.mark.parametrize("zper", [True, False])
def test_forward_matches_oracle(gb, zper):
    B, Z, Y, X = 2, 6, 20, 40
    p = random_params(1)
    x = rng(2).standard_normal((B, 10, Z, Y, X))
    xg = to_gpu_features(x)
    a = gb.Accel(X, Y, Z, B, zperiodic=zper)
    a.set_params(p)
    y = from_gpu(a.forward(xg), B, Z, Y, X)
    xb = from_gpu(xg, B, Z, Y, X, C=10)  # the bf16 features the GPU read
    for b in range(B):
        want, _ = L.forward(p, xb[b], zper=zper)
        err = np.linalg.norm(y[b] - want) / np.linalg.norm(want)
        assert err <= 2e-3, err


def test_forward_many_tiles_per_cta(gb):
    """a volume with a ragged second x-tile (130 cells) and several tiles per persistent CTA, so
    both input boxes and both tensor-memory accumulators are reused"""
    B, Z, Y, X = 1, 8, 40, 130
    p = random_params(11)
    xg = to_gpu_features(rng(12).standard_normal((B, 10, Z, Y, X)))
    a = gb.Accel(X, Y, Z, B)
    a.set_params(p)
    y = from_gpu(a.forward(xg), B, Z, Y, X)[0]
    want, _ = L.forward(p, from_gpu(xg, B, Z, Y, X, C=10)[0])
    assert np.linalg.norm(y - want) / np.linalg.norm(want) <= 2e-3


def test_train_step_matches_oracle_gradient(gb):
    """the loss before the step, and the first Adam move lr g / (|g| + eps) of every parameter
    whose oracle gradient is not negligible has the oracle gradient's sign"""
    B, Z, Y, X = 2, 4, 12, 36
    p = random_params(3)
    x = rng(4).standard_normal((B, 10, Z, Y, X))
    t = rng(5).standard_normal((B, 5, Z, Y, X))
    xg = to_gpu_features(x)
    tg = np.zeros((B, Z, Y, X, 8), dtype=np.float32)
    tg[..., :5] = np.transpose(t, (0, 2, 3, 4, 1))
    tg = torch.from_numpy(tg.reshape(-1, 8)).cuda()
    a = gb.Accel(X, Y, Z, B)
    a.set_params(p)
    lr = 1e-3
    loss = a.train_step(xg, tg, lr)
    p1 = a.get_params().astype(np.float64)
    xb = from_gpu(xg, B, Z, Y, X, C=10)
    want_loss, g = 0.0, np.zeros_like(p)
    for b in range(B):
        lb, gb_ = L.loss_and_grad(p, xb[b], t[b])
        want_loss += lb / B
        g += gb_ / B
    assert abs(loss - want_loss) <= 1e-3 * want_loss
    move = (p - p1) / lr
    o = 0
    for ci, co in zip(L.CH[:-1], L.CH[1:]):
        for n in (co * ci * 27, co):
            gs, ms = g[o:o + n], move[o:o + n]
            big = np.abs(gs) > 0.05 * np.abs(gs).max()
            assert np.all(np.sign(ms[big]) == np.sign(gs[big]))
            assert np.allclose(np.abs(ms[big]), 1.0, rtol=1e-3)
            o += n


TENSORS = ("W1", "b1", "W2", "b2", "W3", "b3")


def tensor_slices():
    """(name, slice) of every weight and bias tensor in the flat parameter layout"""
    out, o = [], 0
    names = iter(TENSORS)
    for ci, co in zip(L.CH[:-1], L.CH[1:]):
        for n in (co * ci * 27, co):
            out.append((next(names), slice(o, o + n)))
            o += n
    return out


def batch_loss_and_grad(p, xb, t, zper=True):
    B = xb.shape[0]
    loss, g = 0.0, np.zeros_like(p)
    for b in range(B):
        lb, gb_ = L.loss_and_grad(p, xb[b], t[b], zper=zper)
        loss += lb / B
        g += gb_ / B
    return loss, g


def train_problem(gb, B, Z, Y, X, zper, seed):
    p = random_params(seed)
    x = rng(seed + 1).standard_normal((B, 10, Z, Y, X))
    t = rng(seed + 2).standard_normal((B, 5, Z, Y, X))
    xg = to_gpu_features(x)
    tg = np.zeros((B, Z, Y, X, 8), dtype=np.float32)
    tg[..., :5] = np.transpose(t, (0, 2, 3, 4, 1))
    tg = torch.from_numpy(tg.reshape(-1, 8)).cuda()
    a = gb.Accel(X, Y, Z, B, zperiodic=zper)
    a.set_params(p)
    return a, p, xg, tg, from_gpu(xg, B, Z, Y, X, C=10), t


@pytest.mark.parametrize("shape,zper", [((2, 4, 12, 36), True), ((1, 3, 10, 130), False)])
def test_train_gradient_matches_oracle_elementwise(gb, shape, zper):
    """the raw gradient of one training step (weight-gradient kernel, tensor-core backward-data
    convolutions through SiLU', loss kernel) against the oracle's backward pass on the same bf16
    features, per tensor: relative L2 <= 1e-2 and every element within 1e-2 of the tensor's
    largest.  (bf16 storage of dY and dZ between the layers bounds the agreement.)  The second
    shape has a ragged second x tile (130 cells) and no z wrap."""
    B, Z, Y, X = shape
    a, p, xg, tg, xb, t = train_problem(gb, B, Z, Y, X, zper, 31)
    loss = a.train_step(xg, tg, 1e-3)
    g_gpu, _, _ = a.train_state()
    want_loss, g = batch_loss_and_grad(p, xb, t, zper)
    assert abs(loss - want_loss) <= 1e-3 * want_loss
    for name, sl in tensor_slices():
        got, want = g_gpu[sl].astype(np.float64), g[sl]
        err = np.linalg.norm(got - want) / np.linalg.norm(want)
        assert err <= 1e-2, (name, err)
        assert np.max(np.abs(got - want)) <= 1e-2 * np.max(np.abs(want)), name


def test_adam_state_over_three_steps_matches_oracle(gb):
    """three training steps on one batch: the gradients, Adam's moments m_t and v_t, and the
    parameters' moves against the oracle's trajectory (its gradients at its own iterates, its
    FP64 Adam with bias corrections 1 - b^t); moves compared where the gradient is not negligible
    (elsewhere Adam's normalised step follows the sign of rounding noise)"""
    B, Z, Y, X = 2, 4, 12, 36
    a, p, xg, tg, xb, t = train_problem(gb, B, Z, Y, X, True, 41)
    lr = 2e-3
    w, m, v = p.copy(), np.zeros_like(p), np.zeros_like(p)
    for step in range(1, 4):
        loss = a.train_step(xg, tg, lr)
        g_gpu, m_gpu, v_gpu = a.train_state()
        want_loss, g = batch_loss_and_grad(w, xb, t)
        w_next, m, v = L.adam(w, g, m, v, step, lr)
        assert abs(loss - want_loss) <= 1e-3 * want_loss, step
        w_gpu = a.get_params().astype(np.float64)
        for name, sl in tensor_slices():
            for got, want, tol, what in ((g_gpu, g, 1e-2, "grad"), (m_gpu, m, 1e-2, "m"), (v_gpu, v, 2e-2, "v")):
                err = np.linalg.norm(got[sl] - want[sl]) / np.linalg.norm(want[sl])
                assert err <= tol, (step, name, what, err)
            big = np.abs(m[sl]) > 0.1 * np.abs(m[sl]).max()
            mv_gpu, mv = (w_gpu - p)[sl][big], (w_next - p)[sl][big]
            assert np.linalg.norm(mv_gpu - mv) <= 2e-2 * np.linalg.norm(mv), (step, name)
        w = w_next


def test_training_reduces_the_loss(gb):
    B, Z, Y, X = 2, 4, 12, 36
    a = gb.Accel(X, Y, Z, B)
    a.set_params(random_params(6))
    x = to_gpu_features(rng(7).standard_normal((B, 10, Z, Y, X)))
    t = torch.zeros((B * Z * Y * X, 8), dtype=torch.float32, device="cuda")
    t[:, :5] = 0.5 * x[:, 5:10].float()   # a learnable target: half the residual channels
    losses = [a.train_step(x, t, 3e-3) for _ in range(60)]
    assert losses[-1] < 0.5 * losses[0], (losses[0], losses[-1])


def channel(seed=3):
    c = cases.channel_case(40, 24, 6, height=0.1, mach=0.6)
    c.state = cases.smooth_random(40, 24, 6, seed=seed, amp=0.02, mach=0.6).state
    return c


def test_features_and_target_match_oracle(gb):
    c = channel()
    bcs = oracle.bc(c.extra["bc"], c.extra["inf"])
    M = oracle.metrics_bc(c.nodes, bcs)
    p = oracle.params(c.gamma, 0.0, 0.72, c.cfl, c.eps, False, 0)
    Qp = oracle.fill_halo_bc(oracle.pad(c.state), M, bcs)
    R = oracle.residual(p, Qp, M)
    dtl = oracle.dt_local(p, Qp, M)
    want, s = L.features(c.state, R, dtl, c.extra["inf"])
    blk = gb.block_for_case(c, precision=gb.FP64)
    a = gb.Accel(c.nx, c.ny, c.nz)
    x = torch.empty((c.cells, 16), dtype=torch.bfloat16, device="cuda")
    a.features(blk, x)
    got = from_gpu(x, 1, c.nz, c.ny, c.nx, C=10)[0]
    assert np.all(np.abs(got - L.bf16(want)) <= 2 ** -7 * np.abs(want) + 1e-30)
    Q0 = blk.get_state().cpu().numpy()
    gb.step([blk], L.K_STEPS)
    t = torch.empty((c.cells, 8), dtype=torch.float32, device="cuda")
    a.target(blk, t)
    tg = from_gpu(t, 1, c.nz, c.ny, c.nx)[0]
    tw = L.target(Q0, blk.get_state().cpu().numpy(), s, c.extra["inf"])
    assert np.linalg.norm(tg - tw) <= 1e-6 * np.linalg.norm(tw)


@pytest.mark.parametrize("precision", [0, 1])
def test_try_keeps_or_restores(gb, precision):
    """zero weights predict no change: the residual does not drop and the state is restored bit
    for bit; random weights are kept only with a lower residual, else restored bit for bit"""
    c = channel(seed=4)
    blk = gb.block_for_case(c, precision=precision)
    gb.step([blk], 3)
    a = gb.Accel(c.nx, c.ny, c.nz)
    a.set_params(np.zeros(gb.ACCEL_NPARAM, dtype=np.float32))
    before = blk.get_state().clone()
    kept, r0, r1 = a.try_update(blk)
    assert not kept and r1 == r0
    assert torch.equal(blk.get_state(), before)
    twin = gb.block_for_case(c, precision=precision)
    gb.step([twin], 3)
    a.set_params(random_params(8, scale=0.05))
    kept, r0, r1 = a.try_update(blk)
    if kept:
        assert r1 < r0
    else:  # nothing else of the block changed either: it steps on exactly like its untouched twin
        assert torch.equal(blk.get_state(), before)
        gb.step([blk], 2)
        gb.step([twin], 2)
        assert torch.equal(blk.get_state(), twin.get_state())
    gb.step([blk], 2)
    assert np.all(np.isfinite(blk.residual_norm()))


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("nsteps", [3, 4])
def test_try_smooth_keeps_or_restores(gb, precision, nsteps):
    """a smoothed try (prediction x alpha, then plain steps) that misses its bar leaves the block bit
    for bit as it was -- state, norms, time steps -- so it steps on exactly like its untouched twin
    (odd step counts swap the mixed path's state buffers inside the try); one that meets it is kept
    exactly when the residual fell below the bar"""
    c = channel(seed=5)
    blk = gb.block_for_case(c, precision=precision)
    twin = gb.block_for_case(c, precision=precision)
    gb.step([blk], 3)
    gb.step([twin], 3)
    a = gb.Accel(c.nx, c.ny, c.nz)
    a.set_params(random_params(8, scale=0.05))
    before, n_before, dt_before = blk.get_state().clone(), blk.residual_norm(), blk.get_dt()
    kept, r0, r1 = a.try_smooth(blk, 0.5, nsteps, 1e-9)  # a bar no try can meet
    assert not kept and np.isfinite(r1)
    assert torch.equal(blk.get_state(), before)
    assert np.array_equal(blk.residual_norm(), n_before) and blk.get_dt() == dt_before
    gb.step([blk], 2)
    gb.step([twin], 2)
    assert torch.equal(blk.get_state(), twin.get_state())
    kept, r0, r1 = a.try_smooth(blk, 0.5, nsteps, 1.0)
    assert kept == (r1 < r0)
    gb.step([blk], 2)
    assert np.all(np.isfinite(blk.residual_norm()))
