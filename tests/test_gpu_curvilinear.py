"""Curvilinear blocks (face area vectors and volumes from grid nodes) on the GPU against the FP64
oracle, on the warped grid x' = x + 0.05 sin(2 pi y) sin(2 pi z) (and cyclic)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1710_09995_gb300 import cases  # noqa: E402


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09995_gb300 import gbcfd
    gbcfd.lib()
    return gbcfd


def oparams(c):
    return oracle.params(c.gamma, c.mu, c.Pr, c.cfl, c.eps, c.viscous, c.limiter)


def per_var(a, b):
    floor = 1e-3 * np.linalg.norm(b[0].ravel())
    return [np.linalg.norm((a[m] - b[m]).ravel()) / max(np.linalg.norm(b[m].ravel()), floor) for m in range(5)]


def warped_case(nx, ny, nz, viscous, seed=3, amp=0.05):
    c = cases.smooth_random(nx, ny, nz, seed=seed, amp=amp, viscous=viscous, mu=3e-3 if viscous else 0.0)
    c.nodes = cases.warped_nodes(nx, ny, nz, 0.05)
    return c


@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-4)])
def test_residual_warped(gb, viscous, precision, tol):
    c = warped_case(70, 19, 12, viscous)
    blk = gb.block_for_case(c, precision=precision)
    R = blk.compute_residual().cpu().numpy()
    ref = oracle.residual(oparams(c), oracle.pad(c.state), oracle.metrics(c.nodes))
    assert max(per_var(R, ref)) <= tol


@pytest.mark.parametrize("viscous", [False, True])
def test_steps_warped_fp64(gb, viscous):
    c = warped_case(40, 19, 12, viscous, seed=5)
    M = oracle.metrics(c.nodes)
    ref, dts, norms = oracle.step(oparams(c), oracle.pad(c.state), M, 5)
    blk = gb.block_for_case(c, precision=gb.FP64)
    gb.step([blk], 5)
    got = blk.get_state().cpu().numpy()
    assert max(per_var(got, oracle.interior(ref))) <= 1e-12
    assert np.allclose(blk.residual_norm(), norms[-1], rtol=1e-11, atol=0)
    assert abs(blk.get_dt() - oracle.dt(oparams(c), ref, M)) <= 1e-13 * dts[0]


def test_steps_warped_mixed(gb):
    c = warped_case(40, 19, 12, True, seed=6)
    ref, _, _ = oracle.step(oparams(c), oracle.pad(c.state), oracle.metrics(c.nodes), 20)
    blk = gb.block_for_case(c, precision=gb.MIXED)
    gb.step([blk], 20)
    err = per_var(blk.get_state().cpu().numpy(), oracle.interior(ref))
    assert err[0] <= 1e-6 and max(err) <= 1e-5, err


@pytest.mark.parametrize("precision", [0, 1])
def test_freestream_preserved_warped(gb, precision):
    c = warped_case(36, 17, 10, True, amp=0.0)
    blk = gb.block_for_case(c, precision=precision)
    R = blk.compute_residual().cpu().numpy()
    h = 1.0 / 36
    assert np.max(np.abs(R)) * h < (1e-13 if precision == 0 else 1e-5)


def test_conservation_warped(gb):
    c = warped_case(36, 17, 10, True, seed=8, amp=0.1)
    V = oracle.metrics(c.nodes)[9, 2:-2, 2:-2, 2:-2]
    blk = gb.block_for_case(c, precision=gb.FP64)
    gb.step([blk], 10)
    got = blk.get_state().cpu().numpy()
    for m in range(5):
        t0, t1 = np.sum(V * c.state[m]), np.sum(V * got[m])
        assert abs(t1 - t0) <= 1e-13 * np.sum(np.abs(V * c.state[m]))


@pytest.mark.parametrize("precision", [0, 1])
def test_multiblock_warped_matches_single(gb, precision):
    """Eight uneven curvilinear blocks (each with its own nodes) equal one block bitwise: the
    metric halos come from the neighbours, so shared faces carry identical area vectors."""
    c = warped_case(40, 24, 16, True, seed=9)
    xs, ys, zs = [0, 27, 40], [0, 9, 24], [0, 5, 16]
    grid = {}
    for a in range(2):
        for b in range(2):
            for e in range(2):
                sub = np.ascontiguousarray(c.state[:, zs[a]:zs[a + 1], ys[b]:ys[b + 1], xs[e]:xs[e + 1]])
                nod = np.ascontiguousarray(c.nodes[:, zs[a]:zs[a + 1] + 1, ys[b]:ys[b + 1] + 1, xs[e]:xs[e + 1] + 1])
                prm = gb.params(c.gamma, c.mu, c.Pr, c.cfl, c.eps, c.viscous, c.limiter, precision)
                blk = gb.Block(sub.shape[3], sub.shape[2], sub.shape[1], prm)
                blk.set_metrics(nodes=torch.from_numpy(nod).cuda())
                grid[(a, b, e)] = (blk, sub)
    for (a, b, e), (blk, _) in grid.items():
        blk.connect("+x", grid[(a, b, (e + 1) % 2)][0])
        blk.connect("+y", grid[(a, (b + 1) % 2, e)][0])
        blk.connect("+z", grid[((a + 1) % 2, b, e)][0])
    for blk, sub in grid.values():
        blk.set_state(torch.from_numpy(sub).cuda())
    single = gb.block_for_case(c, precision=precision)
    gb.step([g[0] for g in grid.values()], 3)
    gb.step([single], 3)
    out = np.zeros_like(c.state)
    for (a, b, e), (blk, _) in grid.items():
        out[:, zs[a]:zs[a + 1], ys[b]:ys[b + 1], xs[e]:xs[e + 1]] = blk.get_state().cpu().numpy()
    want = single.get_state().cpu().numpy()
    assert np.array_equal(out, want), np.max(np.abs(out - want))
