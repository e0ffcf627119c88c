"""Full-size check of the 512 x 512 x 384 warped Navier-Stokes case (Re 1e5, broadband 5%
velocity perturbation on Mach 0.3): the GPU residual of the whole block, in both precisions, is
compared with the FP64 oracle on sampled 8^3 sub-boxes.  Each sample is an exact sub-problem: the
oracle gets the 12^3 window of the state around the box (its 2-cell halo) and the metrics of that
window from the window's own nodes.  One full step then runs on the whole block in each precision
and is compared the same way (a 20^3 window per box).  The 96-block lattice gets the same
treatment after one group step."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

import oracle  # noqa: E402
from paper_1710_09995_gb300 import cases  # noqa: E402


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09995_gb300 import gbcfd
    gbcfd.lib()
    return gbcfd


@pytest.fixture(scope="module")
def case():
    return cases.broadband_warped(512, 512, 384, seed=0, device="cuda")


def sample_boxes(case, nbox=4, size=8, seed=1, edge=4):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(nbox):
        z0 = int(rng.integers(edge, case.nz - size - edge))
        y0 = int(rng.integers(edge, case.ny - size - edge))
        x0 = int(rng.integers(edge, case.nx - size - edge))
        out.append((z0, y0, x0))
    return out


def oracle_box(case, z0, y0, x0, size=8):
    h = 2
    Qp = np.ascontiguousarray(case.state[:, z0 - h:z0 + size + h, y0 - h:y0 + size + h, x0 - h:x0 + size + h])
    nodes = np.ascontiguousarray(case.nodes[:, z0 - h:z0 + size + h + 1, y0 - h:y0 + size + h + 1,
                                            x0 - h:x0 + size + h + 1])
    M = oracle.metrics(nodes)[:, 2:-2, 2:-2, 2:-2]   # metrics of the window's cells = box + halo
    p = oracle.params(case.gamma, case.mu, case.Pr, case.cfl, case.eps, case.viscous, case.limiter)
    return oracle.residual(p, np.ascontiguousarray(Qp), np.ascontiguousarray(M))


@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 1e-3)])
def test_fullsize_warped_residual_on_samples(gb, case, precision, tol):
    """R is a sum of O(1) face fluxes over an O(h) cell, so its rounding error relative to R grows
    like eps / (h |grad F|): at h = 1/512 about 1e-12 with f64 and 1e-4 with f32 fluxes and f32
    metrics (observed 1.6e-12 and 2.6e-4 at worst); the bars are 1e-11 and 1e-3."""
    blk = gb.block_for_case(case, precision=precision)
    R = blk.compute_residual()
    for z0, y0, x0 in sample_boxes(case):
        got = R[:, z0:z0 + 8, y0:y0 + 8, x0:x0 + 8].cpu().numpy()
        ref = oracle_box(case, z0, y0, x0)
        for m in range(5):
            err = np.linalg.norm(got[m] - ref[m]) / max(np.linalg.norm(ref[m]), 1e-3 * np.linalg.norm(ref[0]))
            assert err <= tol, (precision, (z0, y0, x0), m, err)
    del R
    blk.close()
    torch.cuda.empty_cache()


def step_window(case, z0, y0, x0, dt, size=8, margin=6):
    """the oracle's step of a sampled box as an exact sub-problem: the box with a 6-cell margin
    (2 halo cells per stage, 3 stages) and its metrics from the window's own nodes, stepped at
    the block's time step; the margin's outer cells take wrong (wrapped) neighbours, the box does
    not see them"""
    n = size + 2 * margin
    w = np.ascontiguousarray(case.state[:, z0 - margin:z0 - margin + n, y0 - margin:y0 - margin + n,
                                        x0 - margin:x0 - margin + n])
    nodes = np.ascontiguousarray(case.nodes[:, z0 - margin:z0 - margin + n + 1, y0 - margin:y0 - margin + n + 1,
                                            x0 - margin:x0 - margin + n + 1])
    p = oracle.params(case.gamma, case.mu, case.Pr, case.cfl, case.eps, case.viscous, case.limiter)
    ref, _, _ = oracle.step(p, oracle.pad(w), oracle.metrics(nodes), 1, dt_fixed=dt)
    inner = slice(margin, margin + size)
    return oracle.interior(ref)[:, inner, inner, inner], w[:, inner, inner, inner]


@pytest.mark.parametrize("precision", [0, 1])
def test_fullsize_warped_step_on_samples(gb, case, precision):
    """One full SSP-RK3 step of the whole 512 x 512 x 384 block, in the launch configuration the
    benchmark times, against the FP64 oracle on sampled 8^3 boxes (each an exact sub-problem, see
    step_window).  Compared per conserved variable: the new state (FP64 <= 1e-12, mixed <= 1e-5)
    and, more telling, its change over the step (FP64 <= 1e-9, mixed <= 2e-3: the change carries
    the residual's rounding, about 1e-12 and 1e-4 of R with f64 and f32 fluxes and metrics at
    h = 1/512)."""
    blk = gb.block_for_case(case, precision=precision)
    dt = blk.get_dt()
    assert dt > 0
    gb.step([blk], 1)
    norms = blk.residual_norm()
    assert np.all(np.isfinite(norms)) and norms[0] > 0
    q = blk.get_state()
    for z0, y0, x0 in sample_boxes(case, nbox=3, seed=3, edge=8):
        got = q[:, z0:z0 + 8, y0:y0 + 8, x0:x0 + 8].cpu().numpy()
        want, before = step_window(case, z0, y0, x0, dt)
        floor = 1e-3 * np.linalg.norm(want[0])
        e_state = [np.linalg.norm(got[m] - want[m]) / max(np.linalg.norm(want[m]), floor) for m in range(5)]
        dw = want - before
        dfloor = 1e-3 * np.linalg.norm(dw[0]) + 1e-300
        e_change = [np.linalg.norm((got[m] - before[m]) - dw[m]) / max(np.linalg.norm(dw[m]), dfloor)
                    for m in range(5)]
        print(f"warped step p={precision} box={(z0, y0, x0)} state={max(e_state):.2e} change={max(e_change):.2e}")
        if precision == 0:
            assert max(e_state) <= 1e-12 and max(e_change) <= 1e-9, (e_state, e_change)
        else:
            assert max(e_state) <= 1e-5 and max(e_change) <= 2e-3, (e_state, e_change)
    blk.close()
    del q
    torch.cuda.empty_cache()


# ---- the 96-block lattice (4 x 4 x 6, sides 16..160, 1.37e8 cells), Euler at Mach 0.8 ----------

@pytest.fixture(scope="module")
def lattice():
    return cases.lattice_case(device="cuda")


def lattice_windows(lat, nbox=6, size=8, seed=2):
    """sample corners, each box placed across a block interface (and some across the periodic
    wrap): the corner is drawn within 4 cells before a block boundary"""
    rng = np.random.Generator(np.random.PCG64(seed))
    ox, oy, oz = lat.offsets()
    out = []
    for i in range(nbox):
        c = []
        for off in (oz, oy, ox):
            b = off[int(rng.integers(0, len(off) - 1))]
            c.append((b - int(rng.integers(1, 5))) % off[-1])
        out.append(tuple(c))
    out[0] = (oz[-1] - 4, oy[-1] - 4, ox[-1] - 4)  # the corner where the wrap meets in all three
    return out


def window(lat, z0, y0, x0, size, margin):
    N = lat.state.shape[1:]
    idx = [torch.arange(a - margin, a + size + margin, device=lat.state.device) % n for a, n in zip((z0, y0, x0), N)]
    return lat.state[:, idx[0]][:, :, idx[1]][:, :, :, idx[2]].cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1])
def test_fullsize_lattice_group_step(gb, lattice, precision):
    """One group step of the full lattice equals the FP64 oracle on sampled 8^3 boxes.  Each
    sample is an exact sub-problem: the oracle steps the box with a 6-cell margin (2 halo cells
    per stage, 3 stages) at the group's time step, and only the box is compared.  The time step is
    the minimum of the blocks' CFL steps; the FP64 ones are checked against the oracle's on
    sampled blocks.  Bars: FP64 1e-12, mixed 1e-6 density and 1e-5 others (relative L2 per
    variable, floor 1e-3 of density's norm)."""
    lat = lattice
    blocks = gb.blocks_for_lattice(lat, precision)
    dts = [b.get_dt() for b in blocks]
    p = oracle.params(lat.gamma, 0.0, 0.72, lat.cfl, lat.eps, False, 0)
    if precision == 0:
        sl = list(lat.block_slices().values())
        for bi in (0, 37, 95):
            zs, ys, xs = sl[bi]
            q = lat.state[:, zs, ys, xs].cpu().numpy()
            nz_, ny_, nx_ = q.shape[1:]
            M = oracle.metrics(cases.cartesian_nodes(nx_, ny_, nz_, *lat.spacing))
            want = oracle.dt(p, oracle.pad(q), M)
            assert abs(dts[bi] - want) <= 1e-13 * want
    dt = min(dts)
    g = gb.Group(blocks)
    g.tune()
    g.step(1)
    out = gb.gather_lattice(lat, blocks)
    assert abs(blocks[0].get_dt() - blocks[-1].get_dt()) == 0.0
    size, margin = 8, 6
    for z0, y0, x0 in lattice_windows(lat):
        w = window(lat, z0, y0, x0, size, margin)
        n = size + 2 * margin
        M = oracle.metrics(cases.cartesian_nodes(n, n, n, *lat.spacing))
        ref, _, _ = oracle.step(p, oracle.pad(w), M, 1, dt_fixed=dt)
        want = oracle.interior(ref)[:, margin:margin + size, margin:margin + size, margin:margin + size]
        N = out.shape[1:]
        idx = [torch.arange(a, a + size, device=out.device) % m for a, m in zip((z0, y0, x0), N)]
        got = out[:, idx[0]][:, :, idx[1]][:, :, :, idx[2]].cpu().numpy()
        floor = 1e-3 * np.linalg.norm(want[0])
        err = [np.linalg.norm(got[m] - want[m]) / max(np.linalg.norm(want[m]), floor) for m in range(5)]
        if precision == 0:
            assert max(err) <= 1e-12, ((z0, y0, x0), err)
        else:
            assert err[0] <= 1e-6 and max(err) <= 1e-5, ((z0, y0, x0), err)
    g.close()
    for b in blocks:
        b.close()
    del out, blocks
    torch.cuda.empty_cache()
