"""Full-size check of the 512 x 512 x 384 warped Navier-Stokes case (Re 1e5, broadband 5%
velocity perturbation on Mach 0.3): the GPU residual of the whole block, in both precisions, is
compared with the FP64 oracle on sampled 8^3 sub-boxes.  Each sample is an exact sub-problem: the
oracle gets the 12^3 window of the state around the box (its 2-cell halo) and the metrics of that
window from the window's own nodes.  One mixed-precision step then runs on the full block."""
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


def sample_boxes(case, nbox=4, size=8, seed=1):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(nbox):
        z0 = int(rng.integers(4, case.nz - size - 4))
        y0 = int(rng.integers(4, case.ny - size - 4))
        x0 = int(rng.integers(4, case.nx - size - 4))
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


def test_fullsize_warped_mixed_step(gb, case):
    blk = gb.block_for_case(case, precision=gb.MIXED)
    dt0 = blk.get_dt()
    gb.step([blk], 1)
    norms = blk.residual_norm()
    assert np.all(np.isfinite(norms)) and norms[0] > 0
    q = blk.get_state()
    assert bool(torch.isfinite(q).all().item())
    dq = (q[0] - torch.from_numpy(case.state[0]).cuda()).abs().max().item()
    assert 0 < dq < 0.1
    assert dt0 > 0
    blk.close()
