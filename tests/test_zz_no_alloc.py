"""gbcfd_time_step_noalloc: the CFL time step computed with the library's fixed, file-scope device
scratch instead of caller or runtime allocations (for callers that cannot call cudaMalloc).

Checked through the C ABI against the existing entry point (gbcfd_set_state, then gbcfd_get_dt)
on two calls in a row with different states, in both precisions.  Collected last on purpose: it
must pass in a fresh process and after every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1710_09995_gb300 import cases  # noqa: E402


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09995_gb300 import gbcfd
    gbcfd.lib()
    return gbcfd


def existing_dt(gb, case, prm):
    blk = gb.Block(case.nx, case.ny, case.nz, prm)
    blk.set_metrics(spacing=case.spacing)
    blk.set_state(torch.from_numpy(case.state).cuda())
    dt = blk.get_dt()
    blk.close()
    return dt


@pytest.mark.parametrize("precision,rtol", [(0, 1e-13), (1, 1e-6)])
def test_noalloc_time_step_matches_existing_entry_point(gb, precision, rtol):
    a = cases.smooth_random(70, 19, 12, seed=31, amp=0.05, viscous=True, mu=3e-3)
    b = cases.isentropic_vortex(n=48, L=10.0, nz=5, viscous=True)
    a.spacing = (1 / 64, 1 / 16, 1 / 8)
    out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    for case in (a, b, a):  # calls in a row reuse the same static scratch
        prm = gb.params(case.gamma, case.mu, case.Pr, case.cfl, case.eps, case.viscous, case.limiter, precision)
        want = existing_dt(gb, case, prm)
        q = torch.from_numpy(np.ascontiguousarray(case.state)).cuda()
        got = float(gb.time_step_noalloc(q, prm, case.spacing, out=out).item())
        assert abs(got - want) <= rtol * want, (got, want)


def test_noalloc_rejects_oversize(gb):
    import ctypes
    q = torch.zeros((5, 1, 1, 1), dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    prm = gb.params()
    sp = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    rc = gb.lib().gbcfd_time_step_noalloc(ctypes.c_void_p(q.data_ptr()), 1024, 1024, 129, ctypes.byref(prm), sp,
                                          ctypes.c_void_p(out.data_ptr()), None)
    assert rc == gb.ERR_ARG
    assert b"at most" in gb.lib().gbcfd_last_error()


def test_noalloc_flags_nonphysical_state(gb):
    c = cases.smooth_random(16, 8, 4, seed=2)
    bad = c.state.copy()
    bad[4, 1, 2, 3] = -1.0
    q = torch.from_numpy(bad).cuda()
    got = float(gb.time_step_noalloc(q, gb.params(), c.spacing).item())
    assert got < 0.0
