"""The steady-channel path on the GPU against the FP64 oracle: slip-wall and characteristic
far-field ghost cells, halo metrics from reflected nodes, local time steps; on the curvilinear
bump channel (x in [-1, 2], bump 0.1 sin^2(pi x) on the lower wall, stretched towards it)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1710_09995_gb300 import cases  # noqa: E402

G = 1.4


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09995_gb300 import gbcfd
    gbcfd.lib()
    return gbcfd


def per_var(a, b):
    floor = 1e-3 * np.linalg.norm(b[0].ravel())
    return [np.linalg.norm((a[m] - b[m]).ravel()) / max(np.linalg.norm(b[m].ravel()), floor) for m in range(5)]


def channel(nx=40, ny=24, nz=6, height=0.1, mach=0.6, perturb=0.02, seed=3):
    """the bump channel with a smooth seeded perturbation on the free stream, so that every cell
    and every boundary sees a non-trivial state"""
    c = cases.channel_case(nx, ny, nz, height=height, mach=mach)
    if perturb:
        r = cases.smooth_random(nx, ny, nz, seed=seed, amp=perturb, mach=mach)
        c.state = r.state
    return c


def oracle_setup(c):
    bcs = oracle.bc(c.extra["bc"], c.extra["inf"])
    M = oracle.metrics_bc(c.nodes, bcs)
    p = oracle.params(c.gamma, 0.0, 0.72, c.cfl, c.eps, False, 0)
    return bcs, M, p


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-4)])
def test_channel_residual(gb, precision, tol):
    c = channel()
    bcs, M, p = oracle_setup(c)
    ref = oracle.residual(p, oracle.fill_halo_bc(oracle.pad(c.state), M, bcs), M)
    blk = gb.block_for_case(c, precision=precision)
    R = blk.compute_residual().cpu().numpy()
    assert max(per_var(R, ref)) <= tol, per_var(R, ref)


def test_channel_local_steps_fp64(gb):
    """20 local-time-step SSP-RK3 steps: state, residual norms and smallest step"""
    c = channel(seed=5)
    bcs, M, p = oracle_setup(c)
    ref, dts, norms = oracle.step_ex(p, oracle.pad(c.state), M, 20, bcs, local_dt=True)
    blk = gb.block_for_case(c, precision=gb.FP64)
    gb.step([blk], 20)
    got = blk.get_state().cpu().numpy()
    assert max(per_var(got, oracle.interior(ref))) <= 1e-12
    assert np.allclose(blk.residual_norm(), norms[-1], rtol=1e-10, atol=0)
    assert abs(blk.get_dt() - oracle.dt_local(p, oracle.fill_halo_bc(ref, M, bcs), M).min()) <= 1e-12 * dts[0]


def test_channel_local_steps_mixed(gb):
    """50 local-time-step steps on the mixed path (FP32 ghosts and increments): density and
    energy within 1e-6 of the oracle (relative L2), each momentum component within 1e-5 of the
    momentum vector's norm (the transverse components are small, and their FP32 increments'
    error scales with the whole flux; observed 1.3e-5 relative to the w-momentum's own norm)"""
    c = channel(seed=6)
    bcs, M, p = oracle_setup(c)
    ref, _, _ = oracle.step_ex(p, oracle.pad(c.state), M, 50, bcs, local_dt=True)
    blk = gb.block_for_case(c, precision=gb.MIXED)
    gb.step([blk], 50)
    got, want = blk.get_state().cpu().numpy(), oracle.interior(ref)
    err = per_var(got, want)
    mom = np.linalg.norm(want[1:4].ravel())
    emom = [np.linalg.norm((got[m] - want[m]).ravel()) / mom for m in (1, 2, 3)]
    assert err[0] <= 1e-6 and err[4] <= 1e-6 and max(emom) <= 1e-5, (err, emom)


def test_channel_global_step_fp64(gb):
    """boundary conditions with the global time step too"""
    c = channel(seed=7)
    bcs, M, p = oracle_setup(c)
    ref, _, _ = oracle.step_ex(p, oracle.pad(c.state), M, 10, bcs)
    blk = gb.block_for_case(c, precision=gb.FP64, local_dt=False)
    gb.step([blk], 10)
    assert max(per_var(blk.get_state().cpu().numpy(), oracle.interior(ref))) <= 1e-12


@pytest.mark.parametrize("precision", [0, 1])
def test_closed_box_conserves_mass_and_energy(gb, precision):
    """slip walls on all six faces of a Cartesian box: total mass and energy stay constant"""
    n = (36, 20, 12)
    c = cases.smooth_random(*n, seed=4, amp=0.1, mach=0.3)
    prm = gb.params(G, 0.0, 0.72, 0.5, 0.1, False, 0, precision)
    blk = gb.Block(*n, prm)
    for f in gb.FACES:
        blk.set_boundary(f, gb.BC_SLIP_WALL)
    blk.set_metrics(spacing=(1.0 / 36, 0.05, 1.0 / 12))
    blk.set_state(torch.from_numpy(c.state).cuda())
    gb.step([blk], 30)
    q = blk.get_state().cpu().numpy()
    tol = 1e-13 if precision == 0 else 1e-6
    for m in (0, 4):
        assert abs(q[m].sum() - c.state[m].sum()) <= tol * np.abs(c.state[m]).sum()


@pytest.mark.parametrize("precision", [0, 1])
def test_split_channel_equals_single_block(gb, precision):
    """the channel cut into three blocks along x (interfaces connected, boundary faces on the
    outer ones) steps bitwise like the single block, alone and as a group"""
    c = channel(nx=48, ny=16, nz=4, seed=8)
    cuts = [0, 13, 30, 48]
    prm = gb.params(c.gamma, 0.0, 0.72, c.cfl, c.eps, False, 0, precision, True)
    parts = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        blk = gb.Block(b - a, c.ny, c.nz, prm)
        blk.set_metrics(nodes=torch.from_numpy(np.ascontiguousarray(c.nodes[:, :, :, a:b + 1])).cuda())
        parts.append(blk)
    for i, blk in enumerate(parts):
        for f in ("-y", "+y"):
            blk.set_boundary(f, gb.BC_SLIP_WALL)
        blk.connect("+z", blk)
        if i + 1 < len(parts):
            blk.connect("+x", parts[i + 1])
    parts[0].set_boundary("-x", gb.BC_FARFIELD, c.extra["inf"])
    parts[-1].set_boundary("+x", gb.BC_FARFIELD, c.extra["inf"])
    for blk, (a, b) in zip(parts, zip(cuts[:-1], cuts[1:])):
        blk.set_state(torch.from_numpy(np.ascontiguousarray(c.state[:, :, :, a:b])).cuda())
    single = gb.block_for_case(c, precision=precision)
    gb.step(parts, 5)
    gb.step([single], 5)
    want = single.get_state().cpu().numpy()
    got = np.concatenate([blk.get_state().cpu().numpy() for blk in parts], axis=3)
    assert np.array_equal(got, want), np.abs(got - want).max()
    g = gb.Group(parts)
    g.step(3)
    gb.step([single], 3)
    got = np.concatenate([blk.get_state().cpu().numpy() for blk in parts], axis=3)
    assert np.array_equal(got, single.get_state().cpu().numpy())


def test_boundary_argument_errors(gb):
    prm = gb.params(G, 0.0, 0.72, 0.5, 0.1, False, 0, gb.FP64)
    blk = gb.Block(8, 8, 4, prm)
    blk.connect("+z", blk)
    with pytest.raises(gb.GbcfdError):
        blk.set_boundary("-z", gb.BC_SLIP_WALL)                       # connected face
    with pytest.raises(gb.GbcfdError):
        blk.set_boundary("-x", gb.BC_FARFIELD, None)                  # no free stream
    with pytest.raises(gb.GbcfdError):
        blk.set_boundary("-x", gb.BC_FARFIELD, (0.0, 0.5, 0, 0, 1.0))  # rho = 0
    with pytest.raises(gb.GbcfdError):
        blk.set_boundary("-x", 7)                                     # unknown kind
    blk.set_boundary("-y", gb.BC_SLIP_WALL)
    with pytest.raises(gb.GbcfdError):
        blk.connect("-y", blk)                                        # face has a condition
    visc = gb.Block(8, 8, 4, gb.params(G, 1e-3, 0.72, 0.5, 0.1, True, 0, gb.FP64))
    with pytest.raises(gb.GbcfdError):
        visc.set_boundary("-y", gb.BC_SLIP_WALL)                      # viscous block
    with pytest.raises(gb.GbcfdError):
        gb.Block(8, 8, 4, gb.params(G, 1e-3, 0.72, 0.5, 0.1, True, 0, gb.FP64, True))  # local dt + viscous


def test_hybrid_solve_reaches_what_fp64_reaches(gb):
    """on a coarse bump channel the mixed path alone stalls near its FP32 floor (a few 1e-6),
    while the hybrid (mixed, then FP64 from the stalled state) reaches a 1e-8 drop like the
    plain FP64 iteration"""
    from paper_1710_09995_gb300 import learn
    c = cases.channel_case(48, 24, 2, height=0.1, mach=0.5)
    fp64 = learn.solve(c, target=1e-8, precision="fp64", max_seconds=60)
    mixed = learn.solve(c, target=1e-8, precision="mixed", max_seconds=8)
    hybrid = learn.solve(c, target=1e-8, precision="hybrid", max_seconds=60, stall_checks=10)
    assert fp64["reached"] and hybrid["reached"], (fp64["drop"], hybrid["drop"])
    assert not mixed["reached"] and mixed["drop"] > 1e-7
    assert "fp64" in {h[3] for h in hybrid["history"]}
