"""Parity of the CUDA WCNS-E-5 path (the paper's own scheme, Eq. 2, with fourth-order central
viscous terms; gbcfd_wcns_* through the C ABI) with the FP64 CPU oracle on the same seeded inputs.

Bars as for the finite-volume path: FP64 relative L2 <= 1e-12 per conserved variable (residual
and after N steps); mixed (FP32 interpolation, fluxes and derivatives, FP64 state) density
relative L2 <= 1e-5 after 100 steps.  Sizes span several line segments and 16-line tiles with
ragged tails in every direction; the full 256^3 vortex is checked through its exact z-invariance
against the oracle run on one plane of it.
"""
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


def oparams(case, linear=False):
    return oracle.params(case.gamma, case.mu, case.Pr, case.cfl, case.eps, case.viscous, int(bool(linear)))


def per_var(a, b):
    floor = 1e-3 * np.linalg.norm(b[0].ravel())
    return [np.linalg.norm((a[m] - b[m]).ravel()) / max(np.linalg.norm(b[m].ravel()), floor) for m in range(5)]


def ragged(viscous, seed=3, nx=70, ny=19, nz=21, amp=0.05):
    c = cases.smooth_random(nx, ny, nz, seed=seed, amp=amp, viscous=viscous, mu=3e-3 if viscous else 0.0)
    c.spacing = (1.0 / 64, 1.0 / 16, 1.0 / 20)
    return c


@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("linear", [False, True])
def test_residual_fp64(gb, viscous, linear):
    c = ragged(viscous)
    blk = gb.wcns_block_for_case(c, precision=gb.FP64, linear=linear)
    R = blk.compute_residual().cpu().numpy()
    ref = oracle.wcns_residual(oparams(c, linear), c.state, c.spacing)
    assert max(per_var(R, ref)) <= 1e-12


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 2, 5), (5, 17, 4), (60, 3, 61), (118, 7, 2)])
def test_residual_fp64_small_and_ragged(gb, shape):
    """blocks narrower than the 5-cell halo (multiple periodic wraps), one cell, and segment
    splits of 60, 61 and 118 cells"""
    nx, ny, nz = shape
    c = ragged(True, seed=9, nx=nx, ny=ny, nz=nz, amp=0.1)
    blk = gb.wcns_block_for_case(c, precision=gb.FP64)
    R = blk.compute_residual().cpu().numpy()
    ref = oracle.wcns_residual(oparams(c), c.state, c.spacing)
    # a block of one cell is uniform: R is rounding noise (~1e-32) on both sides
    assert np.abs(R - ref).max() <= 1e-12 * max(np.abs(ref).max(), 1.0)


@pytest.mark.parametrize("viscous", [False, True])
def test_residual_mixed(gb, viscous):
    """FP32 edge states and fluxes: the differences of Eq. 2 carry ~1e-7 |F| / h of rounding."""
    c = ragged(viscous)
    blk = gb.wcns_block_for_case(c, precision=gb.MIXED)
    R = blk.compute_residual().cpu().numpy()
    ref = oracle.wcns_residual(oparams(c), c.state, c.spacing)
    assert max(per_var(R, ref)) <= 1e-4


def test_residual_conserves(gb):
    c = ragged(True)
    blk = gb.wcns_block_for_case(c, precision=gb.FP64)
    R = blk.compute_residual().cpu().numpy()
    for m in range(5):
        assert abs(R[m].sum()) < 1e-12 * np.abs(R[m]).sum()


def test_uniform_flow_stays_uniform(gb):
    """Constant data: every edge state is the cell state to rounding (the GPU contracts the
    interpolation's differences into fused multiply-adds, so not bitwise), and the residual
    vanishes to rounding."""
    nx, ny, nz = 40, 18, 9
    Q = cases.conserved(np.full((nz, ny, nx), 1.1), 0.3, -0.2, 0.1, 0.8)
    c = cases.Case("uniform", nx, ny, nz, Q, None, (0.1, 0.12, 0.13), viscous=True, mu=1e-2)
    blk = gb.wcns_block_for_case(c, precision=gb.FP64)
    R = blk.compute_residual().cpu().numpy()
    assert np.abs(R).max() < 1e-12
    blk.step(3)
    assert np.abs(blk.get_state().cpu().numpy() - Q).max() < 1e-14


def test_gaussian_pulse_32_fp64_10_steps(gb):
    """32^3 Euler Gaussian pulse, CFL 0.5, WCNS-E-5 + Roe, 10 SSP-RK3 steps, FP64."""
    c = cases.gaussian_pulse(32, seed=0)
    ref, dts, norms = oracle.wcns_step(oparams(c), c.state, c.spacing, 10)
    blk = gb.wcns_block_for_case(c, precision=gb.FP64)
    blk.step(9)
    got_norm9 = blk.residual_norm()
    blk.step(1)
    got = blk.get_state().cpu().numpy()
    assert max(per_var(got, ref)) <= 1e-12
    assert abs(blk.get_dt() - dts[-1]) <= 1e-13 * dts[-1]
    assert np.allclose(blk.residual_norm(), norms[-1], rtol=1e-11, atol=0)
    assert np.allclose(got_norm9, norms[-2], rtol=1e-11, atol=0)


def test_vortex_ns_fp64_steps(gb):
    c = cases.isentropic_vortex(n=48, nz=6, L=10.0, viscous=True, Re=1e2)
    ref, _, _ = oracle.wcns_step(oparams(c), c.state, c.spacing, 8)
    blk = gb.wcns_block_for_case(c, precision=gb.FP64)
    blk.step(8)
    assert max(per_var(blk.get_state().cpu().numpy(), ref)) <= 1e-12


def test_vortex_ns_mixed_100_steps(gb):
    """The mixed-precision bar: density relative L2 <= 1e-5 after 100 steps."""
    c = cases.isentropic_vortex(n=64, nz=4, L=10.0, viscous=True, Re=1e4)
    ref, _, _ = oracle.wcns_step(oparams(c), c.state, c.spacing, 100)
    blk = gb.wcns_block_for_case(c, precision=gb.MIXED)
    blk.step(100)
    got = blk.get_state().cpu().numpy()
    err = per_var(got, ref)
    assert err[0] <= 1e-5, err


def test_full_size_vortex_256_fp64(gb):
    """Config-2 size (256^3, NS Re 1e4, vortex): the state is z-invariant, so after 2 steps every
    z-plane must equal the oracle run on a single plane (nz = 1; the z derivatives vanish)."""
    c = cases.isentropic_vortex(n=256, L=10.0, viscous=True, Re=1e4)
    blk = gb.wcns_block_for_case(c, precision=gb.FP64)
    blk.step(2)
    got = blk.get_state()
    one = cases.isentropic_vortex(n=256, nz=1, L=10.0, viscous=True, Re=1e4)
    ref, _, _ = oracle.wcns_step(oparams(one), one.state, one.spacing, 2)
    for k in (0, 77, 255):
        assert max(per_var(got[:, k:k + 1].cpu().numpy(), ref)) <= 1e-12
    spread = (got - got[:, :1]).abs().max().item()
    assert spread == 0.0


def test_errors(gb):
    prm = gb.params(local_dt=True)
    with pytest.raises(gb.GbcfdError):
        gb.WcnsBlock(8, 8, 8, prm, (0.1, 0.1, 0.1))
    with pytest.raises(gb.GbcfdError):
        gb.WcnsBlock(8, 8, 8, gb.params(), (0.1, -0.1, 0.1))
    blk = gb.WcnsBlock(8, 8, 8, gb.params(), (0.1, 0.1, 0.1))
    with pytest.raises(gb.GbcfdError) as e:
        blk.step(1)
    assert e.value.code == gb.ERR_STATE


def test_error_codes(gb):
    import ctypes
    L = gb.lib()
    n = ctypes.c_size_t(0)
    prm = gb.params()
    assert L.gbcfd_wcns_required_bytes(0, 4, 4, ctypes.byref(prm), ctypes.byref(n)) == gb.ERR_ARG
    assert L.gbcfd_wcns_required_bytes(4, 4, 4, ctypes.byref(prm), ctypes.byref(n)) == gb.OK
    mem = torch.empty(n.value + 512, dtype=torch.uint8, device="cuda")
    base = mem.data_ptr() + (-mem.data_ptr()) % 256
    h = ctypes.c_void_p(0)
    sp = (ctypes.c_double * 3)(0.1, 0.1, 0.1)
    assert L.gbcfd_wcns_create(4, 4, 4, ctypes.byref(prm), sp, ctypes.c_void_p(base + 8), n.value,
                               ctypes.byref(h)) == gb.ERR_MEMORY
    assert L.gbcfd_wcns_create(4, 4, 4, ctypes.byref(prm), sp, ctypes.c_void_p(base), n.value - 256,
                               ctypes.byref(h)) == gb.ERR_MEMORY


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
def test_nonphysical_state_is_reported(gb, precision):
    c = ragged(False, nx=20, ny=12, nz=8)
    q = c.state.copy()
    q[0, 3, 4, 5] = -0.5  # negative density in one cell
    blk = gb.wcns_block_for_case(c, precision=getattr(gb, precision))
    blk.set_state(torch.from_numpy(q).cuda())
    blk.step(1)
    with pytest.raises(gb.GbcfdError) as e:
        blk.residual_norm()
    assert e.value.code == gb.ERR_NONPHYSICAL
    blk.residual_norm()  # the flag was cleared by the first report


# ---- multi-block lattices (gbcfd_wcns_connect / gbcfd_wcns_step_many) -------------------------
def combined_rms(blocks, cells):
    """the RMS over the whole lattice from the blocks' own RMS norms"""
    s = sum(b.cells * b.residual_norm() ** 2 for b in blocks)
    return np.sqrt(s / cells)


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("viscous", [False, True])
def test_split_lattice_equals_one_block(gb, precision, viscous):
    """a periodic box split into uneven blocks -- one 3 cells wide, thinner than the 5-cell halo,
    so halos cross it into the next block; edges and corners from the diagonal blocks -- advances
    bit for bit like the single periodic block (and, in FP64, matches the oracle)"""
    c = ragged(viscous, seed=5, nx=70, ny=19, nz=21, amp=0.05)
    cuts = ([23, 3, 44], [7, 12], [2, 19])
    prec = getattr(gb, precision)
    one = gb.wcns_block_for_case(c, precision=prec)
    one.step(3)
    blocks = gb.wcns_blocks_for_split(c, cuts, precision=prec)
    gb.wcns_step_many(blocks, 3)
    got = gb.gather_wcns_split(c, cuts, blocks)
    ref = one.get_state()
    assert torch.equal(got, ref), float((got - ref).abs().max())
    assert all(b.get_dt() == one.get_dt() for b in blocks)
    assert np.allclose(combined_rms(blocks, c.cells), one.residual_norm(), rtol=1e-12, atol=0)
    if precision == "FP64":
        want, _, _ = oracle.wcns_step(oparams(c), c.state, c.spacing, 3)
        assert max(per_var(got.cpu().numpy(), want)) <= 1e-12


def test_split_vortex_128_two_by_two_by_two(gb):
    """a larger uneven 2 x 2 x 2 split of the Navier-Stokes vortex (128 x 128 x 8 cells), mixed
    precision, 4 steps: equal to the single block bit for bit"""
    c = cases.isentropic_vortex(n=128, nz=8, L=10.0, viscous=True, Re=1e4)
    cuts = ([40, 88], [101, 27], [3, 5])
    one = gb.wcns_block_for_case(c, precision=gb.MIXED)
    one.step(4)
    blocks = gb.wcns_blocks_for_split(c, cuts, precision=gb.MIXED)
    gb.wcns_step_many(blocks, 4)
    assert torch.equal(gb.gather_wcns_split(c, cuts, blocks), one.get_state())


def test_lone_block_step_many_equals_step(gb):
    c = ragged(True, seed=2, nx=33, ny=9, nz=7)
    a = gb.wcns_block_for_case(c, precision=gb.FP64)
    b = gb.wcns_block_for_case(c, precision=gb.FP64)
    a.step(2)
    gb.wcns_step_many([b], 2)
    assert torch.equal(a.get_state(), b.get_state())
    assert a.get_dt() == b.get_dt()
    assert np.array_equal(a.residual_norm(), b.residual_norm())


def test_step_many_errors(gb):
    c = ragged(False, seed=4, nx=24, ny=10, nz=6)
    cuts = ([10, 14], [10], [6])
    blocks = gb.wcns_blocks_for_split(c, cuts, precision=gb.FP64)
    with pytest.raises(gb.GbcfdError) as e:
        blocks[0].step(1)  # connected to another block
    assert e.value.code == gb.ERR_STATE
    with pytest.raises(gb.GbcfdError) as e:
        gb.wcns_step_many(blocks[:1], 1)  # its +x neighbour is not in the list
    assert e.value.code == gb.ERR_ARG
    with pytest.raises(gb.GbcfdError):
        gb.wcns_step_many([blocks[0], blocks[0]], 1)
    other = gb.WcnsBlock(10, 9, 6, gb.params(), c.spacing)
    with pytest.raises(gb.GbcfdError):
        blocks[0].connect(1, other)  # faces of different sizes
    gb.wcns_step_many(blocks, 1)  # the lattice itself still steps
    # re-connecting a face elsewhere leaves the old neighbour's link stale: refused
    third = gb.wcns_blocks_for_split(c, ([24], [10], [6]), precision=gb.FP64)[0]
    blocks[0].connect(1, third)
    with pytest.raises(gb.GbcfdError) as e:
        gb.wcns_step_many(blocks + [third], 1)
    assert e.value.code == gb.ERR_ARG
