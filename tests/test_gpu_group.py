"""Batched groups (gbcfd_group_*): many uneven blocks advanced with one stage launch per RK stage
and a CUDA graph per step.  A group step must equal gbcfd_step on the same blocks bitwise (the
per-cell arithmetic does not depend on how CTAs are split between blocks), and a lattice of
blocks must equal the FP64 oracle on the assembled global domain."""
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


SMALL = ([21, 40, 16], [17, 33], [9, 25, 14, 20])   # 3 x 2 x 4 = 24 blocks, 77 x 50 x 68 cells


def small_lattice(seed=2, sizes=SMALL):
    return cases.lattice_case(sizes=sizes, seed=seed)


def oparams(lat):
    return oracle.params(lat.gamma, 0.0, 0.72, lat.cfl, lat.eps, False, 0)


def ometrics(lat):
    return oracle.metrics(cases.cartesian_nodes(sum(lat.sx), sum(lat.sy), sum(lat.sz), *lat.spacing))


@pytest.mark.parametrize("precision", [0, 1])
def test_group_equals_step(gb, precision):
    """four steps (both parities of the mixed path twice) through the group's graphs equal
    gbcfd_step on an identical set of blocks bit for bit, state and time step"""
    lat = small_lattice()
    a = gb.blocks_for_lattice(lat, precision)
    b = gb.blocks_for_lattice(lat, precision)
    g = gb.Group(b)
    gb.step(a, 4)
    g.step(4)
    ga, gbb = gb.gather_lattice(lat, a), gb.gather_lattice(lat, b)
    assert torch.equal(ga, gbb), float((ga - gbb).abs().max())
    assert a[0].get_dt() == b[0].get_dt()
    # norms are per-CTA partial sums: the order of the additions follows the CTA split, and on
    # the mixed path each thread's partials are compensated FP32 sums (a few ulp of FP32)
    rtol = 1e-12 if precision == 0 else 1e-6
    for x, y in zip(a, b):
        assert np.allclose(x.residual_norm(), y.residual_norm(), rtol=rtol, atol=0)
    g.close()


def test_lattice_fp64_matches_oracle(gb):
    """the group's FP64 lattice after 3 steps equals the oracle's single periodic block"""
    lat = small_lattice(seed=5)
    q0 = lat.state.numpy()
    M = ometrics(lat)
    ref, dts, norms = oracle.step(oparams(lat), oracle.pad(q0), M, 3)
    blocks = gb.blocks_for_lattice(lat, gb.FP64)
    g = gb.Group(blocks)
    g.step(3)
    got = gb.gather_lattice(lat, blocks).cpu().numpy()
    want = oracle.interior(ref)
    for m in range(5):
        err = np.linalg.norm((got[m] - want[m]).ravel()) / max(np.linalg.norm(want[m].ravel()),
                                                               1e-3 * np.linalg.norm(want[0].ravel()))
        assert err <= 1e-12, (m, err)
    assert abs(blocks[0].get_dt() - oracle.dt(oparams(lat), ref, M)) <= 1e-13 * dts[0]


def test_lattice_mixed_matches_oracle(gb):
    """mixed precision after 20 steps: density within 1e-6, rho u and rho E within 1e-5.  rho v
    and rho w start at zero, so they are made of FP32 increments alone; an increment's relative
    error is the FP32 rounding times the cancellation p / dp (about 70 for a 1e-2 perturbation),
    a few 1e-6 per stage, and their bar is 1e-4 (observed 1.7e-5)."""
    lat = small_lattice(seed=6)
    ref, _, _ = oracle.step(oparams(lat), oracle.pad(lat.state.numpy()), ometrics(lat), 20)
    blocks = gb.blocks_for_lattice(lat, gb.MIXED)
    g = gb.Group(blocks)
    g.tune()
    g.step(20)
    got = gb.gather_lattice(lat, blocks).cpu().numpy()
    want = oracle.interior(ref)
    floor = 1e-3 * np.linalg.norm(want[0].ravel())
    err = [np.linalg.norm((got[m] - want[m]).ravel()) / max(np.linalg.norm(want[m].ravel()), floor)
           for m in range(5)]
    assert err[0] <= 1e-6 and err[1] <= 1e-5 and err[4] <= 1e-5 and max(err[2:4]) <= 1e-4, err


@pytest.mark.parametrize("precision", [0, 1])
def test_tune_keeps_results(gb, precision):
    """every schedule the tuner tries gives the same bits; its choice is one of its candidates"""
    lat = small_lattice(seed=7)
    a = gb.blocks_for_lattice(lat, precision)
    b = gb.blocks_for_lattice(lat, precision)
    ga, gbb = gb.Group(a), gb.Group(b)
    c = gbb.tune()
    assert c >= 1 and gbb.tile_rows in (8, ALT_TILE[precision])
    ga.step(2)
    gbb.step(2)
    assert torch.equal(gb.gather_lattice(lat, a), gb.gather_lattice(lat, b))


ALT_TILE = {0: 11, 1: 4}  # the second tile height compiled for Cartesian Euler blocks, per path


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("tile_rows,ctas,push", [(8, 1, 0), (8, 3, 1), ("alt", 1, 1), ("alt", 2, 0), ("alt", 16, 1)])
def test_every_schedule_gives_the_same_bits(gb, precision, tile_rows, ctas, push):
    """each tile shape the stage kernel is compiled for (32 x 8, and 32 x 11 FP64 / 32 x 4 mixed),
    with several grid splits and with the halo exchange of the stage outputs as launches or folded
    into the stages, advances the lattice (uneven blocks, ragged tiles in x and y) bit for bit
    like gbcfd_step on the same blocks, both parities of the mixed path"""
    ty = ALT_TILE[precision] if tile_rows == "alt" else tile_rows
    lat = small_lattice(seed=9)
    a = gb.blocks_for_lattice(lat, precision)
    b = gb.blocks_for_lattice(lat, precision)
    g = gb.Group(b)
    g.set_schedule(ctas, ty, push)
    assert g.schedule() == (ctas, ty, push)
    gb.step(a, 3)
    g.step(3)
    ga, gbb = gb.gather_lattice(lat, a), gb.gather_lattice(lat, b)
    assert torch.equal(ga, gbb), (ty, ctas, float((ga - gbb).abs().max()))
    assert a[0].get_dt() == b[0].get_dt()
    rtol = 1e-12 if precision == 0 else 1e-6
    for x, y in zip(a, b):
        assert np.allclose(x.residual_norm(), y.residual_norm(), rtol=rtol, atol=0)
    g.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_tiny_blocks_halo_push(gb, precision):
    """a lattice of blocks 2 to 5 cells wide: stages 1 and 2 of the group fill the neighbours'
    halos themselves (cells near two opposite faces push both ways; edge and corner cells into
    the diagonal blocks) and must equal gbcfd_step, whose halos come from the halo kernel, bit
    for bit over both parities of the mixed path"""
    lat = small_lattice(seed=11, sizes=([2, 5, 3], [3, 2], [2, 4]))
    a = gb.blocks_for_lattice(lat, precision)
    b = gb.blocks_for_lattice(lat, precision)
    g = gb.Group(b)
    g.set_schedule(1, 8, 1)
    gb.step(a, 4)
    g.step(4)
    ga, gbb = gb.gather_lattice(lat, a), gb.gather_lattice(lat, b)
    assert torch.equal(ga, gbb), float((ga - gbb).abs().max())
    g.close()


def test_schedule_rejects_uncompiled_shapes(gb):
    lat = small_lattice(seed=9)
    g = gb.Group(gb.blocks_for_lattice(lat, 0))
    with pytest.raises(RuntimeError):
        g.set_schedule(1, 4)   # 32 x 4 is compiled for the mixed path only
    with pytest.raises(RuntimeError):
        g.set_schedule(0, 8)
    with pytest.raises(RuntimeError):
        g.set_schedule(17, 8)
    g.close()
    # a block with an unconnected face (a wall) cannot take the halo fold
    c = cases.channel_case(40, 24, 6, height=0.1, mach=0.6)
    blk = gb.block_for_case(c, precision=0)
    g = gb.Group([blk])
    g.set_schedule(1, 8, 0)
    with pytest.raises(RuntimeError):
        g.set_schedule(1, 8, 1)
    g.close()


def test_group_curvilinear_equals_single(gb):
    """eight curvilinear blocks of a warped grid in one group equal one block stepped alone"""
    nx, ny, nz = 40, 24, 16
    c = cases.smooth_random(nx, ny, nz, seed=9, viscous=True, mu=3e-3)
    c.nodes = cases.warped_nodes(nx, ny, nz, 0.05)
    xs, ys, zs = [0, 27, 40], [0, 9, 24], [0, 5, 16]
    for precision in (0, 1):
        prm = gb.params(c.gamma, c.mu, c.Pr, c.cfl, c.eps, c.viscous, c.limiter, precision)
        grid = {}
        for a in range(2):
            for b in range(2):
                for e in range(2):
                    sub = np.ascontiguousarray(c.state[:, zs[a]:zs[a + 1], ys[b]:ys[b + 1], xs[e]:xs[e + 1]])
                    nod = np.ascontiguousarray(c.nodes[:, zs[a]:zs[a + 1] + 1, ys[b]:ys[b + 1] + 1,
                                                       xs[e]:xs[e + 1] + 1])
                    blk = gb.Block(sub.shape[3], sub.shape[2], sub.shape[1], prm)
                    blk.set_metrics(nodes=torch.from_numpy(nod).cuda())
                    grid[(a, b, e)] = (blk, sub)
        for (a, b, e), (blk, _) in grid.items():
            blk.connect("+x", grid[(a, b, (e + 1) % 2)][0])
            blk.connect("+y", grid[(a, (b + 1) % 2, e)][0])
            blk.connect("+z", grid[((a + 1) % 2, b, e)][0])
        for blk, sub in grid.values():
            blk.set_state(torch.from_numpy(sub).cuda())
        g = gb.Group([v[0] for v in grid.values()])
        g.step(3)
        single = gb.block_for_case(c, precision=precision)
        gb.step([single], 3)
        want = single.get_state().cpu().numpy()
        for (a, b, e), (blk, _) in grid.items():
            got = blk.get_state().cpu().numpy()
            assert np.array_equal(got, want[:, zs[a]:zs[a + 1], ys[b]:ys[b + 1], xs[e]:xs[e + 1]])


def test_group_timing_marks(gb):
    """the timing events bracket the three stage kernels inside the captured step"""
    lat = small_lattice(seed=8)
    blocks = gb.blocks_for_lattice(lat, gb.MIXED)
    ref = gb.blocks_for_lattice(lat, gb.MIXED)
    g = gb.Group(blocks)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
    g.set_timing(ev)
    g.step(1)
    torch.cuda.synchronize()
    t = [ev[i].elapsed_time(ev[i + 1]) for i in range(6)]
    assert all(x >= 0.0 for x in t) and sum(t[1::2]) > 0.0
    gb.step(ref, 1)
    assert torch.equal(gb.gather_lattice(lat, blocks), gb.gather_lattice(lat, ref))


def test_group_rejects_bad_members(gb):
    lat = small_lattice()
    blocks = gb.blocks_for_lattice(lat, gb.FP64)
    with pytest.raises(gb.GbcfdError):
        gb.Group(blocks[:-1])          # a neighbour outside the group
    with pytest.raises(gb.GbcfdError):
        gb.Group(blocks + blocks[:1])  # a block twice
    other = gb.blocks_for_lattice(lat, gb.MIXED)
    with pytest.raises(gb.GbcfdError):
        gb.Group(blocks + other)       # precisions differ
    g = gb.Group(blocks)
    gb.stage(blocks, 1)                # left between stages
    with pytest.raises(gb.GbcfdError):
        g.step(1)
    gb.exchange_halos(blocks)
    gb.stage(blocks, 2)
    gb.exchange_halos(blocks)
    gb.stage(blocks, 3)
    g.step(1)
