"""The host-to-host pipeline (gbcfd_pipe_*, gbcfd_wcns_pipe_create): states in pinned host
memory advanced through a set of identical blocks, with the host-link copies overlapping the
steps.  Its results must equal, bit for bit, the set-state / step / get-state calls on one block
(same kernels, launch shapes and reduction order), and the FP64 results the oracle's to the FP64
bar (1e-12 relative L2 per conserved variable)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1710_09995_gb300 import cases  # noqa: E402

SHAPE = (45, 19, 10)  # two tiles and a ragged tail in x, three in y
SPACING = (1.0 / 45, 1.0 / 19, 1.0 / 10)


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09995_gb300 import gbcfd
    gbcfd.lib()
    return gbcfd


def member(gb, precision, shape=SHAPE):
    nx, ny, nz = shape
    b = gb.Block(nx, ny, nz, gb.params(mu=2e-3, viscous=True, precision=precision)).periodic()
    b.set_metrics(spacing=SPACING)
    return b


def states(n, shape=SHAPE):
    nx, ny, nz = shape
    return [cases.smooth_random(nx, ny, nz, seed=40 + i, amp=0.05, viscous=True, mu=2e-3).state for i in range(n)]


def pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


@pytest.mark.parametrize("precision", [0, 1])
def test_pipe_equals_block_calls_bitwise(gb, precision):
    """7 items over 3 members (every member reused, so every wait on a previous download runs)"""
    qs = states(7)
    members = [member(gb, precision) for _ in range(3)]
    pipe = gb.Pipe(members)
    ins = [pinned(q) for q in qs]
    outs = [torch.empty_like(t).pin_memory() for t in ins]
    norms = [torch.zeros(5, dtype=torch.float64).pin_memory() for _ in ins]
    for q, o, r in zip(ins, outs, norms):
        pipe.submit(q, o, nsteps=2, norms=r)
    pipe.sync()
    ref = member(gb, precision)
    for q, o, r in zip(qs, outs, norms):
        ref.set_state(torch.from_numpy(q).cuda())
        gb.step([ref], 2)
        assert torch.equal(o, ref.get_state().cpu())
        assert np.array_equal(r.numpy(), ref.residual_norm())
    pipe.close()


def test_pipe_fp64_matches_oracle(gb):
    c = cases.smooth_random(*SHAPE, seed=41, amp=0.05, viscous=True, mu=2e-3)
    c.spacing = SPACING
    pipe = gb.Pipe([member(gb, 0) for _ in range(2)])
    qin = pinned(c.state)
    out = torch.empty_like(qin).pin_memory()
    pipe.submit(qin, out, nsteps=3)
    pipe.sync()
    prm = oracle.params(c.gamma, c.mu, c.Pr, c.cfl, c.eps, c.viscous, c.limiter)
    Q, _, _ = oracle.step(prm, oracle.pad(c.state), oracle.metrics(c.grid_nodes()), 3)
    ref = oracle.interior(Q)
    got = out.numpy()
    floor = 1e-3 * np.linalg.norm(ref[0].ravel())
    err = [np.linalg.norm((got[m] - ref[m]).ravel()) / max(np.linalg.norm(ref[m].ravel()), floor) for m in range(5)]
    assert max(err) <= 1e-12, err


def test_pipe_zero_steps_round_trip(gb):
    q = states(1)[0]
    pipe = gb.Pipe([member(gb, 1)])
    qin, out = pinned(q), torch.zeros(q.shape, dtype=torch.float64).pin_memory()
    pipe.submit(qin, out, nsteps=0)
    pipe.sync()
    assert torch.equal(out, qin)


def test_pipe_arguments_checked(gb):
    a, b = member(gb, 0), member(gb, 0)
    other = member(gb, 0, shape=(20, 19, 10))
    mixed = member(gb, 1)
    for bad in ([a, other], [a, mixed], [a, a]):
        with pytest.raises(gb.GbcfdError) as e:
            gb.Pipe(bad)
        assert e.value.code == gb.ERR_ARG
    c1, c2 = member(gb, 0), member(gb, 0)
    c1.connect("+x", c2)
    with pytest.raises(gb.GbcfdError) as e:
        gb.Pipe([c1])
    assert e.value.code == gb.ERR_ARG
    pipe = gb.Pipe([a, b])
    q = states(1)[0]
    good_in, good_out = pinned(q), torch.empty(q.shape, dtype=torch.float64).pin_memory()
    for qi, qo in ((torch.from_numpy(q), good_out), (good_in, torch.empty(q.shape, dtype=torch.float64)),
                   (good_in.cuda(), good_out)):
        with pytest.raises(gb.GbcfdError) as e:
            pipe.submit(qi, qo)
        assert e.value.code == gb.ERR_ARG
    with pytest.raises(gb.GbcfdError) as e:
        pipe.submit(good_in, good_out, nsteps=-1)
    assert e.value.code == gb.ERR_ARG
    pipe.sync()  # nothing was enqueued by the refused calls
    pipe.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_pipe_nonphysical_item_is_reported(gb, precision):
    q = states(2)
    bad = q[1].copy()
    bad[0, 4, 5, 6] = -0.5  # negative density in one cell of the second item
    pipe = gb.Pipe([member(gb, precision) for _ in range(2)])
    ins = [pinned(q[0]), pinned(bad)]
    outs = [torch.empty_like(t).pin_memory() for t in ins]
    for i, o in zip(ins, outs):
        pipe.submit(i, o, nsteps=1)
    with pytest.raises(gb.GbcfdError) as e:
        pipe.sync()
    assert e.value.code == gb.ERR_NONPHYSICAL
    pipe.submit(ins[0], outs[0], nsteps=1)
    pipe.sync()  # the flag was cleared by the first report
    pipe.close()


# ---- the paper's WCNS-E-5 blocks -------------------------------------------------------------

def wcns_member(gb, precision, shape=SHAPE):
    nx, ny, nz = shape
    return gb.WcnsBlock(nx, ny, nz, gb.params(mu=2e-3, viscous=True, precision=precision), SPACING)


@pytest.mark.parametrize("precision", [0, 1])
def test_wcns_pipe_equals_block_calls_bitwise(gb, precision):
    qs = states(5)
    pipe = gb.Pipe([wcns_member(gb, precision) for _ in range(3)])
    ins = [pinned(q) for q in qs]
    outs = [torch.empty_like(t).pin_memory() for t in ins]
    norms = [torch.zeros(5, dtype=torch.float64).pin_memory() for _ in ins]
    for q, o, r in zip(ins, outs, norms):
        pipe.submit(q, o, nsteps=2, norms=r)
    pipe.sync()
    ref = wcns_member(gb, precision)
    for q, o, r in zip(qs, outs, norms):
        ref.set_state(torch.from_numpy(q).cuda())
        ref.step(2)
        assert torch.equal(o, ref.get_state().cpu())
        assert np.array_equal(r.numpy(), ref.residual_norm())
    pipe.close()


def test_wcns_pipe_fp64_matches_oracle(gb):
    c = cases.smooth_random(*SHAPE, seed=42, amp=0.05, viscous=True, mu=2e-3)
    pipe = gb.Pipe([wcns_member(gb, 0) for _ in range(2)])
    qin = pinned(c.state)
    out = torch.empty_like(qin).pin_memory()
    pipe.submit(qin, out, nsteps=2)
    pipe.sync()
    prm = oracle.params(c.gamma, c.mu, c.Pr, c.cfl, c.eps, c.viscous, 0)
    ref, _, _ = oracle.wcns_step(prm, c.state, SPACING, 2)
    got = out.numpy()
    floor = 1e-3 * np.linalg.norm(ref[0].ravel())
    err = [np.linalg.norm((got[m] - ref[m]).ravel()) / max(np.linalg.norm(ref[m].ravel()), floor) for m in range(5)]
    assert max(err) <= 1e-12, err


def test_wcns_pipe_arguments_checked(gb):
    a = wcns_member(gb, 0)
    for bad in ([a, wcns_member(gb, 0, shape=(20, 19, 10))], [a, wcns_member(gb, 1)], [a, a]):
        with pytest.raises(gb.GbcfdError) as e:
            gb.Pipe(bad)
        assert e.value.code == gb.ERR_ARG


@pytest.mark.parametrize("precision", [0, 1])
def test_wcns_pipe_nonphysical_item_is_reported(gb, precision):
    q = states(2)
    bad = q[1].copy()
    bad[0, 4, 5, 6] = -0.5
    pipe = gb.Pipe([wcns_member(gb, precision) for _ in range(2)])
    ins = [pinned(q[0]), pinned(bad)]
    outs = [torch.empty_like(t).pin_memory() for t in ins]
    for i, o in zip(ins, outs):
        pipe.submit(i, o, nsteps=1)
    with pytest.raises(gb.GbcfdError) as e:
        pipe.sync()
    assert e.value.code == gb.ERR_NONPHYSICAL
    pipe.submit(ins[0], outs[0], nsteps=1)
    pipe.sync()
    pipe.close()


# ---- groups of uneven blocks ------------------------------------------------------------------

SMALL = ([21, 40, 16], [17, 33], [9, 25, 14, 20])   # 3 x 2 x 4 = 24 blocks, 77 x 50 x 68 cells


def lattice_item(lat):
    """an item of a group pipeline: the blocks' compact states, concatenated in block order"""
    parts = [lat.state[:, zs, ys, xs].contiguous().reshape(-1) for zs, ys, xs in lat.block_slices().values()]
    return torch.cat(parts).pin_memory()


@pytest.mark.parametrize("precision", [0, 1])
def test_group_pipe_equals_group_calls_bitwise(gb, precision):
    lats = [cases.lattice_case(sizes=SMALL, seed=s) for s in (2, 3, 4, 5)]
    groups = [gb.Group(gb.blocks_for_lattice(lats[0], precision)) for _ in range(3)]
    pipe = gb.Pipe(groups)
    nb = len(groups[0].blocks)
    ins = [lattice_item(lat) for lat in lats]
    outs = [torch.empty_like(t).pin_memory() for t in ins]
    norms = [torch.zeros(5 * nb, dtype=torch.float64).pin_memory() for _ in ins]
    for q, o, r in zip(ins, outs, norms):
        pipe.submit(q, o, nsteps=2, norms=r)
    pipe.sync()
    ref_blocks = gb.blocks_for_lattice(lats[0], precision)
    ref = gb.Group(ref_blocks)
    for lat, o, r in zip(lats, outs, norms):
        for b, (zs, ys, xs) in zip(ref_blocks, lat.block_slices().values()):
            b.set_state(lat.state[:, zs, ys, xs].contiguous().cuda())
        ref.step(2)
        got = torch.cat([b.get_state().reshape(-1) for b in ref_blocks]).cpu()
        assert torch.equal(o, got)
        assert np.array_equal(r.numpy(), np.concatenate([b.residual_norm() for b in ref_blocks]))
    pipe.close()


def test_group_pipe_arguments_checked(gb):
    lat = cases.lattice_case(sizes=SMALL, seed=2)
    other = cases.lattice_case(sizes=([21, 40, 16], [17, 33], [9, 25, 14, 21]), seed=2)
    a = gb.Group(gb.blocks_for_lattice(lat, 1))
    for bad in ([a, gb.Group(gb.blocks_for_lattice(other, 1))], [a, gb.Group(gb.blocks_for_lattice(lat, 0))], [a, a]):
        with pytest.raises(gb.GbcfdError) as e:
            gb.Pipe(bad)
        assert e.value.code == gb.ERR_ARG
