"""gbcfd_op_rate: the arithmetic throughput the FP64 roofline and the FP64 path's choice of
operations rest on.  The FP64 FMA rate must lie near the unit-count peak (152 SMs x 2 FP64 FMA
lanes x 2 flops x 2.07 GHz = 1.2586 TFLOP/s; below it when the clock is lower), FP32 FMAs far
above it, and the Newton reciprocal the FP64 path uses must beat IEEE division."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09995_gb300 import gbcfd
    gbcfd.lib()
    return gbcfd


def test_op_rates(gb):
    dfma = gb.op_rate(gb.OP_DFMA)
    ffma = gb.op_rate(gb.OP_FFMA)
    div = gb.op_rate(gb.OP_DIV)
    rcp = gb.op_rate(gb.OP_RCP_NEWTON)
    rsq = gb.op_rate(gb.OP_RSQRT)
    peak = 1.25856e12  # FP64 flop/s from the unit count and the maximum clock
    assert 0.5 * peak <= 2 * dfma <= 1.05 * peak, 2 * dfma
    assert ffma >= 20 * dfma, (ffma, dfma)
    assert rcp >= 1.2 * div, (rcp, div)  # the reason the FP64 path takes the Newton step
    assert 0 < rsq < dfma and 0 < div < dfma


def test_fp64_instruction_forms(gb):
    """an FP64 FMA of three registers issues faster than an FP64 add or multiply, or an FMA with
    constant-bank operands (measured 598 against 504 G/s)"""
    dfma = gb.op_rate(gb.OP_DFMA)
    for op in (gb.OP_DADD, gb.OP_DMUL, gb.OP_DFMA_CONST):
        r = gb.op_rate(op)
        assert 0.5 * dfma < r <= 1.02 * dfma, (op, r, dfma)


def test_op_rate_rejects_unknown_op(gb):
    with pytest.raises(gb.GbcfdError):
        gb.op_rate(8)
