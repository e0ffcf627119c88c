"""Host logic of bench.py's roofline: the HBM roofline counts the method's FP64-state minimum
of 320 bytes per cell-step (stage 1 reads Q^n and writes Q^1; stages 2 and 3 read the stage
input and Q^n and write the stage output) on both paths, and reports the mixed path's own
layout (f32 shadow and f32 stage increments, 240 bytes per cell-step) beside it."""
import bench


def test_algorithmic_bytes_per_cell_step():
    assert sum(bench.ALGO_BYTES) == 320
    assert bench.ALGO_BYTES == (80, 120, 120)
    assert sum(bench.DESIGN_BYTES["mixed"]) == 240
    assert bench.DESIGN_BYTES["fp64"] == bench.ALGO_BYTES


def test_roofline_arithmetic():
    cells, steps, ms = 1000, 2, 0.5
    res = {"stage_ms": {1: ms * steps, 2: ms * steps, 3: ms * steps}}  # 0.5 ms per launch
    r = bench.roofline("mixed", res, cells, steps, 1000.0, "measured")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["algorithmic_bytes_per_launch"] - cells * 320 / 3) < 1e-6
    assert abs(r["design_bytes_per_launch"] - cells * 240 / 3) < 1e-6
    assert abs(r["achieved"] - round(cells * 320 / 3 / 0.5e-3 / 1e9, 1)) < 1e-9
    assert abs(r["frac"] - round(cells * 320 / 3 / 0.5e-3 / 1e9 / 1000.0, 4)) < 1e-12
    assert r["avg_launch_ms"] == ms
    # curvilinear blocks add their metrics (f32 on the mixed path) to every stage
    w = bench.roofline("mixed", res, cells, steps, 1000.0, "measured", workload="warped512")
    assert abs(w["algorithmic_bytes_per_launch"] - cells * (320 + 3 * 40) / 3) < 1e-6


def test_reference_arm_has_a_sample_for_every_workload():
    """--impl reference times the oracle on a bounded sample of each workload (one step here)"""
    import argparse
    for w in bench.WORKLOADS:
        args = argparse.Namespace(workload=w, side=64)
        cells, step, state, text, metric, unit = bench.reference_sample(args)
        assert cells > 0 and text and unit in ("cell-updates/s", "cells/s")
        out = step(state)
        assert out.shape == state.shape


def test_fp64_alu_peak_and_roofline():
    """the FP64 path is bound by the FP64 pipe: its peak is 152 SMs x 2 FMA lanes x 2 flops x
    2.07 GHz = 1.2586 TFLOP/s (the recipe's nominal 1.25; gbcfd_op_rate measures 1.2524), and the
    roofline divides the flops per cell and stage (from the committed ncu summary, or None when
    that summary predates the kernel source) by the launch time"""
    assert abs(bench.FP64_PEAK_TFLOPS - 1.25856) < 1e-4
    res = {"stage_ms": {1: 1.0, 2: 1.0, 3: 1.0}}
    hbm = {"avg_launch_ms": 1.0, "traffic": None, "frac": 0.01}
    r = bench.fp64_alu_roofline(res, 1000, 1, hbm, workload="lattice96")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["peak"] == bench.FP64_PEAK_TFLOPS
    if r["achieved"] is not None:
        total = sum(r["flops_per_cell"]) * 1000
        assert abs(r["achieved"] - round(total / 3e-3 / 1e12, 4)) < 1e-9
    if r.get("lane_slot_frac") is not None:  # one lane slot per DADD, DMUL or DFMA
        nops = sum(r["ops_per_cell"]) * 1000
        assert abs(r["lane_slot_frac"] - round(nops / 3e-3 / (bench.FP64_PEAK_TFLOPS / 2 * 1e12), 4)) < 1e-9
        assert r["lane_slot_frac"] > r["frac"]


def test_wcns_step_roofline():
    """the WCNS step's figure divides the method's 320 B per cell-step, and the bytes its five
    kernels move by design, by the step's wall time"""
    cells, steps, ms = 1000, 2, 4.0
    res = {"ms": ms}
    r = bench.wcns_step_roofline("mixed", res, cells, steps, 1000.0)
    assert r["algorithmic_bytes_per_cell_step"] == 320
    assert abs(r["achieved"] - round(320 * cells * steps / 4e-3 / 1e9, 1)) < 1e-9
    design = sum(sum(bench.wcns_kernel_bytes("mixed", st).values()) for st in (1, 2, 3))
    assert r["design_bytes_per_cell_step"] == design
    # mixed: prim 44/64/64, viscres 32, x 56, y 60, z 60/80/160 bytes per cell
    assert design == (20 + 24) + (40 + 24) * 2 + 3 * (32 + 56 + 60 + 40) + 20 + 40 + 120
