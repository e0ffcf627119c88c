#!/usr/bin/env python
"""Benchmark of the structured-grid finite-volume hot path on one GB300 (or N replicas).

Default workload: the batched multi-block case, 96 uneven Cartesian blocks (a 4x4x6 periodic
lattice with sides drawn from 16..160, 1.37e8 cells), Euler at Mach 0.8, MUSCL/minmod + Roe,
SSP-RK3 at CFL 0.5, advanced as one group: per step one CUDA graph holding the time step and,
three times, the halo exchange of every block and one fused stage launch for all blocks.  The
headline `value` is the FP64 path (the paper's precision); the mixed path (FP32 reconstruction
and fluxes, FP64 state, update and norms) is timed on the same case beside it, and the 256^3
Navier-Stokes vortex (both paths) and the steady bump channel's wall time to a 1e-6 residual
drop (plain FP64 iteration against the learned-accelerated mixed form) are extra keys of the
same line.  Other workloads: --workload.

Prints one JSON line (rank 0).  Inputs are seeded and synthetic (the paper's meshes are not
available).  `--impl reference` times the FP64 CPU oracle instead (the only reference there is).
"""
import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DEFAULT = 256
PEAK_FALLBACK_GBS = 6800.0
# algorithmic HBM bytes per interior cell for stages 1, 2, 3 (halos excluded): the method's
# minimum with an FP64 state -- stage 1 reads Q^n and writes Q^1, stages 2 and 3 read the stage
# input and Q^n and write the stage output: 80 + 120 + 120 = 320 B per cell-step, both paths
ALGO_BYTES = (40 + 40, 40 + 40 + 40, 40 + 40 + 40)
# the fraction of measured HBM bandwidth the residual/update kernels are meant to reach
HBM_TARGET_FRAC = 0.60
# what each path's own layout moves: the mixed path keeps an f32 shadow S^n and f32 stage
# increments D, so it reads S^n (+ D) and writes D, and only stage 3 touches the f64 state
DESIGN_BYTES = {
    "mixed": (20 + 20, 20 + 20 + 20, 20 + 20 + 40 + 40 + 20),  # S^n, D read; D or Q^{n+1}, S^{n+1} written
    "fp64": ALGO_BYTES,
}
WORKLOADS = {
    "vortex256": "isentropic vortex 256^3, Navier-Stokes Re 1e4 Pr 0.72, MUSCL/minmod + Roe, SSP-RK3 CFL 0.5",
    "warped512": ("warped curvilinear block 512x512x384, Navier-Stokes Re 1e5, 5% broadband velocity on Mach 0.3, "
                  "MUSCL/minmod + Roe, SSP-RK3 CFL 0.5"),
    "accel": ("learned accelerator inference: 3-layer conv3d 10->32->32->5, 3^3 taps, bf16 x bf16 -> f32 on "
              "tcgen05, over the 192x96x64 bump-channel grid (periodic in z)"),
    "channel": ("bump channel 192x96x64 (curvilinear, 10% bump, stretched 1.1 to the wall), Euler, Mach 0.6, "
                "far field in/out, slip walls, local pseudo-time steps to a 1e-6 density-residual drop"),
    "wcns256": ("isentropic vortex 256^3, Navier-Stokes Re 1e4 Pr 0.72, the paper's WCNS-E-5 (Eq. 2, weighted "
                "nonlinear interpolation, Roe edge fluxes) + fourth-order central viscous terms, SSP-RK3 CFL 0.5"),
    "lattice96": ("96 uneven Cartesian blocks (4x4x6 lattice, sides 16..160, seed 4: 506x492x550 = 1.37e8 cells), "
                  "Euler, Mach 0.8 + 1e-2 Fourier perturbation, MUSCL/minmod + Roe, SSP-RK3 CFL 0.5, "
                  "one group: one launch per stage, CUDA graph per step, autotuned grid split"),
}
# metric bytes read per cell and stage on curvilinear blocks (10 fields)
METRIC_BYTES = {"mixed": 40, "fp64": 80}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gbcfd", choices=["gbcfd", "reference"])
    ap.add_argument("--side", type=int, default=N_DEFAULT, help="cells per side of the cubic vortex block")
    ap.add_argument("--workload", default="lattice96", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=None, choices=["both", "mixed", "fp64"],
                    help="default: both for vortex256 (mixed first) and lattice96 (FP64 first), mixed for warped512")
    ap.add_argument("--e2e-steps", type=int, default=None, help="default 20 (3 for the FP64 lattice)")
    ap.add_argument("--no-channel", action="store_true",
                    help="lattice96: skip the bump channel's time-to-drop key (the longest part of the run)")
    ap.add_argument("--no-vortex", action="store_true", help="lattice96: skip the 256^3 vortex key")
    ap.add_argument("--schedule", default=None,
                    help="lattice96: pin the groups' schedule 'ctas_per_sm,tile_rows,halo_push' instead of tuning "
                         "(profiling runs: no tuner launches before the steps)")
    ap.add_argument("--lattice-div", type=int, default=1,
                    help="lattice96: divide every block side by this (same recipe, fewer cells: profiling runs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--target", type=float, default=1e-6, help="channel: residual drop to reach")
    ap.add_argument("--max-seconds", type=float, default=900.0, help="channel: cap per solve")
    return ap.parse_args()


# ---- distributed plumbing (independent replicas; no data-path collective) ------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---- clocks ----------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[4:]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for name, flag in zip(names, r[3][1:]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        loaded = [r for r in rows if r[2] > 200.0] or rows
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "power_w_max": max(r[2] for r in rows), "reasons": sorted(reasons)}


# ---- peaks and profile evidence --------------------------------------------------------------
def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return PEAK_FALLBACK_GBS, "fallback"


def kernel_source_hash(curvi=False):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1710_09995_gb300", "csrc")
    for name in ("stage.cuh", "physics.cuh", "internal.cuh", "vmath.cuh", "stage_inst.cuh") + (("curvi.cuh",) if curvi else ()):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


PROFILE_TAG = {"vortex256": "vortex", "warped512": "warped", "lattice96": "lattice"}


def profiled_traffic(precision, workload="vortex256"):
    """DRAM bytes per stage launch from the committed ncu summary, if it was taken on the
    current kernel source (else None)."""
    v = profiled_numbers(precision, "dram bytes per stage launch at full size", workload)
    return v[0] if v else None


# ---- the GPU arm -----------------------------------------------------------------------------
def time_path(gbcfd, torch, case, precision, steps, warmup, world, device):
    blk = gbcfd.block_for_case(case, precision=gbcfd.MIXED if precision == "mixed" else gbcfd.FP64)
    stream = torch.cuda.current_stream()

    def one_step(evs=None):
        for s in (1, 2, 3):
            if evs is not None:
                evs[s][0].record(stream)
            gbcfd.exchange_halos([blk], stream)
            if evs is not None:
                evs[s][1].record(stream)
            gbcfd.stage([blk], s, stream)
            if evs is not None:
                evs[s][2].record(stream)

    for _ in range(warmup):
        one_step()
    torch.cuda.synchronize()
    events = [{s: [torch.cuda.Event(enable_timing=True) for _ in range(3)] for s in (1, 2, 3)}
              for _ in range(steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    start.record(stream)
    for k in range(steps):
        one_step(events[k])
    stop.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = max_over_ranks(start.elapsed_time(stop), world, device)
    stage_ms = {s: sum(e[s][1].elapsed_time(e[s][2]) for e in events) for s in (1, 2, 3)}
    halo_ms = sum(e[s][0].elapsed_time(e[s][1]) for e in events for s in (1, 2, 3))
    norms = blk.residual_norm()  # also surfaces any device-side error flag
    blk.close()
    return {"ms": ms, "stage_ms": stage_ms, "halo_ms": halo_ms, "launches": 6 * steps, "norms": norms.tolist()}


def schedule_group(g, schedule):
    """the tuner's choice, or the pinned 'ctas_per_sm,tile_rows,halo_push'; returns CTAs per SM"""
    if not schedule:
        return g.tune()
    c, t, p = (int(x) for x in schedule.split(","))
    g.set_schedule(c, t, p)
    return c


def time_group_path(gbcfd, torch, lat, precision, steps, warmup, world, device, schedule=None):
    """The lattice as one group: per step one CUDA graph (time step, then halo exchange and one
    stage launch for all blocks, three times).  Seven events recorded inside the graph time each
    stage kernel; the stream is synchronised after every step to read them (the host gap this
    leaves is inside the timed region)."""
    blocks = gbcfd.blocks_for_lattice(lat, gbcfd.MIXED if precision == "mixed" else gbcfd.FP64, device)
    g = gbcfd.Group(blocks)
    ctas_per_sm = schedule_group(g, schedule)
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
    g.set_timing(marks)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        g.step(1, stream)
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stage_ms = {1: 0.0, 2: 0.0, 3: 0.0}
    halo_ms = 0.0
    barrier(world)
    torch.cuda.synchronize()
    start.record(stream)
    for _ in range(steps):
        g.step(1, stream)
        stream.synchronize()
        for st in (1, 2, 3):
            stage_ms[st] += marks[2 * st - 1].elapsed_time(marks[2 * st])
            halo_ms += marks[2 * st - 2].elapsed_time(marks[2 * st - 1])
    stop.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = max_over_ranks(start.elapsed_time(stop), world, device)
    norms = [b.residual_norm().tolist() for b in blocks]
    _, tile_rows, halo_push = g.schedule()
    g.close()
    for b in blocks:
        b.close()
    return {"ms": ms, "stage_ms": stage_ms, "halo_ms": halo_ms, "launches": 7 * steps, "norms": norms[0],
            "ctas_per_sm": ctas_per_sm, "tile": [32, tile_rows],
            "halo": "folded into stages 1-2" if halo_push else "launch per stage", "blocks": len(blocks)}


def e2e_group_path(gbcfd, torch, lat, precision, steps, world, device, pipelined=True, schedule=None):
    """Through the C ABI with pinned host buffers, every step uploading each block's state,
    advancing the group one SSP-RK3 step and reading back every block's state and residual norms:
    the value is per-block set_state, one group step and per-block get_state / residual_norm calls,
    one after the other (what a time-marching user sees).  With `pipelined`, `pipelined_value`
    runs the steps as independent items of a 3-group gbcfd_pipe instead (an item is the blocks'
    states concatenated)."""
    import gc
    prec = gbcfd.MIXED if precision == "mixed" else gbcfd.FP64
    parts = [lat.state[:, zs, ys, xs].contiguous().cpu() for zs, ys, xs in lat.block_slices().values()]
    nbytes = sum(h.numel() * 8 for h in parts)
    nblk_all = len(parts)
    # serial calls
    blocks = gbcfd.blocks_for_lattice(lat, prec, device)
    g = gbcfd.Group(blocks)
    schedule_group(g, schedule)
    host_in = [h.pin_memory() for h in parts]
    host_out = [torch.empty_like(h).pin_memory() for h in host_in]

    def one():
        for b, h in zip(blocks, host_in):
            b.set_state(h)
        g.step(1)
        for b, h in zip(blocks, host_out):
            b.get_state(h)
        for b in blocks:
            b.residual_norm()

    one()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    torch.cuda.synchronize()
    serial = max_over_ranks(time.perf_counter() - t0, world, device)
    g.close()
    for b in blocks:
        b.close()
    del g, blocks, one, host_in, host_out
    out = {"value": world * lat.cells * steps / serial, "unit": "cell-updates/s",
           "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes + 112 * nblk_all,
           "api": "per block gbcfd_set_state, gbcfd_group_step, per block gbcfd_get_state + gbcfd_residual_norm "
                  "(time marching: each step's state uploaded and read back)", "steps": steps}
    if not pipelined:
        return out
    item = torch.cat([h.reshape(-1) for h in parts]).pin_memory()
    nblk = len(parts)
    del parts  # host memory: the pipeline holds the item and two output buffers (5.5 GB each)
    gc.collect()
    torch.cuda.empty_cache()
    # the pipeline: 3 member groups (tuned alike); downloads are ordered, so two output buffers
    groups = []
    for _ in range(3):
        gg = gbcfd.Group(gbcfd.blocks_for_lattice(lat, prec, device))
        schedule_group(gg, schedule)
        groups.append(gg)
    pipe = gbcfd.Pipe(groups)
    outs = [torch.empty_like(item).pin_memory() for _ in range(2)]
    norms = torch.zeros((max(steps, 3), pipe.norms_numel), dtype=torch.float64).pin_memory()
    for i in range(3):
        pipe.submit(item, outs[i % 2], 1, norms[i])
    pipe.sync()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(steps):
        pipe.submit(item, outs[i % 2], 1, norms[i])
    pipe.sync()
    dt = max_over_ranks(time.perf_counter() - t0, world, device)
    pipe.close()
    for gg in groups:
        gg.close()
        for b in gg.blocks:
            b.close()
    out["pipelined_value"] = world * lat.cells * steps / dt
    out["pipelined_api"] = "gbcfd_pipe_submit x steps + gbcfd_pipe_sync (3 member groups; steps as independent items)"
    return out


def e2e_path(gbcfd, torch, case, precision, steps, world, device):
    """Through the C ABI with pinned host buffers, every step uploading the state, advancing it one
    SSP-RK3 step and reading back the new state and its residual norms: the value is set_state /
    step / get_state / residual_norm calls on one block, one after the other (what a time-marching
    user sees); `pipelined_value` runs the steps as independent items through a 3-block
    gbcfd_pipe instead (host-link copies of neighbouring items overlap the steps)."""
    prec = gbcfd.MIXED if precision == "mixed" else gbcfd.FP64
    host_in = torch.from_numpy(case.state).pin_memory()
    nbytes = case.state.nbytes
    ctrl_bytes = 112  # the control block read by residual_norm
    # serial calls on one block
    blk = gbcfd.block_for_case(case, precision=prec)
    host_out = torch.empty_like(host_in).pin_memory()
    blk.set_state(host_in)
    gbcfd.step([blk], 1)
    blk.get_state(host_out)
    blk.residual_norm()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        blk.set_state(host_in)
        gbcfd.step([blk], 1)
        blk.get_state(host_out)
        blk.residual_norm()
    torch.cuda.synchronize()
    serial = max_over_ranks(time.perf_counter() - t0, world, device)
    blk.close()
    # the pipeline: 3 members, a ring of 3 output buffers, the norms of every item
    members = [gbcfd.block_for_case(case, precision=prec) for _ in range(3)]
    pipe = gbcfd.Pipe(members)
    outs = [torch.empty_like(host_in).pin_memory() for _ in range(3)]
    norms = torch.zeros((max(steps, 3), 5), dtype=torch.float64).pin_memory()
    for i in range(3):
        pipe.submit(host_in, outs[i], 1, norms[i])
    pipe.sync()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(steps):
        pipe.submit(host_in, outs[i % 3], 1, norms[i])
    pipe.sync()
    dt = max_over_ranks(time.perf_counter() - t0, world, device)
    pipe.close()
    for b in members:
        b.close()
    return {"value": world * case.cells * steps / serial, "unit": "cell-updates/s",
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes + ctrl_bytes,
            "api": "gbcfd_set_state + gbcfd_step + gbcfd_get_state + gbcfd_residual_norm per step "
                   "(time marching: each step's state uploaded and read back)",
            "pipelined_value": world * case.cells * steps / dt,
            "pipelined_api": "gbcfd_pipe_submit x steps + gbcfd_pipe_sync (3 member blocks; steps as independent items)",
            "steps": steps}


# GB300 FP64 peak from unit counts and clock: 152 SMs x 2 FP64 FMA lanes per clock x 2 flops x
# 2.07 GHz (the recipe's nominal 1.25 TFLOP/s; gbcfd_op_rate's DFMA chains measure 1.2524)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
ISSUE_PER_CLK = 152 * 4 * 32  # SMs x schedulers x lanes: thread instructions issued per clock


def profiled_numbers(precision, key, workload="vortex256"):
    """numbers of a `key: a b c` line in the committed ncu summary, if it was taken on the current
    kernel source (else None)"""
    path = os.path.join(ROOT, "profiles", f"stage_kernel_{precision}_{PROFILE_TAG[workload]}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m_hash = re.search(r"kernel source hash:\s*([0-9a-f]+)", text)
    m = re.search(re.escape(key) + r":\s*([0-9.eE+ ]+)", text)
    if not m_hash or not m or m_hash.group(1) != kernel_source_hash(workload == "warped512"):
        return None
    return [float(x) for x in m.group(1).split()]


def roofline(precision, res, cells, steps, peak, peak_kind, workload="vortex256"):
    """HBM roofline of the stage kernel: algorithmic bytes per launch / mean launch time.  The
    bytes are the method's FP64-state minimum (ALGO_BYTES); design_* gives the same ratio for
    the bytes the path's own layout moves (smaller on the mixed path)."""
    extra = METRIC_BYTES[precision] if workload == "warped512" else 0
    nbytes = sum((ALGO_BYTES[s - 1] + extra) * cells * steps for s in (1, 2, 3))
    dbytes = sum((DESIGN_BYTES[precision][s - 1] + extra) * cells * steps for s in (1, 2, 3))
    sec = sum(res["stage_ms"].values()) / 1e3
    achieved = nbytes / sec / 1e9
    traffic = profiled_traffic(precision, workload)
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "target_frac": HBM_TARGET_FRAC, "peak_kind": peak_kind,
            "traffic": traffic, "algorithmic_bytes_per_launch": nbytes / (3 * steps),
            "design_bytes_per_launch": dbytes / (3 * steps),
            "design_frac": round(dbytes / sec / 1e9 / peak, 4),
            "kernel": "stage_kernel", "avg_launch_ms": round(sec * 1e3 / (3 * steps), 4)}


def fp64_alu_roofline(res, cells, steps, hbm, workload="vortex256"):
    """FP64-pipe roofline of the FP64 stage kernel: its FP64 flops per cell (2 DFMA + DADD + DMUL,
    counted by ncu per stage) over the launch time, against the part's FP64 peak; and the share of
    the pipe's lane slots its FP64 instructions fill (DADD + DMUL + DFMA per cell against 152 SMs x
    2 lanes x the clock)"""
    flops = profiled_numbers("fp64", "fp64 flops per cell and stage", workload)
    out = {"bound": "alu", "kernel": "stage_kernel", "unit": "TFLOP/s", "peak": FP64_PEAK_TFLOPS,
           "peak_kind": "FP64 FMA lanes x clock (152 SMs x 2 x 2 flops x 2.07 GHz; 1.2524 measured by gbcfd_op_rate)",
           "avg_launch_ms": hbm["avg_launch_ms"],
           "traffic": hbm["traffic"], "hbm_frac": hbm["frac"]}
    ops = profiled_numbers("fp64", "fp64 ops per cell and stage", workload)
    if flops:
        sec = sum(res["stage_ms"].values()) / 1e3
        total = sum(flops[s - 1] * cells * steps for s in (1, 2, 3))
        achieved = total / sec / 1e12
        out.update({"achieved": round(achieved, 4), "frac": round(achieved / FP64_PEAK_TFLOPS, 4),
                    "flops_per_cell": flops})
        if ops:  # FP64 instructions per FMA issue slot (a DADD or DMUL counted as one; they issue at 84% of an FMA's rate)
            nops = sum(ops[s - 1] * cells * steps for s in (1, 2, 3))
            out.update({"lane_slot_frac": round(nops / sec / (FP64_PEAK_TFLOPS / 2 * 1e12), 4),
                        "ops_per_cell": ops})
    else:
        out.update({"achieved": None, "frac": None})
    return out


def issue_estimate(precision, res, cells, steps, sm_mhz, workload="vortex256"):
    """instruction-issue utilisation of the stage kernel: ncu's thread instructions per cell over
    the launch time, against 152 SMs x 4 schedulers x 32 lanes per clock at the sampled clock"""
    inst = profiled_numbers(precision, "thread instructions per cell and stage", workload)
    if not inst or not sm_mhz:
        return None
    total = sum(inst[s - 1] * cells * steps for s in (1, 2, 3))
    rate = total / (sum(res["stage_ms"].values()) / 1e3)
    peak = ISSUE_PER_CLK * sm_mhz * 1e6
    return {"achieved_tinst_per_s": round(rate / 1e12, 3), "peak_tinst_per_s": round(peak / 1e12, 3),
            "frac": round(rate / peak, 4), "instructions_per_cell": inst}


def cpu_model():
    """the host CPU's model name (lscpu or /proc/cpuinfo), for the CPU baseline's record"""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for key in ("Model name:", "Vendor ID:"):
            for line in out.splitlines():
                if line.strip().startswith(key):
                    return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def cpu_baseline_sample(n):
    """The FP64 oracle on the host cores: one SSP-RK3 step of a 256 x 256 x 64 z-slab of the
    (z-invariant) vortex -- exactly a sub-problem of the workload -- best of 2 on all cores, and
    one step of a 256 x 256 x 8 slab on one core."""
    import oracle
    from paper_1710_09995_gb300 import cases
    nz = 64
    c = cases.isentropic_vortex(n=n, L=10.0, nz=nz, viscous=True)
    M = oracle.metrics(c.grid_nodes())
    p = oracle.params(c.gamma, c.mu, c.Pr, c.cfl, c.eps, c.viscous, c.limiter)
    Q = oracle.pad(c.state)
    best = math.inf
    for _ in range(2):
        t0 = time.perf_counter()
        oracle.step(p, Q, M, 1)
        best = min(best, time.perf_counter() - t0)
    cores = oracle.threads()
    c1 = cases.isentropic_vortex(n=n, L=10.0, nz=8, viscous=True)
    M1, Q1 = oracle.metrics(c1.grid_nodes()), oracle.pad(c1.state)
    oracle.set_threads(1)
    t0 = time.perf_counter()
    oracle.step(p, Q1, M1, 1)
    one = c1.cells / (time.perf_counter() - t0)
    oracle.set_threads(cores)
    return {"value": c.cells / best, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"1 SSP-RK3 step (FP64) of a {n}x{n}x{nz} z-slab of the z-invariant vortex, best of 2",
            "value_1core": one, "sample_1core": f"1 SSP-RK3 step of a {n}x{n}x8 z-slab on one thread",
            "cpu": cpu_model()}


def cpu_baseline_warped():
    """The FP64 oracle on the host cores on a bounded sample of the warped 512x512x384 case: one
    SSP-RK3 step of a periodic 128 x 128 x 96 block with the same grid map, perturbation recipe
    and physics (1/16 of the cells), best of 2."""
    import oracle
    from paper_1710_09995_gb300 import cases
    c = cases.broadband_warped(128, 128, 96, seed=0)
    M = oracle.metrics(c.nodes)
    p = oracle.params(c.gamma, c.mu, c.Pr, c.cfl, c.eps, c.viscous, c.limiter)
    Q = oracle.pad(c.state)
    best = math.inf
    for _ in range(2):
        t0 = time.perf_counter()
        oracle.step(p, Q, M, 1)
        best = min(best, time.perf_counter() - t0)
    return {"value": c.cells / best, "unit": "cell-updates/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": "1 SSP-RK3 step (FP64) of a periodic 128x128x96 warped block, same recipe, best of 2"}


def cpu_baseline_lattice():
    """The FP64 oracle on the host cores on a bounded sample of the lattice workload: one SSP-RK3
    step of a periodic 128 x 128 x 96 block with the same state recipe and physics, best of 2."""
    import oracle
    from paper_1710_09995_gb300 import cases
    lat = cases.lattice_case(sizes=([128], [128], [96]), seed=4)
    M = oracle.metrics(cases.cartesian_nodes(128, 128, 96, *lat.spacing))
    p = oracle.params(lat.gamma, 0.0, 0.72, lat.cfl, lat.eps, False, 0)
    Q = oracle.pad(lat.state.numpy())
    best = math.inf
    for _ in range(2):
        t0 = time.perf_counter()
        oracle.step(p, Q, M, 1)
        best = min(best, time.perf_counter() - t0)
    return {"value": lat.cells / best, "unit": "cell-updates/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": "1 SSP-RK3 step (FP64, Euler) of a periodic 128x128x96 block, same recipe, best of 2"}


def run_gbcfd(args):
    world, rank, local = dist_env()
    import torch
    if world > 1:
        dist_init(world, "nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    from paper_1710_09995_gb300 import cases, gbcfd
    gbcfd.lib()
    if args.workload == "lattice96":
        return run_lattice(args, world, rank, local, device, torch, cases, gbcfd)
    if args.workload == "channel":
        return run_channel(args, world, rank, local, device, torch, cases, gbcfd)
    if args.workload == "accel":
        return run_accel(args, world, rank, local, device, torch, gbcfd)
    if args.workload == "wcns256":
        return run_wcns(args, world, rank, local, device, torch, cases, gbcfd)
    if args.workload == "warped512":
        case = cases.broadband_warped(512, 512, 384, seed=0, device=device)
        prec = args.precision or "mixed"
    else:
        case = cases.isentropic_vortex(n=args.side, L=10.0, viscous=True)
        prec = args.precision or "both"
    peak, peak_kind = hbm_peak()
    paths = ["mixed", "fp64"] if prec == "both" else [prec]
    clocks = ClockSampler(local)
    clocks.start()
    results = {p: time_path(gbcfd, torch, case, p, args.steps, args.warmup, world, device) for p in paths}
    clk = clocks.stop()
    head = paths[0]
    e2e = e2e_path(gbcfd, torch, case, head, args.e2e_steps or 20, world, device)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample(args.side) if args.workload == "vortex256" else cpu_baseline_warped()
    if rank != 0:
        return
    r = results[head]
    out = {
        "metric": "cell-updates/s",
        "value": world * case.cells * args.steps / (r["ms"] / 1e3),
        "unit": "cell-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": r["ms"] / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64" if head == "mixed" else "f64",
        "data": ("synthetic (seeded closed-form vortex; the paper's meshes are not available)"
                 if args.workload == "vortex256" else
                 "synthetic (seeded warped grid and Fourier-mode perturbation; the paper's meshes are not available)"),
        "config": {"workload": WORKLOADS[args.workload], "cells": case.cells, "precision": head,
                   "l2": "working set > 1.4 GB >> 129 MB L2, no flush needed",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline(head, r, case.cells, args.steps, peak, peak_kind, args.workload),
        "issue": issue_estimate(head, r, case.cells, args.steps, clk.get("sm_mhz"), args.workload),
        "e2e": e2e,
        "gpu_launches": r["launches"],
        "clocks": clk,
        "cpu_baseline": cpu,
        "halo_ms_per_step": r["halo_ms"] / args.steps,
        "residual_norm": r["norms"],
    }
    for p in paths[1:]:
        rp = results[p]
        hbm = roofline(p, rp, case.cells, args.steps, peak, peak_kind, args.workload)
        out[p] = {"value": world * case.cells * args.steps / (rp["ms"] / 1e3), "unit": "cell-updates/s",
                  "ms_per_step": rp["ms"] / args.steps, "dtype": "f64" if p == "fp64" else "f32+f64",
                  "roofline": fp64_alu_roofline(rp, case.cells, args.steps, hbm, args.workload) if p == "fp64" else hbm,
                  "gpu_launches": rp["launches"]}
    print(json.dumps(out))


def vortex_key(args, world, device, torch, cases, gbcfd):
    """the 256^3 Navier-Stokes vortex, both paths, as a key of the lattice line"""
    peak, peak_kind = hbm_peak()
    case = cases.isentropic_vortex(n=args.side, L=10.0, viscous=True)
    out = {"workload": WORKLOADS["vortex256"], "cells": case.cells, "steps": args.steps, "warmup": args.warmup}
    for p in ("mixed", "fp64"):
        r = time_path(gbcfd, torch, case, p, args.steps, args.warmup, world, device)
        hbm = roofline(p, r, case.cells, args.steps, peak, peak_kind, "vortex256")
        out[p] = {"value": world * case.cells * args.steps / (r["ms"] / 1e3), "unit": "cell-updates/s",
                  "ms_per_step": r["ms"] / args.steps, "dtype": "f64" if p == "fp64" else "f32+f64",
                  "roofline": fp64_alu_roofline(r, case.cells, args.steps, hbm, "vortex256") if p == "fp64" else hbm,
                  "halo_ms_per_step": r["halo_ms"] / args.steps, "gpu_launches": r["launches"]}
    return out


def channel_key(args, device, cases):
    """wall time to a 1e-6 density-residual drop on the steady bump channel (192x96x64): the plain
    FP64 iteration, the mixed path finished on the FP64 path (hybrid) without and with the learned
    accelerator's tries"""
    from paper_1710_09995_gb300 import learn
    case = cases.channel_case(*learn.FULL_GRID, height=0.1, mach=0.6)
    params, info = (learn.load() if os.path.exists(learn.WEIGHTS) else (None, None))
    runs = {"fp64_plain": learn.solve(case, args.target, None, args.max_seconds, precision="fp64", device=device),
            "hybrid_plain": learn.solve(case, args.target, None, args.max_seconds, precision="hybrid", device=device)}
    if params is not None:  # smoothed tries: prediction x alpha, 20 plain steps, kept only if they beat plain
        runs["hybrid_learned"] = learn.solve(case, args.target, params, args.max_seconds, precision="hybrid",
                                             device=device, smooth=20, check=200)
    head = runs.get("hybrid_learned", runs["hybrid_plain"])
    out = {"metric": f"seconds to a {args.target:g} density-residual drop", "unit": "s",
           "workload": WORKLOADS["channel"], "cells": case.cells, "accelerator": info}
    for k, r in runs.items():
        out[k] = {"seconds": r["seconds"], "reached": r["reached"], "steps": r["steps"],
                  "drop": r.get("drop"), **{x: r[x] for x in ("tried", "kept", "smooth") if x in r}}
    plain = runs["fp64_plain"]
    out["speedup_vs_fp64_plain"] = (plain["seconds"] / head["seconds"]
                                    if head["reached"] and plain["reached"] else None)
    return out


def run_lattice(args, world, rank, local, device, torch, cases, gbcfd):
    if args.lattice_div > 1:
        full = cases.lattice_sizes(cases.lattice_seed((4, 4, 6), 16, 160), (4, 4, 6), 16, 160)
        sizes = [[max(8, v // args.lattice_div) for v in s] for s in full]
        lat = cases.lattice_case(sizes=sizes, seed=4, device=device)
    else:
        lat = cases.lattice_case(device=device)
    prec = args.precision or "both"
    paths = ["fp64", "mixed"] if prec == "both" else [prec]
    peak, peak_kind = hbm_peak()
    clocks = ClockSampler(local)
    clocks.start()
    results = {p: time_group_path(gbcfd, torch, lat, p, args.steps, args.warmup, world, device, args.schedule)
               for p in paths}
    clk = clocks.stop()
    head = paths[0]
    e2e_steps = args.e2e_steps if args.e2e_steps is not None else (3 if head == "fp64" else 20)
    e2e = e2e_group_path(gbcfd, torch, lat, head, e2e_steps, world, device, pipelined=head == "mixed",
                         schedule=args.schedule)
    cpu = cpu_baseline_lattice() if rank == 0 and world == 1 and not args.no_cpu_baseline else None
    cells = lat.cells
    del lat
    torch.cuda.empty_cache()
    vortex = None if args.no_vortex else vortex_key(args, world, device, torch, cases, gbcfd)
    channel = None if args.no_channel else channel_key(args, device, cases)
    if rank != 0:
        return
    r = results[head]
    hbm = roofline(head, r, cells, args.steps, peak, peak_kind, "lattice96")
    out = {
        "metric": "cell-updates/s",
        "value": world * cells * args.steps / (r["ms"] / 1e3),
        "unit": "cell-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": r["ms"] / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64" if head == "mixed" else "f64",
        "data": "synthetic (seeded lattice sizes and Fourier-mode phases; the paper's meshes are not available)",
        "config": {"workload": WORKLOADS["lattice96"], "cells": cells, "blocks": r["blocks"], "precision": head,
                   "ctas_per_sm": r["ctas_per_sm"], "tile": r.get("tile"), "halo": r.get("halo"),
                   "l2": "working set > 20 GB >> 129 MB L2, no flush needed",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": fp64_alu_roofline(r, cells, args.steps, hbm, "lattice96") if head == "fp64" else hbm,
        "issue": issue_estimate(head, r, cells, args.steps, clk.get("sm_mhz"), "lattice96"),
        "e2e": e2e,
        "gpu_launches": r["launches"],
        "clocks": clk,
        "cpu_baseline": cpu,
        "halo_ms_per_step": r["halo_ms"] / args.steps,
        "residual_norm": r["norms"],
    }
    for p in paths[1:]:
        rp = results[p]
        hp = roofline(p, rp, cells, args.steps, peak, peak_kind, "lattice96")
        out[p] = {"value": world * cells * args.steps / (rp["ms"] / 1e3), "unit": "cell-updates/s",
                  "ms_per_step": rp["ms"] / args.steps, "dtype": "f64" if p == "fp64" else "f32+f64",
                  "ctas_per_sm": rp["ctas_per_sm"], "tile": rp.get("tile"), "halo": rp.get("halo"),
                  "roofline": fp64_alu_roofline(rp, cells, args.steps, hp, "lattice96") if p == "fp64" else hp,
                  "issue": issue_estimate(p, rp, cells, args.steps, clk.get("sm_mhz"), "lattice96"),
                  "halo_ms_per_step": rp["halo_ms"] / args.steps, "gpu_launches": rp["launches"]}
    if vortex is not None:
        out["vortex256"] = vortex
    if channel is not None:
        out["channel"] = channel
    print(json.dumps(out))


def bf16_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"]), "measured (cuBLAS bf16 burst)"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback"


ACCEL_FLOPS_PER_CELL = 2 * 27 * (10 * 32 + 32 * 32 + 32 * 5)  # useful multiply-adds x 2 per inference


def run_accel(args, world, rank, local, device, torch, gbcfd):
    """The accelerator's forward pass (three tensor-core convolutions) on the full channel grid:
    cells per second and the tensor roofline (useful flops / time against the bf16 peak)."""
    from paper_1710_09995_gb300 import learn
    nx, ny, nz = learn.FULL_GRID
    cells = nx * ny * nz
    acc = gbcfd.Accel(nx, ny, nz, 1, device=device)
    params = learn.load()[0] if os.path.exists(learn.WEIGHTS) else learn.init_params(0)
    acc.set_params(params)
    gen = torch.Generator(device="cpu").manual_seed(0)
    x = torch.randn((cells, 16), generator=gen).to(device=device, dtype=torch.bfloat16)
    y = torch.empty((cells, 8), dtype=torch.float32, device=device)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        acc.forward(x, y, stream)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(args.steps):
        acc.forward(x, y, stream)
    stop.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = max_over_ranks(start.elapsed_time(stop), world, device)
    clk = clocks.stop()
    host_x = x.cpu().pin_memory()
    host_y = torch.empty((cells, 8), dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(min(args.e2e_steps or 20, args.steps)):
        x.copy_(host_x, non_blocking=True)
        acc.forward(x, y, stream)
        host_y.copy_(y, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if rank != 0:
        return
    peak, peak_kind = bf16_peak()
    per = ms / args.steps
    achieved = ACCEL_FLOPS_PER_CELL * cells / (per / 1e3) / 1e12
    out = {
        "metric": "cell inferences/s", "value": world * cells * args.steps / (ms / 1e3), "unit": "cells/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": per,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 x bf16 -> f32",
        "data": "synthetic (random features; trained weights)",
        "config": {"workload": WORKLOADS["accel"], "cells": cells, "l2": "activations 1.2e6 x 64 B per layer"},
        "roofline": {"bound": "tensor", "achieved": round(achieved, 1), "peak": peak, "unit": "TFLOP/s",
                     "frac": round(achieved / peak, 4), "peak_kind": peak_kind, "traffic": None,
                     "kernel": "conv_tc_kernel (3 launches)", "flops_per_cell": ACCEL_FLOPS_PER_CELL},
        "e2e": {"value": world * cells * min(args.e2e_steps or 20, args.steps) / e2e_s, "unit": "cells/s",
                "h2d_bytes_per_step": cells * 16 * 2, "d2h_bytes_per_step": cells * 8 * 4},
        "gpu_launches": 3 * args.steps, "clocks": clk,
        "cpu_baseline": None if (world > 1 or args.no_cpu_baseline) else cpu_baseline_accel(params),
    }
    print(json.dumps(out))


def cpu_baseline_accel(params):
    """the numpy network of the oracle (FP64, bf16-rounded storage) on a 96 x 48 x 4 sample of
    the grid, best of 2"""
    import numpy as np
    from oracle import learn as L
    r = np.random.Generator(np.random.PCG64(0))
    x = r.standard_normal((10, 4, 48, 96))
    p = np.asarray(params, dtype=np.float64)
    best = math.inf
    for _ in range(2):
        t0 = time.perf_counter()
        L.forward(p, x)
        best = min(best, time.perf_counter() - t0)
    return {"value": x[0].size / best, "unit": "cells/s", "cores": 1, "kind": "oracle",
            "sample": "numpy forward (oracle/learn.py, einsum per tap, one thread) of a 96x48x4 volume, best of 2"}


def run_channel(args, world, rank, local, device, torch, cases, gbcfd):
    """Wall time to a residual drop on the steady bump channel: the plain FP64 iteration, the
    mixed path finished on the FP64 path once it stalls (hybrid), and the hybrid with the
    learned accelerator's predictions tried every 200 steps."""
    from paper_1710_09995_gb300 import learn
    case = cases.channel_case(*learn.FULL_GRID, height=0.1, mach=0.6)
    params, info = (learn.load() if os.path.exists(learn.WEIGHTS) else (None, None))
    clocks = ClockSampler(local)
    clocks.start()
    runs = {}
    runs["fp64_plain"] = learn.solve(case, args.target, None, args.max_seconds, precision="fp64", device=device)
    runs["hybrid_plain"] = learn.solve(case, args.target, None, args.max_seconds, precision="hybrid", device=device)
    if params is not None:
        runs["hybrid_learned"] = learn.solve(case, args.target, params, args.max_seconds, precision="hybrid",
                                             device=device, smooth=20, check=200)
    clk = clocks.stop()
    if rank != 0:
        return
    head = runs.get("hybrid_learned", runs["hybrid_plain"])
    for r in runs.values():
        r["history"] = [(t, s, float(f"{d:.3e}"), ph) for t, s, d, ph in r["history"]]
    out = {
        "metric": f"seconds to a {args.target:g} density-residual drop",
        "value": head["seconds"] if head["reached"] else None,
        "unit": "s",
        "n_gpus": world,
        "steps": head["steps"],
        "warmup": 0,
        "ms_per_step": 1e3 * head["seconds"] / max(1, head["steps"]),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic (analytic bump grid, free-stream start; the paper's meshes are not available)",
        "config": {"workload": WORKLOADS["channel"], "cells": case.cells, "target": args.target,
                   "accelerator": info, "parallelism": "replicas" if world > 1 else "single GPU"},
        "speedup_vs_fp64_plain": (runs["fp64_plain"]["seconds"] / head["seconds"]
                                  if head["reached"] and runs["fp64_plain"]["reached"] else None),
        "roofline": None,
        "clocks": clk,
        "runs": runs,
    }
    print(json.dumps(out))


# ---- the paper's own scheme: WCNS-E-5 ----------------------------------------------------------
WCNS_KERNELS = ("prim_kernel", "viscres_kernel", "dir_kernel<x>", "dir_kernel<y>", "dir_kernel<z>")


def wcns_kernel_bytes(precision, stage):
    """algorithmic HBM bytes per interior cell of each WCNS kernel of a stage (T = 4 mixed, 8 FP64):
    prim reads the stage input (f64 on the FP64 path; the f32 shadow and increment on the mixed
    path) and writes 6 primitive fields; viscres reads u, v, w, theta and writes the 4-field
    viscous residual; the x pass reads 5
    primitives and the viscous residual and writes R; y also reads R; z reads R and writes the
    stage output (mixed: D1 / D2, or Q^{n+1} and its shadow; FP64: Q1, Q2, Q^{n+1})"""
    t = 4 if precision == "mixed" else 8
    if precision == "mixed":
        prim_in = 20 if stage == 1 else 40
        z_io = {1: 20, 2: 40, 3: 20 + 40 + 40 + 20}[stage]
    else:
        prim_in = 40
        z_io = {1: 80, 2: 120, 3: 120}[stage]
    return {"prim_kernel": prim_in + 6 * t, "viscres_kernel": 8 * t, "dir_kernel<x>": 14 * t,
            "dir_kernel<y>": 15 * t, "dir_kernel<z>": 10 * t + z_io}


def time_wcns(gbcfd, torch, case, precision, steps, warmup, world, device):
    blk = gbcfd.wcns_block_for_case(case, precision=gbcfd.MIXED if precision == "mixed" else gbcfd.FP64,
                                    device=device)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        blk.step(1, stream)
    marks = [[torch.cuda.Event(enable_timing=True) for _ in range(18)] for _ in range(steps)]
    for ev in marks:
        for e in ev:
            e.record(stream)  # creates the events before the timed region
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    start.record(stream)
    for k in range(steps):
        blk.set_timing(marks[k], created=True)
        blk.step(1, stream)
    stop.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = max_over_ranks(start.elapsed_time(stop), world, device)
    kern = {n: 0.0 for n in WCNS_KERNELS}
    per_stage = {n: [0.0, 0.0, 0.0] for n in WCNS_KERNELS}
    for ev in marks:
        for st in range(3):
            for m, n in enumerate(WCNS_KERNELS):
                t = ev[6 * st + m].elapsed_time(ev[6 * st + m + 1])
                kern[n] += t
                per_stage[n][st] += t
    blk.set_timing(None)
    norms = blk.residual_norm()
    blk.close()
    nlaunch = 3 * (5 if case.viscous else 4) * steps
    return {"ms": ms, "kernel_ms": kern, "kernel_stage_ms": per_stage, "launches": nlaunch, "norms": norms.tolist()}


def time_wcns_split(gbcfd, torch, case, precision, steps, warmup, world, device):
    """the same case as a periodic lattice of 2 x 2 x 2 uneven WCNS blocks advanced together
    (gbcfd_wcns_step_many): the wall time of a step through the multi-block path"""
    n = case.nx
    cuts = ([n * 5 // 16, n - n * 5 // 16], [n * 11 // 16, n - n * 11 // 16], [case.nz // 2, case.nz - case.nz // 2])
    blocks = gbcfd.wcns_blocks_for_split(case, cuts, precision=gbcfd.MIXED if precision == "mixed" else gbcfd.FP64,
                                         device=device)
    stream = torch.cuda.current_stream()
    gbcfd.wcns_step_many(blocks, warmup, stream)
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    start.record(stream)
    gbcfd.wcns_step_many(blocks, steps, stream)
    stop.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = max_over_ranks(start.elapsed_time(stop), world, device)
    for b in blocks:
        b.close()
    return {"value": world * case.cells * steps / (ms / 1e3), "unit": "cell-updates/s",
            "ms_per_step": ms / steps, "steps": steps, "blocks": [list(c) for c in cuts],
            "api": "gbcfd_wcns_connect + gbcfd_wcns_step_many (8 blocks, 5-cell halos across block faces)"}


def wcns_roofline(precision, res, cells, steps, peak, peak_kind):
    """HBM roofline of the WCNS path's dominant kernel: its algorithmic bytes per launch over its
    mean launch time (CUDA events around every launch of the timed region)"""
    name = max(res["kernel_ms"], key=res["kernel_ms"].get)
    nbytes = sum(wcns_kernel_bytes(precision, st)[name] * cells * steps for st in (1, 2, 3))
    sec = res["kernel_ms"][name] / 1e3
    achieved = nbytes / sec / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_kind": peak_kind, "traffic": None,
            "algorithmic_bytes_per_launch": nbytes / (3 * steps), "kernel": name,
            "avg_launch_ms": round(res["kernel_ms"][name] / (3 * steps), 4),
            "share_of_step": round(res["kernel_ms"][name] / max(res["ms"], 1e-9), 4),
            "kernels_ms_per_step": {n: round(v / steps, 4) for n, v in res["kernel_ms"].items()},
            "dominant_ms_per_stage": [round(v / steps, 4) for v in res["kernel_stage_ms"][name]],
            "step": wcns_step_roofline(precision, res, cells, steps, peak)}


def wcns_step_roofline(precision, res, cells, steps, peak):
    """the whole WCNS step against HBM: the method's FP64-state minimum (ALGO_BYTES, 320 B per
    cell-step, as for the block path) and the bytes the path's five kernels move by design (every
    kernel of every stage, wcns_kernel_bytes) over the step's wall time"""
    sec = res["ms"] / 1e3
    algo = sum(ALGO_BYTES) * cells * steps
    design = sum(sum(wcns_kernel_bytes(precision, st).values()) for st in (1, 2, 3)) * cells * steps
    return {"achieved": round(algo / sec / 1e9, 1), "frac": round(algo / sec / 1e9 / peak, 4),
            "algorithmic_bytes_per_cell_step": sum(ALGO_BYTES),
            "design_bytes_per_cell_step": design / (cells * steps),
            "design_achieved": round(design / sec / 1e9, 1), "design_frac": round(design / sec / 1e9 / peak, 4)}


def e2e_wcns(gbcfd, torch, case, precision, steps, world, device):
    """As e2e_path, on WCNS-E-5 blocks: the value through the block calls one after the other,
    `pipelined_value` through a 3-block pipeline (gbcfd_wcns_pipe_create + gbcfd_pipe_submit / _sync)."""
    prec = gbcfd.MIXED if precision == "mixed" else gbcfd.FP64
    host_in = torch.from_numpy(case.state).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    blk = gbcfd.wcns_block_for_case(case, precision=prec, device=device)

    def one():
        blk.set_state(host_in)
        blk.step(1)
        blk.get_state(host_out)
        blk.residual_norm()

    one()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    torch.cuda.synchronize()
    serial = max_over_ranks(time.perf_counter() - t0, world, device)
    blk.close()
    members = [gbcfd.wcns_block_for_case(case, precision=prec, device=device) for _ in range(3)]
    pipe = gbcfd.Pipe(members)
    outs = [torch.empty_like(host_in).pin_memory() for _ in range(3)]
    norms = torch.zeros((max(steps, 3), 5), dtype=torch.float64).pin_memory()
    for i in range(3):
        pipe.submit(host_in, outs[i], 1, norms[i])
    pipe.sync()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(steps):
        pipe.submit(host_in, outs[i % 3], 1, norms[i])
    pipe.sync()
    dt = max_over_ranks(time.perf_counter() - t0, world, device)
    pipe.close()
    for b in members:
        b.close()
    nbytes = case.state.nbytes
    return {"value": world * case.cells * steps / serial, "unit": "cell-updates/s",
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes + 112,
            "api": "gbcfd_wcns_set_state + _step + _get_state + _residual_norm per step "
                   "(time marching: each step's state uploaded and read back)",
            "pipelined_value": world * case.cells * steps / dt,
            "pipelined_api": "gbcfd_pipe_submit x steps + gbcfd_pipe_sync (3 WCNS member blocks; steps as independent items)",
            "steps": steps}


def cpu_baseline_wcns(n):
    """The WCNS oracle (FP64) on the host cores: one SSP-RK3 step of a 256 x 256 x 8 z-slab of the
    z-invariant vortex, best of 2."""
    import oracle
    from paper_1710_09995_gb300 import cases
    nz = 8
    c = cases.isentropic_vortex(n=n, L=10.0, nz=nz, viscous=True)
    p = oracle.params(c.gamma, c.mu, c.Pr, c.cfl, c.eps, c.viscous, 0)
    best = math.inf
    for _ in range(2):
        t0 = time.perf_counter()
        oracle.wcns_step(p, c.state, c.spacing, 1)
        best = min(best, time.perf_counter() - t0)
    return {"value": c.cells / best, "unit": "cell-updates/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"1 SSP-RK3 step (FP64 WCNS-E-5 oracle) of a {n}x{n}x{nz} z-slab of the vortex, best of 2"}


def run_wcns(args, world, rank, local, device, torch, cases, gbcfd):
    case = cases.isentropic_vortex(n=args.side, L=10.0, viscous=True)
    prec = args.precision or "both"
    paths = ["mixed", "fp64"] if prec == "both" else [prec]
    peak, peak_kind = hbm_peak()
    clocks = ClockSampler(local)
    clocks.start()
    steps = {p: (args.steps if p == "mixed" else min(args.steps, 10)) for p in paths}
    results = {p: time_wcns(gbcfd, torch, case, p, steps[p], args.warmup if p == "mixed" else 1, world, device)
               for p in paths}
    split = time_wcns_split(gbcfd, torch, case, paths[0], steps[paths[0]], args.warmup, world, device)
    clk = clocks.stop()
    head = paths[0]
    e2e = e2e_wcns(gbcfd, torch, case, head, args.e2e_steps or 20, world, device)
    cpu = cpu_baseline_wcns(args.side) if rank == 0 and world == 1 and not args.no_cpu_baseline else None
    if rank != 0:
        return
    r = results[head]
    out = {
        "metric": "cell-updates/s", "value": world * case.cells * steps[head] / (r["ms"] / 1e3),
        "unit": "cell-updates/s", "n_gpus": world, "steps": steps[head], "warmup": args.warmup,
        "ms_per_step": r["ms"] / steps[head], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if head == "mixed" else "f64",
        "data": "synthetic (seeded closed-form vortex; the paper's meshes are not available)",
        "config": {"workload": WORKLOADS["wcns256"], "cells": case.cells, "precision": head,
                   "l2": "working set > 1.4 GB >> 129 MB L2, no flush needed",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": wcns_roofline(head, r, case.cells, steps[head], peak, peak_kind),
        "e2e": e2e, "gpu_launches": r["launches"], "clocks": clk, "cpu_baseline": cpu,
        "residual_norm": r["norms"], "multiblock_2x2x2": split,
    }
    for p in paths[1:]:
        rp = results[p]
        out[p] = {"value": world * case.cells * steps[p] / (rp["ms"] / 1e3), "unit": "cell-updates/s",
                  "steps": steps[p], "ms_per_step": rp["ms"] / steps[p], "dtype": "f64",
                  "roofline": wcns_roofline(p, rp, case.cells, steps[p], peak, peak_kind),
                  "gpu_launches": rp["launches"]}
    print(json.dumps(out))


# ---- the reference arm: the FP64 CPU oracle ----------------------------------------------------
def reference_sample(args):
    """The oracle's bounded sample of the workload: (cells, one-step function, initial state,
    sample text, metric, unit).  Every sample has the workload's recipe and physics on fewer cells."""
    import oracle
    from paper_1710_09995_gb300 import cases
    w = args.workload
    cu = ("cell-updates/s", "cell-updates/s")
    if w in ("vortex256", "wcns256"):
        nz = 8
        c = cases.isentropic_vortex(n=args.side, L=10.0, nz=nz, viscous=True)
        p = oracle.params(c.gamma, c.mu, c.Pr, c.cfl, c.eps, c.viscous, c.limiter)
        scheme = "WCNS-E-5 oracle" if w == "wcns256" else "FP64 oracle"
        text = (f"each step: 1 SSP-RK3 step ({scheme}) of a {args.side}x{args.side}x{nz} z-slab of the "
                f"z-invariant {args.side}^3 vortex")
        if w == "wcns256":
            return c.cells, (lambda Q: oracle.wcns_step(p, Q, c.spacing, 1)[0]), c.state, text, *cu
        M = oracle.metrics(c.grid_nodes())
        return c.cells, (lambda Q: oracle.step(p, Q, M, 1)[0]), oracle.pad(c.state), text, *cu
    if w == "warped512":
        c = cases.broadband_warped(128, 128, 96, seed=0)
        p = oracle.params(c.gamma, c.mu, c.Pr, c.cfl, c.eps, c.viscous, c.limiter)
        M = oracle.metrics(c.nodes)
        text = "each step: 1 SSP-RK3 step (FP64 oracle) of a periodic 128x128x96 warped block, same recipe"
        return c.cells, (lambda Q: oracle.step(p, Q, M, 1)[0]), oracle.pad(c.state), text, *cu
    if w == "lattice96":
        lat = cases.lattice_case(sizes=([128], [128], [96]), seed=4)
        p = oracle.params(lat.gamma, 0.0, 0.72, lat.cfl, lat.eps, False, 0)
        M = oracle.metrics(cases.cartesian_nodes(128, 128, 96, *lat.spacing))
        text = "each step: 1 SSP-RK3 step (FP64 oracle, Euler) of a periodic 128x128x96 block, same recipe"
        return lat.cells, (lambda Q: oracle.step(p, Q, M, 1)[0]), oracle.pad(lat.state.numpy()), text, *cu
    if w == "channel":
        # z-invariant flow: a z-slab of the grid is the same problem; the plain FP64 iteration's
        # rate (its seconds to the drop are ~80,000 such steps of the full grid: no bounded run)
        c = cases.channel_case(nz=8)
        p = oracle.params(c.gamma, c.mu, c.Pr, c.cfl, c.eps, c.viscous, c.limiter)
        bcs = oracle.bc(c.extra["bc"], c.extra["inf"])
        M = oracle.metrics_bc(c.nodes, bcs)
        text = ("each step: 1 SSP-RK3 step (FP64 oracle, local time steps, wall and far-field ghost cells) "
                "of a 192x96x8 z-slab of the bump channel; the GPU arm's metric for this workload is "
                "seconds to the 1e-6 drop, which the oracle cannot reach in a bounded run")
        return c.cells, (lambda Q: oracle.step_ex(p, Q, M, 1, bcs, local_dt=True)[0]), oracle.pad(c.state), text, *cu
    if w == "accel":
        import numpy as np
        from oracle import learn as L
        r = np.random.Generator(np.random.PCG64(0))
        x = r.standard_normal((10, 4, 48, 96))
        params = r.standard_normal(L.n_params()) * 0.05
        text = "each step: numpy forward of the network (oracle/learn.py, FP64) on a 96x48x4 volume"
        return 96 * 48 * 4, (lambda X: (L.forward(params, X), X)[1]), x, text, "cell inferences/s", "cells/s"
    raise ValueError(f"no oracle sample for workload {w}")


def run_reference(args):
    """The reference arm: the FP64 CPU oracle as it stands, on the host cores, on a bounded sample
    of the workload per step; rank 0 alone runs and prints."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    cells, step, Q, sample, metric, unit = reference_sample(args)
    for _ in range(args.warmup):
        Q = step(Q)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        Q = step(Q)
    sec = time.perf_counter() - t0
    value = cells * args.steps / sec
    out = {"impl": "reference", "metric": metric, "value": value, "unit": unit,
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOADS[args.workload], "cells": cells, "precision": "fp64"},
           "cpu_baseline": {"value": value, "unit": unit, "cores": oracle.threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_gbcfd(a)
