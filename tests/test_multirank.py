"""bench.py's multi-process plumbing on CPU with gloo, world size 2: the rendezvous, barrier and
max-over-ranks timing of independent replicas, and the reference arm printing one line from
rank 0 only."""
import json
import os
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def torchrun(script_args, port, timeout=300):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port)] + script_args
    env = dict(os.environ, OMP_NUM_THREADS="1")
    return subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=timeout, env=env)


def test_max_over_ranks_and_barrier_gloo(tmp_path):
    script = tmp_path / "ranks.py"
    script.write_text(textwrap.dedent(f"""
        import sys, torch
        sys.path.insert(0, {ROOT!r})
        import bench
        world, rank, local = bench.dist_env()
        assert world == 2
        bench.dist_init(world, "gloo")
        bench.barrier(world)
        t = bench.max_over_ranks(1.5 + rank, world, torch.device("cpu"))
        assert t == 2.5, t
        bench.barrier(world)
        print(f"rank {{rank}} ok {{t}}", flush=True)
    """))
    r = torchrun([str(script)], 29611)
    assert r.returncode == 0, r.stderr[-3000:]
    assert r.stdout.count("ok 2.5") == 2


def test_reference_arm_prints_one_line_from_rank0():
    r = torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--side", "64"],
                 29612)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["cpu_baseline"]["kind"] == "oracle"


def test_reference_arm_wcns_workload():
    r = torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--side", "32",
                  "--workload", "wcns256"], 29613)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert "WCNS" in out["cpu_baseline"]["sample"] and out["value"] > 0
