"""Training and use of the learned convergence accelerator (orchestration over the C ABI; every
step of the solver, the features, the network and the optimiser runs in the library's kernels).

Data: seeded solver trajectories of the bump channel (bump height 5-15%, Mach 0.4-0.7) on a
thin copy of its grid (the flow is invariant along the periodic z direction), run from the free
stream with local pseudo-time steps on the mixed path.  At geometrically spaced steps the
features of the state are stored together with the target, the state change over the next
K = 20 steps.  Training: Adam on random batches of whole snapshots.  Use: plain steps
interleaved with predictions, each kept only if the density residual drops; the mixed path runs
until its FP32 floor, then the FP64 path finishes to the requested drop (or the plain FP64
iteration alone, for comparison).
"""
import argparse
import json
import math
import os
import time

import numpy as np
import torch

from . import cases, gbcfd

K = 20
SNAPSHOTS = (0, 20, 60, 140, 300, 600, 1000, 1600, 2500, 4000, 6000, 9000, 13000, 18000, 25000, 33000)
TRAIN_GRID = (192, 96, 4)
FULL_GRID = (192, 96, 64)
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "accel_bump_channel.npz")


def draw_cases(n, seed=0):
    """n (bump height, Mach) pairs, uniform in [0.05, 0.15] x [0.4, 0.7] (seeded)"""
    r = np.random.Generator(np.random.PCG64(seed))
    return [(float(h), float(m)) for h, m in zip(r.uniform(0.05, 0.15, n), r.uniform(0.4, 0.7, n))]


def channel(grid, height, mach, precision, device=None):
    c = cases.channel_case(*grid, height=height, mach=mach)
    return c, gbcfd.block_for_case(c, precision=precision, device=device)


def generate(n_traj=200, seed=0, grid=TRAIN_GRID, snapshots=SNAPSHOTS, device=None, log=None):
    """features X (bf16 [N][cells][16]) and targets T (f32 [N][cells][8]) on the device"""
    nx, ny, nz = grid
    cells = nx * ny * nz
    n = n_traj * len(snapshots)
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    X = torch.empty((n, cells, 16), dtype=torch.bfloat16, device=dev)
    T = torch.empty((n, cells, 8), dtype=torch.float32, device=dev)
    acc = gbcfd.Accel(nx, ny, nz, 1, device=dev)
    meta = []
    i = 0
    t0 = time.perf_counter()
    for traj, (h, m) in enumerate(draw_cases(n_traj, seed)):
        _, blk = channel(grid, h, m, gbcfd.MIXED, dev)
        g = gbcfd.Group([blk])
        done = 0
        for s in snapshots:
            if s > done:
                g.step(s - done)
                done = s
            acc.features(blk, X[i])
            g.step(K)
            done += K
            acc.target(blk, T[i])
            meta.append({"traj": traj, "height": h, "mach": m, "step": s})
            i += 1
        g.close()
        blk.close()
        if log and (traj + 1) % 20 == 0:
            log(f"trajectories {traj + 1}/{n_traj}, {time.perf_counter() - t0:.1f} s")
    torch.cuda.synchronize()
    return X, T, meta


def init_params(seed=0):
    """He-style initial weights (fan-in 27 x channels), zero biases, last layer scaled down"""
    r = np.random.Generator(np.random.PCG64(seed))
    chans = (10, 32, 32, 5)
    out = []
    for li, (ci, co) in enumerate(zip(chans[:-1], chans[1:])):
        std = math.sqrt(2.0 / (ci * 27)) * (0.1 if li == 2 else 1.0)
        out.append(r.standard_normal(co * ci * 27) * std)
        out.append(np.zeros(co))
    return np.concatenate(out).astype(np.float32)


def train(X, T, iters=3000, batch=4, lr=2e-3, seed=0, grid=TRAIN_GRID, log=None, params=None):
    """Adam with a cosine learning-rate decay; returns (parameters, loss history)"""
    nx, ny, nz = grid
    acc = gbcfd.Accel(nx, ny, nz, batch, device=X.device)
    acc.set_params(init_params(seed) if params is None else params)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    n = X.shape[0]
    losses = []
    for it in range(iters):
        idx = torch.randint(0, n, (batch,), generator=gen).to(X.device)
        xb = X.index_select(0, idx).reshape(-1, 16)
        tb = T.index_select(0, idx).reshape(-1, 8)
        rate = lr * 0.5 * (1.0 + math.cos(math.pi * it / iters))
        losses.append(acc.train_step(xb, tb, rate))
        if log and (it + 1) % 500 == 0:
            log(f"iteration {it + 1}/{iters}, loss {np.mean(losses[-100:]):.4g}")
    return acc.get_params(), losses


def save(path, params, info):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez(path, params=params, info=json.dumps(info))


def load(path=WEIGHTS):
    d = np.load(path)
    return d["params"].astype(np.float32), json.loads(str(d["info"]))


# ---- solving to a residual drop ------------------------------------------------------------------

def _norm(blk):
    return float(blk.residual_norm()[0])


def solve(case, target=1e-6, accel_params=None, max_seconds=900.0, check=200, stall_checks=50,
          precision="hybrid", device=None, log=None, smooth=0, alpha=0.5, alpha_min=0.125, alpha_max=1.0):
    """Pseudo-time iteration of a steady case to RMS(R_rho) <= target x its initial value.

    precision: "fp64" (the plain FP64 iteration), "mixed" (mixed path only; it stalls where the
    Runge-Kutta increments fall below the FP32 resolution of the state, around 1e-5 on the bump
    channel) or "hybrid" (mixed until the density residual has not improved by 10% over
    `stall_checks` checks, or has reached the target, then the FP64 path from that state until the
    FP64 residual confirms the target).  Below its floor the mixed
    iteration still converges the smooth part of the solution (its residual norm is FP32 noise
    there), so a late switch leaves the FP64 path little more than that noise to remove.
    accel_params: network parameters; when given, every `check` steps a prediction is tried (in the
    mixed phase of a hybrid solve; its FP64 finish runs the plain iteration).
    smooth = 0: the bare test (gbcfd_accel_try: kept only if the residual of the predicted state is
    lower; a kept one is followed by another try).  smooth = m > 0: the prediction scaled by alpha
    is followed by m plain steps and kept only if the residual then lies below min(1, rate^m) times
    its value before, rate the plain iteration's per-step factor over the last `check` steps
    (gbcfd_accel_try_smooth); alpha grows (x1.5, up to alpha_max <= 4: beyond 1 the prediction is
    extrapolated along its own direction) after a kept try and halves (down to alpha_min) after a
    rejected one.
    Returns a dict with the wall time, steps, predictions tried/kept and the history."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    prec = gbcfd.FP64 if precision == "fp64" else gbcfd.MIXED
    blk = gbcfd.block_for_case(case, precision=prec, device=dev)
    acc = None
    if accel_params is not None:
        acc = gbcfd.Accel(case.nx, case.ny, case.nz, 1, device=dev)
        acc.set_params(accel_params)
    g = gbcfd.Group([blk])
    g.tune()  # grid split for this block (the timed region starts after it)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.step(1)
    r0 = _norm(blk)
    steps, tried, kept = 1, 0, 0
    hist = [(0.0, 1, 1.0, "fp64" if prec == gbcfd.FP64 else "mixed")]
    best, since = 1.0, 0
    phase = "fp64" if prec == gbcfd.FP64 else "mixed"
    r = 1.0
    r_prev = 1.0
    while True:
        g.step(check)
        steps += check
        r = _norm(blk) / r0
        r_plain = r  # the stall test watches the plain steps' norm, not a kept try's fresh residual
        try_now = acc is not None and (precision != "hybrid" or phase == "mixed")  # the FP64 finish runs plain
        if try_now and smooth > 0:
            rate = (r / r_prev) ** (1.0 / check) if r_prev > 0 and r > 0 else 1.0
            ok, _, r1 = acc.try_smooth(blk, alpha, smooth, min(1.0, rate ** smooth))
            tried += 1
            if ok:
                kept += 1
                steps += smooth
                r = r1 / r0
                alpha = min(alpha_max, 1.5 * alpha)
            else:
                alpha = max(alpha_min, 0.5 * alpha)
        elif try_now:
            while True:
                ok, _, r1 = acc.try_update(blk)
                tried += 1
                if not ok:
                    break
                kept += 1
                r = r1 / r0
                if r <= target:
                    break
        r_prev = r
        el = time.perf_counter() - t0
        hist.append((round(el, 3), steps, r, phase))
        if log and len(hist) % 50 == 0:
            log(f"{phase} {steps} steps {el:.1f} s drop {r:.3e} kept {kept}/{tried}")
        # a hybrid solve is done only when the FP64 path confirms the drop: reaching it on the mixed
        # path's FP32 residual switches to the FP64 path like a stall does
        mixed_phase = precision == "hybrid" and phase == "mixed"
        if (r <= target and not mixed_phase) or el > max_seconds or not math.isfinite(r):
            break
        if r_plain < 0.9 * best:
            best, since = r_plain, 0
        else:
            since += 1
        if mixed_phase and (since >= stall_checks or r <= target):
            q = blk.get_state()
            g.close()
            blk.close()
            blk = gbcfd.block_for_case(case, precision=gbcfd.FP64, device=dev)
            blk.set_state(q)
            g = gbcfd.Group([blk])
            g.tune()
            phase, best, since = "fp64", r, 0
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    out = {"seconds": el, "steps": steps, "drop": r, "reached": bool(r <= target), "tried": tried, "kept": kept,
           "precision": precision, "accelerated": acc is not None, "smooth": smooth,
           "history": hist[:: max(1, len(hist) // 60)]}
    g.close()
    blk.close()
    return out


def main():
    ap = argparse.ArgumentParser(description="train the learned accelerator on bump-channel trajectories")
    ap.add_argument("--trajectories", type=int, default=200)
    ap.add_argument("--iters", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=WEIGHTS)
    a = ap.parse_args()
    gbcfd.lib()
    log = lambda s: print(s, flush=True)
    t0 = time.perf_counter()
    X, T, meta = generate(a.trajectories, a.seed, log=log)
    tg = time.perf_counter() - t0
    params, losses = train(X, T, a.iters, a.batch, a.lr, a.seed, log=log)
    info = {"trajectories": a.trajectories, "snapshots": list(SNAPSHOTS), "grid": list(TRAIN_GRID), "iters": a.iters,
            "batch": a.batch, "lr": a.lr, "seed": a.seed, "generate_seconds": round(tg, 1),
            "train_seconds": round(time.perf_counter() - t0 - tg, 1),
            "loss_first_100": float(np.mean(losses[:100])), "loss_last_100": float(np.mean(losses[-100:]))}
    save(a.out, params, info)
    print(json.dumps(info))


if __name__ == "__main__":
    main()
