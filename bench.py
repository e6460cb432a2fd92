#!/usr/bin/env python3
"""Benchmark of the map-refinement hot path: LiDAR pixels per second for forward + loss +
backward + Adam over a set of keyframes sharing one map, batched (one fused pass over all
keyframes in one CUDA graph) against plain (one launch sequence per keyframe).

Default workload: 12 keyframes of uneven shapes (4x 64x1024, 4x 128x1024, 4x 32x1800) along a
50 m synthetic street trajectory, one map of 500,000 2D Gaussians (seeded synthetic data).
A step is one refinement iteration over all 12 keyframes.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun (N > 1) every rank runs an independent replica of
the workload (weak scaling) and the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LiDAR px/s fwd+bwd (batched vs plain) at depth err ≤1e-3 m vs FP64 oracle"
UNIT = "px/s"
# one FP32 ALU op per lane per clock; ops per Gaussian-pixel evaluation of the forward compositing
# kernel and of the backward adjoint kernel (the per-unit figures of the design)
OPS_PER_EVAL = {"render_fwd": 48.0, "render_bwd": 150.0}
FP32_LANES_PER_SM = 128


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", type=int, default=3)
    p.add_argument("--n-gaussians", type=int, default=None,
                   help="override the workload's primitive count (smaller profiling cases)")
    p.add_argument("--keyframes", type=int, default=None,
                   help="use only the first K keyframes of the workload")
    p.add_argument("--tile", default="auto", help="auto | 16x16 | 8x32 | 32x8 | 4x64")
    p.add_argument("--plain-steps", type=int, default=10)
    p.add_argument("--e2e-steps", type=int, default=50)
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-flush", action="store_true")
    return p.parse_args()


# ----------------------------------------------------------------------------------------------
# distributed plumbing (replicas): rank info, barrier, max over ranks
# ----------------------------------------------------------------------------------------------

def dist_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def dist_init(backend):
    import torch.distributed as dist
    rank, world, _ = dist_info()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend, rank=rank, world_size=world)
    return dist if world > 1 else None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value: float, device="cpu") -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value: float, device="cpu") -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------------------------

CLOCK_FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw",
                "clocks_event_reasons.active", "clocks_event_reasons.hw_slowdown",
                "clocks_event_reasons.hw_thermal_slowdown",
                "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]


class ClockSampler:
    def __init__(self, gpu_id: str | None, period_ms=50):
        self.proc = None
        cmd = ["nvidia-smi", "--query-gpu=" + ",".join(CLOCK_FIELDS),
               "--format=csv,noheader,nounits", "-lms", str(period_ms)]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < len(CLOCK_FIELDS):
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "samples": len(sm), "power_w_max": max(power) if power else None,
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------------------------
# workload
# ----------------------------------------------------------------------------------------------

def build_workload(index, n=None, keyframes=None):
    from paper_2503_17491_gb300 import scenes
    s = scenes.workload(index, n=n)
    views = s.views
    if index == 4:
        views = views[:8]   # the 8 most recent keyframes of the long run's first window
    if keyframes:
        views = views[:keyframes]
    targets = [scenes.render_targets(s, v) for v in views]
    desc = scenes.WORKLOADS[index]
    if n or keyframes:
        desc += f" [reduced: {s.n} primitives, {len(views)} keyframes]"
    return s, views, targets, desc


TRAFFIC_MD = os.path.join(ROOT, "profiles", "render_dram_traffic_12kf_500k.md")


def csrc_digest():
    """sha256 over the library's CUDA sources (names and contents, in name order), 16 hex digits."""
    import glob
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2503_17491_gb300", "csrc")
    files = glob.glob(os.path.join(d, "*.cu")) + glob.glob(os.path.join(d, "*.cuh"))
    for f in sorted(files, key=os.path.basename):
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, tile):
    """DRAM read+write bytes per launch of `kernel` at `tile`, from the committed ncu summary of
    the full workload -- only while the library sources are the ones it was captured from."""
    try:
        with open(TRAFFIC_MD) as f:
            text = f.read()
    except OSError:
        return None
    m = re.search(r"first 16 hex digits\): `([0-9a-f]{16})`", text)
    if not m or m.group(1) != csrc_digest():
        return None
    row = re.search(r"\| `k_%s` \| %s \| (\d+) \| (\d+) \| (\d+) \|" % (kernel, tile), text)
    return int(row.group(3)) if row else None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {"sm_max_mhz": 2070.0}, "fallback"


def cpu_baseline(scene, views, targets, budget_s, seed=0):
    """The FP64 oracle on the host cores: forward + loss + backward of a pixel sample of one
    keyframe (culled mode, per-tile lists built before timing).  Returns a cpu_baseline dict."""
    import oracle
    oracle.build()
    vi = 1 if len(views) > 1 else 0
    v = views[vi]
    t0 = time.perf_counter()
    proj = oracle.project_contract(scene.pos_logit, scene.quat, scene.log_scale, v.T_ws, v.rows,
                                   v.cols, v.elev_min, v.elev_max)
    keys, ids = oracle.bin_pairs(proj, v.rows, v.cols)
    cul = oracle.Culled(keys, ids, v.rows, v.cols, 16, 16)
    t_bin = time.perf_counter() - t0
    params = oracle.split_params(scene.pos_logit, scene.quat, scene.log_scale)
    rng = np.random.default_rng(seed)
    dt, nt = targets[vi]

    def run(k):
        px = np.stack([rng.integers(0, v.rows, k), rng.integers(0, v.cols, k)], 1)
        t = time.perf_counter()
        out = oracle.render(params, proj["flip"], None, v.T_ws, v.rows, v.cols, v.elev_min,
                            v.elev_max, culled=cul, pixels=px)
        L, gD, gN, gO = oracle.loss(out["D"], out["N"], out["O"], dt[px[:, 0], px[:, 1]],
                                    nt[:, px[:, 0], px[:, 1]])
        oracle.render_backward(params, proj["flip"], None, v.T_ws, v.rows, v.cols, v.elev_min,
                               v.elev_max, gD, gN, gO, culled=cul, pixels=px)
        return time.perf_counter() - t

    # grow the sample until it takes about the budget (a small run is dominated by fixed costs)
    k, t = 256, run(256)
    while t < 0.5 * budget_s and k < (1 << 22):
        k = int(min(1 << 22, max(2 * k, 0.9 * k * budget_s / max(t, 1e-6))))
        t = run(k)
    return {"value": k / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"FP64 oracle forward + loss + backward of {k} random pixels of keyframe "
                       f"{vi} ({v.rows}x{v.cols}) of the same workload, culled mode, OpenMP on all "
                       f"host cores; per-tile binning of that keyframe ({t_bin:.2f} s) excluded"),
            "seconds": t}


# ----------------------------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------------------------

def run_ours(args):
    import torch
    from paper_2503_17491_gb300 import api
    from paper_2503_17491_gb300 import build as libbuild

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dist = dist_init("nccl")
    dev = torch.device("cuda", local)
    libbuild.build()

    scene, views, targets_np, desc = build_workload(args.workload, args.n_gaussians,
                                                    args.keyframes)
    pixels = sum(v.rows * v.cols for v in views)
    params0 = [torch.from_numpy(a).to(dev) for a in (scene.pos_logit, scene.quat,
                                                      scene.log_scale)]
    targets = [(torch.from_numpy(d).to(dev), torch.from_numpy(n).to(dev)) for d, n in targets_np]
    max_pairs = api.default_capacity_pairs(scene.n, views)

    # tile shape: autotuned on this workload unless given
    if args.tile == "auto":
        tile, tune = api.autotune_tile(params0, views, targets, max_pairs=max_pairs)
    else:
        tile = tuple(int(x) for x in args.tile.split("x"))
        tune = None
    cfg = api.RenderConfig(tile_h=tile[0], tile_w=tile[1])

    flush_buf = torch.empty(256 << 20, dtype=torch.float32, device=dev)   # 1 GiB > L2

    def flush():
        if not args.no_flush:
            flush_buf.fill_(1.0)

    def timed(step_fn, K):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(K)]
        barrier(dist)
        torch.cuda.synchronize()
        for i in range(K):
            flush()
            evs[i][0].record()
            step_fn()
            evs[i][1].record()
        torch.cuda.synchronize()
        barrier(dist)
        return [a.elapsed_time(b) for a, b in evs]

    # ---- batched: one fused pass over all keyframes, captured in a CUDA graph ---------------
    params = [p.clone() for p in params0]
    ref = api.Refiner(params, views, targets, mode="batched", cfg=cfg, max_pairs=max_pairs)
    ref.step()                                  # eager step: kernel count, status
    torch.cuda.synchronize()
    launches_before = ref.ctx.stats()["kernel_launches"]
    ref.step()
    torch.cuda.synchronize()
    st = ref.ctx.stats()
    launches_per_step = st["kernel_launches"] - launches_before
    status = ref.ctx.status()
    ref.capture(warmup=1)
    for _ in range(args.warmup):
        ref.step()
    torch.cuda.synchronize()
    gpu_uuid = None
    try:
        gpu_uuid = str(torch.cuda.get_device_properties(dev).uuid)
        if not gpu_uuid.startswith("GPU-"):
            gpu_uuid = "GPU-" + gpu_uuid
    except Exception:
        gpu_uuid = None
    sampler = ClockSampler(gpu_uuid)
    t_batched = timed(ref.step, args.steps)
    clocks = sampler.stop()
    ms_batched = sum(t_batched) / len(t_batched)
    ms_max = max_over_ranks(dist, sum(t_batched), dev) / len(t_batched)
    loss_last = float(ref.loss_out)

    # ---- per-kernel times (library events around the two compositing kernels) ----------------
    prof_params = [p.clone() for p in params0]
    pref = api.Refiner(prof_params, views, targets, mode="batched", cfg=cfg, max_pairs=max_pairs)
    pref.ctx.set_profiling(True)
    fwd_ms, bwd_ms, fev, bev, stage_ms = [], [], [], [], []
    for i in range(max(3, min(args.steps, 10)) + 1):
        flush()
        pref.step()
        f, b = pref.ctx.kernel_times()
        s2 = pref.ctx.stats()
        if i == 0:
            continue
        fwd_ms.append(f)
        bwd_ms.append(b)
        fev.append(s2["fwd_evals"])
        bev.append(s2["bwd_evals"])
        stage_ms.append(pref.ctx.stage_times())
    kern = {"render_fwd": (statistics.mean(fwd_ms), statistics.mean(fev)),
            "render_bwd": (statistics.mean(bwd_ms), statistics.mean(bev))}
    dom = max(kern, key=lambda k: kern[k][0])
    peaks, peak_src = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    peak_tops = sms * FP32_LANES_PER_SM * f_max / 1e12
    k_ms, k_ev = kern[dom]
    achieved = k_ev * OPS_PER_EVAL[dom] / (k_ms * 1e-3) / 1e12
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak_tops,
                "unit": "TFLOP/s", "frac": achieved / peak_tops,
                # the committed capture covers the default workload only
                "traffic": (recorded_traffic(dom, f"{tile[0]}x{tile[1]}")
                            if args.workload == 3 and args.n_gaussians is None
                            and args.keyframes is None else None),
                "peak_source": (f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {f_max / 1e6:.0f} "
                                f"MHz ({peak_src} max SM clock), one op per lane per clock"),
                "ops_per_eval": OPS_PER_EVAL[dom], "evals_per_launch": k_ev,
                "launch_ms": k_ms,
                "other_kernel": {k: {"launch_ms": v[0], "evals": v[1]} for k, v in kern.items()
                                 if k != dom}}

    # per-stage times of the same eager steps against the HBM roofline, with each stage's
    # algorithmic bytes (what its definition reads and writes once): n primitives, V keyframes,
    # nv (view, primitive) pairs that touch a tile, M list entries, T tiles, P pixels
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    n, V, nv, M, T = scene.n, len(views), s2["n_touching"], s2["n_pairs"], s2["n_tiles"]
    passes = (max(int(T - 1).bit_length(), 1) + 7) // 8
    stage_bytes = {"projection": 40 * n + 40 * n * V,
                   "range sort": 12 * n * V + 84 * nv,
                   "emission": 20 * nv + 8 * M,
                   "tile sort": 20 * passes * M,
                   "tile ranges": 21 * M + 20 * T,
                   "loss": 52 * pixels,
                   "fused Adam": 304 * n}
    stages = {}
    for name, nbytes in stage_bytes.items():
        vals = [x[name] for x in stage_ms if x.get(name) is not None]
        if not vals:
            continue
        ms = statistics.mean(vals)
        stages[name] = {"ms": ms, "bytes": nbytes, "gbs": nbytes / (ms * 1e-3) / 1e9,
                        "frac": nbytes / (ms * 1e-3) / 1e9 / hbm}

    # ---- plain: one launch sequence per keyframe, no graph ------------------------------------
    plain = None
    if args.plain_steps > 0:
        pparams = [p.clone() for p in params0]
        pl = api.Refiner(pparams, views, targets, mode="plain", cfg=cfg, max_pairs=max_pairs)
        for _ in range(2):
            pl.step()
        t_plain = timed(pl.step, args.plain_steps)
        ms_plain = sum(t_plain) / len(t_plain)
        ms_plain = max_over_ranks(dist, sum(t_plain), dev) / len(t_plain)
        plain = {"value": world * pixels / (ms_plain * 1e-3), "ms_per_step": ms_plain,
                 "steps": args.plain_steps,
                 "note": "one render/loss/backward launch sequence per keyframe, then Adam; "
                         "no CUDA graph"}

    # ---- end to end: host targets in, loss out, through the public API ----------------------
    e2e = None
    if args.e2e_steps > 0:
        host_d = torch.cat([t[0].reshape(-1) for t in targets]).cpu().pin_memory()
        host_n = torch.cat([t[1].reshape(3, -1) for t in targets], 1).cpu().pin_memory()
        host_loss = torch.zeros(1, dtype=torch.float64).pin_memory()

        def e2e_step():
            ref.t_depth.copy_(host_d, non_blocking=True)
            ref.t_normal.copy_(host_n, non_blocking=True)
            ref.step()
            host_loss.copy_(ref.loss_out, non_blocking=True)

        t_e2e = timed(e2e_step, args.e2e_steps)
        ms_e2e = max_over_ranks(dist, sum(t_e2e), dev) / len(t_e2e)
        e2e = {"value": world * pixels / (ms_e2e * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": host_d.numel() * 4 + host_n.numel() * 4,
               "d2h_bytes_per_step": 8, "ms_per_step": ms_e2e,
               "path": "pinned host targets -> splat_refine_step (graph) -> loss to pinned host"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(scene, views, targets_np, args.cpu_seconds)

    if rank != 0:
        return None
    evals_step = st["fwd_evals"] + st["bwd_evals"]
    line = {
        "metric": METRIC, "value": world * pixels / (ms_max * 1e-3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": desc, "n_gaussians": scene.n, "keyframes": len(views),
                   "pixels_per_step": pixels, "tile": f"{tile[0]}x{tile[1]}",
                   "step": "render + loss + backward + Adam over all keyframes",
                   "mode": "batched: one fused pass, one CUDA graph per step",
                   "l2": "flushed between timed steps (1 GiB write)" if not args.no_flush
                   else "not flushed",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "pairs_per_step": st["n_pairs"]},
        "plain": plain,
        "batched_over_plain": (plain["ms_per_step"] / ms_max) if plain else None,
        "gaussian_pixel_evals_per_s": world * evals_step / (ms_max * 1e-3),
        "roofline": roofline,
        "stages": {"unit": "GB/s against the measured HBM copy bandwidth (algorithmic bytes; "
                           "the compositing kernels are in roofline)", **stages},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "status": status,
        "loss": loss_last,
        "autotune": tune,
    }
    return line


# ----------------------------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ----------------------------------------------------------------------------------------------

def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return None
    scene, views, targets_np, desc = build_workload(args.workload, args.n_gaussians,
                                                    args.keyframes)
    K, W = args.steps, args.warmup
    budget = 150.0
    per_step = max(0.05, budget / max(K + W, 1))
    import oracle
    oracle.build()
    vi = 1 if len(views) > 1 else 0
    v = views[vi]
    proj = oracle.project_contract(scene.pos_logit, scene.quat, scene.log_scale, v.T_ws, v.rows,
                                   v.cols, v.elev_min, v.elev_max)
    keys, ids = oracle.bin_pairs(proj, v.rows, v.cols)
    cul = oracle.Culled(keys, ids, v.rows, v.cols, 16, 16)
    params = oracle.split_params(scene.pos_logit, scene.quat, scene.log_scale)
    dt, nt = targets_np[vi]
    rng = np.random.default_rng(0)

    def step(k):
        px = np.stack([rng.integers(0, v.rows, k), rng.integers(0, v.cols, k)], 1)
        t = time.perf_counter()
        out = oracle.render(params, proj["flip"], None, v.T_ws, v.rows, v.cols, v.elev_min,
                            v.elev_max, culled=cul, pixels=px)
        L, gD, gN, gO = oracle.loss(out["D"], out["N"], out["O"], dt[px[:, 0], px[:, 1]],
                                    nt[:, px[:, 0], px[:, 1]])
        oracle.render_backward(params, proj["flip"], None, v.T_ws, v.rows, v.cols, v.elev_min,
                               v.elev_max, gD, gN, gO, culled=cul, pixels=px)
        return time.perf_counter() - t

    # size the per-step sample so that one step takes about per_step (a small sample is
    # dominated by per-call fixed costs, so the size is grown geometrically)
    k, t = 128, step(128)
    while t < 0.5 * per_step and k < (1 << 22):
        k = int(min(1 << 22, max(2 * k, 0.9 * k * per_step / max(t, 1e-6))))
        t = step(k)
    for _ in range(W):
        step(k)
    total = sum(step(k) for _ in range(K))
    value = K * k / total
    sample = (f"per step: FP64 oracle forward + loss + backward of {k} random pixels of keyframe "
              f"{vi} ({v.rows}x{v.cols}), culled mode; binning built once before timing")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": K, "warmup": W, "ms_per_step": 1e3 * total / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "n_gaussians": scene.n, "keyframes": len(views),
                       "pixels_per_step": sum(x.rows * x.cols for x in views),
                       "step": "render + loss + backward + Adam over all keyframes",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "cpu_baseline": {"kind": "oracle", "cores": os.cpu_count(), "sample": sample,
                             "value": value, "unit": UNIT},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    line = run_reference(args) if args.impl == "reference" else run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
