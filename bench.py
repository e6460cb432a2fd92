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
    p.add_argument("--next-rows", action="store_true",
                   help="time the kernels of the next rows (loss modes, map growth, photometric "
                        "normal equations, back-projection) instead; one JSON line per kernel")
    p.add_argument("--next-rows-reps", type=int, default=30)
    p.add_argument("--scan-stride", type=int, default=10,
                   help="workload 4: time every S-th scan of the mapping run")
    p.add_argument("--next-rows-new", type=int, default=50_000)
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


def cpu_baseline(params_np, views, targets, budget_s, images=None, offsets=None, seed=0,
                 acc_pixels=1024):
    """The FP64 oracle on the host cores.

    Timing: forward + loss + backward of a pixel sample of one keyframe (culled mode, per-tile
    lists built before timing), grown until it takes about budget_s.  Returns a cpu_baseline
    dict.

    Accuracy of the measured run: with images = the GPU's packed (depth, normal, alpha) of the
    parameters params_np (the measured run's final state) and offsets the views' first pixels,
    the oracle also composites acc_pixels random pixels of every keyframe from the same
    parameters, and the dict gains "accuracy": max |dD| (blended range <= 100 m), max |dO|, max
    1 - cos(N) over the pixels outside the ambiguity band, and the band count."""
    import oracle
    oracle.build()
    pos_logit, quat, log_scale = params_np
    params = oracle.split_params(pos_logit, quat, log_scale)
    rng = np.random.default_rng(seed)

    def binned(v):
        proj = oracle.project_contract(pos_logit, quat, log_scale, v.T_ws, v.rows, v.cols,
                                       v.elev_min, v.elev_max)
        keys, ids = oracle.bin_pairs(proj, v.rows, v.cols)
        return proj, oracle.Culled(keys, ids, v.rows, v.cols, 16, 16)

    vi = 1 if len(views) > 1 else 0
    v = views[vi]
    t0 = time.perf_counter()
    proj, cul = binned(v)
    t_bin = time.perf_counter() - t0
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
    res = {"value": k / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
           "sample": (f"FP64 oracle forward + loss + backward of {k} random pixels of keyframe "
                      f"{vi} ({v.rows}x{v.cols}) of the same workload, culled mode, OpenMP on all "
                      f"host cores; per-tile binning of that keyframe ({t_bin:.2f} s) excluded"),
           "seconds": t}
    if images is not None:
        gD_img, gN_img, gO_img = images
        worst = {"max_dD_m": 0.0, "max_dO": 0.0, "max_1mcos": 0.0}
        band = compared = 0
        for j, vj in enumerate(views):
            pj, cj = (proj, cul) if j == vi else binned(vj)
            flat = np.sort(rng.choice(vj.rows * vj.cols, min(acc_pixels, vj.rows * vj.cols),
                                      replace=False))
            px = np.stack([flat // vj.cols, flat % vj.cols], 1)
            ref = oracle.render(params, pj["flip"], None, vj.T_ws, vj.rows, vj.cols,
                                vj.elev_min, vj.elev_max, band=oracle.AMBIGUITY_BAND, culled=cj,
                                pixels=px)
            idx = offsets[j] + flat
            ok = ref["band"] == 0
            D, O, N = ref["D"], ref["O"], ref["N"]
            rng_m = np.where(O > 0, D / np.maximum(O, 1e-30), 0.0)
            dD = np.abs(gD_img[idx] - D)[ok & (rng_m <= 100.0)]
            dO = np.abs(gO_img[idx] - O)[ok]
            gN = gN_img[:, idx]
            nr, ng = np.linalg.norm(N, axis=0), np.linalg.norm(gN, axis=0)
            m = ok & (nr > 1e-6)
            cos = np.sum(gN * N, 0)[m] / np.maximum(ng[m] * nr[m], 1e-30)
            worst["max_dD_m"] = max(worst["max_dD_m"], float(dD.max(initial=0)))
            worst["max_dO"] = max(worst["max_dO"], float(dO.max(initial=0)))
            worst["max_1mcos"] = max(worst["max_1mcos"], float((1 - cos).max(initial=0)))
            band += int((~ok).sum())
            compared += len(flat)
        res["accuracy"] = {**worst, "pixels": compared, "band": band,
                           "within_tolerance": (worst["max_dD_m"] <= 1e-3
                                                and worst["max_dO"] <= 1e-5
                                                and worst["max_1mcos"] <= 1e-5),
                           "tolerance": "|dD| <= 1e-3 m (range <= 100 m), |dO| <= 1e-5, "
                                        "1 - cos N <= 1e-5",
                           "what": (f"the measured run's final parameters rendered by the timed "
                                    f"kernels vs the FP64 oracle on {acc_pixels} random pixels "
                                    f"of each of the {len(views)} keyframes")}
    return res


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
    # "plain": every keyframe has its own context, registered before timing (launches only);
    # "plain_reregister": one context that registers each keyframe inside the step (host table
    # rebuild and synchronous upload per keyframe, as per-call splat_render does)
    plains = {}
    if args.plain_steps > 0:
        per_view_pairs = api.default_capacity_pairs(scene.n, [max(views, key=lambda v: v.n_pixels)])
        for mode in ("plain", "plain_reregister"):
            pparams = [p.clone() for p in params0]
            pl = api.Refiner(pparams, views, targets, mode=mode, cfg=cfg, max_pairs=per_view_pairs)
            for _ in range(2):
                pl.step()
            t_plain = timed(pl.step, args.plain_steps)
            ms_plain = max_over_ranks(dist, sum(t_plain), dev) / len(t_plain)
            plains[mode] = {"value": world * pixels / (ms_plain * 1e-3), "ms_per_step": ms_plain,
                            "steps": args.plain_steps}
            pl.close()
            del pl, pparams
        plains["plain"]["note"] = ("one render/loss/backward launch sequence per keyframe on "
                                   "that keyframe's own context (registered before timing), then "
                                   "Adam; no CUDA graph")
        plains["plain_reregister"]["note"] = ("as plain, on one context that registers each "
                                              "keyframe inside the step (host view tables "
                                              "rebuilt and uploaded per keyframe)")
    plain = plains.get("plain")

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
        # the measured run's final parameters, rendered by the same context and kernels
        torch.cuda.synchronize()
        d_img, n_img, a_img = ref.ctx.render(*ref.params)
        torch.cuda.synchronize()
        final = [p.cpu().numpy() for p in ref.params]
        cpu = cpu_baseline(final, views, targets_np, args.cpu_seconds,
                           images=(d_img.cpu().numpy().astype(np.float64),
                                   n_img.cpu().numpy().astype(np.float64),
                                   a_img.cpu().numpy().astype(np.float64)),
                           offsets=ref.ctx.offsets)

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
        "plain_reregister": plains.get("plain_reregister"),
        "batched_over_plain": (plain["ms_per_step"] / ms_max) if plain else None,
        "batched_over_plain_reregister": ((plains["plain_reregister"]["ms_per_step"] / ms_max)
                                          if plains else None),
        "accuracy": cpu.get("accuracy") if cpu else None,
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
# the long incremental mapping run (workload 4)
# ----------------------------------------------------------------------------------------------

def _raycast_scans(scene, idx, workers=8):
    from concurrent.futures import ThreadPoolExecutor
    from paper_2503_17491_gb300 import scenes
    with ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(lambda k: scenes.render_targets(scene, scene.views[k]), idx))


def run_mapping(args):
    """The long incremental mapping run: 300 scans of 128x1024 along a 600 m path; per scan the
    scan is registered as a keyframe, the map grows from it (splat_densify) and 20 refinement
    iterations (splat_refine_step, one fused pass) run over the 8 most recent keyframes, the map
    growing to 3,000,000 primitive slots.  Timed on every S-th scan (S = --scan-stride): each
    timed scan grows the map by S scans' share, so the map reaches 3,000,000 slots at the last
    one, and its window holds the 8 most recent timed scans.  The full run's time is
    extrapolated as S x the timed scans' sum (flagged).  value = pixels refined per second (20 x
    the window's pixels per scan); e2e = the same with each scan's targets copied from pinned
    host memory inside the timed region and the last loss read back."""
    import torch
    from paper_2503_17491_gb300 import api, scenes
    from paper_2503_17491_gb300 import build as libbuild

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dist = dist_init("nccl")
    dev = torch.device("cuda", local)
    libbuild.build()
    S = args.scan_stride
    n_total, iters, window = 3_000_000, 20, 8
    scene = scenes.workload(4, n=1)                 # surfaces and the 300 scan poses
    idx = list(range(0, 300, S))
    n_new = n_total // len(idx)
    t0 = time.perf_counter()
    targets = _raycast_scans(scene, idx)
    t_cast = time.perf_counter() - t0
    P1 = 128 * 1024
    dev_targets = [(torch.from_numpy(d).to(dev), torch.from_numpy(n).to(dev)) for d, n in targets]
    host_targets = [(torch.from_numpy(d).pin_memory(), torch.from_numpy(n).pin_memory())
                    for d, n in targets]
    flush_buf = torch.empty(256 << 20, dtype=torch.float32, device=dev)

    def mapper(shape):
        c = api.RenderConfig(tile_h=shape[0], tile_w=shape[1])
        return api.Mapper(n_total, window, window * P1, n_new, cfg=c, draws=0,
                          max_keyframes=window, device=dev)

    def scan(m, j, e2e):
        if e2e:
            d = host_targets[j][0].to(dev, non_blocking=True)
            n = host_targets[j][1].to(dev, non_blocking=True)
        else:
            d, n = dev_targets[j]
        m.add_keyframe(scene.views[idx[j]], d, n)
        m.refine(iters, read_losses=False)
        if e2e:
            return m.loss_out.to("cpu", non_blocking=True)
        return None

    # tile shape: with --tile auto, the whole run once per shape (untimed, host clock around a
    # synchronised run), the fastest kept -- the map's horizon tiles hold the longest lists, and
    # their length depends on the shape
    autotune = None
    if args.tile == "auto":
        autotune = {}
        for shape in ((16, 16), (8, 32), (32, 8), (4, 64)):
            pm = mapper(shape)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for j in range(len(idx)):
                scan(pm, j, False)
            torch.cuda.synchronize()
            autotune[f"{shape[0]}x{shape[1]}"] = max_over_ranks(
                dist, (time.perf_counter() - t0) * 1e3, dev)
            pm.ctx.close()
            del pm
        tile = min(((16, 16), (8, 32), (32, 8), (4, 64)),
                   key=lambda sh: autotune[f"{sh[0]}x{sh[1]}"])
    else:
        tile = tuple(int(x) for x in args.tile.split("x"))

    # warm-up: a few scans of a throwaway run
    wm = mapper(tile)
    for j in range(min(max(args.warmup, 1), len(idx))):
        scan(wm, j, False)
    torch.cuda.synchronize()
    wm.ctx.close()
    del wm

    def timed_run(e2e):
        m = mapper(tile)
        ms, px = [], []
        barrier(dist)
        torch.cuda.synchronize()
        for j in range(len(idx)):
            if not args.no_flush:
                flush_buf.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            scan(m, j, e2e)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
            px.append(iters * sum(v.rows * v.cols for v in m.views))
        barrier(dist)
        return m, ms, px

    sampler = ClockSampler(None)
    m, ms, px = timed_run(False)
    clocks = sampler.stop()
    total_ms = max_over_ranks(dist, sum(ms), dev)
    value = world * sum(px) / (total_ms * 1e-3)
    status = m.ctx.status()
    st = m.ctx.stats()
    # roofline of the dominant compositing kernel at the final map size (profiled extra steps)
    m.ctx.set_profiling(True)
    fwd, bwd, fev, bev, stage_ms = [], [], [], [], []
    for _ in range(4):
        m.refine(1, read_losses=False)
        f, b = m.ctx.kernel_times()
        s2 = m.ctx.stats()
        fwd.append(f)
        bwd.append(b)
        fev.append(s2["fwd_evals"])
        bev.append(s2["bwd_evals"])
        stage_ms.append(m.ctx.stage_times())
    m.ctx.set_profiling(False)
    stages = {"unit": "ms per refinement iteration at the final map (library events)",
              "render_fwd": statistics.mean(fwd[1:]), "render_bwd": statistics.mean(bwd[1:]),
              **{k: statistics.mean(x[k] for x in stage_ms[1:] if x.get(k) is not None)
                 for k in stage_ms[-1] if stage_ms[-1].get(k) is not None},
              "pairs": s2["n_pairs"], "touching": s2["n_touching"]}
    kern = {"render_fwd": (statistics.mean(fwd[1:]), statistics.mean(fev[1:])),
            "render_bwd": (statistics.mean(bwd[1:]), statistics.mean(bev[1:]))}
    dom = max(kern, key=lambda k: kern[k][0])
    peaks, peak_src = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    peak_tops = sms * FP32_LANES_PER_SM * f_max / 1e12
    k_ms, k_ev = kern[dom]
    achieved = k_ev * OPS_PER_EVAL[dom] / (k_ms * 1e-3) / 1e12
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak_tops,
                "unit": "TFLOP/s", "frac": achieved / peak_tops, "traffic": None,
                "peak_source": (f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {f_max / 1e6:.0f} "
                                f"MHz ({peak_src} max SM clock), one op per lane per clock"),
                "ops_per_eval": OPS_PER_EVAL[dom], "evals_per_launch": k_ev, "launch_ms": k_ms,
                "at": f"final map ({m.n} slots), {len(m.views)} keyframes"}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        torch.cuda.synchronize()
        d_img, n_img, a_img = m.render()
        final = [t[:m.n].cpu().numpy() for t in m.params]
        pos = {id(scene.views[k]): j for j, k in enumerate(idx)}
        win_targets = [targets[pos[id(v)]] for v in m.views]
        cpu = cpu_baseline(final, m.views, win_targets, args.cpu_seconds,
                           images=(d_img.cpu().numpy().astype(np.float64),
                                   n_img.cpu().numpy().astype(np.float64),
                                   a_img.cpu().numpy().astype(np.float64)),
                           offsets=m.ctx.offsets)
    m.ctx.close()
    del m
    me, ms_e, px_e = timed_run(True)
    me.ctx.close()
    e2e_ms = max_over_ranks(dist, sum(ms_e), dev)
    if rank != 0:
        return None
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": len(idx),
        "warmup": args.warmup, "ms_per_step": total_ms / len(idx), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": scenes.WORKLOADS[4], "n_gaussians_final": n_total,
                   "keyframes_per_iteration": window, "iterations_per_scan": iters,
                   "timed_scans": f"every {S}th scan of 300 ({len(idx)} scans), map growing by "
                                  f"{n_new} slots per timed scan",
                   "step": "one scan: register the keyframe, grow the map (splat_densify), 20 "
                           "refinement iterations (render + loss + backward + Adam) over the "
                           "8 most recent keyframes",
                   "loss": "L1 range + self-regularised normals (range-map mode, lambda_n 0.1)",
                   "tile": f"{tile[0]}x{tile[1]}",
                   "l2": "flushed before every timed scan (1 GiB write)" if not args.no_flush
                   else "not flushed",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "target_raycast_s": t_cast},
        "extrapolated": {"run_s": S * total_ms * 1e-3, "scans": 300,
                         "note": f"the full 300-scan run's time as {S} x the sum over the timed "
                                 f"scans (each stands for {S} scans at its map size)"},
        "per_scan_ms": {"first": ms[0], "mid": ms[len(ms) // 2], "last": ms[-1]},
        "stages": stages,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "accuracy": cpu.get("accuracy") if cpu else None,
        "e2e": {"value": world * sum(px_e) / (e2e_ms * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": 16 * P1, "d2h_bytes_per_step": 8,
                "ms_per_step": e2e_ms / len(idx),
                "path": "per scan: pinned host targets -> Mapper.add_keyframe + refine -> loss "
                        "to host"},
        "gpu_launches": st["kernel_launches"],
        "clocks": clocks,
        "status": status,
        "autotune": autotune,
    }


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


def run_next_rows(args):
    """Timing of the kernels beside the refinement step (the "next" rows), on the 12-keyframe /
    500,000-primitive workload, against the measured HBM bandwidth: the loss in both normal
    modes, map growth in both mask modes, the photometric normal equations and back-projection.
    Each kernel is launched through the C ABI on preallocated buffers; L2 is flushed (a 1 GiB
    write) before every timed launch, and the time is the median of CUDA-event intervals around
    the launch alone.  "bytes" are the algorithmic bytes of one launch (what the definition must
    read and write once).  Prints one JSON line per kernel."""
    import ctypes
    import torch
    from paper_2503_17491_gb300 import _lib, api, scenes
    from paper_2503_17491_gb300 import build as libbuild
    libbuild.build()

    def _ptr(t):
        return None if t is None else ctypes.c_void_p(t.data_ptr())

    dev = torch.device("cuda")
    s = scenes.workload(3)
    views = s.views
    targets = [scenes.render_targets(s, v) for v in views]
    P = sum(v.rows * v.cols for v in views)
    ctx = api.SplatContext(s.n + args.next_rows_new, len(views), P,
                           api.default_capacity_pairs(s.n, views))
    ctx.set_views(views)
    params = [torch.from_numpy(a).to(dev) for a in (s.pos_logit, s.quat, s.log_scale)]
    D, N, O = ctx.render(*params)
    Dt = torch.from_numpy(np.concatenate([t[0].ravel() for t in targets])).to(dev)
    Nt = torch.from_numpy(np.concatenate([t[1].reshape(3, -1) for t in targets], 1)).contiguous().to(dev)
    gD, gN, gO = torch.empty_like(D), torch.empty_like(N), torch.empty_like(O)
    L = torch.zeros(1, dtype=torch.float64, device=dev)
    cap = s.n + args.next_rows_new
    grown = [torch.zeros(cap, w, device=dev) for w in (4, 4, 2)]
    pts = torch.empty(3, P, device=dev)
    k1 = 1
    o1 = ctx.offsets[k1]
    P1 = views[k1].rows * views[k1].cols
    T34 = torch.tensor([[1, 0, 0, 0.05], [0, 1, 0, 0.0], [0, 0, 1, 0.0]], dtype=torch.float32,
                       device=dev)
    eqs = torch.zeros(29, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.float32, device=dev)
    lib = ctx.lib
    h = ctx.h

    def loss(mode):
        cfg = api.LossConfig(lambda_n=0.5, lambda_o=0.1, normal_mode=mode).c()
        return lambda: lib.splat_view_loss(h, _ptr(D), _ptr(N), _ptr(O), _ptr(Dt), _ptr(Nt),
                                           ctypes.byref(cfg), _ptr(gD), _ptr(gN), _ptr(gO),
                                           _ptr(L), None)

    def grow(refine):
        cfg = api.DensifyConfig(refine=refine, seed=3).c()
        return lambda: lib.splat_densify(h, _ptr(Dt), _ptr(D), _ptr(O), ctypes.byref(cfg),
                                         args.next_rows_new, _ptr(grown[0]), _ptr(grown[1]),
                                         _ptr(grown[2]), s.n, cap, None)

    def photo():
        return lib.splat_photometric(h, k1, _ptr(D[o1:]), _ptr(O[o1:]), _ptr(Dt[o1:]), _ptr(T34),
                                     0.5, 0.3, _ptr(eqs), None, None)

    def backproject():
        return lib.splat_backproject(h, _ptr(D), _ptr(O), ctypes.c_float(0.5), _ptr(pts), None)

    n_d = args.next_rows_new
    rows = [
        ("k_loss (target normals)", loss(0), P * (9 * 4 + 5 * 4), f"{P} pixels"),
        ("k_loss (range-map normals)", loss(1), P * (6 * 4 + 5 * 4), f"{P} pixels"),
        ("k_grow_* (initialisation masks)", grow(False), P * (4 + 4 + 4) + n_d * 40,
         f"{P} pixels, {n_d} slots"),
        ("k_grow_* (refinement masks)", grow(True), P * (12 + 4 + 4) + n_d * 40,
         f"{P} pixels, {n_d} slots"),
        ("k_photometric", photo, P1 * 12, f"{P1} pixels of one 128x1024 keyframe"),
        ("k_backproject", backproject, P * (8 + 12), f"{P} pixels"),
    ]
    peaks, src = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    for name, fn, nbytes, unit in rows:
        for _ in range(3):
            _lib.check(fn(), name)
        times = []
        for _ in range(args.next_rows_reps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _lib.check(fn(), name)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = float(np.median(times))
        gbs = nbytes / (ms * 1e-3) / 1e9
        print(json.dumps({"kernel": name, "ms": ms, "bytes": nbytes, "units": unit,
                          "gbs": gbs, "peak_gbs": peak, "frac": gbs / peak,
                          "peak_source": src}))



def main():
    args = parse()
    if args.next_rows:
        run_next_rows(args)
        return
    if args.impl == "reference":
        line = run_reference(args)
    elif args.workload == 4:
        line = run_mapping(args)
    else:
        line = run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
