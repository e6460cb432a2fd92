"""Timing of the kernels beside the refinement step, on the 12-keyframe / 500,000-primitive
workload, against the measured HBM bandwidth: the loss in both normal modes, map growth in both
mask modes, the photometric normal equations and back-projection.

    python -m paper_2503_17491_gb300.microbench [--reps 30]

Each kernel is launched through the C ABI on preallocated buffers; L2 is flushed (a 1 GiB write)
before every timed launch, and the time is the median of CUDA-event intervals around the launch
alone.  "bytes" are the algorithmic bytes of one launch (what the definition must read and
write once); GB/s = bytes / time.  Prints one JSON line per kernel.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os

import numpy as np
import torch

from . import _lib, api, scenes

_P = ctypes.c_void_p


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _peak_gbs():
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--reps", type=int, default=30)
    ap.add_argument("--n-new", type=int, default=50_000)
    args = ap.parse_args()
    dev = torch.device("cuda")
    s = scenes.workload(3)
    views = s.views
    targets = [scenes.render_targets(s, v) for v in views]
    P = sum(v.rows * v.cols for v in views)
    ctx = api.SplatContext(s.n + args.n_new, len(views), P,
                           api.default_capacity_pairs(s.n, views))
    ctx.set_views(views)
    params = [torch.from_numpy(a).to(dev) for a in (s.pos_logit, s.quat, s.log_scale)]
    D, N, O = ctx.render(*params)
    Dt = torch.from_numpy(np.concatenate([t[0].ravel() for t in targets])).to(dev)
    Nt = torch.from_numpy(np.concatenate([t[1].reshape(3, -1) for t in targets], 1)).contiguous().to(dev)
    gD, gN, gO = torch.empty_like(D), torch.empty_like(N), torch.empty_like(O)
    L = torch.zeros(1, dtype=torch.float64, device=dev)
    cap = s.n + args.n_new
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
                                         args.n_new, _ptr(grown[0]), _ptr(grown[1]),
                                         _ptr(grown[2]), s.n, cap, None)

    def photo():
        return lib.splat_photometric(h, k1, _ptr(D[o1:]), _ptr(O[o1:]), _ptr(Dt[o1:]), _ptr(T34),
                                     0.5, 0.3, _ptr(eqs), None, None)

    def backproject():
        return lib.splat_backproject(h, _ptr(D), _ptr(O), ctypes.c_float(0.5), _ptr(pts), None)

    n_d = args.n_new
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
    peak, src = _peak_gbs()
    for name, fn, nbytes, unit in rows:
        for _ in range(3):
            _lib.check(fn(), name)
        times = []
        for _ in range(args.reps):
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


if __name__ == "__main__":
    main()
