"""bench.py's CPU legs: the oracle baseline and the in-run accuracy check, with the oracle's own
render standing in for the GPU images (so the check must read zero), and a planted error that
it must report."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2503_17491_gb300 import scenes  # noqa: E402


def test_cpu_baseline_accuracy_reads_zero_on_the_oracles_own_images(oracle_mod):
    s = scenes.workload(0)
    v = s.views[0]
    ref = oracle_mod.full_view(s.pos_logit, s.quat, s.log_scale, v.T_ws, v.rows, v.cols,
                               v.elev_min, v.elev_max)
    images = (ref["D"].ravel(), ref["N"].reshape(3, -1), ref["O"].ravel())
    targets = [scenes.render_targets(s, v)]
    params = (s.pos_logit, s.quat, s.log_scale)
    res = bench.cpu_baseline(params, [v], targets, 0.2, images=images, offsets=[0],
                             acc_pixels=2048)
    acc = res["accuracy"]
    assert res["value"] > 0 and res["kind"] == "oracle"
    assert acc["pixels"] == 2048 and acc["within_tolerance"]
    assert acc["max_dD_m"] < 1e-9 and acc["max_dO"] < 1e-12 and acc["band"] <= 0.01 * 2048
    # an opacity error of 2e-5 on every pixel is reported
    bad = (images[0], images[1], images[2] + 2e-5 * (images[2] > 0))
    acc2 = bench.cpu_baseline(params, [v], targets, 0.2, images=bad, offsets=[0],
                              acc_pixels=2048)["accuracy"]
    assert not acc2["within_tolerance"] and abs(acc2["max_dO"] - 2e-5) < 1e-9
