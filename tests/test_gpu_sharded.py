"""The data-parallel refiner on one GPU (one rank holds every keyframe): its steps equal the
plain per-keyframe refinement's (render, loss, backward accumulated over keyframes, then Adam).
Marked gpu."""
import numpy as np
import pytest
import torch

from paper_2503_17491_gb300 import api, scenes, sharded
from gpu_common import to_dev

pytestmark = pytest.mark.gpu


def test_one_rank_matches_plain_refinement():
    s = scenes.workload(3, n=20_000)
    views = s.views[:4]
    targets = [scenes.render_targets(s, v) for v in views]
    tt = [(torch.from_numpy(d).cuda(), torch.from_numpy(n).cuda()) for d, n in targets]
    pa = [t.clone() for t in to_dev(s)]
    pb = [t.clone() for t in to_dev(s)]
    plain = api.Refiner(pa, views, tt, mode="plain")
    shard = sharded.ShardedRefiner(pb, views, tt)
    assert shard.world == 1 and shard.split == [[0, 1, 2, 3]]
    la = [float(plain.step()) for _ in range(3)]
    lb = [float(shard.step()) for _ in range(3)]
    torch.cuda.synchronize()
    assert lb == pytest.approx(la, rel=1e-4)
    for a, b in zip(pa, pb):
        np.testing.assert_allclose(a.cpu().numpy(), b.cpu().numpy(), rtol=0, atol=1e-4)
