"""Checkpoint and resume of the refinement state (map parameters, Adam moments, step count)."""
import pytest
import torch

from paper_2503_17491_gb300 import api, scenes


def _map(n, seed):
    g = torch.Generator().manual_seed(seed)
    params = (torch.randn(n, 4, generator=g), torch.randn(n, 4, generator=g),
              torch.randn(n, 2, generator=g))
    state = api.adam_state(n, "cpu")
    for t in state[:6]:
        t.copy_(torch.randn(t.shape, generator=g))
    state[6].fill_(7)
    return params, state


def test_round_trip_new_tensors(tmp_path):
    params, state = _map(50, 0)
    path = tmp_path / "ck.pt"
    api.save_checkpoint(path, params, state, {"n": 50, "note": "x"})
    p2, s2, extra = api.load_checkpoint(path, device="cpu")
    assert extra == {"n": 50, "note": "x"}
    for a, b in zip(params + state, p2 + s2):
        assert torch.equal(a, b)


def test_load_in_place_keeps_storage(tmp_path):
    params, state = _map(40, 1)
    path = tmp_path / "ck.pt"
    api.save_checkpoint(path, params, state)
    dst_p, dst_s = _map(40, 2)
    ptrs = [t.data_ptr() for t in dst_p + dst_s]
    p2, s2, _ = api.load_checkpoint(path, dst_p, dst_s)
    assert [t.data_ptr() for t in p2 + s2] == ptrs
    for a, b in zip(params + state, dst_p + dst_s):
        assert torch.equal(a, b)


def test_load_rejects_other_shapes(tmp_path):
    params, state = _map(30, 3)
    path = tmp_path / "ck.pt"
    api.save_checkpoint(path, params, state)
    other_p, other_s = _map(31, 4)
    with pytest.raises(ValueError):
        api.load_checkpoint(path, other_p, other_s)


@pytest.mark.gpu
def test_refiner_resume_repeats_the_steps(tmp_path):
    """Steps taken after resuming from a checkpoint repeat the steps taken after it was written,
    through the same captured graph (within the run-to-run spread of the backward's float
    atomics)."""
    import numpy as np
    s = scenes.workload(3, n=20_000)
    views = s.views[:3]
    tt = [(torch.from_numpy(d).cuda(), torch.from_numpy(n).cuda())
          for d, n in (scenes.render_targets(s, v) for v in views)]
    params = [torch.from_numpy(a).cuda() for a in (s.pos_logit, s.quat, s.log_scale)]
    r = api.Refiner(params, views, tt, mode="batched")
    r.capture(warmup=0)
    for _ in range(3):
        r.step()
    path = tmp_path / "ck.pt"
    r.save(path)
    after = [float(r.step()) for _ in range(4)]
    snap = [t.cpu().numpy() for t in r.params]
    r.load(path)
    assert int(r.state[-1]) == 3
    again = [float(r.step()) for _ in range(4)]
    torch.cuda.synchronize()
    assert again == pytest.approx(after, rel=1e-4)
    for a, b in zip(snap, r.params):
        np.testing.assert_allclose(a, b.cpu().numpy(), rtol=0, atol=1e-4)
