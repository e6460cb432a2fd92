"""GPU forward parity through the C ABI: binning bit-exact, images within tolerance of the FP64
oracle, robustness cases.  Marked gpu."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2503_17491_gb300 import api, scenes
from gpu_common import (check_lists, compare_images, make_ctx, oracle_view, to_dev)

pytestmark = pytest.mark.gpu

TILES = [(16, 16), (8, 32), (32, 8), (4, 64)]


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def _render(scene, views, tile=(16, 16), max_pairs=None):
    ctx = make_ctx(scene.n, views, tile, max_pairs)
    pl, q, ls = to_dev(scene)
    d, n, a = ctx.render(pl, q, ls)
    torch.cuda.synchronize()
    return ctx, d.cpu().numpy(), n.cpu().numpy(), a.cpu().numpy()


@pytest.mark.parametrize("tile", TILES)
def test_workload0_lists_and_images(tile):
    s = scenes.workload(0)
    v = s.views[0]
    ctx, d, n, a = _render(s, s.views, tile)
    assert ctx.status() == 0
    assert check_lists(ctx, s, s.views, tile) > 500
    ref, *_ = oracle_view(s, v, tile)
    st = compare_images(d, n, a, ref, f"workload0 {tile}")
    assert st["covered"] > 1000


def test_workload1_full_image():
    """100k primitives on a street, 64x1024, random pose: lists bit-exact, every pixel compared."""
    s = scenes.workload(1)
    v = s.views[0]
    ctx, d, n, a = _render(s, s.views)
    assert ctx.status() == 0
    check_lists(ctx, s, s.views)
    ref, *_ = oracle_view(s, v)
    st = compare_images(d, n, a, ref, "workload1")
    assert st["covered"] > 0.5 * v.n_pixels
    assert st["band"] < 0.01 * v.n_pixels


@pytest.mark.parametrize("tile", [(16, 16), (4, 64)])
def test_ragged_image_and_tiles(tile):
    """Image sizes that are not multiples of the tile (partial last tile row and column), a
    posed sensor, near and far primitives."""
    s = scenes.tiny_scene(300, 5, rows=37, cols=250, fov_deg=30, dist=(0.6, 60.0),
                          log_scale=(-3.0, -0.7))
    s.views[0].T_ws = scenes.random_pose(np.random.default_rng(2), 1.0, 20.0)
    ctx, d, n, a = _render(s, s.views, tile)
    check_lists(ctx, s, s.views, tile)
    ref, *_ = oracle_view(s, s.views[0], tile)
    compare_images(d, n, a, ref, "ragged")


def test_seam_and_pole_cases():
    """Primitives across the +-pi seam, over the pole, and around the sensor."""
    rng = np.random.default_rng(8)
    pts, nrm = [], []
    for _ in range(40):   # behind the sensor, straddling azimuth pi
        p = np.array([-rng.uniform(1, 20), rng.uniform(-0.3, 0.3), rng.uniform(-2, 2)])
        pts.append(p)
        nrm.append(-p + rng.normal(0, 0.3, 3))
    for _ in range(20):   # overhead and underfoot
        p = np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), rng.choice([-1, 1]) * rng.uniform(0.5, 3)])
        pts.append(p)
        nrm.append(np.array([0, 0, 1.0]) + rng.normal(0, 0.2, 3))
    for _ in range(20):   # very near
        p = rng.normal(0, 0.4, 3)
        pts.append(p)
        nrm.append(rng.normal(size=3))
    pl, q, ls = scenes.gaussians_on(np.array(pts), np.array(nrm), rng, log_scale=(-2.0, -0.9))
    view = scenes.View(np.eye(4), 48, 360, scenes.deg(-60), scenes.deg(60))
    s = scenes.Scene("seam", pl, q, ls, [view])
    ctx, d, n, a = _render(s, s.views)
    check_lists(ctx, s, s.views)
    ref, *_ = oracle_view(s, view)
    compare_images(d, n, a, ref, "seam/pole")
    assert a.reshape(48, 360)[:, :3].max() > 0 and a.reshape(48, 360)[:, -3:].max() > 0


def test_batched_views_lists_and_bitwise_equal_to_single():
    """Several views of uneven shapes in one call: lists bit-exact against the oracle's per-view
    lists, and every view's image bit-identical to rendering that view alone."""
    s = scenes.workload(3, n=20_000)
    views = [s.views[0], s.views[2], s.views[1], s.views[5]]
    ctx, d, n, a = _render(s, views)
    check_lists(ctx, s, views)
    pl, q, ls = to_dev(s)
    for k, v in enumerate(views):
        c1 = make_ctx(s.n, [v])
        d1, n1, a1 = c1.render(pl, q, ls)
        o = ctx.offsets[k]
        P = v.n_pixels
        np.testing.assert_array_equal(d[o:o + P], d1.cpu().numpy())
        np.testing.assert_array_equal(a[o:o + P], a1.cpu().numpy())
        np.testing.assert_array_equal(n[:, o:o + P], n1.cpu().numpy())


def _sampled_parity(s, views, n_rand=8192, rows_per_view=4, seed=0, label="", tile=(16, 16)):
    ctx, d, n, a = _render(s, views, tile)
    assert ctx.status() == 0
    rng = np.random.default_rng(seed)
    per = max(n_rand // len(views), 256)
    stats = []
    for k, v in enumerate(views):
        r = rng.integers(0, v.rows, per)
        c = rng.integers(0, v.cols, per)
        full = rng.choice(v.rows, min(rows_per_view, v.rows), replace=False)
        rr = np.concatenate([r, np.repeat(full, v.cols)])
        cc = np.concatenate([c, np.tile(np.arange(v.cols), len(full))])
        px = np.stack([rr, cc], 1)
        ref, *_ = oracle_view(s, v, pixels=px)
        idx = ctx.offsets[k] + rr * v.cols + cc
        stats.append(compare_images(d[idx], n[:, idx], a[idx], ref, f"{label} view {k}"))
    return ctx, stats


def test_workload2_full_size_sampled():
    """1M primitives, 128x2048: sampled pixels + 4 full rows, each composited by the oracle."""
    s = scenes.workload(2)
    ctx, stats = _sampled_parity(s, s.views, label="workload2")
    st = ctx.stats()
    assert st["n_pairs"] > s.n
    assert sum(x["covered"] for x in stats) > 0.5 * sum(x["pixels"] for x in stats)


@pytest.mark.parametrize("tile", TILES)
def test_workload3_full_size_batched_sampled(tile):
    """The batched workload at full size (500k primitives, 12 uneven views) in one call, with
    every tile shape the benchmark's autotuner can pick."""
    s = scenes.workload(3)
    _sampled_parity(s, s.views, n_rand=12 * 1024, rows_per_view=2, label=f"workload3 {tile}",
                    tile=tile)


@pytest.mark.parametrize("tile", TILES)
def test_workload3_lists_bit_exact(tile):
    s = scenes.workload(3)
    ctx, *_ = _render(s, s.views, tile)
    assert check_lists(ctx, s, s.views, tile) > 10 * s.n


@pytest.mark.parametrize("tile", [(16, 16), (8, 32)])
def test_primitives_below_alpha_min_take_no_tiles(tile):
    """Primitives whose opacity stays below alpha_min everywhere (o < 0.999 alpha_min, Sec. 3.2.3
    reading) reach no pixel and take no tile: among them the empty slots the map growth writes
    (world origin, unit scale, logit -30, here at the sensor itself) and opacities on both sides
    of the threshold.  Lists bit-exact against the oracle, images within tolerance."""
    s = scenes.workload(0)
    i = np.arange(s.n)
    amin = 1.0 / 255.0
    s.pos_logit[i % 7 == 0, 3] = -30.0
    empty = i % 7 == 1
    s.pos_logit[empty] = (0.0, 0.0, 0.0, -30.0)
    s.quat[empty] = (1.0, 0.0, 0.0, 0.0)
    s.log_scale[empty] = 0.0
    for k, f in ((2, 0.9985), (3, 0.995), (4, 1.0005)):
        o = f * amin
        s.pos_logit[i % 11 == k, 3] = math.log(o / (1.0 - o))
    ctx, d, n, a = _render(s, s.views, tile)
    assert ctx.status() == 0
    check_lists(ctx, s, s.views, tile)
    rec = ctx.pair_records(s.n)
    assert (rec["count"][(i % 7 <= 1) | (i % 11 == 3)] == 0).all()
    ref, *_ = oracle_view(s, s.views[0], tile)
    compare_images(d, n, a, ref, f"below alpha_min {tile}")


def test_empty_and_single():
    v = scenes.View(np.eye(4), 16, 64, scenes.deg(-10), scenes.deg(10))
    ctx = make_ctx(4, [v])
    z4 = torch.zeros(0, 4, device="cuda")
    d, n, a = ctx.render(z4, z4.clone(), torch.zeros(0, 2, device="cuda"))
    torch.cuda.synchronize()
    assert float(a.abs().max()) == 0 and float(d.abs().max()) == 0
    s = scenes.tiny_scene(1, 3, rows=16, cols=64)
    ctx2, d, n, a = _render(s, s.views)
    ref, *_ = oracle_view(s, s.views[0])
    compare_images(d, n, a, ref, "single")


def test_nonfinite_input_sets_status():
    s = scenes.tiny_scene(50, 1)
    s.pos_logit[3, 0] = np.nan
    s.quat[7] = 0.0
    ctx, d, n, a = _render(s, s.views)
    assert ctx.status() & api._lib.SPLAT_STATUS_NONFINITE
    assert np.isfinite(d).all() and np.isfinite(a).all()
    rec = ctx.pair_records(s.n)
    assert rec["invalid"][3] and rec["invalid"][7] and rec["count"][3] == 0
    assert ctx.status() == 0   # reading clears it


def test_capacity_overflow_sets_status():
    s = scenes.workload(0)
    ctx, d, n, a = _render(s, s.views, max_pairs=100)
    assert ctx.status() & api._lib.SPLAT_STATUS_CAPACITY
    assert ctx.stats()["n_pairs"] == 100
    assert np.isfinite(d).all()


def test_invalid_arguments_are_rejected():
    v = scenes.View(np.eye(4), 16, 64, scenes.deg(-10), scenes.deg(10))
    ctx = make_ctx(4, [v])
    bad = scenes.View(np.eye(4) * 2, 16, 64, scenes.deg(-10), scenes.deg(10))
    with pytest.raises(api._lib.SplatError):
        ctx.set_views([bad])
    with pytest.raises(api._lib.SplatError):
        ctx.set_views([scenes.View(np.eye(4), 1, 64, -0.1, 0.1)])
    with pytest.raises(api._lib.SplatError):
        ctx.set_views([scenes.View(np.eye(4), 16, 64, 0.2, 0.1)])
    T = np.eye(4)
    T[0, 3] = math.inf
    with pytest.raises(api._lib.SplatError):
        ctx.set_views([scenes.View(T, 16, 64, -0.1, 0.1)])


def test_workload4_map_size_batched_sampled():
    """The long mapping run's largest state: a 3,000,000-primitive map and its 8 most recent
    128x1024 scans (mid-trajectory) in one batched call; sampled pixels of three scans are
    composited by the oracle."""
    s = scenes.workload(4, n=3_000_000)
    views = s.views[100:108]
    ctx, d, n, a = _render(s, views)
    assert ctx.status() == 0
    rng = np.random.default_rng(4)
    for k in (0, 3, 7):
        v = views[k]
        r = rng.integers(0, v.rows, 2048)
        c = rng.integers(0, v.cols, 2048)
        rr = np.concatenate([r, np.full(v.cols, v.rows // 2)])
        cc = np.concatenate([c, np.arange(v.cols)])
        ref, *_ = oracle_view(s, v, pixels=np.stack([rr, cc], 1))
        idx = ctx.offsets[k] + rr * v.cols + cc
        compare_images(d[idx], n[:, idx], a[idx], ref, f"workload4 scan {k}")
