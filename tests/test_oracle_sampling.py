"""Pins of the oracle's keyframe sampling (Sec. 3.3: a geometric-distribution scheme that picks
the newest keyframe with probability at least 40 % and older ones progressively less often) and
of the Philox-4x32-10 generator it draws from (its published definition; no reference output
vectors are used, so the generator is pinned by its statistics)."""
import math

import numpy as np
import pytest

import oracle


def _words(n, seed=7):
    out = np.zeros((n, 4), np.uint64)
    for i in range(n):
        out[i] = oracle.philox4x32_10((i, 3, 0, 0), (seed, 0))
    return out


def test_philox_words_are_uniform():
    w = _words(20_000).ravel()
    counts = np.bincount((w >> np.uint64(26)).astype(np.int64), minlength=64)
    exp = w.size / 64
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 63 + 6 * math.sqrt(2 * 63), chi2
    assert w.max() < 2 ** 32


def test_philox_avalanche():
    """Flipping one counter or key bit flips about half of the 128 output bits."""
    rng = np.random.default_rng(0)
    flips = []
    for _ in range(400):
        ctr = [int(x) for x in rng.integers(0, 2 ** 32, 4)]
        key = [int(x) for x in rng.integers(0, 2 ** 32, 2)]
        a = oracle.philox4x32_10(ctr, key)
        which = int(rng.integers(0, 6))
        bit = 1 << int(rng.integers(0, 32))
        if which < 4:
            ctr[which] ^= bit
        else:
            key[which - 4] ^= bit
        b = oracle.philox4x32_10(ctr, key)
        flips.append(sum(bin(x ^ y).count("1") for x, y in zip(a, b)))
    assert abs(np.mean(flips) - 64.0) < 2.0, np.mean(flips)
    assert min(flips) > 30


@pytest.mark.parametrize("n_views,p", [(8, 0.4), (3, 0.4), (12, 0.6)])
def test_sampling_follows_the_truncated_geometric_law(n_views, p):
    """Age frequencies over 12,000 single draws match p (1 - p)^a / Z within 4 sigma, the newest
    view's share is at least p, and it decreases with age."""
    n = 12_000
    ages = np.zeros(n_views)
    for step in range(n):
        act = oracle.sample_active_views(n_views, 1, p, 99, step)
        ages[n_views - 1 - int(np.flatnonzero(act)[0])] += 1
    P = np.array([p * (1 - p) ** a for a in range(n_views)])
    P /= P.sum()
    sigma = np.sqrt(n * P * (1 - P))
    assert (np.abs(ages - n * P) <= 4 * sigma + 1).all(), (ages, n * P)
    assert ages[0] / n >= p - 4 * sigma[0] / n
    assert (np.diff(P) < 0).all()


def test_thresholds_and_determinism():
    thr = oracle.view_sampling_thresholds(8, 0.4)
    assert len(thr) == 7 and all(a < b for a, b in zip(thr, thr[1:])) and thr[-1] < 2 ** 32
    assert thr[0] == math.floor(0.4 / (1 - 0.6 ** 8) * 2 ** 32)
    a = oracle.sample_active_views(8, 4, 0.4, 1234, 17)
    b = oracle.sample_active_views(8, 4, 0.4, 1234, 17)
    assert (a == b).all() and 1 <= a.sum() <= 4
    assert oracle.sample_active_views(5, 3, 1.0, 5, 0).tolist() == [False] * 4 + [True]
