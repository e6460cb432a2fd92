"""bench.py reads the DRAM bytes of its dominant kernel from the committed ncu summary; this
checks that every row of that summary parses and that a stale summary is not used."""
import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _rows():
    with open(bench.TRAFFIC_MD) as f:
        text = f.read()
    digest = re.search(r"first 16 hex digits\): `([0-9a-f]{16})`", text).group(1)
    rows = re.findall(r"\| `k_(render_fwd|render_bwd)` \| (\d+x\d+) \| (\d+) \| (\d+) \| (\d+) \|",
                      text)
    return digest, rows


def test_summary_rows_are_consistent():
    digest, rows = _rows()
    assert len(rows) == 8   # two kernels x four tile shapes
    for _, _, rd, wr, tot in rows:
        assert int(rd) + int(wr) == int(tot)


def test_traffic_is_read_only_for_the_sources_it_was_taken_on(monkeypatch):
    digest, rows = _rows()
    kernel, tile, _, _, tot = rows[0]
    monkeypatch.setattr(bench, "csrc_digest", lambda: digest)
    assert bench.recorded_traffic(kernel, tile) == int(tot)
    monkeypatch.setattr(bench, "csrc_digest", lambda: "0" * 16)
    assert bench.recorded_traffic(kernel, tile) is None


def test_summary_matches_the_current_sources():
    digest, _ = _rows()
    if bench.csrc_digest() != digest:
        pytest.skip("the library sources changed since the capture: bench reports no traffic")
    assert bench.recorded_traffic("render_fwd", "8x32") is not None
