"""Host-side bookkeeping of bench.py (no GPU): the workload it describes, the
work it counts, the Table 1 check it prints and the gating of the committed
DRAM-traffic figures on the kernel sources they were taken on."""
import json
import os
import sys

import pytest

import golden_io
from oracle import flm, partitions

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("k", [12, 17, 33, 41])
def test_band_and_terms_match_the_oracle(k):
    assert bench.band(k) == list(flm.band(k))
    # the sweep keeps one more square term at odd k: the mu_{k-1} term reaches z^{2k-3} (Sec. 4.2)
    assert bench.n_terms("square", k) == flm.n_terms("square", k) + (k % 2)
    assert bench.n_terms("triangular", k) == flm.n_terms("triangular", k)
    if k == 33:
        assert len(bench.band(k)) == 62 and max(r for r, _ in bench.band(k)) == 16


def test_motzkin_table():
    M = bench.motzkin_table(20)
    assert M[:21] == [partitions.motzkin(j) for j in range(21)]


def test_strip_updates_counts_every_factor_output():
    # width 1: one factor per row (1 state) and the identity read-out (1 state)
    assert bench.strip_updates("square", 1, [5], 10, 3) == (4 * 1 + 1) * 10 * 3
    # width 3, square: NCNNN space of 3 points has M_2 = 2 states, the excepted
    # spaces M_2 + M_1 = 3; row = two excepted outputs then one NCNNN output;
    # read-out: T_1^last -> M_1 = 1, T_2^last -> M_0 = 1
    M = bench.motzkin_table(5)
    row = 2 * (M[2] + M[1]) + M[2]
    assert bench.strip_updates("square", 3, [3, 4], 7, 2) == (3 * row + 2 * 2) * 7 * 2
    # triangular: every factor maps the NCNNN space to itself
    assert bench.strip_updates("triangular", 3, [4], 7, 2) == (3 * 3 * M[2] + 2) * 7 * 2


def test_table1_reader_is_the_fixture():
    assert bench.table1() == golden_io.table1()
    t = bench.table1()
    assert len(t["alpha"]) == len(t["beta"]) == 80 and t["alpha"][0] == t["beta"][0] == 1


def test_traffic_used_only_for_the_fingerprinted_sources(tmp_path, monkeypatch):
    sha = bench.gather_source_sha()
    assert len(sha) == 16 and int(sha, 16) >= 0
    entry = {"dram_bytes_per_launch": 123, "source_sha": sha}
    stale = {"dram_bytes_per_launch": 456, "source_sha": "0" * 16}
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps({"a": entry, "b": stale}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "gather_source_sha", lambda: sha)
    assert bench.load_traffic("a")["dram_bytes_per_launch"] == 123
    assert bench.load_traffic("b") is None
    assert bench.load_traffic("missing") is None


def test_committed_traffic_file_names_its_sources():
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for key, ent in d.items():
        assert key.startswith("gather_kernel:") and ent["dram_bytes_per_launch"] > 0
        assert os.path.exists(os.path.join(ROOT, ent["from"]))


def test_tile_names():
    assert bench.tile_name(4) == "register gather kernel, 4 rows/warp"
    assert "32 rows/block, 40 KB ring, 2 edge(s) per stage, 2 chunk(s) per thread" in bench.tile_name(
        32 | (40 << 12) | (2 << 20) | (2 << 24))
    assert bench.tile_name(64 | (8 << 20) | (2 << 28)).endswith("narrow blocks")
    assert bench.tile_name(64 | (1 << 28)).endswith("wide blocks")
