"""Host logic of bench.py's roofline fields: the algorithmic floor, the
achieved bandwidth and fraction of one kernel kind from the library's
profiling rows, and the rule that a stored ncu traffic figure is used only
for the sources and the tile shape it was measured on."""
import json
import os

import pytest

import bench


def test_floor_bytes_closed_form():
    """Each level l = 0 .. L-1 reads and writes every live record and its one
    int32 once; the live range at level l is N - F(l-1), F(m) = 2^m - 1,
    F(-1) = 0.  So the sum is 2 (S + 4) (L N - sum_{m=0}^{L-2} (2^m - 1))."""
    for n, s in [(1, 12), (2, 12), (10, 8), (1000, 12), (10**7, 12), (10**8, 16)]:
        L = n.bit_length()
        dropped = (2 ** (L - 1) - 1) - (L - 1) if L >= 2 else 0
        assert bench.floor_bytes(n, s) == pytest.approx(2 * (s + 4) * (L * n - dropped), rel=1e-12)
    # 1e8 float4 (27 levels) and 1e7 float3 (24 levels) in GB
    assert bench.floor_bytes(10**8, 16) / 1e9 == pytest.approx(105.3, abs=0.05)
    assert bench.floor_bytes(10**7, 12) / 1e9 == pytest.approx(7.41, abs=0.01)


def test_kernel_roofline_of_an_hbm_kind():
    steps, n = 20, 10**8
    row = {"name": "radix_pass", "ms": steps * 11.7, "bytes": steps * 12 * 32.0 * n,
           "launches": steps * 12}
    shapes = {"partition": (512, 13, 2), "radix": (256, 13, 3)}
    r = bench.kernel_roofline(row, steps, n, 6794.1, "measured", shapes)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(12 * 32.0 * n / 11.7e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6794.1)
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(32.0 * n)
    stored = json.load(open(os.path.join(bench.ROOT, "profiles", "radix_pass_traffic.json")))
    if stored["kernel_hash"] == bench.kernel_hash("radix_pass"):
        assert r["traffic"] == pytest.approx(stored["by_shape"]["256x13x3"] * n)
    else:
        assert r["traffic"] is None  # measured on other sources: not reused


def test_kernel_roofline_of_the_issue_bound_local_finish(monkeypatch):
    """The local finish is rated against the warp-instruction issue peak
    (four schedulers per SM, one instruction each per cycle): achieved =
    stored warp instructions per point x points / CUDA-event time; without a
    stored count for its current sources the fraction is null, not guessed."""
    steps, n = 20, 10**8
    row = {"name": "local_finish", "ms": steps * 6.68, "bytes": 0.0, "launches": steps}
    monkeypatch.setattr(bench, "issue_peak_ginst", lambda device=0: (4 * 152 * 2070e6 / 1e9, "test"))
    counters = {"warp_instructions_per_point": 53.0, "dram_bytes_per_point": 38.0}
    monkeypatch.setattr(bench, "stored_counters", lambda name, kind: counters)
    r = bench.kernel_roofline(row, steps, n, 6799.6, "measured", {})
    assert r["bound"] == "alu" and r["unit"] == "Gwarp-inst/s"
    assert r["peak"] == pytest.approx(1258.56)
    assert r["achieved"] == pytest.approx(53.0 * n / 6.68e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 1258.56)
    assert 0.6 < r["frac"] < 0.7
    assert r["ms_per_step"] == pytest.approx(6.68)
    monkeypatch.setattr(bench, "stored_counters", lambda name, kind: None)
    r = bench.kernel_roofline(row, steps, n, 6799.6, "measured", {})
    assert r["achieved"] is None and r["frac"] is None and r["traffic"] is None


def test_stored_traffic_only_for_its_tile_shape():
    assert bench.traffic_per_launch("radix_pass", 1e6, {"radix": (999, 1, 1)}) is None
    assert bench.traffic_per_launch("partition_pass", 1e6, {"partition": (999, 1, 1)}) is None


def test_code_only_drops_comments_and_layout():
    src = 'int a = 1; // one\n/* two\n lines */  char* s = "a // b /* c */";\n  char q = \'"\';'
    assert bench.code_only(src) == 'int a = 1; char* s = "a // b /* c */"; char q = \'"\';'
    assert bench.code_only("x\n\n\t y") == "x y"


def test_kernel_hash_follows_included_headers(tmp_path, monkeypatch):
    """A code change in a header that a kernel's file includes changes its
    hash; a comment, or a change to a file it does not include, does not."""
    import shutil

    src = os.path.join(bench.ROOT, "paper_2211_00120_gb300", "csrc")
    dst = tmp_path / "paper_2211_00120_gb300" / "csrc"
    shutil.copytree(src, dst)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_hash("radix_pass")
    assert len(h0) == 16 and h0 == bench.kernel_hash("radix_pass")
    with open(dst / "kdb_serve.cu", "a") as f:  # not included by kdb_lists.cu
        f.write("\nstatic int unrelated_code = 0;\n")
    assert bench.kernel_hash("radix_pass") == h0
    with open(dst / "kdb_segsort.cuh", "a") as f:  # included: a comment only
        f.write("\n// a comment\n/* and another */\n")
    assert bench.kernel_hash("radix_pass") == h0
    with open(dst / "kdb_segsort.cuh", "a") as f:  # included: code
        f.write("\nstatic int changed_code = 1;\n")
    assert bench.kernel_hash("radix_pass") != h0
    assert bench.kernel_hash("no_such_kind") == ""
