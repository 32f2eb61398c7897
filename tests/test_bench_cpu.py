"""Host logic of the benchmark that decides what runs: the serving stream's
choice of warps per query by batch size (CPU only)."""
import os
import sys
from types import SimpleNamespace

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _sb(lat):
    """small_batch-like table: lat[W] = {b: p50 ms}."""
    return {W: {**{f"b{b}_p50_ms": v for b, v in row.items()}, "cfg": SimpleNamespace(W=W, T=96 // W)}
            for W, row in lat.items()}


def test_w_policy_takes_the_fastest_w_per_size_and_merges_ranges():
    # the 10M x 96 measurement: W = 8 leads up to 256 queries, W = 2 at 1,024
    sb = _sb({1: {16: 0.325, 256: 0.313, 1024: 0.316},
              2: {16: 0.182, 256: 0.185, 1024: 0.205},
              4: {16: 0.129, 256: 0.135, 1024: 0.254},
              8: {16: 0.092, 256: 0.100, 1024: 0.318}})
    pol = bench.w_policy(sb)
    assert [(b, c.W) for b, c in pol] == [(256, 8), (1024, 2)]


def test_w_policy_keeps_one_warp_where_it_wins():
    sb = _sb({1: {16: 0.10, 256: 0.10, 1024: 0.10},
              8: {16: 0.09, 256: 0.20, 1024: 0.50}})
    assert [(b, c.W) for b, c in bench.w_policy(sb)] == [(16, 8)]
    sb = _sb({1: {16: 0.05, 256: 0.05, 1024: 0.05}, 8: {16: 0.09, 256: 0.20, 1024: 0.50}})
    assert bench.w_policy(sb) == []


def test_serving_picks_the_first_range_that_holds_the_batch():
    pol = [(16, "w8"), (256, "w4"), (1024, "w2")]
    assert [bench.pick_cfg(pol, s, "w1") for s in (1, 16, 17, 256, 257, 1024, 1025, 2048)] == \
        ["w8", "w8", "w4", "w4", "w2", "w2", "w1", "w1"]
    assert bench.pick_cfg(None, 5, "w1") == "w1" and bench.pick_cfg([], 5, "w1") == "w1"


def test_profiled_traffic_follows_the_kernel_code(tmp_path):
    """The committed ncu summary's DRAM bytes are reported only for the
    captured form and point and while the library's code (comments aside)
    hashes to the captured value."""
    import shutil
    root = tmp_path / "repo"
    shutil.copytree(os.path.join(ROOT, "paper_2601_08528_b300", "csrc"), root / "paper_2601_08528_b300" / "csrc")
    h0 = bench.csrc_hash(str(root))
    assert h0 == bench.csrc_hash()
    f = root / "paper_2601_08528_b300" / "csrc" / "svf_dev.cuh"
    f.write_text(f.read_text() + "\n// a comment changes nothing\n/* nor does\n   this */\n")
    assert bench.csrc_hash(str(root)) == h0
    f.write_text(f.read_text() + "\nnamespace svf { constexpr int kProbe = 1; }\n")
    assert bench.csrc_hash(str(root)) != h0
    # the committed capture counts while its recorded source hash is the code's
    txt = open(os.path.join(ROOT, "profiles", "search_kernel_unit96_10M.md")).read()
    sha = [ln.split(": ", 1)[1].strip() for ln in txt.splitlines() if ln.startswith("source_sha: ")]
    assert len(sha) == 1
    current = sha[0] == bench.csrc_hash()
    assert (bench.profiled_traffic("fp8+rerank", 64, 40) is not None) == current
    assert bench.profiled_traffic("fp8+rerank", 64, 72) is None      # another launch point
    assert bench.profiled_traffic("bf16+rerank", 64, 40) is None     # another form
