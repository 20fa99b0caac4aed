"""Host-side logic of bench.py, without a GPU: the roofline arithmetic of the
bench line, the committed counters it reads, and the kernel-source hash that
voids them when the step kernel changes."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def committed_counters():
    with open(os.path.join(ROOT, "profiles", "step_counters.json")) as fh:
        return json.load(fh)


@pytest.fixture
def counters_current(monkeypatch):
    """The committed counters as if the step-kernel sources still hashed to
    the captured state (whether they do is the bench's check, at run time)."""
    rec = committed_counters()
    monkeypatch.setattr(bench, "library_source_hash", lambda: rec["source_sha256"])
    return rec


def test_committed_counters_cover_the_bench_kernels():
    rec = committed_counters()
    kinds = {(e["field"], e["kernel"]) for e in rec["entries"]}
    assert ("f64", "auto") in kinds and ("f64", "fp64") in kinds
    for e in rec["entries"]:
        assert e["dram_bytes_per_update"] > 0 and e["warp_inst_per_update"] > 0


def test_source_hash_ignores_comments_and_layout(tmp_path, monkeypatch):
    """Comments and whitespace do not change the hash; code does."""
    csrc = tmp_path / "paper_2604_11008_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "bench.py").write_text("")
    (csrc / "lcs_step_x.cu").write_text("int a = 1; // one\n")
    (csrc / "k.cuh").write_text("/* block */ int b = 2;\n")
    monkeypatch.setattr(bench, "__file__", str(tmp_path / "bench.py"))
    h0 = bench.library_source_hash()
    (csrc / "lcs_step_x.cu").write_text("int a =   1;  // another comment\n\n")
    (csrc / "k.cuh").write_text("int b = 2; /* moved */\n")
    assert bench.library_source_hash() == h0
    (csrc / "k.cuh").write_text("int b = 3;\n")
    assert bench.library_source_hash() != h0


def test_counters_are_void_when_the_sources_change(counters_current, monkeypatch):
    assert bench.measured_counters("scale_256", "f64", "auto", 16777216, (256, 1, 3)) is not None
    monkeypatch.setattr(bench, "library_source_hash", lambda: "0" * 64)
    assert bench.measured_counters("scale_256", "f64", "auto", 16777216, (256, 1, 3)) is None


def test_counters_match_only_their_configuration(counters_current):
    assert bench.measured_counters("scale_256", "f64", "auto", 16777216, (128, 1, 3)) is None
    assert bench.measured_counters("precision_512", "f64", "auto", 10**8, (256, 1, 3)) is None


def test_step_roofline_arithmetic(counters_current):
    """achieved = algorithmic bytes / mean step-kernel time; frac against the
    given peak; traffic = per-update DRAM bytes x particles + field bytes;
    issue ceiling = SMs x 4 schedulers x the sampled clock."""
    n, N = 16777216, 256
    cnt = bench.measured_counters("scale_256", "f64", "auto", n, (256, 1, 3))
    prof = {"step": (12.0, 10), "tail": (0.24, 10), "sort": (0.6, 1)}
    clk = {"sm_mhz": 2000.0}
    r = bench.step_roofline("scale_256", "f64", "auto", n, N, True, (256, 1, 3), prof, 6000.0,
                            "measured", clk, 150)
    alg = n * 2 * (48 + 8 + 4) + 24 * N ** 3
    t = 1.2e-3
    assert r["algorithmic_bytes"] == alg
    assert r["achieved"] == pytest.approx(alg / t / 1e9, rel=1e-3)
    assert r["frac"] == pytest.approx(alg / t / 1e9 / 6000.0, rel=1e-3)
    assert r["traffic"] == int(cnt["dram_bytes_per_update"] * n + cnt["dram_field_bytes"])
    peak = 150 * 4 * 2000e6
    assert r["issue"]["frac"] == pytest.approx(cnt["warp_inst_per_update"] * n / t / peak,
                                               rel=1e-3)
    assert r["kernel_share"] == pytest.approx(12.0 / 12.84, rel=1e-3)


def test_single_rank_reduction_is_the_identity():
    assert bench.aggregate_over_ranks(12.5, 1000) == (12.5, 1000)
