"""Host logic of bench.py that needs no GPU: the graph-quality formula, the
recall record's comparison with the sequential oracle, the stored oracle
recall it reads, and the rule that ties the committed ncu traffic to the
search kernel's source."""
import argparse
import math

import bench
from paper_1602_06819_gb300 import inputs


def test_quality_q_is_the_oracle_formula(orc):
    for e_c, n, n_a, k in [(900_000, 100_000, 25_600, 10), (10_000, 1000, 1000, 10), (0, 50, 7, 3)]:
        assert math.isclose(bench.quality_q(e_c, n, n_a, k), orc.quality_q(e_c, n, n_a, k), rel_tol=1e-12)


def test_recall_record_holds_batches_to_the_oracle_within_0_01():
    seq = {"edge_recall": 0.86, "inserted_recall": 0.88}
    ok = bench.recall_record(0.865, 0.889, 0.6, 125_600, seq)
    assert ok["delta_vs_oracle"]["within"] and not ok["target_met"]
    far = bench.recall_record(0.865, 0.869, 0.6, 125_600, seq)
    assert not far["delta_vs_oracle"]["within"]
    assert "delta_vs_oracle" not in bench.recall_record(0.9, 0.9, 0.7, 10, None)


def test_sequential_oracle_recall_reads_the_fixture():
    args = argparse.Namespace(speedup=4.0, expansion=5.0, depth=2, storage="fp32", order="none")
    rec = bench.sequential_oracle_recall(args, inputs.PLAIN_D128, 25_600)
    assert rec is not None and 0.0 < rec["edge_recall"] < 1.0 and 0.0 < rec["inserted_recall"] < 1.0
    assert bench.sequential_oracle_recall(args, inputs.PLAIN_D128, 12_345) is None
    other = argparse.Namespace(speedup=8.0, expansion=5.0, depth=2, storage="fp32", order="none")
    assert bench.sequential_oracle_recall(other, inputs.PLAIN_D128, 25_600) is None


def test_traffic_only_for_the_captured_source(monkeypatch):
    text = open(bench.SEARCH_PROFILE).read()
    committed = [ln for ln in text.splitlines() if ln.startswith("traffic_bytes_per_launch:")][0]
    traffic, src = bench.profiled_traffic()
    if traffic is not None:   # the summary was taken on the current source
        assert traffic == float(committed.split(":")[1]) and src.startswith("profiles/")
    monkeypatch.setattr(bench, "search_source_hash", lambda: "0" * 16)
    assert bench.profiled_traffic() == (None, None)


def test_source_hash_ignores_comments_and_spacing(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1602_06819_gb300" / "csrc"
    csrc.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "SEARCH_SOURCES", ["a.cuh"])
    (csrc / "a.cuh").write_text("int x = 1;  // one\n/* block */ int y;\n")
    h1 = bench.search_source_hash()
    (csrc / "a.cuh").write_text("int   x = 1;\n\n int y; // another comment\n")
    assert bench.search_source_hash() == h1
    (csrc / "a.cuh").write_text("int x = 2; int y;\n")
    assert bench.search_source_hash() != h1


def _bench(*args, env=None):
    import json
    import os
    import subprocess
    import sys
    e = dict(os.environ, **(env or {}))
    out = subprocess.run([sys.executable, os.path.join(os.path.dirname(bench.__file__), "bench.py"), *args],
                         capture_output=True, text=True, timeout=600, env=e)
    assert out.returncode == 0, out.stderr[-2000:]
    return [json.loads(ln) for ln in out.stdout.splitlines() if ln.startswith("{")]


def test_reference_arm_prints_one_line_on_the_host():
    """The reference arm is the oracle on the host cores: one JSON line with
    the line's metric, the oracle as cpu_baseline and an e2e that moves no
    bytes; it needs no GPU."""
    lines = _bench("--impl", "reference", "--workload", "small", "--steps", "2", "--warmup", "3")
    assert len(lines) == 1
    ln = lines[0]
    assert ln["impl"] == "reference" and ln["metric"] == bench.METRIC and ln["unit"] == bench.UNIT
    assert ln["higher_is_better"] is True and ln["steps"] == 2 and ln["warmup"] == 3
    assert ln["value"] > 0 and ln["cpu_baseline"]["value"] == ln["value"]
    assert ln["cpu_baseline"]["kind"] == "oracle" and ln["cpu_baseline"]["cores"] == 1
    assert ln["e2e"] == {"value": ln["value"], "unit": ln["unit"], "h2d_bytes_per_step": 0,
                         "d2h_bytes_per_step": 0}
    assert ln["config"]["workload"] == "gmm-d16-n1k+1k-k10-batch1"


def test_reference_arm_other_ranks_print_nothing():
    assert _bench("--impl", "reference", "--workload", "small", "--steps", "2", "--warmup", "3",
                  env={"RANK": "1", "WORLD_SIZE": "2"}) == []


def test_extra_records_fail_in_place(capsys):
    """An auxiliary record that raises leaves its error in the line instead
    of losing the line."""
    assert bench.guarded("x", lambda a, b=0: a + b, 2, b=3) == 5

    def boom():
        raise RuntimeError("out of memory")
    assert bench.guarded("precision", boom) == {"error": "RuntimeError: out of memory"}
    assert "precision record failed" in capsys.readouterr().err
