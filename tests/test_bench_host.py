"""Host-side logic of bench.py, without a GPU: the batched workload's
per-group arithmetic, the DRAM-traffic record's validity check, and the
reference arm's JSON line (the CPU oracle on a small sample)."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("d,h,expect", [
    (8, 0.5, ("mixed", 0.05)), (8, 1.0, ("mixed", 0.05)), (8, 2.0, ("mixed_f64", 0.05)),
    (8, 4.0, ("mixed_f64", 0.02)), (32, 0.5, ("mixed", 0.05)), (32, 1.0, ("mixed", 0.05)),
    (32, 2.0, ("mixed", 0.05)), (32, 4.0, ("mixed_f64", 0.05)), (128, 0.5, ("mixed", 0.05)),
    (128, 1.0, ("mixed", 0.05)), (128, 2.0, ("mixed", 0.05)), (128, 4.0, ("mixed", 0.05)),
])
def test_batch_group_rules(d, h, expect):
    """d / h^2 <= 2: FP64 decompositions and factorization; <= 0.5: also
    eps_c 0.02; every group keeps the workload's sample budget."""
    W = bench.BATCH_WL
    prec, eps_c, r_max = bench.group_precision(d, h, W["eps_c"], W["r_max"])
    assert (prec, eps_c) == expect
    assert r_max == W["r_max"]


def test_workload_keys():
    assert bench.IMAGE_WL["eps_c"] == 0.01 and bench.IMAGE_WL["eps_c_orderings"] == 0.05
    assert bench.WL["n"] == 65536 and bench.WL["d"] == 8


def test_traffic_record_follows_the_kernel_source(monkeypatch):
    rec = open(os.path.join(ROOT, "profiles", "sample_tc_traffic.txt")).read()
    sha = [ln.split()[1] for ln in rec.splitlines() if ln.startswith("kernel_source_sha1")][0]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: sha)
    v = bench._traffic()
    assert isinstance(v, int) and v > 0
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 40)
    assert bench._traffic() is None   # another kernel source: no traffic figure


def test_reference_arm_line(monkeypatch, capsys):
    """`--impl reference` prints one JSON line with the contract's keys; a
    512-point sample keeps this test short."""
    monkeypatch.setattr(bench, "CPU_SAMPLE_N", 512)

    class A:
        steps, warmup = 1, 0

    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    bench.run_reference(A())
    out = capsys.readouterr().out.strip().splitlines()
    assert len(out) == 1
    d = json.loads(out[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "s"
    assert d["higher_is_better"] is False and d["value"] > 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["timed_n"] == 512 and cb["cores"] >= 1
    assert "n=512" in cb["sample"]


def test_reference_arm_silent_on_other_ranks(monkeypatch, capsys):
    class A:
        steps, warmup = 1, 0

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
