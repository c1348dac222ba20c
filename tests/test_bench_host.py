"""CPU checks of bench.py's host side: the reference arm (the FP64 oracle timed
on the host cores) prints one JSON line carrying every key of the benchmark
contract, and the oracle baseline extrapolates from a stored oracle run only
when that run is of the same workload. Both run on a small workload (n = 1024,
tol 1e-6) so that they finish in seconds."""

import argparse
import contextlib
import io
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import dcg_synth as S  # noqa: E402

SMALL_TOL6 = S.RBFSequence(**{**S.SMALL_1024.__dict__, "tol": 1e-6})


@pytest.fixture
def small_cfg(monkeypatch):
    monkeypatch.setattr(bench, "CFG", SMALL_TOL6)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    return SMALL_TOL6


def test_golden_lookup_matches_workload_and_tolerance(monkeypatch):
    monkeypatch.setattr(bench, "CFG", S.DENSE_16384)
    total, src = bench._golden_total_matvecs()
    assert src == "tests/golden/dense_16384_oracle.json" and total > 0
    # the stored small run was taken at tol 1e-6; the small workload's own
    # tolerance (1e-8) must not borrow its matvec count
    monkeypatch.setattr(bench, "CFG", S.SMALL_1024)
    assert bench._golden_total_matvecs() == (None, None)
    monkeypatch.setattr(bench, "CFG", SMALL_TOL6)
    total, src = bench._golden_total_matvecs()
    assert src == "tests/golden/small_1024_tol1e-6_oracle.json"
    with open(os.path.join(ROOT, src)) as f:
        assert total == json.load(f)["total_defcg_matvecs"]


def test_reference_arm_prints_the_contract_line(small_cfg):
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.reference_arm(argparse.Namespace(steps=2, warmup=1))
    lines = [l for l in buf.getvalue().splitlines() if l.strip()]
    assert len(lines) == 1
    out = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in out, key
    assert out["impl"] == "reference" and out["metric"] == bench.METRIC
    assert out["steps"] == 2 and out["warmup"] == 1 and out["n_gpus"] == 1
    assert out["higher_is_better"] is False and out["unit"] == "s/sequence"
    assert out["value"] > 0
    assert out["config"]["workload"] == small_cfg.name and out["config"]["n"] == small_cfg.n
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == out["value"] and cb["cores"] >= 1
    assert f"n={small_cfg.n}" in cb["sample"] and "small_1024_tol1e-6_oracle.json" in cb["sample"]
    e2e = out["e2e"]
    assert e2e["value"] == out["value"] and e2e["unit"] == out["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_cpu_baseline_is_bounded_and_extrapolated(small_cfg):
    cb = bench.cpu_baseline(samples=2, min_seconds=0.05)
    assert cb["kind"] == "oracle" and cb["unit"] == "s/sequence" and cb["value"] > 0
    assert cb["cores"] >= 1
    assert f"n={small_cfg.n}" in cb["sample"]
    assert "extrapolated by matvec count" in cb["sample"]
