"""Host-side pieces of bench.py that need no GPU: the measured-traffic figure
is taken from the committed ncu summary only while the kernel sources hash to
the value that summary records; the reference arm (the FP64 oracle on the
host cores) prints its contract line."""
import json
import os
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_source_hash_is_stable_and_hex():
    h = bench._source_hash()
    assert h == bench._source_hash()
    assert len(h) == 16 and int(h, 16) >= 0


def test_traffic_reported_only_for_the_profiled_sources(monkeypatch):
    t = bench._profiled_traffic()
    assert t is None or t > 0
    monkeypatch.setattr(bench, "_source_hash", lambda: "0" * 16)
    assert bench._profiled_traffic() is None


def test_peaks_read_from_measured_file():
    peak, kind = bench._peaks()
    assert peak > 1000 and kind in ("measured", "fallback")


def test_reference_arm_line_on_cpu():
    """bench.py --impl reference runs the FP64 oracle on the host (no GPU) and
    prints one JSON line with the contract's keys, its own cpu_baseline and an
    e2e that moves no bytes."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "3",
                          "--warmup", "3", "--reference-seconds", "2"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["higher_is_better"] is True
    assert d["steps"] == 3 and d["warmup"] == 3 and d["value"] > 0
    assert d["value"] == pytest.approx(d["config"]["nx"] * d["config"]["sample_rows"] * 3
                                       / (d["ms_per_step"] * 3 / 1e3) / 1e6, rel=1e-9)
    c = d["cpu_baseline"]
    assert c["kind"] == "oracle" and c["value"] == d["value"] and c["cores"] >= 1 and c["cpu"]
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
