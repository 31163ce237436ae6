"""bench.py end to end on the GPU with small step counts: one JSON line with
the keys and units the measurement contract asks for, consistent with each
other."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_has_the_contract_keys():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "40", "--warmup", "3",
                          "--batch-steps", "8", "--no-cpu-baseline"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "clocks",
              "gpu_launches", "batched", "single_case_storage", "data_variants"):
        assert k in d, k
    assert d["unit"] == "MLUPS" and d["steps"] == 40 and d["warmup"] == 3 and d["gpu_launches"] == 40
    N = d["config"]["nx"] * d["config"]["ny"]
    assert d["value"] == pytest.approx(N * 40 / (d["ms_per_step"] * 40 / 1e3) / 1e6, rel=1e-9)
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["achieved"] == pytest.approx(160 * N / (d["ms_per_step"] * 1e-3) / 1e9)
    e = d["e2e"]
    assert e["unit"] == "MLUPS" and 0 < e["value"] <= d["value"] * 1.05
    assert e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    b = d["batched"]
    assert b["cases"] == 64 and b["value"] > 0 and b["sequential_fp32"] > 0 and b["batched_fp32"] > 0
    assert set(b["tile"]) == {"periodic", "walls"}
    assert d["clocks"] is None or "sm_mhz" in d["clocks"]
    v = d["data_variants"]
    for k in ("perf-2048-drop", "perf-2048-eq29", "impact-2400x600-open-top"):
        assert v[k]["value"] > 0 and v[k]["unit"] == "MLUPS", k
    assert set(v["impact_tooling_us"]) == {"spreading_radius", "laplace_jump", "probe_1000"}
    assert all(t > 0 for t in v["impact_tooling_us"].values())
