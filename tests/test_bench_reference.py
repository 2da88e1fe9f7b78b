"""The benchmark's reference arm: the FP64 oracle timed for exactly --steps steps after
--warmup untimed ones, printed as the same JSON line as the GPU arm (CPU only)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["unit"] == "mapping iters/s" and d["dtype"] == "f64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "whole 640x480 view" in d["cpu_baseline"]["sample"]


def test_reference_arm_samples_a_band_of_rows_on_a_short_budget():
    sys.path.insert(0, ROOT)
    import bench
    rate, cb, ms = bench.oracle_reference_run(2, 1, budget_s=0.5)
    assert rate > 0 and ms > 0
    assert "rows [" in cb["sample"] and "scaled to full-view steps" in cb["sample"]
