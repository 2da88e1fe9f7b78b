"""The benchmark's JSON line (a short run on the GPU): every field of the contract, with the
types and relations it promises."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line():
    out = subprocess.run([sys.executable, "bench.py", "--steps", "20", "--warmup", "3", "--no-extra",
                          "--no-cpu-baseline", "--px", "4,4"], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-3000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "e2e", "gpu_launches", "roofline", "clocks"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 20 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["scaling"] == "weak" and d["vs_baseline"] is None and d["dtype"] == "f32"
    assert d["value"] > 0 and abs(d["value"] * d["ms_per_step"] / 1e3 - 1.0) < 1e-6
    assert d["config"]["workload"].startswith("aerial2m") and d["config"]["K"] == 16 and "l2" in d["config"]
    assert d["config"]["storage"] == "f16"
    e = d["e2e"]
    assert 0 < e["value"] < d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] > 10_000_000 and e["d2h_bytes_per_step"] > 5_000_000
    # per step: the projection and the live-item compaction (2), the 11 kernels of gs_bin_sort at
    # 16 x 1280x720, the fused forward + backward compositing, and the backward projection (live
    # items, per-Gaussian sums and chain rule, the pose reduction)
    assert d["gpu_launches"] == 20 * (2 + 11 + 1 + 3)
    assert d["roofline"]["kernel"] == "raster_fwd_l1_bwd"
    r = d["roofline"]
    assert r["bound"] in ("alu", "hbm") and r["unit"] in ("TFLOP/s", "GB/s")
    assert 0 < r["frac"] < 1.5 and abs(r["achieved"] / r["peak"] - r["frac"]) < 1e-9
    c = d["clocks"]
    assert c["samples"] >= 1 and c["sm_mhz"] and c["sm_max_mhz"]
