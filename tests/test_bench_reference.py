"""The benchmark's reference arm: the FP64 oracle timed for exactly --steps steps after
--warmup untimed ones, printed as the same JSON line as the GPU arm (CPU only). The oracle's
inputs are shrunk here (a 20k-Gaussian, 2-view, 320x180 aerial scene) so the test runs in
seconds; the line and the sampling logic are those of the full workload."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _small_inputs(monkeypatch):
    import bench
    import scenes
    full = scenes.make_scene
    monkeypatch.setattr(scenes, "make_scene", lambda name: full(name, n=20000, K=2, W=320, H=180, f=225.0))
    return bench


def test_reference_arm_line(monkeypatch):
    bench = _small_inputs(monkeypatch)
    args = bench.parse(["--impl", "reference", "--steps", "3", "--warmup", "1", "--ref-seconds", "600"])
    d = bench.reference_line(args, 1)
    assert d["impl"] == "reference" and d["steps"] == 3 and d["warmup"] == 1
    assert d["value"] > 0 and d["unit"] == "mapping iters/s" and d["dtype"] == "f64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("aerial2m") and d["config"]["K"] == 16
    # a generous budget: every step is a whole view
    assert "rows [0, 180) of one 320x180 view" in d["cpu_baseline"]["sample"]


def test_reference_arm_samples_a_band_of_rows_on_a_short_budget(monkeypatch):
    bench = _small_inputs(monkeypatch)
    rate, cb, ms = bench.oracle_reference_run(2, 1, budget_s=1e-3)
    assert rate > 0 and ms > 0
    assert "rows [80, 96) of one 320x180 view" in cb["sample"] and "1/2 views" in cb["sample"]
