"""Per-output error of the GPU path against the FP64 oracle, per storage precision.

Prints one line per (workload, storage): max |error| of RGB, depth and T over the pixels
without a threshold-adjacent decision, the number of such pixels, and the relative L2
error of every gradient tensor. Asserts the parity bar (1e-4 max-abs, 1e-3 relative L2).
"""
import numpy as np
import pytest

import oracle
from scenes import make_scene, random_image
from tests.gpu_common import GRAD_RTOL, IMG_ATOL, check_images, gpu_render, rel_l2, to_np, torch_mods

pytestmark = pytest.mark.gpu

CASES = [
    ("fwd10k 320x240", lambda: make_scene("fwd10k"), "f32"),
    ("map100k 640x480", lambda: make_scene("map100k"), "f32"),
    ("map100k 640x480", lambda: make_scene("map100k"), "bf16"),
    ("window 20k K=3 160x120", lambda: make_scene("window500k", n=20000, K=3, W=160, H=120, f=130.0), "bf16"),
    ("aerial 30k K=2 320x180", lambda: make_scene("aerial2m", n=30000, K=2, W=320, H=180, f=225.0), "f16"),
]


@pytest.mark.parametrize("label,mk,storage", CASES)
def test_error_report(label, mk, storage):
    torch, api = torch_mods()
    dt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[storage]
    s = mk()
    stored = [torch.as_tensor(a).to(dt).float().numpy() for a in s.params()[1:]]
    params = (s.means,) + tuple(stored)
    orc = oracle.forward(params, s.cams, s.W, s.H)
    r, g, ct, out = gpu_render(s.params(), s.cams, s.W, s.H, dtype=dt)
    o = to_np(out)
    check_images(o, orc)
    clean = orc["near"] == 0
    err = {k: float(np.abs(o[k].astype(np.float64) - orc[k])[(clean[:, None] if k == "rgb" else clean)
                                                           if k != "rgb" else np.broadcast_to(clean[:, None], o[k].shape)].max())
           for k in ("rgb", "depth", "T")}
    gr, gd = random_image(41, (s.K, 3, s.H, s.W)), random_image(42, (s.K, s.H, s.W))
    og = oracle.backward(params, s.cams, s.W, s.H, orc["lists"], gr, gd)
    grads = to_np(r.backward(g, ct, out, torch.as_tensor(gr).cuda(), torch.as_tensor(gd).cuda()))
    gerr = {k: rel_l2(grads[k], og[k]) for k in ("means", "log_scales", "quats", "opacity_logits", "rgb", "pose")}
    print(f"\nERRORS | {label} | {storage} | rgb {err['rgb']:.2e} | depth {err['depth']:.2e} | T {err['T']:.2e} | "
          f"near px {int((orc['near'] > 0).sum())} | " + " | ".join(f"{k} {v:.1e}" for k, v in gerr.items()))
    assert max(err.values()) <= IMG_ATOL
    assert max(gerr.values()) < GRAD_RTOL
