"""The index-checking debug build (GS_DEBUG=1) renders and differentiates exactly like the
release build and reports no failed index check on a valid workload."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, ".")
from scenes import make_scene, random_image
from paper_2509_06433_gb300 import api
s = make_scene("window500k", n=20000, K=3, W=160, H=120, f=130.0)
g = api.Gaussians.from_numpy(s.params())
ct = torch.as_tensor(s.cams).cuda()
r = api.Rasterizer(s.W, s.H, s.K, s.N)
r.plan(g, ct)
out = r.render(g, ct)
gr = torch.as_tensor(random_image(1, (s.K, 3, s.H, s.W))).cuda()
gd = torch.as_tensor(random_image(2, (s.K, s.H, s.W))).cuda()
grads = r.backward(g, ct, out, gr, gd)
code, err, total, _ = r.status()
np.savez(sys.argv[1], err=err, **{k: v.cpu().numpy() for k, v in out.items()},
         **{"g_" + k: v.cpu().numpy() for k, v in grads.items()})
"""


def run(path, debug):
    env = dict(os.environ)
    env.pop("GS_DEBUG", None)
    if debug:
        env["GS_DEBUG"] = "1"
    res = subprocess.run([sys.executable, "-c", SCRIPT, path], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=600)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-2000:]
    return np.load(path)


def test_debug_build_equals_release_build(tmp_path):
    from paper_2509_06433_gb300.build import build
    build(debug=True)
    rel = run(str(tmp_path / "rel.npz"), False)
    dbg = run(str(tmp_path / "dbg.npz"), True)
    assert int(dbg["err"]) == 0 and int(rel["err"]) == 0
    for k in rel.files:
        assert np.array_equal(rel[k], dbg[k]), k
