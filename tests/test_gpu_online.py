"""Online mapping of a key-frame sequence (insertion + windowed mapping graph with Adam) on
the GPU: every frame's view converges, empty slots stay untouched, and the reported PSNR /
SSIM equal the metric oracle's on the same rendered images."""
import numpy as np
import pytest

from oracle import metrics as OM
from scenes import make_scene

pytestmark = pytest.mark.gpu


def test_turn_sequence_converges():
    import torch
    from paper_2509_06433_gb300 import api, online
    s = make_scene("turn_room", n=100_000, K=4, W=336, H=188, f=130.0)
    g = api.Gaussians.from_numpy(s.params())
    cams = torch.as_tensor(s.cams.reshape(-1, 16)).cuda().contiguous()
    r = api.Rasterizer(s.W, s.H, s.K, s.N)
    r.plan(g, cams)
    kf = r.render(g, cams)
    cover = 1.0 - kf["T"]
    depth = torch.where(cover > 0.5, kf["depth"] / cover.clamp_min(1e-6), torch.zeros_like(cover))
    frames = [(kf["rgb"][k].contiguous(), depth[k].contiguous(), cams[k].contiguous()) for k in range(s.K)]
    C = 60_000
    m = online.OnlineMapper(s.W, s.H, capacity=C, window=3)
    rec = online.map_sequence(m, frames, iters_per_frame=60, eval_every=20, thresholds=(20.0, 25.0))
    assert m.count == sum(rc["added"] for rc in rec) and 0 < m.count < C
    for rc in rec:
        assert rc["curve"][-1][2] >= 25.0, rc["curve"]
        assert rc["t_reach"][20.0] is not None
        times = [c[0] for c in rc["curve"]]
        assert all(b > a for a, b in zip(times, times[1:]))
    assert not m.overflowed()
    # slots past the map's count were never touched
    assert torch.all(m.g.opacity_logits[m.count:] == online.EMPTY_LOGIT)
    assert torch.all(m.g.means[m.count:] == 0)
    # the GPU metrics of the final render against the metric oracle
    out = m.render(cams[-1])
    x = out["rgb"].cpu().numpy()
    y = kf["rgb"][-1:].cpu().numpy()
    p, q = online.evaluate(m, kf["rgb"][-1], cams[-1])
    assert abs(p - OM.psnr(x, y)[0]) < 1e-3
    assert abs(q - OM.ssim(x, y)[0][0]) < 1e-4
