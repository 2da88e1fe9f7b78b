"""Map dump / load round trip (CPU): every array bit for bit, 16-bit storage kept as is."""
import numpy as np
import torch

from paper_2509_06433_gb300 import api, checkpoint
from scenes import make_scene


def test_round_trip_float32_and_16_bit(tmp_path):
    s = make_scene("fwd10k", n=500)
    for dt in (torch.float32, torch.bfloat16, torch.float16):
        g = api.Gaussians.from_numpy(s.params(), device="cpu", dtype=dt)
        cams = torch.as_tensor(s.cams)
        p = str(tmp_path / f"map_{str(dt)[6:]}.npz")
        checkpoint.save(p, g, cams, sh_degree=None)
        g2, c2, extras = checkpoint.load(p, device="cpu")
        for n in ("means", "log_scales", "quats", "opacity_logits", "rgb"):
            a, b = getattr(g, n), getattr(g2, n)
            assert a.dtype == b.dtype and a.shape == b.shape
            assert torch.equal(a.view(torch.int16) if a.element_size() == 2 else a,
                               b.view(torch.int16) if b.element_size() == 2 else b), n
        assert torch.equal(c2, cams) and extras["adam_state"] is None and extras["sh_degree"] is None


def test_round_trip_with_optimiser_state(tmp_path):
    s = make_scene("fwd10k", n=300)
    g = api.Gaussians.from_numpy(s.params(), device="cpu", dtype=torch.bfloat16)

    class Opt:  # the fields checkpoint reads from api.MapOptimizer
        pass
    opt = Opt()
    opt.state = torch.arange(2 * 14 * 300 + 1, dtype=torch.float32)
    opt.storage = g
    opt.masters = api.Gaussians.from_numpy(s.params(), device="cpu")
    p = str(tmp_path / "map.npz")
    checkpoint.save(p, g, optimizer=opt, sh_degree=2)
    g2, c2, extras = checkpoint.load(p, device="cpu")
    assert c2 is None and extras["sh_degree"] == 2
    assert torch.equal(extras["adam_state"], opt.state)
    assert torch.equal(extras["masters"].means, opt.masters.means)
    np.testing.assert_array_equal(g2.rgb.float().numpy(), g.rgb.float().numpy())
