"""GPU PSNR / SSIM against the FP64 metric oracle (per image, and the SSIM map per pixel)."""
import numpy as np
import pytest

from oracle import metrics as OM

pytestmark = pytest.mark.gpu


def mods():
    import torch
    from paper_2509_06433_gb300 import api
    return torch, api


def pair(seed, shape, noise):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, shape).astype(np.float32)
    # smooth structure plus noise, so SSIM is neither ~0 nor ~1
    y = np.clip(x + rng.normal(0, noise, shape), 0, 1).astype(np.float32)
    return x, y


@pytest.mark.parametrize("shape,noise", [((3, 3, 480, 640), 0.05), ((2, 3, 37, 53), 0.2), ((1, 1, 16, 16), 0.1),
                                         ((1, 3, 376, 672), 0.02)])
def test_psnr_ssim_match_oracle(shape, noise):
    torch, api = mods()
    x, y = pair(sum(shape), shape, noise)
    xd, yd = torch.as_tensor(x).cuda(), torch.as_tensor(y).cuda()
    ps = api.gs_psnr(xd, yd).cpu().numpy()
    smap = torch.empty_like(xd)
    ss = api.gs_ssim(xd, yd, ssim_map=smap).cpu().numpy()
    ref_p = OM.psnr(x, y)
    ref_s, ref_map = OM.ssim(x, y)
    assert np.abs(ps - ref_p).max() < 1e-4, (ps, ref_p)
    assert np.abs(ss - ref_s).max() < 1e-5, (ss, ref_s)
    # per pixel: FP32 moments, variance by E[x^2] - mu^2, amplified by at most 1 / C2
    assert np.abs(smap.cpu().numpy() - ref_map).max() < 2e-3


def test_metric_edge_cases():
    torch, api = mods()
    x = torch.rand(2, 3, 40, 24, device="cuda")
    assert torch.isinf(api.gs_psnr(x, x)).all()
    assert torch.allclose(api.gs_ssim(x, x), torch.ones(2, device="cuda"), atol=1e-5)
    # data range 255: the same images scaled by 255 give the same PSNR and SSIM
    y = (x + 0.05 * torch.randn_like(x)).clamp(0, 1)
    p1, p2 = api.gs_psnr(x, y), api.gs_psnr(x * 255, y * 255, data_range=255.0)
    assert torch.allclose(p1, p2, atol=1e-3)
    s1, s2 = api.gs_ssim(x, y), api.gs_ssim(x * 255, y * 255, data_range=255.0)
    assert torch.allclose(s1, s2, atol=1e-4)
    # deterministic
    assert torch.equal(api.gs_ssim(x, y), s1) and torch.equal(api.gs_psnr(x, y), p1)
    from paper_2509_06433_gb300._lib import GsError
    with pytest.raises(GsError):
        api.gs_psnr(x, y, data_range=0.0)
