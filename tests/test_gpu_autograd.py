"""The torch.autograd.Function wrappers: gradients equal the C-ABI backward bit for bit and
the FP64 oracle within the parity tolerance; a directional finite difference through the
Function agrees in the colours; the pose-only form gives the same pose gradient; a second
render before the backward is refused."""
import numpy as np
import pytest

import oracle
from scenes import make_scene, random_image
from tests.gpu_common import GRAD_RTOL, rel_l2, torch_mods

pytestmark = pytest.mark.gpu


def _setup(n=3000, W=96, H=64, f=80.0):
    torch, api = torch_mods()
    s = make_scene("map100k", n=n, W=W, H=H, f=f)
    g = api.Gaussians.from_numpy(s.params())
    cams = torch.as_tensor(s.cams).cuda()
    r = api.Rasterizer(s.W, s.H, s.K, s.N, pair_capacity=1 << 18)
    r.plan(g, cams)
    wr = torch.as_tensor(random_image(31, (s.K, 3, s.H, s.W))).cuda()
    wd = torch.as_tensor(random_image(32, (s.K, s.H, s.W))).cuda()
    return torch, api, s, g, cams, r, wr, wd


def _leaves(torch, g):
    return [t.clone().requires_grad_(True) for t in (g.means, g.log_scales, g.quats, g.opacity_logits, g.rgb)]


def test_autograd_gradients_equal_the_abi_backward_and_the_oracle():
    torch, api, s, g, cams, r, wr, wd = _setup()
    from paper_2509_06433_gb300 import autograd as ga
    leaves = _leaves(torch, g)
    xi = torch.zeros((s.K, 6), device="cuda", requires_grad=True)
    rgb, depth, T = ga.render(r, *leaves, cams, xi)
    ((rgb * wr).sum() + (depth * wd).sum()).backward()
    out = r.render(g, cams)
    ref = r.backward(g, cams, out, wr.contiguous(), wd.contiguous())
    for name, leaf in zip(("means", "log_scales", "quats", "opacity_logits", "rgb"), leaves):
        assert torch.equal(leaf.grad, ref[name]), name
    assert torch.equal(xi.grad, ref["pose"])
    o = oracle.forward(s.params(), s.cams, s.W, s.H)
    og = oracle.backward(s.params(), s.cams, s.W, s.H, o["lists"], wr.cpu().numpy().astype(np.float64),
                         wd.cpu().numpy().astype(np.float64))
    for name, leaf in zip(("means", "log_scales", "quats", "opacity_logits", "rgb"), leaves):
        assert rel_l2(leaf.grad.cpu().numpy(), og[name]) < GRAD_RTOL, name
    assert rel_l2(xi.grad.cpu().numpy(), og["pose"]) < GRAD_RTOL


def test_directional_finite_difference_of_the_render_in_the_colours():
    """The render is linear in the colours (no decision depends on them), so a central
    difference through the Function is exact up to FP32 rounding. (In the geometric
    parameters the render jumps wherever a pixel crosses the alpha = 1/255 contour, so their
    gradients are checked against the oracle, whose own pins use guarded differences.)"""
    torch, api, s, g, cams, r, wr, wd = _setup()
    from paper_2509_06433_gb300 import autograd as ga
    leaves = _leaves(torch, g)
    rgb, depth, T = ga.render(r, *leaves, cams)
    ((rgb * wr).sum() + (depth * wd).sum()).backward()
    gen = torch.Generator(device="cuda").manual_seed(4)
    d = torch.randn(leaves[4].shape, generator=gen, device="cuda")
    h = 1e-2
    vals = []
    for sgn in (1.0, -1.0):
        p = [t.detach().clone() for t in leaves]
        p[4] = p[4] + sgn * h * d
        with torch.no_grad():
            a, b, _ = ga.render(r, *p, cams)
            vals.append(((a.double() * wr.double()).sum() + (b.double() * wd.double()).sum()).item())
    fd = (vals[0] - vals[1]) / (2 * h)
    an = (leaves[4].grad.double() * d.double()).sum().item()
    assert abs(fd - an) <= 1e-4 * abs(an) + 1e-4, (fd, an)


def test_pose_only_render_gives_the_full_renders_pose_gradient():
    torch, api, s, g, cams, r, wr, wd = _setup()
    from paper_2509_06433_gb300 import autograd as ga
    xi = torch.zeros((s.K, 6), device="cuda", requires_grad=True)
    rgb, depth, _ = ga.render_pose(r, g, cams, xi)
    ((rgb * wr).sum() + (depth * wd).sum()).backward()
    leaves = _leaves(torch, g)
    xi2 = torch.zeros((s.K, 6), device="cuda", requires_grad=True)
    rgb2, depth2, _ = ga.render(r, *leaves, cams, xi2)
    ((rgb2 * wr).sum() + (depth2 * wd).sum()).backward()
    assert torch.equal(xi.grad, xi2.grad)
    assert torch.count_nonzero(xi.grad).item() > 0


def test_second_render_before_backward_is_refused():
    torch, api, s, g, cams, r, wr, wd = _setup()
    from paper_2509_06433_gb300 import autograd as ga
    leaves = _leaves(torch, g)
    rgb, depth, _ = ga.render(r, *leaves, cams)
    ga.render(r, *[t.detach() for t in leaves], cams)
    with pytest.raises(RuntimeError, match="rendered again"):
        (rgb.sum() + depth.sum()).backward()
    with pytest.raises(ValueError):
        ga.render(r, *leaves, cams, torch.ones((s.K, 6), device="cuda"))
