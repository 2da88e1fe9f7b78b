"""The mapping loop on the GPU: the Adam step against the FP64 oracle (FP32 masters and
reduced-storage copies), the captured mapping iteration with its optimiser against eager
execution and its loss going down, and key-frame insertion against the oracle."""
import numpy as np
import pytest

import oracle
from oracle import mapping as om
from scenes import make_scene, random_image
from tests.gpu_common import torch_mods

pytestmark = pytest.mark.gpu

LR = {"means": 1e-3, "log_scales": 5e-3, "quats": 1e-3, "opacity_logits": 5e-2, "rgb": 2.5e-3}


@pytest.mark.parametrize("color_width", [3, 48])  # RGB, or SH coefficients of degree 3
def test_adam_steps_match_the_oracle(color_width):
    torch, api = torch_mods()
    rng = np.random.default_rng(0)
    N = 3001
    widths = om.WIDTHS[:-1] + (color_width,)
    p0 = {k: rng.normal(size=(N, w)).astype(np.float32).reshape((N,) if w == 1 else (N, w))
          for k, w in zip(om.GROUPS, widths)}
    masters = api.Gaussians(*(torch.as_tensor(p0[k]).cuda() for k in om.GROUPS))
    store = api.Gaussians(masters.means.clone(), *(masters_t.to(torch.bfloat16) for masters_t in
                                                    (masters.log_scales, masters.quats, masters.opacity_logits,
                                                     masters.rgb)))
    state = torch.zeros(api.gs_map_adam_state_size(N, color_width), device="cuda")
    assert state.numel() == 2 * (11 + color_width) * N + 1
    ref = {k: p0[k].astype(np.float64) for k in om.GROUPS}
    m = {k: np.zeros_like(v) for k, v in ref.items()}
    v = {k: np.zeros_like(x) for k, x in ref.items()}
    for t in range(1, 4):
        g = {k: rng.normal(size=p0[k].shape).astype(np.float32) for k in om.GROUPS}
        gt = {k: torch.as_tensor(g[k]).cuda() for k in om.GROUPS}
        api.gs_map_adam_step(masters, gt, state, LR, 0.9, 0.999, 1e-8, storage=store)
        om.adam_step(ref, g, m, v, t, LR, 0.9, 0.999, 1e-8)
    torch.cuda.synchronize()
    assert state[-1].item() == 3.0
    for k in om.GROUPS:
        got = getattr(masters, k).cpu().numpy().astype(np.float64)
        np.testing.assert_allclose(got, ref[k], rtol=0, atol=2e-6 * max(1.0, np.abs(ref[k]).max()))
        st = getattr(store, k)
        if k == "means":  # an FP32 storage copy of the means (a separate array) receives the values as they are
            assert torch.equal(st, masters.means)
        else:  # BF16 copies: the masters rounded to nearest
            assert torch.equal(st, getattr(masters, k).to(torch.bfloat16)), k


def test_mapping_step_with_adam_graph_equals_eager_and_reduces_the_loss():
    torch, api = torch_mods()
    from paper_2509_06433_gb300.tracking import MappingStep
    s = make_scene("map100k", n=20000, W=160, H=120, f=130.0)
    t = s.target
    cams = torch.as_tensor(s.cams).cuda()
    r = api.Rasterizer(s.W, s.H, s.K, s.N, pair_capacity=1 << 20)
    tgt = r.render(api.Gaussians.from_numpy(t.params()), cams)
    losses = {}
    finals = {}
    for graph in (True, False):
        g = api.Gaussians.from_numpy(s.params())
        r.plan(g, cams)
        opt = api.MapOptimizer(g, lr={"means": 1e-3})
        m = MappingStep(r, g, cams, tgt["rgb"].clone(), tgt["depth"].clone(), graph=graph, optimizer=opt)
        ls = []
        for _ in range(25):
            m.replay()
            ls.append(m.loss.item())
        losses[graph] = ls
        finals[graph] = [x.clone() for x in (g.means, g.log_scales, g.quats, g.opacity_logits, g.rgb)]
        assert r.status()[0] == 0
    assert losses[True] == losses[False]
    for a, b in zip(finals[True], finals[False]):
        assert torch.equal(a, b)
    assert losses[True][-1] < 0.8 * losses[True][0], losses[True]


def test_keyframe_insertion_matches_the_oracle():
    torch, api = torch_mods()
    rng = np.random.default_rng(5)
    s = make_scene("map100k", n=5000, W=160, H=120, f=130.0)
    cam = s.cams[0]
    r = api.Rasterizer(s.W, s.H, 1, s.N, pair_capacity=1 << 18)
    g = api.Gaussians.from_numpy(s.params())
    ct = torch.as_tensor(s.cams).cuda()
    r.plan(g, ct)
    out = r.render(g, ct)
    depth = rng.uniform(0.5, 6.0, (s.H, s.W)).astype(np.float32)
    depth[rng.uniform(size=depth.shape) < 0.1] = 0.0
    rgb = rng.uniform(size=(3, s.H, s.W)).astype(np.float32)
    T = out["T"][0].cpu().numpy()
    cap = 4000
    dst = api.Gaussians(*(torch.full(shape, -7.0, device="cuda") for shape in
                          ((cap, 3), (cap, 3), (cap, 4), (cap,), (cap, 3))))
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    first = 10
    api.gs_keyframe_insert(ct[0], torch.as_tensor(rgb).cuda(), torch.as_tensor(depth).cuda(), out["T"][0], dst,
                           first, count, stride=3, near=0.2, t_min=0.3, scale_factor=0.5, logit0=-1.0)
    torch.cuda.synchronize()
    ref = om.keyframe_gaussians(rgb, depth, cam, stride=3, near=0.2, T=T, t_min=0.3, scale_factor=0.5, logit0=-1.0)
    n = int(count.item())
    assert n == len(ref[0]) > 50
    got = [x.cpu().numpy() for x in (dst.means, dst.log_scales, dst.quats, dst.opacity_logits, dst.rgb)]
    assert np.all(got[0][:first] == -7.0) and np.all(got[0][first + n:] == -7.0)
    for a, b, tol in zip(got, ref, (2e-5, 2e-6, 0, 0, 0)):
        np.testing.assert_allclose(a[first:first + n], b, rtol=tol, atol=tol * 10)
    # capacity: only the room left is written
    count.zero_()
    api.gs_keyframe_insert(ct[0], torch.as_tensor(rgb).cuda(), torch.as_tensor(depth).cuda(), None, dst,
                           cap - 5, count, stride=3)
    torch.cuda.synchronize()
    assert int(count.item()) == 5


def test_host_mapping_step_equals_device_step():
    """HostMappingStep (copies from pinned host buffers, the iteration, copies back; one graph)
    returns the device MappingStep's gradients and loss bit for bit, and follows new host inputs."""
    torch, api = torch_mods()
    from paper_2509_06433_gb300.tracking import HostMappingStep, MappingStep
    s = make_scene("map100k", n=20_000, W=160, H=120, f=130.0)
    t = s.target
    cams = torch.as_tensor(s.cams).cuda()
    r = api.Rasterizer(s.W, s.H, 1, s.N)
    gt = api.Gaussians.from_numpy(t.params())
    r.plan(gt, cams)
    tgt = r.render(gt, cams)
    rgb_t, depth_t = tgt["rgb"].clone(), tgt["depth"].clone()
    g = api.Gaussians.from_numpy(s.params())
    r.plan(g, cams)
    dev = MappingStep(r, g, cams, rgb_t, depth_t, graph=True)
    dev.replay()
    host = HostMappingStep(r, api.Gaussians(*(torch.as_tensor(a) for a in s.params())), cams.cpu(), rgb_t.cpu(),
                           depth_t.cpu(), graph=True)
    host.replay()
    torch.cuda.synchronize()
    for k, v in dev.grads.items():
        assert torch.equal(host.host_out[k], v.cpu()), k
    assert host.host_out["loss"].item() == dev.loss.item()
    # new host inputs are picked up by the next replay
    host.host_in["rgb"].mul_(0.5)
    host.replay()
    torch.cuda.synchronize()
    assert host.host_out["loss"].item() != dev.loss.item()
    h2d, d2h = host.transfer_bytes()
    # the packed inputs start on 256-byte boundaries: at most 255 bytes of padding per array
    assert 0 <= h2d - 4 * (s.N * 14 + 16 + 4 * s.W * s.H) < 6 * 256 and d2h == 4 * (s.N * 14 + 6 + 1)


def test_host_mapping_step_reduced_storage():
    """HostMappingStep with FP16 Gaussians on the host (packed in their storage precision)
    equals the device MappingStep on the same FP16 map bit for bit."""
    torch, api = torch_mods()
    from paper_2509_06433_gb300.tracking import HostMappingStep, MappingStep
    s = make_scene("aerial2m", n=20_000, K=2, W=160, H=96, f=110.0)
    cams = torch.as_tensor(s.cams).cuda()
    r = api.Rasterizer(s.W, s.H, s.K, s.N)
    g = api.Gaussians.from_numpy(s.params(), dtype=torch.float16)
    r.plan(g, cams)
    rgb_t = torch.as_tensor(random_image(61, (s.K, 3, s.H, s.W), 0.0, 1.0)).cuda()
    depth_t = torch.as_tensor(random_image(62, (s.K, s.H, s.W), 0.0, 8.0)).cuda()
    dev = MappingStep(r, g, cams, rgb_t, depth_t, graph=True)
    dev.replay()
    host_g = api.Gaussians(*(t.cpu() for t in (g.means, g.log_scales, g.quats, g.opacity_logits, g.rgb)))
    host = HostMappingStep(r, host_g, cams.cpu(), rgb_t.cpu(), depth_t.cpu(), graph=True)
    assert host.dev_in["quats"].dtype == torch.float16 and host.dev_in["means"].dtype == torch.float32
    host.replay()
    torch.cuda.synchronize()
    for k, v in dev.grads.items():
        assert torch.equal(host.host_out[k], v.cpu()), k
    assert host.host_out["loss"].item() == dev.loss.item()
    h2d, _ = host.transfer_bytes()
    assert 0 <= h2d - (s.N * (12 + 11 * 2) + 4 * s.K * (16 + 4 * s.W * s.H)) < 6 * 256
