"""Tracking and captured iterations on the GPU: the on-device pose update against the
SE(3) exponential, convergence of render-based tracking from a perturbed pose, and
CUDA-graph replays of tracking and mapping iterations against eager execution."""
import math

import numpy as np
import pytest
import scipy.linalg
from scipy.spatial.transform import Rotation

from scenes import make_scene
from scenes.generate import perturb_pose
from tests.gpu_common import GRAD_RTOL, rel_l2, torch_mods

pytestmark = pytest.mark.gpu


def _T(cam):
    T = np.eye(4)
    T[:3, :3] = np.asarray(cam[4:13], np.float64).reshape(3, 3)
    T[:3, 3] = cam[13:16]
    return T


def _twist(xi):
    M = np.zeros((4, 4))
    rho, phi = xi[:3], xi[3:]
    M[:3, :3] = [[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]]
    M[:3, 3] = rho
    return M


def test_pose_adam_step_is_the_se3_exponential_on_the_left():
    torch, api = torch_mods()
    rng = np.random.default_rng(3)
    K = 3
    cams = np.zeros((K, 16), np.float32)
    for k in range(K):
        cams[k, :4] = (500, 500, 320, 240)
        cams[k, 4:13] = Rotation.random(random_state=rng).as_matrix().reshape(9)
        cams[k, 13:16] = rng.normal(0, 1, 3)
    grad = rng.normal(0, 1, (K, 6)).astype(np.float32)
    lr_rho, lr_phi, eps = 0.02, 0.05, 1e-8
    ct = torch.as_tensor(cams).cuda()
    gt = torch.as_tensor(grad).cuda()
    st = torch.zeros((K, 16), device="cuda")
    api.gs_pose_adam_step(ct, gt, st, lr_rho, lr_phi, 0.9, 0.999, eps, zero_grad=True)
    out = ct.cpu().numpy()
    assert torch.count_nonzero(gt).item() == 0
    for k in range(K):
        # first Adam step: m_hat = g, v_hat = g^2 -> xi = -lr g / (|g| + eps)
        lr = np.array([lr_rho] * 3 + [lr_phi] * 3)
        xi = -lr * grad[k] / (np.abs(grad[k]) + eps)
        expect = scipy.linalg.expm(_twist(xi)) @ _T(cams[k])
        got = _T(out[k])
        np.testing.assert_allclose(got, expect, atol=2e-6)
        np.testing.assert_allclose(got[:3, :3] @ got[:3, :3].T, np.eye(3), atol=2e-6)


def _pose_error(cam, ref):
    dR = _T(cam)[:3, :3] @ _T(ref)[:3, :3].T
    ang = math.degrees(np.linalg.norm(Rotation.from_matrix(dR).as_rotvec()))
    # camera centres c = -R^T t
    c = -_T(cam)[:3, :3].T @ _T(cam)[:3, 3]
    c0 = -_T(ref)[:3, :3].T @ _T(ref)[:3, 3]
    return ang, float(np.linalg.norm(c - c0))


def test_tracking_recovers_a_perturbed_pose():
    torch, api = torch_mods()
    from paper_2509_06433_gb300.tracking import Tracker
    s = make_scene("track300k", n=60_000, W=320, H=240, f=260.0)
    g = api.Gaussians.from_numpy(s.params())
    true_cam = torch.as_tensor(s.cams).cuda()
    r = api.Rasterizer(s.W, s.H, 1, s.N)
    r.plan(g, true_cam)
    obs = r.render(g, true_cam)
    start = s.track_cams.copy()
    cams = torch.as_tensor(start).cuda()
    tr = Tracker(g, cams, s.W, s.H, obs["rgb"].clone(), obs["depth"].clone(), lr_rho=2e-3, lr_phi=2e-3)
    a0, t0 = _pose_error(start[0], s.cams[0])
    tr.run(100)
    torch.cuda.synchronize()
    assert tr.status()[0] == 0
    a1, t1 = _pose_error(cams.cpu().numpy()[0], s.cams[0])
    assert a0 > 1.5 and t0 > 0.04
    assert a1 < 0.25 * a0 and t1 < 0.25 * t0, (a0, t0, a1, t1)


def test_graph_replay_equals_eager_for_tracking_and_mapping():
    torch, api = torch_mods()
    from paper_2509_06433_gb300.tracking import MappingStep, Tracker
    s = make_scene("window500k", n=20_000, K=3, W=160, H=120, f=130.0)
    g = api.Gaussians.from_numpy(s.params())
    cams = torch.as_tensor(s.cams).cuda()
    t = s.target
    r = api.Rasterizer(s.W, s.H, s.K, s.N, pair_capacity=1 << 20)
    tgt = r.render(api.Gaussians.from_numpy(t.params()), cams)
    steps = {}
    for graph in (True, False):
        m = MappingStep(r, g, cams, tgt["rgb"].clone(), tgt["depth"].clone(), graph=graph)
        m.replay()
        torch.cuda.synchronize()
        steps[graph] = {k: v.clone() for k, v in m.grads.items()}
    for k in steps[True]:
        assert torch.equal(steps[True][k], steps[False][k]), k
    poses = {}
    for graph in (True, False):
        c = torch.as_tensor(np.stack([perturb_pose(c, np.random.default_rng(1), 1.0, 0.02) for c in s.cams])).cuda()
        tr = Tracker(g, c, s.W, s.H, tgt["rgb"].clone(), tgt["depth"].clone(), graph=graph)
        tr.run(10)
        torch.cuda.synchronize()
        poses[graph] = c.clone()
    assert torch.equal(poses[True], poses[False])


def test_batched_bf16_window_gradients_match_per_view_fp32_sum():
    """The K-view batched launch with BF16 storage equals the sum of K single-view launches
    on the dequantised (FP32) attributes."""
    torch, api = torch_mods()
    s = make_scene("window500k", n=20_000, K=4, W=160, H=120, f=130.0)
    gb = api.Gaussians.from_numpy(s.params(), dtype=torch.bfloat16)
    deq = api.Gaussians(gb.means, gb.log_scales.float(), gb.quats.float(), gb.opacity_logits.float(),
                        gb.rgb.float())
    cams = torch.as_tensor(s.cams).cuda()
    rng = np.random.default_rng(5)
    grgb = torch.as_tensor(rng.normal(size=(s.K, 3, s.H, s.W)).astype(np.float32)).cuda()
    gdep = torch.as_tensor(rng.normal(size=(s.K, s.H, s.W)).astype(np.float32)).cuda()
    rb = api.Rasterizer(s.W, s.H, s.K, s.N, pair_capacity=1 << 20)
    ob = rb.render(gb, cams)
    batched = rb.backward(gb, cams, ob, grgb, gdep)
    total = None
    for k in range(s.K):
        r1 = api.Rasterizer(s.W, s.H, 1, s.N, pair_capacity=1 << 19)
        o1 = r1.render(deq, cams[k:k + 1].contiguous())
        assert torch.equal(o1["rgb"][0], ob["rgb"][k])
        g1 = r1.backward(deq, cams[k:k + 1].contiguous(), o1, grgb[k:k + 1].contiguous(), gdep[k:k + 1].contiguous())
        if total is None:
            total = {kk: v.clone() for kk, v in g1.items() if kk != "pose"}
        else:
            for kk in total:
                total[kk] += g1[kk]
        np.testing.assert_allclose(g1["pose"].cpu().numpy()[0], batched["pose"].cpu().numpy()[k], rtol=1e-4, atol=1e-6)
    for kk in total:
        assert rel_l2(batched[kk].cpu().numpy(), total[kk].cpu().numpy()) < 1e-5, kk
