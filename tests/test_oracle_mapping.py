"""Pins of the mapping-loop oracle (oracle/mapping.py): Adam against closed forms of its
recursion, key-frame back-projection against re-projection through the camera."""
import numpy as np

from oracle import mapping as om
from scenes.generate import camera_array, look_at


def _params(rng, n):
    return {k: rng.normal(size=(n, w)).reshape((n,) if w == 1 else (n, w)) for k, w in zip(om.GROUPS, om.WIDTHS)}


def _zeros_like(p):
    return {k: np.zeros_like(v) for k, v in p.items()}


LR = {"means": 1e-3, "log_scales": 5e-3, "quats": 1e-3, "opacity_logits": 5e-2, "rgb": 2.5e-3}


def test_adam_constant_gradient_moves_lr_per_step():
    # with a constant gradient g the bias-corrected moments are exactly g and g^2 at every step
    rng = np.random.default_rng(0)
    p0 = _params(rng, 50)
    g = _params(rng, 50)
    p = {k: v.copy() for k, v in p0.items()}
    m, v = _zeros_like(p), _zeros_like(p)
    for t in range(1, 6):
        om.adam_step(p, g, m, v, t, LR, eps=1e-8)
    for k in om.GROUPS:
        np.testing.assert_allclose(p[k], p0[k] - 5 * LR[k] * g[k] / (np.abs(g[k]) + 1e-8), rtol=0, atol=1e-12)


def test_adam_gradient_then_zero():
    rng = np.random.default_rng(1)
    p0 = _params(rng, 20)
    g = _params(rng, 20)
    b1, b2, eps = 0.9, 0.999, 1e-8
    p = {k: val.copy() for k, val in p0.items()}
    m, v = _zeros_like(p), _zeros_like(p)
    om.adam_step(p, g, m, v, 1, LR, b1, b2, eps)
    om.adam_step(p, _zeros_like(g), m, v, 2, LR, b1, b2, eps)
    for k in om.GROUPS:
        step1 = LR[k] * g[k] / (np.abs(g[k]) + eps)
        # m_hat_2 = b1 g / (1 + b1), v_hat_2 = b2 g^2 / (1 + b2)
        step2 = LR[k] * (b1 / (1 + b1)) * g[k] / (np.abs(g[k]) * np.sqrt(b2 / (1 + b2)) + eps)
        np.testing.assert_allclose(p[k], p0[k] - step1 - step2, rtol=0, atol=1e-12)


def test_keyframe_gaussians_reproject_to_their_pixels():
    rng = np.random.default_rng(2)
    H, W = 40, 52
    R, t = look_at(np.array([0.3, -0.2, -1.0]), np.array([0.1, 1.0, 0.2]))
    cam = np.asarray(camera_array(45.0, 47.0, 26.5, 19.0, R, t), np.float64)
    depth = rng.uniform(0.5, 6.0, (H, W))
    depth[rng.uniform(size=(H, W)) < 0.2] = 0.0  # invalid depth
    T = rng.uniform(size=(H, W))
    rgb = rng.uniform(size=(3, H, W))
    stride = 3
    means, ls, qs, lg, col = om.keyframe_gaussians(rgb, depth, cam, stride=stride, T=T, t_min=0.4,
                                                   scale_factor=0.5, logit0=-0.5)
    ys, xs = np.meshgrid(np.arange(0, H, stride), np.arange(0, W, stride), indexing="ij")
    ys, xs = ys.ravel(), xs.ravel()
    keep = (depth[ys, xs] > 0.2) & (T[ys, xs] > 0.4)
    ys, xs = ys[keep], xs[keep]
    assert len(means) == keep.sum() > 10
    R = cam[4:13].reshape(3, 3)
    pc = means @ R.T + cam[13:16]
    # the stored (binary32) rotation is orthonormal to ~1e-7, and the back-projection takes
    # R^T as its inverse: the round trip holds to that level
    np.testing.assert_allclose(cam[0] * pc[:, 0] / pc[:, 2] + cam[2], xs + 0.5, atol=1e-4)
    np.testing.assert_allclose(cam[1] * pc[:, 1] / pc[:, 2] + cam[3], ys + 0.5, atol=1e-4)
    np.testing.assert_allclose(pc[:, 2], depth[ys, xs], rtol=1e-6)
    np.testing.assert_allclose(np.exp(ls[:, 0]), 0.5 * stride * depth[ys, xs] / (0.5 * (cam[0] + cam[1])), rtol=1e-12)
    assert np.all(ls[:, 0] == ls[:, 1]) and np.all(ls[:, 1] == ls[:, 2])
    np.testing.assert_array_equal(qs, np.tile([1.0, 0, 0, 0], (len(qs), 1)))
    assert np.all(lg == -0.5)
    np.testing.assert_array_equal(col, rgb[:, ys, xs].T)
