"""FP64 oracle of the mapping loop around the rasterizer (plain numpy).

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only the tests, the smoke check and the
CPU-baseline legs of the benchmark use it; the CUDA library never does.

The paper's mapping optimiser updates the Gaussian map by comparing rendered images with the
key-frames (Sec. II-B) and grows the map from new key-frames; it names neither the
optimiser nor how Gaussians are created. Readings taken here (3DGS-lineage practice):

* the optimiser is Adam with bias correction, one learning rate per parameter group
  (means, log-scales, quaternions, opacity logits, colours), applied to FP32 master values;
* a key-frame adds one Gaussian per sampled pixel (every ``stride``-th pixel in x and y, at
  the pixel centre) whose depth is valid (> near) and, when a transmittance image of the
  current map is given, where that transmittance exceeds ``t_min`` (the map does not yet
  cover the pixel): mean = the pixel centre back-projected to its depth, isotropic log-scale
  ln(scale_factor * stride * depth / f) with f the mean of fx and fy, identity quaternion,
  opacity logit ``logit0``, colour = the pixel's RGB. New Gaussians are appended in row-major
  pixel order. (Densification and pruning heuristics are not in the paper: these are proposed.)
"""
from __future__ import annotations

import numpy as np

GROUPS = ("means", "log_scales", "quats", "opacity_logits", "rgb")
WIDTHS = (3, 3, 4, 1, 3)


def adam_step(params: dict, grads: dict, m: dict, v: dict, t: int, lr: dict, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015, Algorithm 1) on every group, in place; t is the step
    number of this update (1 for the first). Returns the updated params."""
    c1 = 1.0 - beta1 ** t
    c2 = 1.0 - beta2 ** t
    for k in GROUPS:
        g = np.asarray(grads[k], np.float64)
        m[k] = beta1 * m[k] + (1.0 - beta1) * g
        v[k] = beta2 * v[k] + (1.0 - beta2) * g * g
        mhat = m[k] / c1
        vhat = v[k] / c2
        params[k] = params[k] - lr[k] * mhat / (np.sqrt(vhat) + eps)
    return params


def keyframe_gaussians(rgb, depth, cam, stride=4, near=0.2, T=None, t_min=0.5, scale_factor=0.5, logit0=0.0):
    """New Gaussians of one key-frame: rgb [3,H,W], depth [H,W], cam = 16 floats
    (fx, fy, cx, cy, R row-major, t; world -> camera). Returns the five parameter arrays."""
    rgb = np.asarray(rgb, np.float64)
    depth = np.asarray(depth, np.float64)
    cam = np.asarray(cam, np.float64).reshape(16)
    fx, fy, cx, cy = cam[:4]
    R = cam[4:13].reshape(3, 3)
    t = cam[13:16]
    H, W = depth.shape
    ys, xs = np.meshgrid(np.arange(0, H, stride), np.arange(0, W, stride), indexing="ij")
    ys, xs = ys.reshape(-1), xs.reshape(-1)  # row-major
    d = depth[ys, xs]
    keep = d > near
    if T is not None:
        keep &= np.asarray(T, np.float64)[ys, xs] > t_min
    ys, xs, d = ys[keep], xs[keep], d[keep]
    pc = np.stack([(xs + 0.5 - cx) / fx * d, (ys + 0.5 - cy) / fy * d, d], axis=1)
    means = (pc - t) @ R  # R^T (p_c - t), row by row
    f = 0.5 * (fx + fy)
    ls = np.repeat(np.log(scale_factor * stride * d / f)[:, None], 3, axis=1)
    quats = np.tile(np.array([1.0, 0.0, 0.0, 0.0]), (len(d), 1))
    logits = np.full(len(d), float(logit0))
    colours = rgb[:, ys, xs].T
    return means, ls, quats, logits, colours
