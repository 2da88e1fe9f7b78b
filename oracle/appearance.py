"""FP64 oracle of view-dependent colour by spherical harmonics (plain numpy), and the
K-view render / backward built on it.

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only the tests, the smoke check and the
CPU-baseline legs of the benchmark use it; the CUDA library never does.

Sec. II-A: Gaussian splatting models view-dependent colour with spherical harmonics, which
GS-SLAM variants drop (Sec. II-B). The paper gives no formula; the reading taken here is the
one of the Gaussian-splatting work it cites:

* a Gaussian holds (D + 1)^2 coefficient triples (D = degree 0..3), ordered by band l and
  then m = -l..l, each an RGB triple;
* the basis is the real spherical harmonics WITH the Condon-Shortley phase: for m > 0
  sqrt(2) Re Y_l^m, for m < 0 sqrt(2) Im Y_l^|m|, for m = 0 Y_l^0, Y_l^m the complex
  orthonormal harmonics; evaluated at the unit direction u = (mu - C) / |mu - C| from the
  camera centre C = -R^T t to the Gaussian mean. Each basis function is written below as
  its polynomial in (x, y, z) on the unit sphere;
* colour = max(sum_i Y_i(u) f_i + 1/2, 0) per channel (the SH0 mapping at D = 0:
  colour = f_0 / (2 sqrt(pi)) + 1/2);
* gradients: zero where the clamp is active (raw < 0); the direction's gradient flows to the
  mean and, through C, to the pose. Under the left perturbation T <- Exp(xi) T the world
  direction is R^T (p_c + rho) to first order, so d(colour)/d(phi) = 0 and
  dL/drho = R dL/du_world.
"""
from __future__ import annotations

import math

import numpy as np

import oracle

PI = math.pi
# normalisation constants of the real harmonics (closed forms)
C0 = 0.5 / math.sqrt(PI)                    # l = 0
C1 = math.sqrt(3.0 / (4.0 * PI))            # l = 1
C2A = 0.5 * math.sqrt(15.0 / PI)            # l = 2, |m| = 1, 2 (xy, yz, xz)
C2B = 0.25 * math.sqrt(5.0 / PI)            # l = 2, m = 0
C2C = 0.25 * math.sqrt(15.0 / PI)           # l = 2, m = 2 (x^2 - y^2)
C3A = 0.25 * math.sqrt(35.0 / (2.0 * PI))   # l = 3, |m| = 3
C3B = 0.5 * math.sqrt(105.0 / PI)           # l = 3, m = -2 (xyz)
C3C = 0.25 * math.sqrt(21.0 / (2.0 * PI))   # l = 3, |m| = 1
C3D = 0.25 * math.sqrt(7.0 / PI)            # l = 3, m = 0
C3E = 0.25 * math.sqrt(105.0 / PI)          # l = 3, m = 2


def n_coeffs(degree: int) -> int:
    return (degree + 1) ** 2


def sh_basis(u, degree: int) -> np.ndarray:
    """Real SH (Condon-Shortley phase) at unit vectors u [M, 3]; returns [M, (degree + 1)^2]."""
    u = np.asarray(u, np.float64)
    x, y, z = u[:, 0], u[:, 1], u[:, 2]
    cols = [np.full_like(x, C0)]
    if degree >= 1:
        cols += [-C1 * y, C1 * z, -C1 * x]
    if degree >= 2:
        cols += [C2A * x * y, -C2A * y * z, C2B * (2 * z * z - x * x - y * y), -C2A * x * z,
                 C2C * (x * x - y * y)]
    if degree >= 3:
        cols += [-C3A * y * (3 * x * x - y * y), C3B * x * y * z, -C3C * y * (4 * z * z - x * x - y * y),
                 C3D * z * (2 * z * z - 3 * x * x - 3 * y * y), -C3C * x * (4 * z * z - x * x - y * y),
                 C3E * z * (x * x - y * y), -C3A * x * (x * x - 3 * y * y)]
    return np.stack(cols, axis=1)


def sh_basis_grad(u, degree: int) -> np.ndarray:
    """Gradient in (x, y, z) of each polynomial of sh_basis; returns [M, (degree + 1)^2, 3]."""
    u = np.asarray(u, np.float64)
    x, y, z = u[:, 0], u[:, 1], u[:, 2]
    o = np.zeros_like(x)
    g = [(o, o, o)]
    if degree >= 1:
        g += [(o, o - C1, o), (o, o, o + C1), (o - C1, o, o)]
    if degree >= 2:
        g += [(C2A * y, C2A * x, o), (o, -C2A * z, -C2A * y), (-2 * C2B * x, -2 * C2B * y, 4 * C2B * z),
              (-C2A * z, o, -C2A * x), (2 * C2C * x, -2 * C2C * y, o)]
    if degree >= 3:
        g += [(-6 * C3A * x * y, -3 * C3A * (x * x - y * y), o),
              (C3B * y * z, C3B * x * z, C3B * x * y),
              (2 * C3C * x * y, -C3C * (4 * z * z - x * x - 3 * y * y), -8 * C3C * y * z),
              (-6 * C3D * x * z, -6 * C3D * y * z, C3D * (6 * z * z - 3 * x * x - 3 * y * y)),
              (-C3C * (4 * z * z - 3 * x * x - y * y), 2 * C3C * x * y, -8 * C3C * x * z),
              (2 * C3E * x * z, -2 * C3E * y * z, C3E * (x * x - y * y)),
              (-3 * C3A * (x * x - y * y), 6 * C3A * x * y, o)]
    return np.stack([np.stack(t, axis=1) for t in g], axis=1)


def camera_centre(cam) -> np.ndarray:
    cam = np.asarray(cam, np.float64).reshape(16)
    R = cam[4:13].reshape(3, 3)
    return -R.T @ cam[13:16]


def sh_colour(coeffs, means, cam, degree: int):
    """Colour [N, 3] of every Gaussian seen from camera cam (16 floats); also returns the
    unclamped value [N, 3]."""
    f = np.asarray(coeffs, np.float64).reshape(len(means), n_coeffs(degree), 3)
    d = np.asarray(means, np.float64) - camera_centre(cam)
    u = d / np.linalg.norm(d, axis=1, keepdims=True)
    raw = np.einsum("ni,nic->nc", sh_basis(u, degree), f) + 0.5
    return np.maximum(raw, 0.0), raw


def sh_colour_bwd(coeffs, means, cam, degree: int, d_rgb):
    """Reverse mode of sh_colour: (d_coeffs [N, nc, 3], d_means [N, 3], d_rho [3])."""
    N = len(means)
    f = np.asarray(coeffs, np.float64).reshape(N, n_coeffs(degree), 3)
    cam = np.asarray(cam, np.float64).reshape(16)
    R = cam[4:13].reshape(3, 3)
    d = np.asarray(means, np.float64) - camera_centre(cam)
    r = np.linalg.norm(d, axis=1, keepdims=True)
    u = d / r
    Y = sh_basis(u, degree)
    raw = np.einsum("ni,nic->nc", Y, f) + 0.5
    g = np.asarray(d_rgb, np.float64) * (raw >= 0.0)
    d_coeffs = Y[:, :, None] * g[:, None, :]
    # dL/du = sum_c g_c sum_i f_ic grad Y_i, projected on the tangent plane and divided by |d|
    du = np.einsum("nc,nic,nij->nj", g, f, sh_basis_grad(u, degree))
    dd = (du - u * np.sum(du * u, axis=1, keepdims=True)) / r
    return d_coeffs, dd, R @ dd.sum(axis=0)


def forward_sh(params, cams, W, H, degree: int, tile=oracle.TILE):
    """K-view oracle render with SH colour: params = (means, log_scales, quats, logits, coeffs).
    Each view renders with its own colours; returns the stacked outputs and per-view lists."""
    means, ls, qs, lg, coeffs = params
    cams = np.asarray(cams).reshape(-1, 16)  # the discrete mirror rounds it to binary32 itself
    outs, lists, colours = [], [], []
    for k in range(cams.shape[0]):
        col, _ = sh_colour(coeffs, means, cams[k].astype(np.float64), degree)
        o = oracle.forward((means, ls, qs, lg, col), cams[k:k + 1], W, H, tile)
        outs.append(o)
        lists.append(o["lists"])
        colours.append(col)
    res = {key: np.concatenate([o[key] for o in outs]) for key in outs[0] if key not in ("lists", "total_evals")}
    res["lists"], res["colours"] = lists, colours
    return res


def backward_sh(params, cams, W, H, degree: int, fwd, dL_drgb, dL_ddepth, dL_dT=None, tile=oracle.TILE):
    """Gradients of the SH render: means, log_scales, quats, opacity_logits summed over views,
    coefficients [N, nc, 3], pose [K, 6] (geometry plus the colour's direction term)."""
    means, ls, qs, lg, coeffs = params
    cams = np.asarray(cams).reshape(-1, 16)
    K, N = cams.shape[0], len(means)
    out = {"means": np.zeros((N, 3)), "log_scales": np.zeros((N, 3)), "quats": np.zeros((N, 4)),
           "opacity_logits": np.zeros(N), "rgb": np.zeros((N, n_coeffs(degree), 3)), "pose": np.zeros((K, 6))}
    for k in range(K):
        col = fwd["colours"][k]
        gT = None if dL_dT is None else dL_dT[k:k + 1]
        g = oracle.backward((means, ls, qs, lg, col), cams[k:k + 1], W, H, fwd["lists"][k], dL_drgb[k:k + 1],
                            dL_ddepth[k:k + 1], gT, tile)
        dc, dm, drho = sh_colour_bwd(coeffs, means, cams[k].astype(np.float64), degree, g["rgb"])
        for key in ("means", "log_scales", "quats", "opacity_logits"):
            out[key] += g[key]
        out["means"] += dm
        out["rgb"] += dc
        out["pose"][k] = g["pose"][0]
        out["pose"][k, :3] += drho
    return out
