"""Pins of the spherical-harmonics colour oracle: the basis against scipy's complex
harmonics, orthonormality by quadrature, the addition theorem, the SH0 mapping, and the
reverse mode against central finite differences. CPU only."""
import math

import numpy as np
import pytest

from oracle import appearance as A


def unit_dirs(seed, n):
    v = np.random.default_rng(seed).normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def test_basis_matches_scipy_real_harmonics():
    special = pytest.importorskip("scipy.special")
    u = unit_dirs(1, 64)
    theta = np.arccos(np.clip(u[:, 2], -1, 1))   # polar angle from +z
    phi = np.arctan2(u[:, 1], u[:, 0])            # azimuth from +x
    Y = A.sh_basis(u, 3)
    i = 0
    for l in range(4):
        for m in range(-l, l + 1):
            c = special.sph_harm_y(l, abs(m), theta, phi)
            ref = (math.sqrt(2) * c.imag) if m < 0 else (c.real if m == 0 else math.sqrt(2) * c.real)
            assert np.abs(Y[:, i] - ref).max() < 1e-13, (l, m)
            i += 1


def test_basis_orthonormal_by_quadrature():
    # Gauss-Legendre in cos(theta) x uniform phi integrates products of degree <= 6 exactly
    xg, wg = np.polynomial.legendre.leggauss(12)
    nphi = 16
    phi = 2 * np.pi * np.arange(nphi) / nphi
    ct, ph = np.meshgrid(xg, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    u = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=-1).reshape(-1, 3)
    w = (wg[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).reshape(-1)
    Y = A.sh_basis(u, 3)
    G = (Y * w[:, None]).T @ Y
    assert np.abs(G - np.eye(16)).max() < 1e-12


def test_addition_theorem_and_sh0():
    u = unit_dirs(2, 50)
    Y = A.sh_basis(u, 3)
    for l in range(4):
        band = Y[:, l * l:(l + 1) * (l + 1)]
        assert np.abs((band ** 2).sum(axis=1) - (2 * l + 1) / (4 * np.pi)).max() < 1e-13
    # degree 0: colour = f0 / (2 sqrt(pi)) + 1/2, whatever the direction; clamped at 0
    means = np.random.default_rng(3).normal(size=(20, 3)) + [0, 0, 4]
    f = np.random.default_rng(4).normal(size=(20, 1, 3))
    cam = np.array([300, 300, 160, 120, 1, 0, 0, 0, 1, 0, 0, 0, 1, 0.1, -0.2, 0.3], np.float64)
    col, raw = A.sh_colour(f, means, cam, 0)
    assert np.abs(raw - (f[:, 0] / (2 * np.sqrt(np.pi)) + 0.5)).max() < 1e-15
    assert np.array_equal(col, np.maximum(raw, 0))


def test_direction_is_from_camera_centre():
    # a Gaussian straight ahead of the camera (on its optical axis) sees u = R^T (0, 0, 1):
    # with R = identity, band-1 colour = C1 f_(1,0) only
    cam = np.array([300, 300, 160, 120, 1, 0, 0, 0, 1, 0, 0, 0, 1, 0.5, -0.25, 2.0], np.float64)
    centre = A.camera_centre(cam)
    assert np.allclose(centre, [-0.5, 0.25, -2.0])
    means = np.array([[-0.5, 0.25, 3.0]])
    f = np.zeros((1, 4, 3))
    f[0, 2] = [0.1, 0.2, 0.3]
    col, _ = A.sh_colour(f, means, cam, 1)
    assert np.allclose(col[0], 0.5 + A.C1 * np.array([0.1, 0.2, 0.3]), atol=1e-15)


@pytest.mark.parametrize("degree", [0, 1, 2, 3])
def test_colour_reverse_mode_matches_finite_differences(degree):
    rng = np.random.default_rng(10 + degree)
    N = 6
    nc = A.n_coeffs(degree)
    means = rng.normal(size=(N, 3)) + [0, 0, 4]
    f = rng.normal(size=(N, nc, 3)) * 0.3
    f[:, 0] += 1.0  # keep the colours away from the clamp
    th = 0.3
    R = np.array([[np.cos(th), 0, np.sin(th)], [0, 1, 0], [-np.sin(th), 0, np.cos(th)]])
    cam = np.concatenate([[300, 300, 160, 120], R.reshape(-1), [0.1, -0.2, 0.3]])
    g = rng.normal(size=(N, 3))
    L = lambda f_, m_, c_: np.sum(A.sh_colour(f_, m_, c_, degree)[0] * g)  # noqa: E731
    dc, dm, drho = A.sh_colour_bwd(f, means, cam, degree, g)
    h = 1e-6
    for n in range(N):
        for j in range(3):
            e = np.zeros_like(means)
            e[n, j] = h
            fd = (L(f, means + e, cam) - L(f, means - e, cam)) / (2 * h)
            assert abs(fd - dm[n, j]) < 1e-7 * max(1.0, abs(fd)), (n, j)
        for i in range(nc):
            e = np.zeros_like(f)
            e[n, i, 1] = h
            fd = (L(f + e, means, cam) - L(f - e, means, cam)) / (2 * h)
            assert abs(fd - dc[n, i, 1]) < 1e-7
    # pose: rho moves the camera-space points by +rho, i.e. t -> t + rho with R fixed
    for j in range(3):
        cp, cm = cam.copy(), cam.copy()
        cp[13 + j] += h
        cm[13 + j] -= h
        fd = (L(f, means, cp) - L(f, means, cm)) / (2 * h)
        assert abs(fd - drho[j]) < 1e-7 * max(1.0, abs(fd)), j


def test_clamp_blocks_the_gradient():
    means = np.array([[0.0, 0.0, 4.0]])
    f = np.zeros((1, 1, 3))
    f[0, 0] = [-5.0, 1.0, -5.0]  # channels 0 and 2 clamp
    cam = np.array([300, 300, 160, 120, 1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0], np.float64)
    col, raw = A.sh_colour(f, means, cam, 0)
    assert col[0, 0] == 0 and col[0, 2] == 0 and col[0, 1] > 0.5
    dc, _, _ = A.sh_colour_bwd(f, means, cam, 0, np.ones((1, 3)))
    assert dc[0, 0, 0] == 0 and dc[0, 0, 2] == 0 and dc[0, 0, 1] == pytest.approx(A.C0)


def _sh_scene(degree, seed=31):
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(seed)
    N, W, H, f = 10, 40, 32, 40.0
    means = rng.uniform((-0.5, -0.4, 2.0), (0.5, 0.4, 4.0), (N, 3))
    ls = rng.normal(-2.0, 0.3, (N, 3))
    qs = rng.normal(size=(N, 4))
    lg = rng.normal(0.0, 1.0, N)
    coeffs = rng.normal(0, 0.3, (N, A.n_coeffs(degree), 3))
    coeffs[:, 0] += 0.5
    params = tuple(np.asarray(a, np.float32) for a in (means, ls, qs, lg, coeffs))
    R = Rotation.from_rotvec([0.05, -0.08, 0.03]).as_matrix()
    cam = np.concatenate([[f, f * 1.05, 21.0, 15.5], R.reshape(-1), [0.03, -0.02, 0.1]]).astype(np.float32)
    return params, cam[None], W, H


@pytest.mark.parametrize("degree", [1, 3])
def test_sh_render_gradients_match_finite_differences(degree):
    params, cams, W, H = _sh_scene(degree)
    p64 = [np.asarray(a, np.float64) for a in params]
    base = A.forward_sh(params, cams, W, H, degree)
    rng = np.random.default_rng(5)
    wr, wd = rng.normal(size=base["rgb"].shape), rng.normal(size=base["depth"].shape)
    g = A.backward_sh(p64, cams, W, H, degree, base, wr, wd)
    h = 1e-6

    def L_at(pp, c=cams):
        o = A.forward_sh(pp, c, W, H, degree)
        same = np.array_equal(o["evals"], base["evals"]) and np.array_equal(o["last"], base["last"])
        return float((o["rgb"] * wr).sum() + (o["depth"] * wd).sum()), same

    for bi, name in ((4, "rgb"), (0, "means")):
        an = g[name].reshape(-1)
        scale = np.abs(an).max()
        checked = 0
        for j in range(an.size):
            pp = [a.copy() for a in p64]
            flat = pp[bi].reshape(-1)
            flat[j] += h
            Lp, okp = L_at(pp)
            flat[j] -= 2 * h
            Lm, okm = L_at(pp)
            if not (okp and okm):
                continue
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - an[j]) <= 2e-6 * scale + 1e-5 * abs(an[j]), (name, j, fd, an[j])
            checked += 1
        assert checked >= 0.9 * an.size
    # pose translation rho: t -> t + rho (R fixed) moves p_c by rho and the camera centre by -R^T rho
    for j in range(3):
        vals = []
        for s in (1, -1):
            c = cams.astype(np.float64).copy()
            c[0, 13 + j] += s * h
            vals.append(L_at(p64, c)[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g["pose"][0, j]) <= 2e-6 * np.abs(g["pose"]).max() + 1e-5 * abs(fd), j


def test_sh_translation_gradient_equals_summed_mean_gradient():
    # translating the world by delta is translating the camera by -delta: geometry and view
    # directions alike, so sum_g dL/dmean_g = R^T dL/drho also with view-dependent colour
    params, cams, W, H = _sh_scene(2, seed=32)
    fwd = A.forward_sh(params, cams, W, H, 2)
    rng = np.random.default_rng(6)
    g = A.backward_sh(params, cams, W, H, 2, fwd, rng.normal(size=fwd["rgb"].shape), rng.normal(size=fwd["depth"].shape))
    R = cams[0, 4:13].astype(np.float64).reshape(3, 3)
    # exact for orthonormal R; the binary32 rotation is orthonormal to ~1e-8, which the view
    # direction (mu - C with C = -R^T t) feels, unlike the geometry
    np.testing.assert_allclose(g["means"].sum(0), R.T @ g["pose"][0, :3], rtol=1e-7, atol=1e-12)
