"""Pins of the metric oracle (PSNR, SSIM) against closed forms, brute force and an
independent library filter (scipy.ndimage). CPU only."""
import numpy as np
import pytest

from oracle import metrics as M


def rand_images(seed, shape=(2, 3, 37, 29)):
    return np.random.default_rng(seed).uniform(0.0, 1.0, shape)


def test_psnr_closed_forms():
    x = rand_images(1) * 0.5 + 0.2
    # a constant offset delta: MSE = delta^2, PSNR = -20 log10(delta)
    assert np.allclose(M.psnr(x, x + 0.01), 40.0, atol=1e-9)
    assert np.allclose(M.psnr(x, x - 0.1, data_range=2.0), 20.0 * np.log10(2.0 / 0.1), atol=1e-9)
    # half the pixels off by d, half exact: MSE = d^2 / 2
    y = x.copy()
    y[:, :, :, ::2] += 0.02
    frac = np.mean(np.arange(x.shape[-1]) % 2 == 0)
    assert np.allclose(M.psnr(x, y), 10 * np.log10(1.0 / (0.02 ** 2 * frac)), atol=1e-9)
    assert np.all(np.isinf(M.psnr(x, x)))


def test_window_matches_scipy_gaussian_filter():
    ndimage = pytest.importorskip("scipy.ndimage")
    x = rand_images(2)
    got = M.window_mean(x)
    # scipy's kernel: exp(-r^2 / (2 sigma^2)) on |r| <= int(truncate sigma + 0.5), normalised;
    # truncate = 5 / 1.5 gives the 11 taps, mode constant 0 the zero padding
    for b in range(x.shape[0]):
        for c in range(x.shape[1]):
            ref = ndimage.gaussian_filter(x[b, c], sigma=1.5, mode="constant", cval=0.0, truncate=5.0 / 1.5)
            assert np.abs(got[b, c] - ref).max() < 1e-13
    w = M.gaussian_window()
    assert w.shape == (11,) and abs(w.sum() - 1) < 1e-15 and np.allclose(w, w[::-1])
    assert np.argmax(w) == 5


def test_ssim_identity_and_symmetry():
    x, y = rand_images(3), rand_images(4)
    s, m = M.ssim(x, x)
    assert np.abs(m - 1.0).max() < 1e-12 and np.allclose(s, 1.0, atol=1e-12)
    s1, m1 = M.ssim(x, y)
    s2, m2 = M.ssim(y, x)
    assert np.abs(m1 - m2).max() < 1e-15
    assert np.all(m1 <= 1.0 + 1e-12) and np.all(m1 >= -1.0 - 1e-12)
    assert np.all(s1 < 0.5)  # independent noise images are dissimilar


def test_ssim_constant_images_interior_closed_form():
    # constant planes a and b: away from the border (>= 5 px) the window sees no padding,
    # mu = (a, b), all variances 0, so SSIM = (2ab + C1) / (a^2 + b^2 + C1)
    a, b = 0.3, 0.7
    x = np.full((1, 1, 30, 24), a)
    y = np.full((1, 1, 30, 24), b)
    _, m = M.ssim(x, y)
    c1 = 0.01 ** 2
    assert np.abs(m[0, 0, 5:-5, 5:-5] - (2 * a * b + c1) / (a * a + b * b + c1)).max() < 1e-12
    # at the border the zero padding lowers both means and adds variance: a different value
    assert abs(m[0, 0, 0, 0] - (2 * a * b + c1) / (a * a + b * b + c1)) > 1e-3


def test_ssim_affine_pair_closed_form():
    # y = alpha x + beta: mu_y = alpha mu_x + beta, s_y^2 = alpha^2 s_x^2, s_xy = alpha s_x^2
    # (interior pixels, where the window sees no padding)
    x = rand_images(5, (1, 2, 40, 33))
    alpha, beta = 0.6, 0.25
    y = alpha * x + beta
    _, m = M.ssim(x, y)
    mx = M.window_mean(x)
    vx = M.window_mean(x * x) - mx * mx
    my = alpha * mx + beta
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    ref = ((2 * mx * my + c1) * (2 * alpha * vx + c2)) / ((mx * mx + my * my + c1) * ((1 + alpha ** 2) * vx + c2))
    assert np.abs(m - ref)[..., 5:-5, 5:-5].max() < 1e-10


def test_ssim_brute_force_pixels():
    # per pixel: explicit 11 x 11 window with weights w_a w_b and zero outside the image
    x, y = rand_images(6, (1, 1, 20, 17)), rand_images(7, (1, 1, 20, 17))
    _, m = M.ssim(x, y)
    w = M.gaussian_window()
    H, W = x.shape[-2:]
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    for (i, j) in [(0, 0), (3, 16), (10, 8), (19, 2), (7, 0)]:
        sx = sy = sxx = syy = sxy = 0.0
        for a in range(11):
            for b in range(11):
                r, c = i + a - 5, j + b - 5
                if 0 <= r < H and 0 <= c < W:
                    wt = w[a] * w[b]
                    u, v = x[0, 0, r, c], y[0, 0, r, c]
                    sx += wt * u
                    sy += wt * v
                    sxx += wt * u * u
                    syy += wt * v * v
                    sxy += wt * u * v
        vx, vy, cxy = sxx - sx * sx, syy - sy * sy, sxy - sx * sy
        ref = ((2 * sx * sy + c1) * (2 * cxy + c2)) / ((sx * sx + sy * sy + c1) * (vx + vy + c2))
        assert abs(m[0, 0, i, j] - ref) < 1e-12, (i, j)
