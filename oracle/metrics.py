"""FP64 oracle of the map-accuracy metrics (plain numpy).

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only the tests, the smoke check and the
CPU-baseline legs of the benchmark use it; the CUDA library never does.

Sec. IV measures map accuracy by PSNR and SSIM of rendered views against the key-frames and
map-generation speed by the time each new frame takes to reach its final PSNR / SSIM. The
paper gives no formula for either metric; the readings taken here are the standard ones
used by the Gaussian-splatting literature it builds on:

* PSNR of one image (all channels) = 10 log10(R^2 / MSE), R = the data range (1 for
  images in [0, 1]); MSE = 0 gives +inf.
* SSIM (Wang et al. 2004) per pixel and channel from local statistics under an 11 x 11
  Gaussian window (sigma 1.5, taps normalised to sum 1), the image taken as 0 outside its
  border (zero padding, output the same size as the input):
      SSIM = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2)),
  s_x^2 = E[x^2] - mu_x^2, s_xy = E[xy] - mu_x mu_y, C1 = (0.01 R)^2, C2 = (0.03 R)^2;
  an image's SSIM is the mean over its channels and pixels.
"""
from __future__ import annotations

import numpy as np

SSIM_SIZE = 11
SSIM_SIGMA = 1.5
SSIM_K1 = 0.01
SSIM_K2 = 0.03


def psnr(x, y, data_range=1.0):
    """PSNR of each image of x, y [B, C, H, W] (or [C, H, W]); returns [B]."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    if x.ndim == 3:
        x, y = x[None], y[None]
    mse = ((x - y) ** 2).reshape(x.shape[0], -1).mean(axis=1)
    with np.errstate(divide="ignore"):
        return 10.0 * np.log10(data_range ** 2 / mse)


def gaussian_window(size=SSIM_SIZE, sigma=SSIM_SIGMA):
    """1D Gaussian taps centred on the middle tap, normalised to sum 1."""
    r = np.arange(size, dtype=np.float64) - (size // 2)
    w = np.exp(-(r * r) / (2.0 * sigma * sigma))
    return w / w.sum()


def window_mean(img, size=SSIM_SIZE, sigma=SSIM_SIGMA):
    """Weighted local mean of each plane of img [..., H, W] under the separable window, zero outside."""
    w = gaussian_window(size, sigma)
    h = size // 2
    a = np.asarray(img, np.float64)
    H, W = a.shape[-2:]
    pad = [(0, 0)] * (a.ndim - 2) + [(h, h), (h, h)]
    p = np.pad(a, pad)
    rows = sum(w[i] * p[..., :, i:i + W] for i in range(size))      # along x
    return sum(w[i] * rows[..., i:i + H, :] for i in range(size))  # along y


def ssim(x, y, data_range=1.0, size=SSIM_SIZE, sigma=SSIM_SIGMA):
    """SSIM of each image of x, y [B, C, H, W] (or [C, H, W]); returns (per-image mean [B], map [B, C, H, W])."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    if x.ndim == 3:
        x, y = x[None], y[None]
    c1 = (SSIM_K1 * data_range) ** 2
    c2 = (SSIM_K2 * data_range) ** 2
    mx, my = window_mean(x, size, sigma), window_mean(y, size, sigma)
    sxx = window_mean(x * x, size, sigma) - mx * mx
    syy = window_mean(y * y, size, sigma) - my * my
    sxy = window_mean(x * y, size, sigma) - mx * my
    m = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
    return m.reshape(m.shape[0], -1).mean(axis=1), m
