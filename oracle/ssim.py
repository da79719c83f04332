"""Oracle of SSIM, the structural-similarity index the paper reports beside
PSNR and LPIPS (Sec. 4, metrics; the index of Wang et al. 2004), plain numpy
in FP64.

TEST INFRASTRUCTURE. Only ``tests/`` (and ``__graft_entry__.smoke()``) may
import this module; the product package never does, and nothing here is
shared with the CUDA path.

For images x, y with values in [0, L] (L = 1 here), at every pixel whose
window lies inside the image:
    mu_x = sum_w g(w) x(w),  sigma_x^2 = sum_w g(w) x(w)^2 - mu_x^2,
    sigma_xy = sum_w g(w) x(w) y(w) - mu_x mu_y,
    SSIM = (2 mu_x mu_y + C1) (2 sigma_xy + C2)
           / ((mu_x^2 + mu_y^2 + C1) (sigma_x^2 + sigma_y^2 + C2)),
with g the 11 x 11 Gaussian window of standard deviation 1.5 normalised to
sum 1, C1 = (0.01 L)^2 and C2 = (0.03 L)^2 (Wang et al.'s constants). The
image's SSIM is the mean over those pixels and the colour channels.

Border reading: only windows wholly inside the image count ("valid"). The
3DGS training code pads with zeros instead ("same"); ``mode="same"`` gives
that form.
"""
from __future__ import annotations

import numpy as np

WINDOW = 11
SIGMA = 1.5
K1, K2 = 0.01, 0.03


def gaussian_window(size: int = WINDOW, sigma: float = SIGMA) -> np.ndarray:
    """1-D Gaussian weights of the separable window, summing to 1."""
    r = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    w = np.exp(-(r * r) / (2.0 * sigma * sigma))
    return w / w.sum()


def _filter(img: np.ndarray, w: np.ndarray, mode: str) -> np.ndarray:
    """Weighted window sums of a 2-D image: one 1-D convolution along each axis
    (the window is symmetric, so convolution and correlation agree)."""
    k = len(w)
    if mode == "same":
        pad = k // 2
        img = np.pad(img, pad, mode="constant")
    rows = np.apply_along_axis(lambda v: np.convolve(v, w, mode="valid"), 1, img)
    return np.apply_along_axis(lambda v: np.convolve(v, w, mode="valid"), 0, rows)


def ssim_map(x: np.ndarray, y: np.ndarray, data_range: float = 1.0, mode: str = "valid") -> np.ndarray:
    """Per-pixel SSIM of two single-channel images (H x W)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    if x.shape != y.shape or x.ndim != 2:
        raise ValueError("ssim_map: two H x W images of the same shape")
    if mode not in ("valid", "same"):
        raise ValueError("ssim_map: mode is 'valid' or 'same'")
    if mode == "valid" and min(x.shape) < WINDOW:
        raise ValueError("ssim_map: images smaller than the window have no valid pixel")
    w = gaussian_window()
    c1 = (K1 * data_range) ** 2
    c2 = (K2 * data_range) ** 2
    mu_x = _filter(x, w, mode)
    mu_y = _filter(y, w, mode)
    sxx = _filter(x * x, w, mode) - mu_x * mu_x
    syy = _filter(y * y, w, mode) - mu_y * mu_y
    sxy = _filter(x * y, w, mode) - mu_x * mu_y
    num = (2.0 * mu_x * mu_y + c1) * (2.0 * sxy + c2)
    den = (mu_x * mu_x + mu_y * mu_y + c1) * (sxx + syy + c2)
    return num / den


def ssim(x: np.ndarray, y: np.ndarray, data_range: float = 1.0, mode: str = "valid") -> float:
    """Mean SSIM of two images, H x W or H x W x C (channels averaged)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    if x.ndim == 2:
        return float(ssim_map(x, y, data_range, mode).mean())
    if x.ndim != 3 or x.shape != y.shape:
        raise ValueError("ssim: H x W or H x W x C images of the same shape")
    return float(np.mean([ssim_map(x[..., c], y[..., c], data_range, mode).mean() for c in range(x.shape[2])]))
