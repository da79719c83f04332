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


def _filter_adjoint(m: np.ndarray, w: np.ndarray, shape, mode: str) -> np.ndarray:
    """Adjoint of ``_filter``: spreads each output pixel's value back over its
    window (a full convolution with the symmetric window, cropped in the
    'same' mode to undo the zero padding)."""
    k = len(w)
    cols = np.apply_along_axis(lambda v: np.convolve(v, w, mode="full"), 0, m)
    full = np.apply_along_axis(lambda v: np.convolve(v, w, mode="full"), 1, cols)
    if mode == "same":
        pad = k // 2
        full = full[pad:pad + shape[0], pad:pad + shape[1]]
    return full


def ssim_grad(x: np.ndarray, y: np.ndarray, data_range: float = 1.0, mode: str = "valid") -> np.ndarray:
    """Gradient of the mean SSIM of two single-channel images with respect to x.

    With the window sums m_x = g * x, E_xx = g * x^2, E_xy = g * (x y) of each
    pixel p, SSIM_p = A1 A2 / (B1 B2), A1 = 2 m_x m_y + C1,
    A2 = 2 (E_xy - m_x m_y) + C2, B1 = m_x^2 + m_y^2 + C1,
    B2 = E_xx - m_x^2 + E_yy - m_y^2 + C2. Its partial derivatives in
    (m_x, E_xx, E_xy) are spread back over each window (the adjoint of the
    window sum) and chained through dE_xx/dx = 2x, dE_xy/dx = y. The D-SSIM
    loss (1 - SSIM) / 2 has minus half this gradient."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    w = gaussian_window()
    c1 = (K1 * data_range) ** 2
    c2 = (K2 * data_range) ** 2
    mx = _filter(x, w, mode)
    my = _filter(y, w, mode)
    exx = _filter(x * x, w, mode)
    eyy = _filter(y * y, w, mode)
    exy = _filter(x * y, w, mode)
    a1 = 2.0 * mx * my + c1
    a2 = 2.0 * (exy - mx * my) + c2
    b1 = mx * mx + my * my + c1
    b2 = exx - mx * mx + eyy - my * my + c2
    s = a1 * a2 / (b1 * b2)
    npix = s.size
    d_mx = (2.0 * my * a2 - 2.0 * my * a1) / (b1 * b2) - s * (2.0 * mx / b1 - 2.0 * mx / b2)
    d_exx = -s / b2
    d_exy = 2.0 * a1 / (b1 * b2)
    g_m = _filter_adjoint(d_mx / npix, w, x.shape, mode)
    g_xx = _filter_adjoint(d_exx / npix, w, x.shape, mode)
    g_xy = _filter_adjoint(d_exy / npix, w, x.shape, mode)
    return g_m + 2.0 * x * g_xx + y * g_xy
