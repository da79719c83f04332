"""Pins of the SSIM oracle (the index of Wang et al. 2004 that the paper
reports, Sec. 4 metrics) against what the definition fixes: identity, the
closed form of constant images, symmetry and range, and a brute-force
evaluation of every window with directly built 2-D weights on tiny images
(which catches a wrong window, normalisation, orientation or border)."""
import math

import numpy as np
import pytest

from oracle import ssim as S

C1 = (0.01) ** 2
C2 = (0.03) ** 2


def _brute_map(x, y, mode="valid"):
    """SSIM at every pixel by explicit sums over the 11 x 11 window, with the
    2-D weights exp(-(u^2 + v^2) / (2 * 1.5^2)) normalised by their own sum."""
    h, w = x.shape
    r = 5
    wts = np.array([[math.exp(-((u - r) ** 2 + (v - r) ** 2) / (2 * 1.5 ** 2)) for v in range(11)]
                    for u in range(11)])
    wts /= wts.sum()
    if mode == "valid":
        centres = [(i, j) for i in range(r, h - r) for j in range(r, w - r)]
        oh, ow = h - 2 * r, w - 2 * r
    else:
        centres = [(i, j) for i in range(h) for j in range(w)]
        oh, ow = h, w
    out = np.zeros(oh * ow)
    for k, (i, j) in enumerate(centres):
        mx = my = exx = eyy = exy = 0.0
        for u in range(11):
            for v in range(11):
                a, b = i + u - r, j + v - r
                if 0 <= a < h and 0 <= b < w:
                    xv, yv = x[a, b], y[a, b]
                else:  # zero padding
                    xv = yv = 0.0
                g = wts[u, v]
                mx += g * xv
                my += g * yv
                exx += g * xv * xv
                eyy += g * yv * yv
                exy += g * xv * yv
        sx, sy, sxy = exx - mx * mx, eyy - my * my, exy - mx * my
        out[k] = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sx + sy + C2))
    return out.reshape(oh, ow)


def test_identical_images_score_one():
    x = np.random.default_rng(0).random((24, 31, 3))
    assert S.ssim(x, x) == pytest.approx(1.0, abs=1e-12)


def test_constant_images_closed_form():
    # no variance: the structure factor is C2 / C2, the luminance one (2ab + C1) / (a^2 + b^2 + C1)
    for a, b in ((0.2, 0.7), (0.0, 1.0), (0.5, 0.5), (0.9, 0.1)):
        x = np.full((16, 20), a)
        y = np.full((16, 20), b)
        want = (2 * a * b + C1) / (a * a + b * b + C1)
        m = S.ssim_map(x, y)
        assert m.shape == (6, 10)
        np.testing.assert_allclose(m, want, rtol=0, atol=1e-12)


def test_symmetric_and_bounded():
    rng = np.random.default_rng(1)
    x, y = rng.random((20, 22)), rng.random((20, 22))
    assert S.ssim(x, y) == pytest.approx(S.ssim(y, x), abs=1e-15)
    m = S.ssim_map(x, y)
    assert np.all(m <= 1.0 + 1e-12) and np.all(m >= -1.0 - 1e-12)
    # an inverted image is anti-correlated: below zero on noise
    assert S.ssim(x, 1.0 - x) < 0.0


@pytest.mark.parametrize("mode", ["valid", "same"])
def test_brute_force_windows(mode):
    rng = np.random.default_rng(2)
    x = rng.random((14, 13))
    y = np.clip(x + rng.normal(0, 0.1, x.shape), 0, 1)
    np.testing.assert_allclose(S.ssim_map(x, y, mode=mode), _brute_map(x, y, mode), rtol=0, atol=1e-12)


def test_window_weights():
    w = S.gaussian_window()
    assert len(w) == 11 and w.sum() == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose(w, w[::-1], rtol=0, atol=0)
    # centre over edge: exp(5^2 / (2 * 1.5^2))
    assert w[5] / w[0] == pytest.approx(math.exp(25 / 4.5), rel=1e-12)


def test_channels_are_averaged():
    rng = np.random.default_rng(3)
    x, y = rng.random((15, 15, 3)), rng.random((15, 15, 3))
    want = np.mean([S.ssim(x[..., c], y[..., c]) for c in range(3)])
    assert S.ssim(x, y) == pytest.approx(want, abs=1e-15)


def test_rejects_images_smaller_than_the_window():
    with pytest.raises(ValueError):
        S.ssim_map(np.zeros((10, 40)), np.zeros((10, 40)))


@pytest.mark.parametrize("mode", ["valid", "same"])
def test_gradient_matches_central_differences(mode):
    rng = np.random.default_rng(4)
    x = rng.random((15, 14))
    y = np.clip(x + rng.normal(0, 0.15, x.shape), 0, 1)
    g = S.ssim_grad(x, y, mode=mode)
    h = 1e-6
    for (i, j) in ((0, 0), (3, 7), (7, 6), (14, 13), (10, 2)):
        xp, xm = x.copy(), x.copy()
        xp[i, j] += h
        xm[i, j] -= h
        fd = (S.ssim_map(xp, y, mode=mode).mean() - S.ssim_map(xm, y, mode=mode).mean()) / (2 * h)
        assert g[i, j] == pytest.approx(fd, rel=1e-6, abs=1e-10), (i, j)


def test_gradient_vanishes_at_identity():
    # SSIM is at its maximum 1 when x = y
    x = np.random.default_rng(5).random((16, 16))
    np.testing.assert_allclose(S.ssim_grad(x, x), 0.0, atol=1e-12)
