"""gs_ssim and gs_loss_l1_dssim (through the C ABI) against the FP64 SSIM
oracle (oracle/ssim.py, pinned in test_ssim_pins.py) and the L1 oracle.

Tolerances: the mean SSIM within 2e-5 (FP32 window sums of values in [0, 1],
accumulated in double), gradients within 1e-3 of the per-tensor maximum (the
gradient tolerance of the other parity tests), the loss within 1e-5.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from oracle import ssim as S
from paper_2412_13547_b300 import raster as R
from paper_2412_13547_b300 import scenes

import gpu_util as U

pytestmark = pytest.mark.gpu

SSIM_TOL = 2e-5
GRAD_TOL = 1e-3


def _images(w, h, seed):
    """A rendered-looking image (smooth field plus noise) and a target close to it."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:h, 0:w]
    base = np.stack([0.5 + 0.4 * np.sin(xx / (7.0 + c) + yy / (11.0 - c)) for c in range(3)], -1)
    img = np.clip(base + rng.normal(0, 0.05, base.shape), 0, 1)
    tgt = np.clip(base + rng.normal(0, 0.08, base.shape), 0, 1)
    return img.astype(np.float32), tgt.astype(np.float32)


def _cam(w, h):
    return scenes.look_at(scenes.orbit_eye(3.0, 10.0, 10.0), width=w, height=h)


CASES = [(40, 23, R.Dilation(1, 0, 0)), (131, 97, R.Dilation(1, 0, 0)), (300, 170, R.Dilation(2, 1, 0)),
         (257, 199, R.Dilation(3, 2, 1))]


def test_ssim_u8_target_matches_its_fp32_values():
    """An 8-bit target gives the SSIM, the gradient and the D-SSIM loss of the
    FP32 target holding t * (1/255) (the per-pixel results bit for bit, the
    sums up to the order of their atomic additions), and the oracle's SSIM of it."""
    w, h, dil = 300, 170, R.Dilation(2, 1, 0)
    cam = _cam(w, h)
    w_ds, h_ds, _, _ = R.gs_grid(cam, dil)
    _, tgt = _images(w, h, 3)
    img, _ = _images(w_ds, h_ds, 4)
    t8 = np.clip(np.rint(tgt.astype(np.float64) * 255.0), 0, 255).astype(np.uint8)
    t8f = t8.astype(np.float32) * np.float32(1.0 / 255.0)
    ws = torch.empty(R.gs_ssim_workspace_size(cam, dil), dtype=torch.uint8, device=U.DEV)
    ti = torch.tensor(img, device=U.DEV)
    res = []
    for target in (torch.tensor(t8, device=U.DEV), torch.tensor(t8f, device=U.DEV)):
        out = torch.zeros(1, device=U.DEV)
        g = torch.zeros((h_ds, w_ds, 3), device=U.DEV)
        R.gs_ssim(cam, dil, ti, target, out, ws, d_img=g, mode=R.SSIM_SAME)
        dl = torch.zeros((h_ds, w_ds, 3), device=U.DEV)
        loss = torch.zeros(1, device=U.DEV)
        R.gs_loss_l1_dssim(cam, dil, ti, target, 0.2, dl, loss, ws)
        res.append((out.item(), g.cpu().numpy(), loss.item(), dl.cpu().numpy()))
    assert abs(res[0][0] - res[1][0]) <= 1e-6 and abs(res[0][2] - res[1][2]) <= 1e-6 * abs(res[1][2])
    np.testing.assert_array_equal(res[0][1], res[1][1])
    np.testing.assert_array_equal(res[0][3], res[1][3])
    ref = S.ssim(img.astype(np.float64), _lattice(t8f.astype(np.float64), dil, w_ds, h_ds), mode="same")
    assert abs(res[0][0] - ref) < SSIM_TOL


def _lattice(tgt_hr, dil, w_ds, h_ds):
    return tgt_hr[dil.oy::dil.d, dil.ox::dil.d][:h_ds, :w_ds]


@pytest.mark.parametrize("mode", [R.SSIM_VALID, R.SSIM_SAME], ids=["valid", "same"])
@pytest.mark.parametrize("w,h,dil", CASES, ids=[f"{c[0]}x{c[1]}d{c[2].d}" for c in CASES])
def test_ssim_and_gradient_against_oracle(w, h, dil, mode):
    cam = _cam(w, h)
    w_ds, h_ds, _, _ = R.gs_grid(cam, dil)
    _, tgt = _images(w, h, 1)
    img, _ = _images(w_ds, h_ds, 2)
    if mode == R.SSIM_VALID and min(w_ds, h_ds) < 11:
        pytest.skip("no valid window")
    ws = torch.empty(R.gs_ssim_workspace_size(cam, dil), dtype=torch.uint8, device=U.DEV)
    out = torch.zeros(1, device=U.DEV)
    g = torch.full((h_ds, w_ds, 3), 7.0, device=U.DEV)
    R.gs_ssim(cam, dil, torch.tensor(img, device=U.DEV), torch.tensor(tgt, device=U.DEV), out, ws, d_img=g, mode=mode)
    torch.cuda.synchronize()
    y = _lattice(tgt.astype(np.float64), dil, w_ds, h_ds)
    x = img.astype(np.float64)
    sm = "valid" if mode == R.SSIM_VALID else "same"
    ref = S.ssim(x, y, mode=sm)
    assert abs(out.item() - ref) < SSIM_TOL, (out.item(), ref)
    gref = np.stack([S.ssim_grad(x[..., c], y[..., c], mode=sm) for c in range(3)], -1) / 3.0
    assert U.grad_report("d_img", g.cpu().numpy(), gref) < GRAD_TOL


def test_ssim_rejects_small_valid_lattices_and_bad_modes():
    cam = _cam(20, 30)
    ws = torch.empty(R.gs_ssim_workspace_size(cam, R.Dilation()), dtype=torch.uint8, device=U.DEV)
    img = torch.zeros(30, 20, 3, device=U.DEV)
    out = torch.zeros(1, device=U.DEV)
    with pytest.raises(R.GsError):
        R.gs_ssim(cam, R.Dilation(2, 0, 0), img[:15, :10].contiguous(), img, out, ws, mode=R.SSIM_VALID)
    with pytest.raises(R.GsError):
        R.gs_ssim(cam, R.Dilation(), img, img, out, ws, mode=2)


def test_identical_images_give_one_and_zero_gradient():
    cam = _cam(64, 48)
    img, _ = _images(64, 48, 3)
    t = torch.tensor(img, device=U.DEV)
    ws = torch.empty(R.gs_ssim_workspace_size(cam, R.Dilation()), dtype=torch.uint8, device=U.DEV)
    out = torch.zeros(1, device=U.DEV)
    g = torch.empty_like(t)
    R.gs_ssim(cam, R.Dilation(), t, t, out, ws, d_img=g, mode=R.SSIM_SAME)
    torch.cuda.synchronize()
    assert abs(out.item() - 1.0) < 1e-6
    assert float(g.abs().max()) < 1e-6


@pytest.mark.parametrize("lam", [0.0, 0.2, 1.0])
def test_l1_dssim_loss_against_oracle(lam):
    w, h = 300, 170
    cam = _cam(w, h)
    dil = R.Dilation(2, 1, 1)
    w_ds, h_ds, _, _ = R.gs_grid(cam, dil)
    _, tgt = _images(w, h, 4)
    img, _ = _images(w_ds, h_ds, 5)
    ws = torch.empty(R.gs_ssim_workspace_size(cam, dil), dtype=torch.uint8, device=U.DEV)
    loss = torch.zeros(1, device=U.DEV)
    dl = torch.empty(h_ds, w_ds, 3, device=U.DEV)
    R.gs_loss_l1_dssim(cam, dil, torch.tensor(img, device=U.DEV), torch.tensor(tgt, device=U.DEV), lam, dl, loss, ws)
    torch.cuda.synchronize()
    l1, gl1 = orc.loss_l1(img, tgt, orc.as_camera(cam), orc.as_dilation(dil))
    x = img.astype(np.float64)
    y = _lattice(tgt.astype(np.float64), dil, w_ds, h_ds)
    s = S.ssim(x, y, mode="same")
    gs_ = np.stack([S.ssim_grad(x[..., c], y[..., c], mode="same") for c in range(3)], -1) / 3.0
    assert abs(loss.item() - ((1 - lam) * l1 + lam * (1 - s))) < 1e-5
    assert U.grad_report("dl", dl.cpu().numpy(), (1 - lam) * gl1 - lam * gs_) < GRAD_TOL


def test_train_steps_with_dssim_loss():
    """TrainStep and BatchTrainStep with lambda = 0.2: the loss they record is
    (1 - lambda) L1 + lambda (1 - SSIM) of the image they rendered (oracle
    evaluation of that image), and the step moves the parameters."""
    from paper_2412_13547_b300.pipeline import AdamConfig, BatchTrainStep, Rasterizer, TrainStep
    s, cam, tgt = scenes.workload_small()
    p32 = U.params_np(s)
    dil = R.Dilation(2, 1, 0)
    p = U.gpu_params(p32)
    w_ds, h_ds, tx, ty = R.gs_grid(cam, dil)
    rast = Rasterizer(p.n, capacity=1 << 16, max_tiles=tx * ty)
    step = TrainStep(p, rast, AdamConfig(), max_pixels=w_ds * h_ds, dssim_lambda=0.2)
    t = torch.tensor(tgt, device=U.DEV)
    before = p.means.clone()
    loss = step(cam, dil, t)
    torch.cuda.synchronize()
    img = step.img[:3 * w_ds * h_ds].view(h_ds, w_ds, 3).cpu().numpy().astype(np.float64)
    l1, _ = orc.loss_l1(img, tgt, orc.as_camera(cam), orc.as_dilation(dil))
    y = _lattice(tgt.astype(np.float64), dil, w_ds, h_ds)
    assert abs(loss.item() - (0.8 * l1 + 0.2 * (1 - S.ssim(img, y, mode="same")))) < 1e-5
    assert bool((p.means != before).any())
    # the batched step: two views, the same loss per view
    p2 = U.gpu_params(p32)
    cam2 = scenes.look_at(scenes.orbit_eye(4.0, 120.0, 30.0), width=96, height=80)
    tg2 = [t, torch.tensor(scenes.target_image(96, 80, 3), device=U.DEV)]
    bs = BatchTrainStep(p2, [cam, cam2], tg2, d=2, dssim_lambda=0.2, optimize=False)
    bs.render_pass(0)
    torch.cuda.synchronize()
    for i, c in enumerate([cam, cam2]):
        d = bs._dil(0, i)
        w2, h2, _, _ = R.gs_grid(c, d)
        im = bs.img[i].view(-1)[:3 * w2 * h2].view(h2, w2, 3).cpu().numpy().astype(np.float64)
        tt = tg2[i].cpu().numpy().astype(np.float64)
        l1, _ = orc.loss_l1(im, tt, orc.as_camera(c), orc.as_dilation(d))
        ref = 0.8 * l1 + 0.2 * (1 - S.ssim(im, _lattice(tt, d, w2, h2), mode="same"))
        assert abs(bs.loss[i].item() - ref) < 1e-5
