"""The precision form against the FP64 truth: SH coefficients stored in BF16 or
FP16 (rounded to nearest from the FP32 parameters), blend and accumulation in
FP32, compared per output with the FP64 oracle of the unrounded FP32
parameters, on the 1920x1080 / 1M-Gaussian scene and the 3840x2160 /
3M-Gaussian scene at d = 2 (64 sampled tiles each; every Gaussian projected).

The bounds are derived, not fitted:
* colour of Gaussian i: |rgb(stored) - rgb(FP32)| <= u sum_k |Y_k(dir_i)| |sh_ik|
  (u the unit roundoff of the storage type, 2^-8 for BF16 and 2^-11 for FP16:
  each coefficient moves by at most u of itself; FP16 coefficients below its
  normal range move by at most 2^-25), and the clamp at zero only shrinks the
  difference;
* image: a pixel is a convex combination of colours (the blend weights do not
  depend on colour and sum to 1 - T_final), so its storage error is at most the
  largest colour error of the Gaussians of its tile; with FP32 arithmetic the
  GPU's error is within that plus the 1e-4 image tolerance;
* gradients and densification statistics: within the effect of storage alone
  (the FP64 oracle run on the stored coefficients against the FP64 oracle on
  the FP32 ones, per tensor relative to its maximum) plus the 1e-3 gradient
  tolerance (triangle inequality).
The measured errors and the storage-only effects are recorded per output
(gpu_util.REPORT, written out with GS_PARITY_REPORT).
"""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2412_13547_b300 import raster as R
from paper_2412_13547_b300 import scenes

import gpu_util as U

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4
GRAD_TOL = 1e-3
UNIT_ROUNDOFF = {torch.bfloat16: 2.0 ** -8, torch.float16: 2.0 ** -11}
NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")


def _camera_centre(cam):
    Rm = np.asarray(cam.R, np.float64).reshape(3, 3)
    return -Rm.T @ np.asarray(cam.T, np.float64).reshape(3)


def _colour_bound(p64, rows, cam, u):
    """u sum_k |Y_k(dir)| |sh_k| per Gaussian and channel (rows only)."""
    c = _camera_centre(cam)
    deg = int(round(np.sqrt(p64["sh"].shape[1]))) - 1
    out = np.zeros((rows.size, 3))
    for j, g in enumerate(rows):
        d = p64["means"][g] - c
        Y = np.abs(orc.sh_basis(deg, d / np.linalg.norm(d)))
        # relative rounding u of each coefficient, and half the smallest FP16 subnormal step
        # (2^-25) for coefficients below the normal range
        out[j] = u * (Y[:, None] * np.abs(p64["sh"][g])).sum(0) + 2.0 ** -25 * Y.sum()
    return out


@pytest.mark.parametrize("sh_dtype", [torch.bfloat16, torch.float16], ids=["bf16", "fp16"])
@pytest.mark.parametrize("workload", ["hd", "uhd"])
def test_storage_error_against_fp64_of_fp32_parameters(workload, sh_dtype):
    scene, cam, _ = scenes.workload_hd() if workload == "hd" else scenes.workload_uhd()
    p32 = U.params_np(scene)
    dil = R.Dilation(2, 1, 0)
    ocam, odil = orc.as_camera(cam), orc.as_dilation(dil)
    out, rast, p, (img, t_final, last) = U.run_forward(p32, cam, dil, sh_dtype=sh_dtype)
    w_ds, h_ds, tx, ty = out["grid"]
    u = UNIT_ROUNDOFF[sh_dtype]
    # FP64 truth of the FP32 parameters, and the FP64 oracle of the stored coefficients
    p64 = U.params_f64(p32)
    p64s = dict(p64)
    p64s["sh"] = p.sh_store.float().cpu().numpy().astype(np.float64)
    o = orc.project(p64, ocam, odil)
    os_ = orc.project(p64s, ocam, odil)
    rng = np.random.default_rng(4 if workload == "hd" else 5)
    nonempty = np.nonzero(out["ranges"][:, 1] > out["ranges"][:, 0])[0]
    tiles = np.sort(rng.choice(nonempty, 64, replace=False)).astype(np.int32)
    # the lists depend on geometry only: the same for every storage type
    sv, sr = orc.bin_tiles(out["rects"], U.gpu_depth_bits(out), tx, tiles)
    of = orc.render_fwd(o, sv, sr, ocam, odil, (0.0, 0.0, 0.0), tile_ids=tiles)
    ofs = orc.render_fwd(os_, sv, sr, ocam, odil, (0.0, 0.0, 0.0), tile_ids=tiles)
    mask = np.zeros(tx * ty, bool)
    mask[tiles] = True
    flagged = ((o["flags"] | os_["flags"]) & orc.FLAG_AMBIGUOUS) != 0
    pm = U.tile_pixel_mask(mask, w_ds, h_ds, tx, dil.tile) & ~of["ambiguous"] & ~ofs["ambiguous"]
    ids = np.unique(sv)
    # colours: storage error within its analytic bound
    bound_rgb = _colour_bound(p64, ids, cam, u)
    drgb = np.abs(os_["rgb"][ids] - o["rgb"][ids])
    assert (drgb <= bound_rgb * (1 + 1e-9) + 1e-12).all()
    # image: storage error within the largest colour error, GPU error within that + 1e-4
    storage_img = np.abs(ofs["img"] - of["img"])[pm].max()
    gpu_img = np.abs(out["img"] - of["img"])[pm].max()
    assert storage_img <= drgb.max() + 1e-12
    assert gpu_img <= drgb.max() + IMG_TOL, (gpu_img, drgb.max())
    key = f"{workload}/{str(sh_dtype).replace('torch.', '')}"
    U.REPORT[U.report_key(f"{key}:image")] = dict(gpu_vs_fp64=float(gpu_img), storage_only=float(storage_img),
                                              colour_bound=float(bound_rgb.max()), colour_err=float(drgb.max()),
                                              pixels=int(pm.sum()))
    # backward of a fixed upstream gradient on the sampled tiles (an L1 loss would add sign
    # flips where the render sits within the storage error of the target)
    dl = rng.standard_normal(out["img"].shape) * 1e-3
    dl[~pm] = 0.0
    rast.render_bwd(cam, dil, (0.0, 0.0, 0.0), t_final, last, torch.tensor(dl, dtype=torch.float32, device=U.DEV))
    torch.cuda.synchronize()
    og = orc.render_bwd(o, sv, sr, ocam, odil, dl.astype(np.float32), tile_ids=tiles)
    ogs = orc.render_bwd(os_, sv, sr, ocam, odil, dl.astype(np.float32), tile_ids=tiles)
    g2d = rast.grad2d.cpu().numpy()
    gg = U.split_grad2d(g2d)
    for k in ("dxy", "dconic", "dopacity", "drgb"):
        st = U.max_rel(ogs[k], og[k])
        err = U.grad_report(f"{key}:{k}", gg[k], og[k])
        U.REPORT[U.report_key(f"{key}:{k}")]["storage_only"] = st
        assert err <= st + GRAD_TOL, (k, err, st)
    # parameter gradients and densification statistics, on the Gaussians of the sampled tiles
    # (a colour clamp that the rounding moves across zero changes that Gaussian's SH gradient
    # discontinuously: such rows are counted and left out)
    clamp_flip = ((o["rgb"] > 0) != (os_["rgb"] > 0)).any(1)
    rows = np.nonzero((np.abs(g2d).sum(1) > 0) & ~flagged & ~clamp_flip & (o["tiles_touched"] > 0))[0]
    grads = [torch.empty(tuple(t.shape), dtype=torch.float32, device=U.DEV) for t in p.tensors()]
    pos, col = torch.zeros(p.n, device=U.DEV), torch.zeros(p.n, device=U.DEV)
    cnt = torch.zeros(p.n, dtype=torch.int32, device=U.DEV)
    R.gs_project_bwd(p.means, p.log_scales, p.quats, p.opacity_logits, p.sh_store, cam, dil, rast.tiles_touched,
                     rast.grad2d, *grads, pos, col, cnt)
    torch.cuda.synchronize()
    sub = {k: v[rows] for k, v in p64.items()}
    subs = {k: v[rows] for k, v in p64s.items()}
    ref = orc.project_bwd(sub, ocam, odil, {k: v[rows] for k, v in og.items()})
    refs = orc.project_bwd(subs, ocam, odil, {k: v[rows] for k, v in ogs.items()})
    for i, name in enumerate(NAMES):
        st = U.max_rel(refs[name], ref[name])
        err = U.grad_report(f"{key}:d_{name}", grads[i].cpu().numpy()[rows], ref[name])
        U.REPORT[U.report_key(f"{key}:d_{name}")]["storage_only"] = st
        assert err <= st + GRAD_TOL, (name, err, st)
    rp, rc, rn = np.zeros(rows.size), np.zeros(rows.size), np.zeros(rows.size, np.int32)
    orc.densify_stats(o["tiles_touched"][rows], {k: v[rows] for k, v in og.items()}, rp, rc, rn)
    sp, sc, sn = np.zeros(rows.size), np.zeros(rows.size), np.zeros(rows.size, np.int32)
    orc.densify_stats(o["tiles_touched"][rows], {k: v[rows] for k, v in ogs.items()}, sp, sc, sn)
    for name, gpu, r64, s64 in (("pos_acc", pos, rp, sp), ("col_acc", col, rc, sc)):
        st = U.max_rel(s64, r64)
        err = U.grad_report(f"{key}:{name}", gpu.cpu().numpy()[rows], r64)
        U.REPORT[U.report_key(f"{key}:{name}")]["storage_only"] = st
        assert err <= st + GRAD_TOL, (name, err, st)
    U.REPORT[U.report_key(f"{key}:rows")] = dict(compared=int(rows.size), clamp_flipped=int(clamp_flip[ids].sum()),
                                             gaussians_in_tiles=int(ids.size))
