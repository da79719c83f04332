"""Parity of the CUDA path (through the C ABI) against the FP64 oracle.

Staged as the method is: projection (continuous values within FP32 rounding,
integer radius/rect/tile counts exact except where the oracle flags a decision
within rounding distance of its threshold), binning (bit-exact: the oracle's
binning of the GPU's own FP32 rects and depth bits), blending (image within
1e-4 abs), backward (gradients within 1e-3 of the per-tensor maximum), and
the full step. Tolerances: images 1e-4 max abs,
gradients 1e-3 relative, keys/sort order/ranges bit-exact.
"""
import math

import numpy as np
import pytest
import torch

from oracle import lowp
from oracle import oracle as orc
from paper_2412_13547_b300 import raster as R
from paper_2412_13547_b300 import scenes
from paper_2412_13547_b300.pipeline import (AdamConfig, BatchTrainStep, GaussianParams, Rasterizer, TrainStep,
                                            image_buffers)

import gpu_util as U

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4
GRAD_TOL = 1e-3


def scene_small():
    s, cam, tgt = scenes.workload_small()
    return U.params_np(s), cam, tgt


def scene_sh3(w=160, h=120):
    s = scenes.small_scene(3000, index=11, sh_degree=3, log_scale_mean=-2.6)
    s.sh[:, 1:, :] = np.random.default_rng(5).normal(0, 0.1, s.sh[:, 1:, :].shape)
    cam = scenes.look_at(scenes.orbit_eye(3.0, 60.0, 25.0), width=w, height=h)
    return U.params_np(s), cam, scenes.target_image(w, h, 11)


def scene_clusters(n=40000, w=1280, h=720, index=5):
    s = scenes.cluster_scene(n, index=index, log_scale_mean=-3.6)
    cam = scenes.look_at(scenes.orbit_eye(2.6, 30.0, 20.0), width=w, height=h)
    return U.params_np(s), cam, scenes.target_image(w, h, index)


DILATIONS = [R.Dilation(1, 0, 0), R.Dilation(2, 1, 0), R.Dilation(2, 0, 1, 1), R.Dilation(4, 3, 3),
             R.Dilation(1, 0, 0, tile=8), R.Dilation(2, 1, 1, tile=32), R.Dilation(3, 2, 0)]


def _dil_id(d):
    return f"d{d.d}o{d.ox}{d.oy}m{d.center_mode}t{d.tile}"


# ---------------------------------------------------------------------------
# Projection
# ---------------------------------------------------------------------------

def check_projection(p32, cam, dil, out, sh_f64=None):
    p64 = U.params_f64(p32)
    if sh_f64 is not None:
        p64["sh"] = sh_f64
    o = orc.project(p64, orc.as_camera(cam), orc.as_dilation(dil))
    flagged = (o["flags"] & orc.FLAG_AMBIGUOUS) != 0
    ok = ~flagged
    assert flagged.mean() < 0.02, flagged.mean()
    np.testing.assert_array_equal(out["radii"][ok], o["radius"][ok])
    np.testing.assert_array_equal(out["rects"][ok], o["rect"][ok])
    np.testing.assert_array_equal(out["tiles_touched"][ok], o["tiles_touched"][ok])
    vis = ok & (o["tiles_touched"] > 0)
    g = U.gpu_proj_as_oracle(out)
    assert np.abs(g["xy"][vis] - o["xy"][vis]).max(initial=0) < 1e-4
    cmax = np.abs(o["conic"][vis]).max(1, initial=0)[:, None]
    assert (np.abs(g["conic"][vis] - o["conic"][vis]) <= 2e-5 * cmax + 1e-12).all()
    assert np.abs(g["opacity"][vis] - o["opacity"][vis]).max(initial=0) < 1e-6
    assert np.abs(g["rgb"][vis] - o["rgb"][vis]).max(initial=0) < 2e-5
    assert (np.abs(g["depth"][vis] - o["depth"][vis]) <= 1e-6 * o["depth"][vis]).all()
    return o


@pytest.mark.parametrize("dil", DILATIONS, ids=_dil_id)
def test_projection_parity_small(dil):
    p32, cam, _ = scene_small()
    out, *_ = U.run_forward(p32, cam, dil)
    check_projection(p32, cam, dil, out)


@pytest.mark.parametrize("sh_dtype", [torch.float32, torch.bfloat16, torch.float16])
def test_projection_parity_sh3_storage(sh_dtype):
    p32, cam, _ = scene_sh3()
    dil = R.Dilation(2, 1, 0)
    out, _, p, _ = U.run_forward(p32, cam, dil, sh_dtype=sh_dtype)
    # the oracle sees exactly the stored (rounded) coefficients
    sh_f64 = p.sh_store.float().cpu().numpy().astype(np.float64)
    check_projection(p32, cam, dil, out, sh_f64=sh_f64)


# ---------------------------------------------------------------------------
# Binning: bit-exact
# ---------------------------------------------------------------------------

def check_binning(out):
    w_ds, h_ds, tx, ty = out["grid"]
    keys, vals, ranges = orc.bin_sort(out["rects"], out["tiles_touched"].astype(np.int64), U.gpu_depth_bits(out),
                                      tx, ty)
    assert out["k"] == len(vals) == int(out["tiles_touched"].astype(np.int64).sum())
    np.testing.assert_array_equal(out["sorted_ids"], vals)
    np.testing.assert_array_equal(out["ranges"], ranges)
    np.testing.assert_array_equal(U.gpu_keys(out), keys)


@pytest.mark.parametrize("dil", DILATIONS, ids=_dil_id)
def test_binning_bitexact_small(dil):
    p32, cam, _ = scene_small()
    out, *_ = U.run_forward(p32, cam, dil)
    check_binning(out)


@pytest.mark.parametrize("dil", [R.Dilation(1, 0, 0), R.Dilation(2, 1, 1), R.Dilation(1, 0, 0, tile=8)], ids=_dil_id)
def test_binning_bitexact_many_pairs(dil):
    """Millions of pairs, thousands of tiles: several sort blocks, two tile passes."""
    p32, cam, _ = scene_clusters()
    out, *_ = U.run_forward(p32, cam, dil)
    assert out["k"] > 1_000_000 or dil.d > 1
    check_binning(out)


@pytest.mark.parametrize("dil", [R.Dilation(1, 0, 0, tile=8), R.Dilation(2, 1, 0, tile=8)], ids=_dil_id)
def test_binning_bitexact_both_paths(dil):
    """2560x1440 with 8 px tiles: d=1 gives 320x180 tiles (long rows for the
    tile-level scatter), d=2 160x90. Both must equal the oracle bit for bit."""
    p32, cam, _ = scene_clusters(n=60000, w=2560, h=1440, index=6)
    out, *_ = U.run_forward(p32, cam, dil)
    check_binning(out)


@pytest.mark.parametrize("dil", [R.Dilation(1, 0, 0), R.Dilation(2, 1, 1, bin_shift=2)],
                         ids=["d1", "d2shift2"])
def test_binning_from_projection_keys_is_identical(dil):
    """gs_project's depth keys (the float bits of a visible Gaussian's depth,
    all ones for a culled one) given to gs_bin_sort give the same lists, ranges
    and pair count, bit for bit, as its own pass over the splat records."""
    p32, cam, _ = scene_clusters()
    p = U.gpu_params(p32)
    n = p.n
    btx, bty = R.gs_bin_grid(cam, dil)
    splats = torch.zeros(n, R.SPLAT_FLOATS, device=U.DEV)
    radii = torch.zeros(n, dtype=torch.int32, device=U.DEV)
    rects = torch.zeros(n, 4, dtype=torch.int32, device=U.DEV)
    tiles = torch.zeros(n, dtype=torch.int32, device=U.DEV)
    # a key array that is 4- but not 16-byte aligned (a row of a batch's key matrix can be)
    keys = torch.full((n + 1,), 7, dtype=torch.int32, device=U.DEV)[1:]
    R.gs_project(p.means, p.log_scales, p.quats, p.opacity_logits, p.sh_store, cam, dil, splats, radii, rects, tiles,
                 depth_keys=keys)
    k = int(tiles.to(torch.int64).sum().item())
    cap = k + 1000
    aligned = torch.empty_like(keys)
    aligned.copy_(keys)
    res = []
    for use_keys in (None, keys, aligned):
        ws = torch.empty(R.gs_bin_sort_workspace_size(n, cap, btx, bty), dtype=torch.uint8, device=U.DEV)
        ids = torch.full((cap,), -1, dtype=torch.int32, device=U.DEV)
        rng = torch.full((btx * bty, 2), -1, dtype=torch.int32, device=U.DEV)
        num = torch.zeros(1, dtype=torch.int64, device=U.DEV)
        R.gs_bin_sort(n, rects, tiles, splats, btx, bty, ws, cap, ids, rng, num, depth_keys=use_keys)
        torch.cuda.synchronize()
        res.append((num.item(), ids[:k].cpu().numpy(), rng.cpu().numpy()))
    for r in res[1:]:
        assert r[0] == res[0][0] == k
        np.testing.assert_array_equal(r[1], res[0][1])
        np.testing.assert_array_equal(r[2], res[0][2])
    kb = keys.cpu().numpy().view(np.uint32)
    vis = tiles.cpu().numpy() > 0
    depth_bits = splats[:, 9].cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(kb[vis], np.minimum(depth_bits[vis], 0xFFFFFFFE))
    assert (kb[~vis] == 0xFFFFFFFF).all() and (~vis).any()


def test_binning_equal_depths_keep_index_order():
    """Gaussians with identical depth bits: ties ordered by index."""
    n = 64
    rng = np.random.default_rng(3)
    p = dict(means=np.c_[rng.uniform(-0.3, 0.3, (n, 2)), np.zeros(n)].astype(np.float32),
             log_scales=np.full((n, 3), -2.0, np.float32),
             quats=np.tile([1, 0, 0, 0], (n, 1)).astype(np.float32),
             opacity_logits=np.zeros(n, np.float32), sh=np.zeros((n, 1, 3), np.float32))
    cam = scenes.Cam(R=np.eye(3), T=np.array([0.0, 0.0, 3.0]), fx=60.0, fy=60.0, cx=47.5, cy=31.5, width=96,
                     height=64)
    out, *_ = U.run_forward(p, cam, R.Dilation())
    assert len(np.unique(out["splats"][:, 9])) == 1
    check_binning(out)


# ---------------------------------------------------------------------------
# Blend forward / backward on the same lists
# ---------------------------------------------------------------------------

def render_case(p32, cam, dil, bg=(0.1, 0.2, 0.3), sh_dtype=torch.float32):
    out, rast, p, bufs = U.run_forward(p32, cam, dil, bg, sh_dtype=sh_dtype)
    p64 = U.params_f64(p32)
    # the oracle sees exactly the stored (rounded) coefficients
    p64["sh"] = p.sh_store.float().cpu().numpy().astype(np.float64)
    o = orc.project(p64, orc.as_camera(cam), orc.as_dilation(dil))
    # Gaussians the two sides cull differently get no exact comparison: their tiles are excluded
    cull_diff = (o["tiles_touched"] > 0) != (out["tiles_touched"] > 0)
    of = orc.render_fwd(o, out["sorted_ids"], out["ranges"], orc.as_camera(cam), orc.as_dilation(dil), bg)
    w_ds, h_ds, tx, ty = out["grid"]
    bad_tiles = np.zeros(tx * ty, bool)
    for g in np.nonzero(cull_diff)[0]:
        rc = out["rects"][g] if out["tiles_touched"][g] > 0 else o["rect"][g]
        for yy in range(rc[1], rc[3] + 1):
            bad_tiles[yy * tx + rc[0]: yy * tx + rc[2] + 1] = True
    excl = of["ambiguous"] | U.tile_pixel_mask(bad_tiles, w_ds, h_ds, tx, dil.tile)
    return out, rast, p, bufs, o, of, excl


def check_counts_outside(out, rast, o, cam, dil, excl, bg=(0.1, 0.2, 0.3)):
    """Blend counts (entries evaluated, entries blended, replayed list prefix).
    Over the tiles with no excluded pixel they must equal the oracle's exactly:
    the GPU renders again with the other tiles' lists emptied, the oracle
    blends only the kept tiles (same lists). Over the whole image they may
    differ only at excluded pixels, each by at most its tile's list length."""
    w_ds, h_ds, tx, ty = out["grid"]
    ys, xs = np.nonzero(excl)
    tile_of_px = (ys // dil.tile) * tx + xs // dil.tile
    bad = np.zeros(tx * ty, bool)
    bad[tile_of_px] = True
    lens = (out["ranges"][:, 1].astype(np.int64) - out["ranges"][:, 0].astype(np.int64))[:tx * ty]
    slack = int(lens[tile_of_px].sum())
    of_all = orc.render_fwd(o, out["sorted_ids"], out["ranges"], orc.as_camera(cam), orc.as_dilation(dil), bg)
    for i in (0, 1):
        ref = of_all["n_eval"] if i == 0 else of_all["n_blend"]
        assert abs(int(out["counts"][i]) - ref) <= slack, (i, int(out["counts"][i]), ref, slack)
    keep_tiles = np.nonzero(~bad)[0].astype(np.int32)
    print(f"counts: {keep_tiles.size} of {tx * ty} tiles without an excluded pixel; whole-image slack {slack}")
    if keep_tiles.size == 0:
        return
    ranges = rast.ranges.clone()
    ranges[:tx * ty][torch.tensor(bad, device=U.DEV)] = 0
    img, tf, last = image_buffers(h_ds, w_ds, U.DEV)
    counts = torch.zeros(3, dtype=torch.int64, device=U.DEV)
    R.gs_render_fwd(rast.n, rast.splats, rast.sorted_ids, ranges, cam, dil, bg, img, tf, last, counts)
    torch.cuda.synchronize()
    c = counts.cpu().numpy()
    # the oracle's ranges are indexed like its tile_ids
    of = orc.render_fwd(o, out["sorted_ids"], out["ranges"][keep_tiles], orc.as_camera(cam), orc.as_dilation(dil),
                        bg, tile_ids=keep_tiles)
    kp = ~U.tile_pixel_mask(bad, w_ds, h_ds, tx, dil.tile)
    assert c[0] == of["n_eval"], (c[0], of["n_eval"])
    assert c[1] == of["n_blend"], (c[1], of["n_blend"])
    assert c[2] == int(of["last"][kp].astype(np.int64).sum())


@pytest.mark.parametrize("dil", DILATIONS, ids=_dil_id)
def test_render_fwd_parity(dil):
    p32, cam, _ = scene_small()
    out, rast, p, bufs, o, of, excl = render_case(p32, cam, dil)
    # pixels where a gate value (alpha vs 1/255 or 0.99, transmittance vs 1e-4) lies within the
    # oracle's margin of its threshold may legitimately branch the other way in FP32
    assert excl.mean() < 5e-3
    keep = ~excl
    assert np.abs(out["img"] - of["img"])[keep].max() < IMG_TOL
    assert np.abs(out["t_final"] - of["t_final"])[keep].max() < 1e-5
    np.testing.assert_array_equal(out["last"][keep], of["last"][keep])
    # the backward's replay work: the sum of the pixels' last positions in their tile lists
    assert out["counts"][2] == int(out["last"].astype(np.int64).sum())
    check_counts_outside(out, rast, o, cam, dil, excl)


def scene_needles(n=1500, w=203, h=157, index=17):
    """Thin, rotated, mostly opaque Gaussians (aspect ratios up to ~50): their
    gate ellipses cover a small part of their bounding boxes, which is where the
    blend kernels' per-warp-block ellipse test skips work."""
    rng = np.random.default_rng(index)
    s = scenes.small_scene(n, index=index, sh_degree=0, log_scale_mean=-2.4)
    ls = np.stack([rng.normal(-1.9, 0.3, n), rng.normal(-5.2, 0.5, n), rng.normal(-3.5, 0.8, n)], 1)
    s.log_scales = ls.astype(np.float32)
    q = rng.normal(size=(n, 4))
    s.quats = (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(np.float32)
    # opacities from barely above the 1/255 gate to nearly 1
    s.opacity_logits = rng.uniform(-5.5, 5.0, n).astype(np.float32)
    cam = scenes.look_at(scenes.orbit_eye(2.8, 40.0, 30.0), width=w, height=h)
    return U.params_np(s), cam


@pytest.mark.parametrize("dil", [R.Dilation(1, 0, 0), R.Dilation(2, 1, 0), R.Dilation(1, 0, 0, tile=8),
                                 R.Dilation(2, 0, 1, tile=32), R.Dilation(3, 2, 1)], ids=_dil_id)
def test_render_fwd_parity_needles(dil):
    """No pixel that passes the gate is skipped: the blend order, counts and
    images equal the oracle's, which evaluates every pixel against every entry."""
    p32, cam = scene_needles()
    out, rast, p, bufs, o, of, excl = render_case(p32, cam, dil)
    assert excl.mean() < 5e-3
    keep = ~excl
    assert out["counts"][1] > 0
    assert np.abs(out["img"] - of["img"])[keep].max() < IMG_TOL
    np.testing.assert_array_equal(out["last"][keep], of["last"][keep])
    check_counts_outside(out, rast, o, cam, dil, excl)
    out, rast, p, o, og, g2d, excl = backward_case(p32, cam, dil)
    gg = U.split_grad2d(g2d)
    for k in ("dxy", "dconic", "dopacity", "drgb"):
        assert U.grad_report(k, gg[k], og[k]) < GRAD_TOL, (k, U.max_rel(gg[k], og[k]))


@pytest.mark.parametrize("sh_dtype", [torch.float32, torch.bfloat16, torch.float16])
def test_render_fwd_parity_sh3_ragged(sh_dtype):
    """SH degree 3 on ragged image sizes, with the SH stored in FP32, BF16 or
    FP16 (the oracle is given the stored coefficients): image within 1e-4,
    last index exact, and the 2D gradients within 1e-3."""
    p32, cam, _ = scene_sh3(131, 97)
    for dil in [R.Dilation(1, 0, 0), R.Dilation(2, 1, 1), R.Dilation(3, 0, 2, tile=8)]:
        out, rast, p, bufs, o, of, excl = render_case(p32, cam, dil, sh_dtype=sh_dtype)
        keep = ~excl
        assert np.abs(out["img"] - of["img"])[keep].max() < IMG_TOL
        np.testing.assert_array_equal(out["last"][keep], of["last"][keep])
    out, rast, p, o, og, g2d, excl = backward_case(p32, cam, R.Dilation(2, 1, 0), sh_dtype=sh_dtype)
    gg = U.split_grad2d(g2d)
    for k in ("dxy", "dconic", "dopacity", "drgb"):
        assert U.grad_report(k, gg[k], og[k]) < GRAD_TOL, k


@pytest.mark.parametrize("tile,ppts", [(8, (1, 2)), (16, (1, 2, 4)), (32, (2, 4))])
def test_launch_shape_does_not_change_results(tile, ppts):
    """pixels_per_thread is a launch shape: the forward is bit-identical across it
    and the backward differs only by the order of floating-point atomics."""
    p32, cam, _ = scene_sh3(131, 97)
    dil = R.Dilation(2, 1, 0, tile=tile)
    p = U.gpu_params(p32)
    w_ds, h_ds, tx, ty = R.gs_grid(cam, dil)
    outs = []
    for ppt in ppts:
        rast = Rasterizer(p.n, capacity=1 << 16, max_tiles=tx * ty, pixels_per_thread=ppt)
        rast.project(p, cam, dil)
        rast.bin_checked(cam, dil)
        img, tf, last = image_buffers(h_ds, w_ds)
        counts = torch.zeros(3, dtype=torch.int64, device=U.DEV)
        rast.render(cam, dil, (0.1, 0.2, 0.3), img, tf, last, counts)
        dl = torch.tensor(np.random.default_rng(0).standard_normal((h_ds, w_ds, 3)) * 1e-3, dtype=torch.float32,
                          device=U.DEV)
        rast.render_bwd(cam, dil, (0.1, 0.2, 0.3), tf, last, dl)
        torch.cuda.synchronize()
        outs.append([img.cpu().numpy(), tf.cpu().numpy(), last.cpu().numpy(), counts.cpu().numpy(),
                     rast.grad2d.cpu().numpy()])
    for o in outs[1:]:
        for a, b in zip(o[:4], outs[0][:4]):
            np.testing.assert_array_equal(a, b)
        assert U.max_rel(o[4], outs[0][4]) < 1e-5


def test_longest_first_order_does_not_change_results():
    """gs_tile_order only reorders the CTAs: forward bit-identical, backward equal
    up to the order of floating-point atomics; the order is a permutation."""
    p32, cam, _ = scene_sh3(200, 150)
    dil = R.Dilation(1, 0, 0)
    p = U.gpu_params(p32)
    w_ds, h_ds, tx, ty = R.gs_grid(cam, dil)
    outs = []
    for lf in (False, True):
        rast = Rasterizer(p.n, capacity=1 << 17, max_grid=(tx, ty), longest_first=lf)
        rast.project(p, cam, dil)
        rast.bin_checked(cam, dil)
        img, tf, last = image_buffers(h_ds, w_ds)
        rast.render(cam, dil, (0.2, 0.2, 0.2), img, tf, last)
        dl = torch.tensor(np.random.default_rng(1).standard_normal((h_ds, w_ds, 3)) * 1e-3, dtype=torch.float32,
                          device=U.DEV)
        rast.render_bwd(cam, dil, (0.2, 0.2, 0.2), tf, last, dl)
        torch.cuda.synchronize()
        outs.append((img.cpu().numpy(), tf.cpu().numpy(), last.cpu().numpy(), rast.grad2d.cpu().numpy()))
        if lf:
            order = rast.tile_order[:tx * ty].cpu().numpy()
            assert sorted(order.tolist()) == list(range(tx * ty))
            lens = (rast.ranges[:, 1] - rast.ranges[:, 0]).cpu().numpy()[order]
            # non-increasing up to the bucketing (8 buckets per octave)
            assert np.all(lens[:-1] + 1 >= (lens[1:] + 1) * 0.875)
    for a, b in zip(outs[0][:3], outs[1][:3]):
        np.testing.assert_array_equal(a, b)
    assert U.max_rel(outs[1][3], outs[0][3]) < 1e-5


@pytest.mark.parametrize("shift", [0, 2])
def test_forward_reuses_the_backward_order_of_the_same_view(shift):
    """After a backward, the next forward of the same camera and grid (another lattice
    offset) launches in that backward's order (no order kernel): results bit-identical to the
    list-length order; another camera gets the list-length order again."""
    p32, cam, _ = scene_sh3(200, 150)
    p = U.gpu_params(p32)
    d0, d1 = R.Dilation(2, 0, 0, bin_shift=shift), R.Dilation(2, 1, 1, bin_shift=shift)
    w_ds, h_ds, tx, ty = R.gs_grid(cam, d1)
    grid = R.gs_bin_grid(cam, R.Dilation(2, 0, 0, bin_shift=0))
    bg = (0.2, 0.2, 0.2)
    rast = Rasterizer(p.n, capacity=1 << 17, max_grid=grid)
    rast.project(p, cam, d0)
    rast.bin_checked(cam, d0)
    assert rast.fwd_order_kernels == 1
    w0, h0, _, _ = R.gs_grid(cam, d0)
    img, tf, last = image_buffers(h0, w0)
    rast.render(cam, d0, bg, img, tf, last)
    dl = torch.tensor(np.random.default_rng(1).standard_normal((h0, w0, 3)) * 1e-3, dtype=torch.float32,
                      device=U.DEV)
    rast.render_bwd(cam, d0, bg, tf, last, dl)
    bwd_order = rast.bwd_order[:tx * ty].clone()
    rast.project(p, cam, d1)
    rast.bin_checked(cam, d1)
    assert rast.fwd_order_kernels == 0
    np.testing.assert_array_equal(rast.tile_order[:tx * ty].cpu().numpy(), bwd_order.cpu().numpy())
    outs = []
    for r in (rast, Rasterizer(p.n, capacity=1 << 17, max_grid=grid)):
        if r is not rast:
            r.project(p, cam, d1)
            r.bin_checked(cam, d1)
            assert r.fwd_order_kernels == 1
        img, tf, last = image_buffers(h_ds, w_ds)
        r.render(cam, d1, bg, img, tf, last)
        torch.cuda.synchronize()
        outs.append((img.cpu().numpy(), tf.cpu().numpy(), last.cpu().numpy()))
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)
    assert sorted(rast.tile_order[:tx * ty].cpu().numpy().tolist()) == list(range(tx * ty))
    # another camera: the list-length order
    cam2 = scenes.look_at(scenes.orbit_eye(3.0, 40.0, 15.0), width=200, height=150)
    rast.render_bwd(cam, d1, bg, tf, last, torch.zeros(h_ds, w_ds, 3, device=U.DEV))
    rast.project(p, cam2, d1)
    rast.bin_checked(cam2, d1)
    assert rast.fwd_order_kernels == 1


def _tile_max_last(last, tile, tx, ty):
    h, w = last.shape
    pad = np.zeros((ty * tile, tx * tile), np.int64)
    pad[:h, :w] = last
    return pad.reshape(ty, tile, tx, tile).max(axis=(1, 3)).reshape(-1)


@pytest.mark.parametrize("shift", [0, 2])
def test_backward_order_by_last(shift):
    """gs_tile_order_by_last_batch: a permutation of all blend tiles of all
    views, non-increasing (up to the 8-per-octave bucketing) in the largest
    `last` of each tile, also with coarse binning, where the tiles of one
    binning tile share a list length but not their work."""
    p32, cam, _ = scene_clusters(20000, 400, 256)
    cams = [cam, scenes.look_at(scenes.orbit_eye(2.6, 150.0, 35.0), width=301, height=207)]
    dils = [R.Dilation(2, 1, 0, bin_shift=shift), R.Dilation(1, 0, 0, bin_shift=shift)]
    keys, total = [], 0
    views, alive = [], []
    for c, d in zip(cams, dils):
        out, rast, p, (img, tf, last) = U.run_forward(p32, c, d)
        w_ds, h_ds, tx, ty = R.gs_grid(c, d)
        keys.append(_tile_max_last(out["last"].astype(np.int64), d.tile, tx, ty))
        views.append(R.View(c, d, ranges=rast.ranges, last=last))
        total += tx * ty
        alive.append((rast, last))
    order = torch.full((total,), -1, dtype=torch.int32, device=U.DEV)
    R.gs_tile_order_by_last_batch(views, order)
    torch.cuda.synchronize()
    o = order.cpu().numpy()
    assert sorted(o.tolist()) == list(range(total))
    k = np.concatenate(keys)[o]
    assert k.max() > 0
    assert np.all(k[:-1] + 1 >= (k[1:] + 1) * 0.875)
    with pytest.raises(ValueError):
        R.gs_tile_order_by_last_batch(views, order[:total - 1])
    # the forward's order of the same views is a permutation too
    R.gs_tile_order_batch([R.View(v.cam, v.dil, ranges=v.ranges) for v in views], order)
    torch.cuda.synchronize()
    assert sorted(order.cpu().numpy().tolist()) == list(range(total))


def backward_case(p32, cam, dil, seed=0, bg=(0.1, 0.2, 0.3), sh_dtype=torch.float32):
    out, rast, p, (img, t_final, last), o, of, excl = render_case(p32, cam, dil, bg, sh_dtype)
    rng = np.random.default_rng(seed)
    dl = rng.standard_normal(out["img"].shape) * 1e-3
    dl[excl] = 0.0
    dl_t = torch.tensor(dl, dtype=torch.float32, device=U.DEV)
    rast.render_bwd(cam, dil, bg, t_final, last, dl_t)
    torch.cuda.synchronize()
    g2d = rast.grad2d.cpu().numpy()
    og = orc.render_bwd(o, out["sorted_ids"], out["ranges"], orc.as_camera(cam), orc.as_dilation(dil),
                        dl.astype(np.float32).astype(np.float64), bg)
    return out, rast, p, o, og, g2d, excl


@pytest.mark.parametrize("dil", DILATIONS, ids=_dil_id)
def test_render_bwd_parity(dil):
    p32, cam, _ = scene_small()
    out, rast, p, o, og, g2d, excl = backward_case(p32, cam, dil)
    gg = U.split_grad2d(g2d)
    for k in ("dxy", "dconic", "dopacity", "drgb"):
        assert U.grad_report(k, gg[k], og[k]) < GRAD_TOL, (k, U.max_rel(gg[k], og[k]))
    assert np.all(g2d[:, 9:] == 0.0)


def test_render_bwd_parity_sh3():
    p32, cam, _ = scene_sh3()
    out, rast, p, o, og, g2d, excl = backward_case(p32, cam, R.Dilation(2, 0, 1))
    gg = U.split_grad2d(g2d)
    for k in ("dxy", "dconic", "dopacity", "drgb"):
        assert U.grad_report(k, gg[k], og[k]) < GRAD_TOL, k


@pytest.mark.parametrize("sh_dtype", [torch.float32, torch.bfloat16, torch.float16])
def test_project_bwd_parity(sh_dtype):
    p32, cam, _ = scene_sh3()
    dil = R.Dilation(2, 1, 0)
    out, rast, p, o, og, g2d, excl = backward_case(p32, cam, dil)
    flagged = (o["flags"] & orc.FLAG_AMBIGUOUS) != 0
    g2d[flagged] = 0.0
    rast.grad2d.copy_(torch.tensor(g2d, device=U.DEV))
    pp = U.gpu_params(p32, sh_dtype)
    grads = [torch.empty_like(t, dtype=torch.float32) for t in pp.tensors()]
    R.gs_project_bwd(pp.means, pp.log_scales, pp.quats, pp.opacity_logits, pp.sh_store, cam, dil, rast.tiles_touched,
                     rast.grad2d, *grads)
    torch.cuda.synchronize()
    p64 = U.params_f64(p32)
    p64["sh"] = pp.sh_store.float().cpu().numpy().astype(np.float64)
    ref = orc.project_bwd(p64, orc.as_camera(cam), orc.as_dilation(dil), U.split_grad2d(g2d))
    for name, g in zip(("means", "log_scales", "quats", "opacity_logits", "sh"), grads):
        assert U.grad_report(name, g.cpu().numpy(), ref[name]) < GRAD_TOL, (name, U.max_rel(g.cpu().numpy(), ref[name]))


# ---------------------------------------------------------------------------
# Loss, densification statistics, Adam
# ---------------------------------------------------------------------------

def test_loss_l1_parity():
    _, cam, tgt = scene_small()
    for dil in [R.Dilation(1, 0, 0), R.Dilation(2, 1, 0), R.Dilation(3, 2, 1)]:
        w_ds, h_ds, _, _ = R.gs_grid(cam, dil)
        img = np.random.default_rng(1).uniform(0, 1, (h_ds, w_ds, 3)).astype(np.float32)
        t_img = torch.tensor(img, device=U.DEV)
        t_tgt = torch.tensor(tgt, device=U.DEV)
        dl = torch.empty_like(t_img)
        loss = torch.zeros(1, device=U.DEV)
        R.gs_loss_l1(cam, dil, t_img, t_tgt, dl, loss)
        L, g = orc.loss_l1(img, tgt, orc.as_camera(cam), orc.as_dilation(dil))
        assert abs(loss.item() - L) < 1e-6 * max(1.0, L)
        np.testing.assert_allclose(dl.cpu().numpy(), g, rtol=1e-6, atol=1e-12)


def _u8_target(tgt):
    """An 8-bit target and the FP32 values the kernels read for it (t * (1/255),
    1/255 rounded to FP32, the product rounded to FP32)."""
    t8 = np.clip(np.rint(np.asarray(tgt, np.float64) * 255.0), 0, 255).astype(np.uint8)
    return t8, t8.astype(np.float32) * np.float32(1.0 / 255.0)


def test_loss_l1_parity_u8_target():
    """An 8-bit target: the oracle on the values the header defines, and the
    FP32 path given those values, agree with the 8-bit path (the gradient bit
    for bit; the loss up to the order of its atomic sums)."""
    _, cam, tgt = scene_small()
    t8, t8f = _u8_target(tgt)
    assert t8f.dtype == np.float32 and np.abs(t8f - tgt).max() <= 0.5 / 255 + 1e-7
    for dil in [R.Dilation(1, 0, 0), R.Dilation(2, 1, 0), R.Dilation(3, 2, 1)]:
        w_ds, h_ds, _, _ = R.gs_grid(cam, dil)
        img = np.random.default_rng(2).uniform(0, 1, (h_ds, w_ds, 3)).astype(np.float32)
        img[0, 0] = t8f[dil.oy, dil.ox]  # a zero residual: sign(0) = 0 in both paths
        t_img = torch.tensor(img, device=U.DEV)
        outs = []
        for target in (torch.tensor(t8, device=U.DEV), torch.tensor(t8f, device=U.DEV)):
            dl = torch.empty_like(t_img)
            loss = torch.zeros(1, device=U.DEV)
            R.gs_loss_l1(cam, dil, t_img, target, dl, loss)
            outs.append((loss.item(), dl.cpu().numpy()))
        assert abs(outs[0][0] - outs[1][0]) <= 1e-6 * outs[1][0]
        np.testing.assert_array_equal(outs[0][1], outs[1][1])
        assert np.all(outs[0][1][0, 0] == 0.0)
        L, g = orc.loss_l1(img, t8f.astype(np.float64), orc.as_camera(cam), orc.as_dilation(dil))
        assert abs(outs[0][0] - L) < 1e-6 * max(1.0, L)
        np.testing.assert_allclose(outs[0][1], g, rtol=1e-6, atol=1e-12)


@pytest.mark.parametrize("u8", [False, True], ids=["f32_target", "u8_target"])
@pytest.mark.parametrize("dil", [R.Dilation(1, 0, 0), R.Dilation(2, 1, 0, bin_shift=2)], ids=["d1", "d2s2"])
def test_render_fwd_l1_equals_the_separate_calls(dil, u8):
    """gs_render_fwd_l1 = gs_render_fwd + gs_loss_l1 (image, T, last and dL/dimg bit for bit, the loss
    up to the order of its sums) and leaves the 2D-gradient rows zeroed."""
    p32, cam, tgt = scene_sh3(200, 150)
    p = U.gpu_params(p32)
    w_ds, h_ds, tx, ty = R.gs_grid(cam, dil)
    rast = Rasterizer(p.n, capacity=1 << 18, max_grid=R.gs_bin_grid(cam, dil))
    rast.project(p, cam, dil)
    rast.bin_checked(cam, dil)
    target = torch.tensor(scenes.quantize_u8(tgt) if u8 else tgt, device=U.DEV)
    bg = (0.2, 0.3, 0.1)
    img, tf, last = image_buffers(h_ds, w_ds)
    rast.render(cam, dil, bg, img, tf, last)
    dl = torch.empty_like(img)
    loss = torch.zeros(1, device=U.DEV)
    R.gs_loss_l1(cam, dil, img, target, dl, loss)
    img2, tf2, last2 = image_buffers(h_ds, w_ds)
    dl2 = torch.full_like(img, 7.0)
    loss2 = torch.full((1,), 5.0, device=U.DEV)
    rast.grad2d.fill_(3.0)
    counts = torch.zeros(3, dtype=torch.int64, device=U.DEV)
    rast.render_l1(cam, dil, bg, img2, tf2, last2, target, dl2, loss2, counts=counts)
    torch.cuda.synchronize()
    for a, b in ((img, img2), (tf, tf2), (last, last2), (dl, dl2)):
        assert torch.equal(a, b)
    assert abs(loss.item() - loss2.item()) <= 1e-6 * loss.item()
    assert int(torch.count_nonzero(rast.grad2d).item()) == 0
    assert counts[0].item() > 0
    # without the zeroing the rows are left alone
    rast.grad2d.fill_(3.0)
    rast.render_l1(cam, dil, bg, img2, tf2, last2, target, dl2, loss2, zero_grad2d=False)
    torch.cuda.synchronize()
    assert bool((rast.grad2d == 3.0).all())


def test_densify_stats_parity():
    p32, cam, _ = scene_small()
    out, rast, p, o, og, g2d, excl = backward_case(p32, cam, R.Dilation(2, 1, 1))
    n = p.n
    pos = torch.zeros(n, device=U.DEV)
    col = torch.zeros(n, device=U.DEV)
    cnt = torch.zeros(n, dtype=torch.int32, device=U.DEV)
    for _ in range(2):
        R.gs_densify_stats(n, rast.tiles_touched, rast.grad2d, pos, col, cnt)
    # fused path of the projection backward gives the same accumulation
    pos2, col2, cnt2 = torch.zeros_like(pos), torch.zeros_like(col), torch.zeros_like(cnt)
    grads = [torch.empty_like(t, dtype=torch.float32) for t in p.tensors()]
    R.gs_project_bwd(p.means, p.log_scales, p.quats, p.opacity_logits, p.sh_store, cam, R.Dilation(2, 1, 1),
                     rast.tiles_touched, rast.grad2d, *grads, pos2, col2, cnt2)
    torch.cuda.synchronize()
    rp, rc, rn = np.zeros(n), np.zeros(n), np.zeros(n, np.int32)
    gg = U.split_grad2d(g2d)
    for _ in range(2):
        orc.densify_stats(out["tiles_touched"], gg, rp, rc, rn)
    np.testing.assert_allclose(pos.cpu().numpy(), rp, rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(col.cpu().numpy(), rc, rtol=1e-6, atol=1e-12)
    np.testing.assert_array_equal(cnt.cpu().numpy(), rn)
    np.testing.assert_allclose(pos2.cpu().numpy() * 2, rp, rtol=1e-6, atol=1e-12)
    np.testing.assert_array_equal(cnt2.cpu().numpy() * 2, rn)


@pytest.mark.parametrize("masked", [False, True])
def test_adam_parity(masked):
    rng = np.random.default_rng(7)
    shapes = [(1001, 3), (1001, 4), (1001,), (1001, 16, 3)]
    params = [rng.standard_normal(s).astype(np.float32) for s in shapes]
    mask = (rng.uniform(size=1001) < 0.6).astype(np.uint8) if masked else None
    dev = [dict(param=torch.tensor(x, device=U.DEV), grad=torch.zeros(x.shape, device=U.DEV),
                m=torch.zeros(x.shape, device=U.DEV), v=torch.zeros(x.shape, device=U.DEV), lr=1e-2 * (i + 1))
           for i, x in enumerate(params)]
    # the shadow mirrors the parameter; rows the mask skips keep their old copy
    shadow = dev[3]["param"].to(torch.bfloat16)
    dev[3]["shadow"] = shadow
    ref = [dict(p=x.astype(np.float64), m=np.zeros(x.shape), v=np.zeros(x.shape)) for x in params]
    mask_t = None if mask is None else torch.tensor(mask, device=U.DEV)
    for step in range(1, 4):
        for i, x in enumerate(params):
            g = rng.standard_normal(x.shape).astype(np.float32)
            dev[i]["grad"].copy_(torch.tensor(g))
            orc.adam(ref[i]["p"], g.astype(np.float64), ref[i]["m"], ref[i]["v"], 1e-2 * (i + 1), 0.9, 0.999, 1e-8,
                     step, row_mask=mask)
        R.gs_adam(dev, 0.9, 0.999, 1e-8, step, row_mask=mask_t)
    torch.cuda.synchronize()
    for i in range(len(params)):
        np.testing.assert_allclose(dev[i]["param"].cpu().numpy(), ref[i]["p"], rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(dev[i]["m"].cpu().numpy(), ref[i]["m"], rtol=1e-5, atol=1e-7)
    np.testing.assert_array_equal(shadow.float().cpu().numpy(),
                                  dev[3]["param"].to(torch.bfloat16).float().cpu().numpy())


# ---------------------------------------------------------------------------
# The full step against the oracle's own pipeline
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dil", [R.Dilation(1, 0, 0), R.Dilation(2, 1, 0)], ids=_dil_id)
def test_full_step_parity(dil):
    p32, cam, tgt = scene_small()
    bg = (0.0, 0.0, 0.0)
    ref = orc.forward_backward(U.params_f64(p32), orc.as_camera(cam), orc.as_dilation(dil), tgt, bg)
    p = U.gpu_params(p32)
    w_ds, h_ds, tx, ty = R.gs_grid(cam, dil)
    rast = Rasterizer(p.n, capacity=len(ref["vals"]) + 1000, max_tiles=tx * ty)
    step = TrainStep(p, rast, AdamConfig(), max_pixels=w_ds * h_ds, bg=bg, fused=False)
    before = [t.clone() for t in p.tensors()]
    loss = step(cam, dil, torch.tensor(tgt, device=U.DEV))
    torch.cuda.synchronize()
    assert abs(loss.item() - ref["loss"]) < 1e-5
    img = step.img[:3 * w_ds * h_ds].view(h_ds, w_ds, 3).cpu().numpy()
    diff = np.abs(img - ref["fwd"]["img"]).max(-1)
    # excluded: pixels whose FP64 gate values lie within the oracle's margin of a threshold, and
    # the tiles of Gaussians whose radius or rect differs between the FP32 and FP64 projections
    # (their lists may differ); every other pixel within 1e-4
    proj = ref["proj"]
    gpu = dict(rects=rast.rects.cpu().numpy(), radii=rast.radii.cpu().numpy(),
               ranges=rast.ranges[:tx * ty].cpu().numpy())
    bad_tiles, _ = U.flagged_tiles(proj, gpu, tx)
    # and the tiles whose lists differ (two depths whose FP32 order differs from the FP64 one)
    ids = rast.sorted_ids[:rast.num_pairs()].cpu().numpy().view(np.uint32)
    granges = gpu["ranges"].view(np.uint32)
    for t in range(tx * ty):
        a = ids[granges[t, 0]:granges[t, 1]]
        b = ref["vals"][ref["ranges"][t, 0]:ref["ranges"][t, 1]]
        if a.shape != b.shape or (a != b).any():
            bad_tiles[t] = True
    excl = ref["fwd"]["ambiguous"] | U.tile_pixel_mask(bad_tiles, w_ds, h_ds, tx, dil.tile)
    print(f"full step: {excl.mean():.4%} of pixels excluded ({bad_tiles.sum()} of {tx * ty} tiles)")
    assert excl.mean() < 0.1
    assert diff[~excl].max() < IMG_TOL
    assert rast.num_pairs() == len(ref["vals"])
    for name, g in zip(("means", "log_scales", "quats", "opacity_logits", "sh"), step.grads):
        assert U.grad_report(name, g.cpu().numpy(), ref["grads"][name]) < GRAD_TOL, name
    # Adam moved every visible Gaussian's parameters
    moved = (p.means != before[0]).any(1).cpu().numpy()
    assert moved[ref["proj"]["tiles_touched"] > 0].mean() > 0.5


def lowp_spacing(v, dtype):
    """The step of the 16-bit type at the values v (float64), away from zero."""
    lo, hi, _ = lowp.neighbours(np.asarray(v, np.float32), "bf16" if dtype == torch.bfloat16 else "f16")
    return np.abs(hi - lo)


def assert_lowp_close(a, b, dtype, min_exact=0.999):
    """Two low-precision results of the same update computed with different FP32
    rounding: equal, or (where the FP32 values straddle a rounding decision)
    one step of the type apart."""
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    assert (a == b).mean() >= min_exact, (a == b).mean()
    assert (np.abs(a - b) <= lowp_spacing(b, dtype) * (1 + 1e-12)).all()


@pytest.mark.parametrize("sh_dtype,sparse,master", [(torch.float32, False, False), (torch.bfloat16, False, True),
                                                    (torch.bfloat16, False, False), (torch.float16, False, False),
                                                    (torch.float16, True, False), (torch.float32, True, False)],
                         ids=["fp32", "bf16-master", "bf16", "fp16", "fp16-sparse", "fp32-sparse"])
def test_fused_project_bwd_adam_matches_unfused(sh_dtype, sparse, master):
    """gs_project_bwd_adam equals gs_project_bwd followed by gs_adam (parameters,
    moments, SH storage, gradients, densification statistics) when both are
    given the same 2D gradients, three steps in a row: up to FP32 rounding of the
    gradient arithmetic, which the two kernels may contract differently. SH kept
    only in BF16/FP16 draws the same stochastic-rounding bits in both paths: equal
    but where that FP32 rounding straddles a rounding decision."""
    p32, cam, tgt = scene_sh3()
    dil = R.Dilation(2, 1, 0)
    out, rast, p, (img, tf, last) = U.run_forward(p32, cam, dil, sh_dtype=sh_dtype, master=master)
    dl = torch.tensor(np.random.default_rng(2).standard_normal(img.shape) * 1e-3, dtype=torch.float32, device=U.DEV)
    rast.render_bwd(cam, dil, (0.0, 0.0, 0.0), tf, last, dl)
    lrs = [1e-3, 5e-3, 1e-3, 5e-2, 2.5e-3]
    seed = 77
    lowp_mode = sh_dtype != torch.float32 and not master
    sets = []
    for _ in range(2):
        ps = [t.clone() for t in p.tensors()]
        sets.append(dict(p=ps, m=[torch.zeros_like(t, dtype=torch.float32) for t in ps],
                         v=[torch.zeros_like(t, dtype=torch.float32) for t in ps],
                         shadow=p.sh_store.clone() if master else None,
                         stats=[torch.zeros(p.n, device=U.DEV), torch.zeros(p.n, device=U.DEV),
                                torch.zeros(p.n, dtype=torch.int32, device=U.DEV)]))
    mask = (rast.tiles_touched > 0).to(torch.uint8) if sparse else None
    for step in (1, 2, 3):
        # unfused: gradients, then the multi-tensor Adam
        a = sets[0]
        store = a["shadow"] if a["shadow"] is not None else a["p"][4]
        g = [torch.empty_like(t, dtype=torch.float32) for t in a["p"]]
        R.gs_project_bwd(*a["p"][:4], store, cam, dil, rast.tiles_touched, rast.grad2d, *g, *a["stats"])
        ent = [dict(param=a["p"][i], grad=g[i], m=a["m"][i], v=a["v"][i], lr=lrs[i], sr_seed=seed) for i in range(5)]
        if a["shadow"] is not None:
            ent[4]["shadow"] = a["shadow"]
        R.gs_adam(ent, 0.9, 0.999, 1e-15, step, row_mask=mask)
        # fused
        b = sets[1]
        storeb = b["shadow"] if b["shadow"] is not None else b["p"][4]
        gout = [torch.full_like(t, 7.0, dtype=torch.float32) for t in b["p"]]
        R.gs_project_bwd_adam(b["p"], b["m"], b["v"], lrs, 0.9, 0.999, 1e-15, step, storeb, cam, dil,
                              rast.tiles_touched, rast.grad2d, sparse=sparse, sh_shadow=b["shadow"],
                              pos_acc=b["stats"][0], col_acc=b["stats"][1], count=b["stats"][2], grads_out=gout,
                              sr_seed=seed)
        torch.cuda.synchronize()
        for x, y in zip(gout, g):
            assert U.max_rel(x.cpu().numpy(), y.cpu().numpy()) < 1e-6
    for key, rtol in (("p", 1e-6), ("m", 1e-5), ("v", 1e-5), ("stats", 1e-6)):
        for i, (x, y) in enumerate(zip(sets[0][key], sets[1][key])):
            a, b = x.float().cpu().numpy(), y.float().cpu().numpy()
            if key == "p" and i == 4 and lowp_mode:
                assert_lowp_close(b, a, sh_dtype)
                # and the SH moved (the rounding is not stuck at the stored values)
                assert (a != p.sh_store.float().cpu().numpy()).mean() > 0.05
                continue
            assert U.max_rel(a, b) < rtol, key
    if sets[0]["shadow"] is not None:
        a, b = sets[0]["shadow"].float().cpu().numpy(), sets[1]["shadow"].float().cpu().numpy()
        # BF16 copies of parameters equal to FP32 rounding: equal or one BF16 step apart
        assert (np.abs(a - b) <= np.abs(b) * 2.0 ** -7 + 1e-30).all()


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_adam_lowp_parity(dtype):
    """gs_adam on a parameter kept only in BF16/FP16 against the oracle (FP64
    Adam from the stored values, rounded to FP32, then stochastically with the
    same hash stream), three steps, each from the GPU's state. The FP32 update
    of the kernel (SFU square root and division) and the oracle's differ by a
    few FP32 ulps, which flips a rounding decision only when the random bits
    fall between the two: equal elsewhere, one step of the type apart there."""
    from oracle import lowp as L
    name = "bf16" if dtype == torch.bfloat16 else "f16"
    rng = np.random.default_rng(8)
    shape = (1001, 16, 3)
    p = torch.tensor(rng.standard_normal(shape) * 0.3, dtype=torch.float32).to(dtype).to(U.DEV)
    m = torch.tensor(rng.standard_normal(shape) * 1e-2, dtype=torch.float32, device=U.DEV)
    v = torch.tensor(rng.uniform(1e-5, 1e-4, shape), dtype=torch.float32, device=U.DEV)
    lr, seed = 1e-3, 12345
    moved = 0.0
    for step in (1, 2, 3):
        g = (rng.standard_normal(shape) * 1e-2).astype(np.float32)
        st = p.float().cpu().numpy().astype(np.float64)
        mm = m.cpu().numpy().astype(np.float64)
        vv = v.cpu().numpy().astype(np.float64)
        ref = L.adam_lowp(st, g, mm, vv, lr, 0.9, 0.999, 1e-15, step, name, seed)
        R.gs_adam([dict(param=p, grad=torch.tensor(g, device=U.DEV), m=m, v=v, lr=lr, sr_seed=seed, row_width=48)],
                  0.9, 0.999, 1e-15, step)
        torch.cuda.synchronize()
        out = p.float().cpu().numpy().astype(np.float64)
        assert_lowp_close(out, ref, dtype)
        np.testing.assert_allclose(m.cpu().numpy(), mm, rtol=1e-5, atol=1e-9)
        np.testing.assert_allclose(v.cpu().numpy(), vv, rtol=1e-5, atol=1e-12)
        moved = max(moved, float((out != st).mean()))
    assert moved > 0.3


def test_adam_lowp_fp16_range_edges():
    """FP16 kept parameters across its range: subnormals and zero, both ends of
    the normal range and the largest finite value (where rounding up
    saturates), against the oracle's rounding of the same update."""
    from oracle import lowp as L
    base = np.array([0.0, 1e-7, 3e-6, 6.0e-5, 6.2e-5, 1e-3, 1.0, 1000.0, 6.0e4, 65504.0])
    vals = np.concatenate([base, -base])
    rng = np.random.default_rng(12)
    x = np.repeat(vals, 64)
    p = torch.tensor(x, dtype=torch.float32).to(torch.float16).to(U.DEV)
    g = rng.standard_normal(x.size).astype(np.float32)
    m = torch.zeros(x.size, device=U.DEV)
    v = torch.zeros(x.size, device=U.DEV)
    st = p.float().cpu().numpy().astype(np.float64)
    mm, vv = np.zeros(x.size), np.zeros(x.size)
    for lr in (1e-6,):
        ref = L.adam_lowp(st, g, mm, vv, lr, 0.9, 0.999, 1e-15, 1, "f16", 321)
        R.gs_adam([dict(param=p, grad=torch.tensor(g, device=U.DEV), m=m, v=v, lr=lr, sr_seed=321)],
                  0.9, 0.999, 1e-15, 1)
        torch.cuda.synchronize()
        out = p.float().cpu().numpy().astype(np.float64)
        assert np.isfinite(out).all() and np.abs(out).max() <= 65504.0
        assert_lowp_close(out, ref, torch.float16, min_exact=0.99)
        # values far below the update's size move by whole steps in both directions
        assert (out[np.abs(x) < 1e-5] != st[np.abs(x) < 1e-5]).any()


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_fused_lowp_against_oracle(dtype):
    """The fused optimizer pass with the SH kept only in BF16/FP16, against
    the oracle: projection backward from the stored coefficients (gradients
    within 1e-3) and the low-precision Adam step of oracle/lowp.py (same hash
    stream; equal but where the kernel's FP32 update and the oracle's straddle
    a rounding decision, then one step apart). Moments start from a seeded
    state of the gradients' scale, so the update is smooth in the gradient."""
    name = "bf16" if dtype == torch.bfloat16 else "f16"
    p32, cam, _ = scene_sh3()
    dil = R.Dilation(2, 1, 0)
    out, rast, p, o, og, g2d, excl = backward_case(p32, cam, dil, sh_dtype=dtype)
    flagged = (o["flags"] & orc.FLAG_AMBIGUOUS) != 0
    rows = np.nonzero((out["tiles_touched"] > 0) & ~flagged)[0]
    p64 = U.params_f64(p32)
    p64["sh"] = p.sh_store.float().cpu().numpy().astype(np.float64)
    ref = orc.project_bwd({k: v[rows] for k, v in p64.items()}, orc.as_camera(cam), orc.as_dilation(dil),
                          {k: v[rows] for k, v in og.items()})
    lrs = [1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3]
    seed, step = 99, 4
    rng = np.random.default_rng(3)
    m0, v0 = [], []
    for nm, t in zip(("means", "log_scales", "quats", "opacity_logits", "sh"), p.tensors()):
        sc = float(np.sqrt(np.mean(ref[nm] ** 2))) or 1.0
        m0.append(rng.normal(0.0, sc, tuple(t.shape)).astype(np.float32))
        v0.append((sc * sc * rng.uniform(0.5, 2.0, tuple(t.shape))).astype(np.float32))
    m = [torch.tensor(x, device=U.DEV) for x in m0]
    v = [torch.tensor(x, device=U.DEV) for x in v0]
    stored = p64["sh"].copy()
    gout = [torch.zeros(tuple(t.shape), dtype=torch.float32, device=U.DEV) for t in p.tensors()]
    R.gs_project_bwd_adam(p.tensors(), m, v, lrs, 0.9, 0.999, 1e-15, step, p.sh_store, cam, dil,
                          rast.tiles_touched, rast.grad2d, grads_out=gout, sr_seed=seed)
    torch.cuda.synchronize()
    for i, nm in enumerate(("means", "log_scales", "quats", "opacity_logits", "sh")):
        assert U.grad_report(nm, gout[i].cpu().numpy()[rows], ref[nm]) < GRAD_TOL, nm
    g_full = np.zeros_like(stored)
    g_full[rows] = ref["sh"]
    mm, vv = m0[4].astype(np.float64), v0[4].astype(np.float64)
    want = lowp.adam_lowp(stored, g_full, mm, vv, lrs[4], 0.9, 0.999, 1e-15, step, name, seed)
    got = p.sh_store.float().cpu().numpy().astype(np.float64)
    assert_lowp_close(got[rows], want[rows], dtype, min_exact=0.99)
    assert (got[rows] != stored[rows]).mean() > 0.3
    np.testing.assert_allclose(m[4].cpu().numpy()[rows], mm[rows], rtol=1e-3, atol=1e-3 * np.abs(mm).max())


# ---------------------------------------------------------------------------
# Edge cases
# ---------------------------------------------------------------------------

def _camera_centre(cam):
    """-R^T T evaluated as the library does (double, then FP32)."""
    Rm = np.asarray(cam.R, np.float32).reshape(-1).astype(np.float64)
    T = np.asarray(cam.T, np.float32).reshape(-1).astype(np.float64)
    return np.array([-(Rm[j] * T[0] + Rm[3 + j] * T[1] + Rm[6 + j] * T[2]) for j in range(3)], np.float32)


@pytest.mark.parametrize("views", [1, 2])
def test_gaussian_at_the_camera_centre_stays_finite(views):
    """A Gaussian exactly at the camera centre is culled (depth 0); its view
    direction has zero length. The fused optimizer passes (one view, and the
    batched form) must leave every parameter and moment finite."""
    p32, cam, tgt = scene_sh3()
    p32 = {k: v.copy() for k, v in p32.items()}
    p32["means"][0] = _camera_centre(cam)
    p = U.gpu_params(p32)
    cams = [cam, scenes.look_at(scenes.orbit_eye(3.0, 150.0, 20.0), width=cam.width, height=cam.height)][:views]
    targets = [torch.tensor(scenes.target_image(c.width, c.height, 11 + i), device=U.DEV) for i, c in enumerate(cams)]
    step = BatchTrainStep(p, cams, targets, d=2)
    for ph in range(3):
        step.run(ph)
    torch.cuda.synchronize()
    assert not step.overflowed()
    for t in list(p.tensors()) + step.m + step.v:
        assert bool(torch.isfinite(t).all())
    assert int(step.vis_count[0].item()) == 0


def test_empty_and_all_culled():
    _, cam, _ = scene_small()
    bg = (0.25, 0.5, 0.75)
    for n, z in [(0, 0.0), (50, 10.0)]:
        rng = np.random.default_rng(0)
        # camera at radius 4 looking at the origin: push everything behind it
        eye = np.array(scenes.orbit_eye(4.0, 30.0, 20.0))
        p = dict(means=(eye * 1.5 + rng.uniform(-0.1, 0.1, (n, 3))).astype(np.float32),
                 log_scales=np.full((n, 3), -2.0, np.float32), quats=rng.standard_normal((n, 4)).astype(np.float32),
                 opacity_logits=np.zeros(n, np.float32), sh=np.zeros((n, 1, 3), np.float32))
        if n == 0:
            p = {k: v[:0] for k, v in p.items()}
            p["sh"] = np.zeros((0, 1, 3), np.float32)
            out = dict()
            w_ds, h_ds, tx, ty = R.gs_grid(cam, R.Dilation())
            rast = Rasterizer(1, capacity=16, max_tiles=tx * ty)
            rast.n = 0
            R.gs_bin_sort(0, rast.rects, rast.tiles_touched, rast.splats, tx, ty, rast.workspace, 16,
                          rast.sorted_ids, rast.ranges, rast.num_pairs_dev)
            img, tf, last = image_buffers(h_ds, w_ds)
            R.gs_render_fwd(0, rast.splats, rast.sorted_ids, rast.ranges, cam, R.Dilation(), bg, img, tf, last)
            torch.cuda.synchronize()
            assert rast.num_pairs() == 0
            np.testing.assert_allclose(img.cpu().numpy(), np.broadcast_to(bg, img.shape), atol=0)
            continue
        out, *_ = U.run_forward(p, cam, R.Dilation(), bg)
        assert out["k"] == 0 and (out["radii"] == 0).all()
        np.testing.assert_allclose(out["img"], np.broadcast_to(bg, out["img"].shape), atol=1e-7)
        assert (out["t_final"] == 1.0).all() and (out["last"] == 0).all()


def test_one_gaussian_covering_every_tile():
    p = dict(means=np.zeros((1, 3), np.float32), log_scales=np.full((1, 3), 0.5, np.float32),
             quats=np.array([[1, 0, 0, 0]], np.float32), opacity_logits=np.array([2.0], np.float32),
             sh=np.full((1, 1, 3), 0.3, np.float32))
    cam = scenes.look_at(scenes.orbit_eye(4.0, 0.0, 0.0), width=200, height=150)
    for dil in [R.Dilation(1, 0, 0), R.Dilation(2, 1, 1)]:
        out, rast, p_, bufs, o, of, excl = render_case(p, cam, dil)
        w_ds, h_ds, tx, ty = out["grid"]
        assert out["k"] == tx * ty
        check_binning(out)
        assert np.abs(out["img"] - of["img"])[~excl].max() < IMG_TOL


def test_capacity_overflow_then_regrow():
    p32, cam, _ = scene_small()
    dil = R.Dilation()
    out_ok, *_ = U.run_forward(p32, cam, dil)
    k = out_ok["k"]
    out, rast, p, bufs = U.run_forward(p32, cam, dil, bg=(0.5, 0.5, 0.5), capacity=k // 2)
    assert out["k"] == k and rast.capacity < k
    assert (out["ranges"] == 0).all()
    np.testing.assert_allclose(out["img"], 0.5, atol=1e-7)
    rast.ensure_capacity(k)
    rast.bin(cam, dil)
    torch.cuda.synchronize()
    assert (rast.ranges[: out["ranges"].shape[0]].cpu().numpy().view(np.uint32) == out_ok["ranges"]).all()


def test_pair_count_high_water_mark_is_sticky():
    """num_pairs_max keeps the largest pair count of all calls: an overflowing
    call followed by a smaller one still shows the overflow."""
    p32, cam, _ = scene_small()
    dil = R.Dilation()
    out, rast, p, bufs = U.run_forward(p32, cam, dil)
    k = out["k"]
    tx, ty = R.gs_bin_grid(cam, dil)
    mx = torch.zeros(1, dtype=torch.int64, device=U.DEV)
    num = torch.zeros(1, dtype=torch.int64, device=U.DEV)
    for cap in (k // 2, k + 10):
        ws = torch.empty(R.gs_bin_sort_workspace_size(p.n, cap, tx, ty), dtype=torch.uint8, device=U.DEV)
        ids = torch.empty(cap, dtype=torch.int32, device=U.DEV)
        R.gs_bin_sort(p.n, rast.rects, rast.tiles_touched, rast.splats, tx, ty, ws, cap, ids, rast.ranges, num,
                      num_pairs_max=mx)
    # a call on nothing visible: K = 0 does not lower the mark
    empty = torch.zeros_like(rast.tiles_touched)
    R.gs_bin_sort(p.n, rast.rects, empty, rast.splats, tx, ty, ws, k + 10, ids, rast.ranges, num, num_pairs_max=mx)
    torch.cuda.synchronize()
    assert num.item() == 0 and mx.item() == k


def test_deterministic_forward():
    p32, cam, _ = scene_sh3()
    a, *_ = U.run_forward(p32, cam, R.Dilation(2, 1, 0))
    b, *_ = U.run_forward(p32, cam, R.Dilation(2, 1, 0))
    for k in ("splats", "sorted_ids", "ranges", "img", "t_final", "last"):
        np.testing.assert_array_equal(a[k], b[k])


# ---------------------------------------------------------------------------
# autograd.Function
# ---------------------------------------------------------------------------

def test_autograd_matches_oracle_gradient():
    from paper_2412_13547_b300.pipeline import rasterize
    p32, cam, _ = scene_sh3(96, 80)
    dil = R.Dilation(2, 1, 0)
    p = U.gpu_params(p32)
    ts = [t.clone().requires_grad_(True) for t in p.tensors()]
    rng = np.random.default_rng(0)
    w_ds, h_ds, _, _ = R.gs_grid(cam, dil)
    wts = torch.tensor(rng.standard_normal((h_ds, w_ds, 3)), dtype=torch.float32, device=U.DEV)
    img, _, _ = rasterize(*ts, cam, dil)
    (img * wts).sum().backward()
    o = orc.project(U.params_f64(p32), orc.as_camera(cam), orc.as_dilation(dil))
    out, *_ = U.run_forward(p32, cam, dil)
    np.testing.assert_allclose(img.detach().cpu().numpy(), out["img"], atol=0)
    og = orc.render_bwd(o, out["sorted_ids"], out["ranges"], orc.as_camera(cam), orc.as_dilation(dil),
                        wts.cpu().numpy().astype(np.float64))
    ref = orc.project_bwd(U.params_f64(p32), orc.as_camera(cam), orc.as_dilation(dil), og)
    for name, t in zip(("means", "log_scales", "quats", "opacity_logits", "sh"), ts):
        assert U.grad_report(name, t.grad.cpu().numpy(), ref[name]) < GRAD_TOL, name


def test_autograd_rejects_parameters_changed_in_place():
    """The parameters go through save_for_backward: changing one in place
    between the forward and the backward (an optimizer step) is an error, not
    a silent gradient at the changed values."""
    from paper_2412_13547_b300.pipeline import rasterize
    p32, cam, _ = scene_sh3(64, 48)
    p = U.gpu_params(p32)
    ts = [t.clone().requires_grad_(True) for t in p.tensors()]
    img, _, _ = rasterize(*ts, cam, R.Dilation(2, 1, 0))
    with torch.no_grad():
        ts[0].add_(1e-3)
    with pytest.raises(RuntimeError, match="inplace"):
        img.sum().backward()


def test_autograd_finite_differences_hd_64_params():
    """1920x1080, 1M Gaussians, d=2: the autograd.Function gradient of a random
    linear loss against FP64 central differences (the oracle's forward with the
    lists held fixed) on 64 sampled parameters."""
    from paper_2412_13547_b300.pipeline import rasterize
    scene, cam, _ = scenes.workload_hd()
    p32 = U.params_np(scene)
    dil = R.Dilation(2, 1, 0)
    ocam, odil = orc.as_camera(cam), orc.as_dilation(dil)
    out, *_ = U.run_forward(p32, cam, dil)
    w_ds, h_ds, tx, ty = out["grid"]
    p64 = U.params_f64(p32)
    o = orc.project(p64, ocam, odil)
    of = orc.render_fwd(o, out["sorted_ids"], out["ranges"], ocam, odil)
    rng = np.random.default_rng(1)
    w = rng.standard_normal((h_ds, w_ds, 3))
    w[of["ambiguous"]] = 0.0
    p = U.gpu_params(p32)
    ts = [t.clone().requires_grad_(True) for t in p.tensors()]
    img, _, _ = rasterize(*ts, cam, dil)
    (img * torch.tensor(w, dtype=torch.float32, device=U.DEV)).sum().backward()
    grads = {name: t.grad.cpu().numpy() for name, t in zip(("means", "log_scales", "quats", "opacity_logits", "sh"), ts)}
    ok = (out["tiles_touched"] > 0) & ((o["flags"] & orc.FLAG_AMBIGUOUS) == 0) & (out["tiles_touched"] < 400)
    names = ["means"] * 3 + ["log_scales"] * 3 + ["quats"] * 4 + ["opacity_logits"] + ["sh"] * 48
    picks = rng.choice(np.nonzero(ok)[0], 64, replace=False)
    fd, an, grp = [], [], []
    for g in picks:
        k = int(rng.integers(len(names)))
        name = names[k]
        elem = k - names.index(name)
        rc = out["rects"][g]
        tiles = np.array([yy * tx + xx for yy in range(rc[1], rc[3] + 1) for xx in range(rc[0], rc[2] + 1)], np.int32)
        sub_v = np.concatenate([out["sorted_ids"][out["ranges"][t, 0]:out["ranges"][t, 1]] for t in tiles])
        lens = np.array([out["ranges"][t, 1] - out["ranges"][t, 0] for t in tiles], np.int64)
        sub_r = np.c_[np.r_[0, np.cumsum(lens)[:-1]], np.cumsum(lens)].astype(np.uint32)
        pm = U.tile_pixel_mask(np.isin(np.arange(tx * ty), tiles), w_ds, h_ds, tx, dil.tile)
        vals = []
        for sgn in (1.0, -1.0):
            one = {kk: vv[g:g + 1].copy() for kk, vv in p64.items()}
            flat = one[name].reshape(-1)
            h = 1e-6 * max(1.0, abs(flat[elem]))
            flat[elem] += sgn * h
            po = orc.project(one, ocam, odil)
            pr = {kk: o[kk].copy() for kk in ("xy", "conic", "opacity", "rgb", "depth")}
            for kk in pr:
                pr[kk][g] = po[kk][0]
            im = orc.render_fwd(pr, sub_v, sub_r, ocam, odil, tile_ids=tiles)["img"]
            vals.append(float(np.sum((w * im)[pm])))
        fd.append((vals[0] - vals[1]) / (2 * h))
        an.append(float(grads[name].reshape(len(p32["means"]), -1)[g, elem]))
        grp.append(name)
    fd, an, grp = np.array(fd), np.array(an), np.array(grp)
    for name in set(grp):
        sel = grp == name
        scale = np.abs(fd[sel]).max()
        assert np.abs(an[sel] - fd[sel]).max() <= GRAD_TOL * scale + 1e-9, (name, an[sel], fd[sel])


# ---------------------------------------------------------------------------
# Full size: 3840x2160, 3M Gaussians, in the launch configuration of the bench
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d,ox,oy", [(2, 1, 0), (4, 3, 1)])
def test_uhd_sampled_tiles_parity(d, ox, oy):
    scene, cam, tgt = scenes.workload_uhd()
    p32 = U.params_np(scene)
    dil = R.Dilation(d, ox, oy)
    out, rast, p, (img, t_final, last) = U.run_forward(p32, cam, dil)
    w_ds, h_ds, tx, ty = out["grid"]
    rng = np.random.default_rng(d)
    # tiles with content, sampled uniformly
    nonempty = np.nonzero(out["ranges"][:, 1] > out["ranges"][:, 0])[0]
    tiles = np.sort(rng.choice(nonempty, 12, replace=False)).astype(np.int32)
    # binning of those tiles, bit-exact against the oracle's per-tile lists of the GPU rects
    sv, sr = orc.bin_tiles(out["rects"], U.gpu_depth_bits(out), tx, tiles)
    for k, t in enumerate(tiles):
        np.testing.assert_array_equal(out["sorted_ids"][out["ranges"][t, 0]:out["ranges"][t, 1]],
                                      sv[sr[k, 0]:sr[k, 1]])
    # projection of every Gaussian
    o = check_projection(p32, cam, dil, out)
    # blend of the sampled tiles
    of = orc.render_fwd(o, sv, sr, orc.as_camera(cam), orc.as_dilation(dil), (0.0, 0.0, 0.0), tile_ids=tiles)
    mask = np.zeros(tx * ty, bool)
    mask[tiles] = True
    pm = U.tile_pixel_mask(mask, w_ds, h_ds, tx, dil.tile) & ~of["ambiguous"]
    assert np.abs(out["img"] - of["img"])[pm].max() < IMG_TOL
    np.testing.assert_array_equal(out["last"][pm], of["last"][pm])
    # backward restricted to the sampled tiles (dL/dimg zero elsewhere)
    dl = rng.standard_normal(out["img"].shape) * 1e-3
    dl[~pm] = 0.0
    rast.render_bwd(cam, dil, (0.0, 0.0, 0.0), t_final, last, torch.tensor(dl, dtype=torch.float32, device=U.DEV))
    torch.cuda.synchronize()
    og = orc.render_bwd(o, sv, sr, orc.as_camera(cam), orc.as_dilation(dil), dl.astype(np.float32), tile_ids=tiles)
    gg = U.split_grad2d(rast.grad2d.cpu().numpy())
    for k in ("dxy", "dconic", "dopacity", "drgb"):
        assert U.grad_report(k, gg[k], og[k]) < GRAD_TOL, k
    check_fused_pass_against_oracle(p, p32, cam, dil, rast, o, og, seed=d)


def check_fused_pass_against_oracle(p, p32, cam, dil, rast, o, og, seed, step=10):
    """gs_project_bwd_adam at full size, in the bench's launch configuration,
    against the oracle's projection backward (of the oracle's own 2D gradients),
    densification statistics and Adam, on the Gaussians the sampled tiles
    touch (every other row has a zero 2D gradient). The moments start from a
    seeded state of the gradients' scale, so the update is smooth in the
    gradient (a first step from zero moments moves by lr * sign(g), which a
    gradient near zero may flip)."""
    names = ("means", "log_scales", "quats", "opacity_logits", "sh")
    lrs = [1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3]
    b1, b2, eps = 0.9, 0.999, 1e-15
    ocam, odil = orc.as_camera(cam), orc.as_dilation(dil)
    g2d = rast.grad2d.cpu().numpy()
    flagged = (o["flags"] & orc.FLAG_AMBIGUOUS) != 0
    rows = np.nonzero((np.abs(g2d).sum(1) > 0) & ~flagged & (o["tiles_touched"] > 0))[0]
    assert rows.size > 100
    p64 = U.params_f64(p32)
    sub = {k: v[rows] for k, v in p64.items()}
    og_sub = {k: v[rows] for k, v in og.items()}
    ref = orc.project_bwd(sub, ocam, odil, og_sub)
    rng = np.random.default_rng(seed)
    m0, v0 = [], []
    for name, t in zip(names, p.tensors()):
        sc = float(np.sqrt(np.mean(ref[name] ** 2))) or 1.0
        m0.append(rng.normal(0.0, sc, tuple(t.shape)).astype(np.float32))
        v0.append((sc * sc * rng.uniform(0.5, 2.0, tuple(t.shape))).astype(np.float32))
    m = [torch.tensor(x, device=U.DEV) for x in m0]
    v = [torch.tensor(x, device=U.DEV) for x in v0]
    before = [t.detach().cpu().numpy().copy() for t in p.tensors()]
    gout = [torch.zeros_like(t) for t in p.tensors()]
    pos, col = torch.zeros(p.n, device=U.DEV), torch.zeros(p.n, device=U.DEV)
    cnt = torch.zeros(p.n, dtype=torch.int32, device=U.DEV)
    R.gs_project_bwd_adam(p.tensors(), m, v, lrs, b1, b2, eps, step, p.sh_store, cam, dil, rast.tiles_touched,
                          rast.grad2d, pos_acc=pos, col_acc=col, count=cnt, grads_out=gout)
    torch.cuda.synchronize()
    rp, rc, rn = np.zeros(rows.size), np.zeros(rows.size), np.zeros(rows.size, np.int32)
    orc.densify_stats(o["tiles_touched"][rows], og_sub, rp, rc, rn)
    assert U.grad_report("pos_acc", pos.cpu().numpy()[rows], rp) < GRAD_TOL
    assert U.grad_report("col_acc", col.cpu().numpy()[rows], rc) < GRAD_TOL
    np.testing.assert_array_equal(cnt.cpu().numpy()[rows], rn)
    for i, name in enumerate(names):
        g = gout[i].cpu().numpy()[rows]
        assert U.grad_report(name, g, ref[name]) < GRAD_TOL, name
        pr, mr, vr = (before[i][rows].astype(np.float64), m0[i][rows].astype(np.float64),
                      v0[i][rows].astype(np.float64))
        orc.adam(pr, ref[name], mr, vr, lrs[i], b1, b2, eps, step)
        dp = p.tensors()[i].detach().cpu().numpy()[rows].astype(np.float64) - before[i][rows]
        dr = pr - before[i][rows]
        ulp = np.abs(before[i][rows]).astype(np.float64) * 2.0 ** -22
        assert (np.abs(dp - dr) <= GRAD_TOL * np.abs(dr).max() + ulp).all(), name
        assert U.grad_report(name + "_m", m[i].cpu().numpy()[rows], mr) < GRAD_TOL, name


@pytest.mark.parametrize("d,ox,oy,shift", [(2, 1, 0, 2), (4, 3, 1, 1)])
def test_uhd_bench_binning_gives_the_same_step(d, ox, oy, shift):
    """The bench bins the 4K step with coarser tiles (16 << shift: 64 at d = 2, 32 at d = 4) and
    filters per blend tile. At full size its image and final transmittance are bit-identical to
    the per-tile binning checked against the oracle above, and its 2D gradients equal up to the
    order of floating-point atomics."""
    scene, cam, _ = scenes.workload_uhd()
    p32 = U.params_np(scene)
    res = []
    for s in (0, shift):
        dil = R.Dilation(d, ox, oy, bin_shift=s)
        out, rast, p, (img, t_final, last) = U.run_forward(p32, cam, dil)
        dl = np.random.default_rng(d).standard_normal(out["img"].shape) * 1e-3
        rast.render_bwd(cam, dil, (0.0, 0.0, 0.0), t_final, last,
                        torch.tensor(dl, dtype=torch.float32, device=U.DEV))
        torch.cuda.synchronize()
        res.append((out["img"], out["t_final"], out["counts"], rast.grad2d.cpu().numpy()))
        del out, rast, p, img, t_final, last
    np.testing.assert_array_equal(res[1][0], res[0][0])
    np.testing.assert_array_equal(res[1][1], res[0][1])
    # the blends evaluated depend on the lists' lengths; the blends taken do not
    assert res[1][2][1] == res[0][2][1]
    assert U.max_rel(res[1][3], res[0][3]) < 1e-5
