"""Coarse binning (GsDilation.bin_shift): pairs formed with tiles of
tile << bin_shift, every blend tile filtering its binning tile's list down to
its own. The blend tile lists are then the same lists in the same order, so
the forward is bit for bit the one of bin_shift 0 (itself pinned to the
oracle), the backward differs only by the order of float atomics, and `last`
maps onto the blend-tile index exactly.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2412_13547_b300 import raster as R
from paper_2412_13547_b300 import scenes

import gpu_util as U

pytestmark = pytest.mark.gpu
BG = (0.1, 0.2, 0.3)


def _scene(kind):
    if kind == "small":
        s, cam, _ = scenes.workload_small()
        return U.params_np(s), cam
    s = scenes.cluster_scene(40000, index=5, log_scale_mean=-3.6, packed_frac=0.2, packed_radius=0.25)
    cam = scenes.look_at(scenes.orbit_eye(2.6, 30.0, 20.0), width=643, height=365)
    return U.params_np(s), cam


# (scene, tile, bin_shift, d, pixels per thread): every launch shape of the blend,
# including CTAs wider than a staging batch (tile 32 at 2 pixels per thread)
CASES = [("small", 16, 1, 1, 0), ("small", 8, 1, 2, 0), ("small", 8, 1, 1, 1), ("clusters", 16, 1, 1, 0),
         ("clusters", 16, 2, 2, 0), ("clusters", 16, 1, 2, 1), ("clusters", 16, 1, 1, 4), ("clusters", 8, 2, 1, 0),
         ("clusters", 8, 1, 3, 0), ("clusters", 32, 1, 1, 2), ("clusters", 32, 1, 2, 4)]


def _ids(c):
    return f"{c[0]}-t{c[1]}-s{c[2]}-d{c[3]}-ppt{c[4]}"


def _fine_index_of(out_c, out_f, dil, grid):
    """Map each pixel's `last` (position + 1 in its binning tile's list) to the
    position + 1 in its blend tile's list."""
    w_ds, h_ds, tx, ty = grid
    s = dil.bin_shift
    btx = (tx + (1 << s) - 1) >> s
    rect_f = out_f["splats"][:, 12:16].copy().view(np.int32)
    last = out_c["last"].astype(np.int64)
    mapped = np.zeros_like(last)
    T = dil.tile
    for v in range(h_ds):
        for u in range(w_ds):
            if last[v, u] == 0:
                continue
            ftx, fty = u // T, v // T
            ct = (fty >> s) * btx + (ftx >> s)
            a, b = out_c["ranges"][ct]
            ids = out_c["sorted_ids"][a:a + last[v, u]]
            r = rect_f[ids]
            keep = (r[:, 0] <= ftx) & (ftx <= r[:, 2]) & (r[:, 1] <= fty) & (fty <= r[:, 3])
            assert keep[-1], "the last blended entry must belong to the blend tile"
            mapped[v, u] = int(keep.sum())
    return mapped


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_coarse_binning_gives_the_same_render(case):
    kind, tile, shift, d, ppt = case
    p32, cam = _scene(kind)
    dil0 = R.Dilation(d, d - 1, 0, tile=tile)
    dil1 = R.Dilation(d, d - 1, 0, tile=tile, bin_shift=shift)
    out0, rast0, p, bufs0 = U.run_forward(p32, cam, dil0, BG, ppt=ppt)
    out1, rast1, _, bufs1 = U.run_forward(p32, cam, dil1, BG, ppt=ppt)
    # projection: identical record (with the blend rect), rects and counts at the binning tiles
    np.testing.assert_array_equal(out1["splats"], out0["splats"])
    np.testing.assert_array_equal(out1["radii"], out0["radii"])
    r0 = out0["rects"]
    vis = out0["tiles_touched"] > 0
    np.testing.assert_array_equal(out1["rects"][vis], r0[vis] >> shift)
    area = (out1["rects"][:, 2] - out1["rects"][:, 0] + 1) * (out1["rects"][:, 3] - out1["rects"][:, 1] + 1)
    np.testing.assert_array_equal(out1["tiles_touched"][vis], area[vis])
    np.testing.assert_array_equal(out1["tiles_touched"][~vis], 0)
    assert out1["k"] < out0["k"]
    # binning of the coarse rects: bit-exact against the oracle's binning of the same rects
    btx, bty = R.gs_bin_grid(cam, dil1)
    _, vals, ranges = orc.bin_sort(out1["rects"], out1["tiles_touched"].astype(np.int64), U.gpu_depth_bits(out1),
                                   btx, bty)
    assert out1["k"] == len(vals)
    np.testing.assert_array_equal(out1["sorted_ids"], vals)
    np.testing.assert_array_equal(out1["ranges"], ranges)
    # forward: bit for bit
    np.testing.assert_array_equal(out1["img"], out0["img"])
    np.testing.assert_array_equal(out1["t_final"], out0["t_final"])
    np.testing.assert_array_equal(out1["counts"], out0["counts"])
    np.testing.assert_array_equal(_fine_index_of(out1, out0, dil1, out0["grid"]), out0["last"].astype(np.int64))
    # backward: the same sums in another order
    rng = np.random.default_rng(4)
    dl = torch.tensor(rng.standard_normal(out0["img"].shape) * 1e-3, dtype=torch.float32, device=U.DEV)
    rast0.render_bwd(cam, dil0, BG, bufs0[1], bufs0[2], dl)
    rast1.render_bwd(cam, dil1, BG, bufs1[1], bufs1[2], dl)
    torch.cuda.synchronize()
    g0, g1 = rast0.grad2d.cpu().numpy(), rast1.grad2d.cpu().numpy()
    assert np.abs(g0).max() > 0
    for sl in (slice(0, 2), slice(2, 5), slice(5, 6), slice(6, 9)):
        assert U.max_rel(g1[:, sl], g0[:, sl]) < 1e-5, sl


def test_coarse_binning_in_a_batch():
    """Batched views with bin_shift 1: each view's forward equals its one-view
    render at bin_shift 0."""
    p32, cam = _scene("clusters")
    cams = [cam, scenes.look_at(scenes.orbit_eye(2.6, 140.0, 35.0), width=401, height=233)]
    dils = [R.Dilation(1, 0, 0, bin_shift=1), R.Dilation(2, 1, 1, bin_shift=1)]
    p = U.gpu_params(p32)
    n = p.n
    views = []
    for c, dl in zip(cams, dils):
        w_ds, h_ds, tx, ty = R.gs_grid(c, dl)
        btx, bty = R.gs_bin_grid(c, dl)
        views.append(R.View(c, dl, splats=torch.zeros(n, R.SPLAT_FLOATS, device=U.DEV),
                            radii=torch.zeros(n, dtype=torch.int32, device=U.DEV),
                            rects=torch.zeros(n, 4, dtype=torch.int32, device=U.DEV),
                            tiles_touched=torch.zeros(n, dtype=torch.int32, device=U.DEV),
                            ranges=torch.zeros(btx * bty, 2, dtype=torch.int32, device=U.DEV),
                            img=torch.zeros(h_ds, w_ds, 3, device=U.DEV), t_final=torch.zeros(h_ds, w_ds, device=U.DEV),
                            last=torch.zeros(h_ds, w_ds, dtype=torch.int32, device=U.DEV)))
    R.gs_project_batch(p.means, p.log_scales, p.quats, p.opacity_logits, p.sh_store, views)
    torch.cuda.synchronize()
    for v in views:
        btx, bty = R.gs_bin_grid(v.cam, v.dil)
        k = int(v.tiles_touched.to(torch.int64).sum().item())
        ws = torch.empty(R.gs_bin_sort_workspace_size(n, k + 16, btx, bty), dtype=torch.uint8, device=U.DEV)
        v.sorted_ids = torch.empty(k + 16, dtype=torch.int32, device=U.DEV)
        R.gs_bin_sort(n, v.rects, v.tiles_touched, v.splats, btx, bty, ws, k + 16, v.sorted_ids, v.ranges,
                      torch.zeros(1, dtype=torch.int64, device=U.DEV))
    total = sum(R.gs_grid(v.cam, v.dil)[2] * R.gs_grid(v.cam, v.dil)[3] for v in views)
    order = torch.zeros(total, dtype=torch.int32, device=U.DEV)
    t = R.ViewTable(views)
    R.gs_tile_order_batch(t, order)
    R.gs_render_fwd_batch(n, t, BG, tile_order=order)
    torch.cuda.synchronize()
    assert sorted(order.cpu().numpy().tolist()) == list(range(total))
    for v, c, dl in zip(views, cams, dils):
        ref, *_ = U.run_forward(p32, c, R.Dilation(dl.d, dl.ox, dl.oy), BG)
        np.testing.assert_array_equal(v.img.cpu().numpy().astype(np.float64), ref["img"])
        np.testing.assert_array_equal(v.t_final.cpu().numpy().astype(np.float64), ref["t_final"])
