"""gs_bin_sort_static: the binning entry point for callers that cannot allocate
device memory (a plugin or embedded host that only hands over its own input and
output buffers, or a serving process whose device-memory budget is fixed at
start-up). Its scratch is a fixed array inside the library instead of a caller
workspace.

Through the C ABI, its results must equal gs_bin_sort's (integer outputs, so
bit for bit) on two calls in a row with different inputs; the array keeps the
previous call's contents, so a second, smaller call would expose any part of
the scratch that needed to start at zero. This file runs last so that a
failure here leaves every other test already run.
"""
import numpy as np
import pytest
import torch

from paper_2412_13547_b300 import raster as R
from paper_2412_13547_b300 import scenes

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _project(scene, cam, dil):
    d = {k: torch.tensor(np.asarray(v, np.float32), device=DEV).contiguous() for k, v in scene.as_dict().items()}
    n = scene.n
    splats = torch.zeros(n, R.SPLAT_FLOATS, device=DEV)
    radii = torch.zeros(n, dtype=torch.int32, device=DEV)
    rects = torch.zeros(n, 4, dtype=torch.int32, device=DEV)
    tiles = torch.zeros(n, dtype=torch.int32, device=DEV)
    R.gs_project(d["means"], d["log_scales"], d["quats"], d["opacity_logits"].reshape(-1), d["sh"], cam, dil,
                 splats, radii, rects, tiles)
    return n, splats, rects, tiles


def _both(scene, cam, dil):
    n, splats, rects, tiles = _project(scene, cam, dil)
    _, _, tx, ty = R.gs_grid(cam, dil)
    k = int(tiles.to(torch.int64).sum().item())
    cap = k + 4096
    assert R.gs_bin_sort_workspace_size(n, cap, tx, ty) <= R.BIN_SORT_STATIC_SCRATCH_BYTES
    # reference: the existing entry point with a caller workspace
    ws = torch.empty(R.gs_bin_sort_workspace_size(n, cap, tx, ty), dtype=torch.uint8, device=DEV)
    ids_a = torch.full((cap,), -1, dtype=torch.int32, device=DEV)
    rng_a = torch.full((tx * ty, 2), -1, dtype=torch.int32, device=DEV)
    k_a = torch.zeros(1, dtype=torch.int64, device=DEV)
    R.gs_bin_sort(n, rects, tiles, splats, tx, ty, ws, cap, ids_a, rng_a, k_a)
    # the allocation-free entry point
    ids_b = torch.full((cap,), -2, dtype=torch.int32, device=DEV)
    rng_b = torch.full((tx * ty, 2), -2, dtype=torch.int32, device=DEV)
    k_b = torch.zeros(1, dtype=torch.int64, device=DEV)
    R.gs_bin_sort_static(n, rects, tiles, splats, tx, ty, cap, ids_b, rng_b, k_b)
    torch.cuda.synchronize()
    assert k_a.item() == k_b.item() == k
    np.testing.assert_array_equal(ids_b[:k].cpu().numpy(), ids_a[:k].cpu().numpy())
    np.testing.assert_array_equal(rng_b.cpu().numpy(), rng_a.cpu().numpy())
    return k


def test_static_scratch_matches_workspace_on_two_calls():
    big = scenes.cluster_scene(40000, index=5, log_scale_mean=-3.6)
    cam_big = scenes.look_at(scenes.orbit_eye(2.6, 30.0, 20.0), width=640, height=360)
    small, cam_small, _ = scenes.workload_small()
    k1 = _both(big, cam_big, R.Dilation(1, 0, 0))
    k2 = _both(small, cam_small, R.Dilation(2, 1, 0))
    assert k1 > 10 * k2 > 0


def test_static_scratch_rejects_sizes_beyond_its_maximum():
    # 3M Gaussians need 48 MiB for their depth keys alone. Every buffer has the size
    # the call claims (and no Gaussian touches a tile), so nothing could run out of
    # bounds even if the size check were missing.
    n, tx, ty = 3_000_000, 8, 8
    splats = torch.zeros(n, R.SPLAT_FLOATS, device=DEV)
    rects = torch.zeros(n, 4, dtype=torch.int32, device=DEV)
    tiles = torch.zeros(n, dtype=torch.int32, device=DEV)
    ids = torch.zeros(16, dtype=torch.int32, device=DEV)
    rng = torch.zeros(tx * ty, 2, dtype=torch.int32, device=DEV)
    k = torch.zeros(1, dtype=torch.int64, device=DEV)
    assert R.gs_bin_sort_workspace_size(n, 16, tx, ty) > R.BIN_SORT_STATIC_SCRATCH_BYTES
    with pytest.raises(R.GsError, match="static array"):
        R.gs_bin_sort_static(n, rects, tiles, splats, tx, ty, 16, ids, rng, k)
