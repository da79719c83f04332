"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
the FP64 oracle on the same seeded inputs, and compare what is unique."""
import numpy as np
import torch

from oracle import oracle as orc
from paper_2412_13547_b300 import raster as R
from paper_2412_13547_b300.pipeline import GaussianParams, Rasterizer, image_buffers

DEV = "cuda"


def params_np(scene_or_dict):
    d = scene_or_dict.as_dict() if hasattr(scene_or_dict, "as_dict") else scene_or_dict
    return {k: np.asarray(v, np.float32) for k, v in d.items()}


def params_f64(p32):
    return {k: np.asarray(v, np.float64) for k, v in p32.items()}


def gpu_params(p32, sh_dtype=torch.float32, master=False):
    return GaussianParams.from_arrays(p32, DEV, sh_dtype, master=master)


def run_forward(p32, cam, dil, bg=(0.0, 0.0, 0.0), sh_dtype=torch.float32, capacity=None, ppt=0, master=False):
    """GPU project + bin + blend. Returns numpy outputs and the rasterizer."""
    p = gpu_params(p32, sh_dtype, master)
    w_ds, h_ds, tx, ty = R.gs_grid(cam, dil)
    btx, bty = R.gs_bin_grid(cam, dil)
    rast = Rasterizer(p.n, capacity=capacity or 1 << 16, device=DEV, max_grid=(btx, bty), pixels_per_thread=ppt)
    rast.project(p, cam, dil)
    if capacity is None:
        rast.bin_checked(cam, dil)
    else:
        rast.bin(cam, dil)
    img, t_final, last = image_buffers(h_ds, w_ds, DEV)
    counts = torch.zeros(3, dtype=torch.int64, device=DEV)
    rast.render(cam, dil, bg, img, t_final, last, counts)
    torch.cuda.synchronize()
    k = rast.num_pairs()
    ntile = btx * bty
    out = dict(
        splats=rast.splats.cpu().numpy(), radii=rast.radii.cpu().numpy(), rects=rast.rects.cpu().numpy(),
        tiles_touched=rast.tiles_touched.cpu().numpy(), k=k,
        sorted_ids=rast.sorted_ids[:min(k, rast.capacity)].cpu().numpy().view(np.uint32),
        ranges=rast.ranges[:ntile].cpu().numpy().view(np.uint32),
        img=img.cpu().numpy().astype(np.float64), t_final=t_final.cpu().numpy().astype(np.float64),
        last=last.cpu().numpy().view(np.uint32), counts=counts.cpu().numpy(), grid=(w_ds, h_ds, tx, ty))
    return out, rast, p, (img, t_final, last)


def gpu_proj_as_oracle(out):
    """The GPU's FP32 projection in the oracle's record format (FP64 values)."""
    s = out["splats"].astype(np.float64)
    return dict(xy=np.c_[s[:, 0] + s[:, 10], s[:, 1] + s[:, 11]], conic=s[:, 2:5].copy(), opacity=s[:, 5].copy(),
                rgb=s[:, 6:9].copy(), depth=s[:, 9].copy(), rect=out["rects"], tiles_touched=out["tiles_touched"])


def gpu_depth_bits(out):
    return np.ascontiguousarray(out["splats"][:, 9].astype(np.float32).view(np.uint32))


def gpu_keys(out):
    """64-bit keys implied by the GPU's (ranges, sorted ids)."""
    ranges, ids = out["ranges"], out["sorted_ids"]
    dbits = gpu_depth_bits(out).astype(np.uint64)
    keys = np.zeros(len(ids), np.uint64)
    for t in range(ranges.shape[0]):
        a, b = int(ranges[t, 0]), int(ranges[t, 1])
        if b > a:
            keys[a:b] = (np.uint64(t) << np.uint64(32)) | dbits[ids[a:b]]
    return keys


def max_rel(a, b):
    """max |a - b| / max |b| (per-tensor relative error)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    scale = np.abs(b).max()
    if scale == 0:
        return float(np.abs(a).max())
    return float(np.abs(a - b).max() / scale)


def split_grad2d(g):
    g = np.asarray(g, np.float64)
    return dict(dxy=g[:, 0:2], dconic=g[:, 2:5], dopacity=g[:, 5], drgb=g[:, 6:9])


def flagged_tiles(orc_proj, gpu_out, tiles_x):
    """Tiles whose lists may differ between FP64 and FP32 rects (flagged Gaussians)."""
    bad = np.zeros(gpu_out["ranges"].shape[0], bool)
    diff = np.nonzero((orc_proj["rect"] != gpu_out["rects"]).any(1) |
                      (orc_proj["radius"] != gpu_out["radii"]))[0]
    for g in diff:
        for rc in (orc_proj["rect"][g], gpu_out["rects"][g]):
            if rc[2] >= rc[0]:
                for ty in range(rc[1], rc[3] + 1):
                    bad[ty * tiles_x + rc[0]: ty * tiles_x + rc[2] + 1] = True
    return bad, diff


def tile_pixel_mask(tile_flags, w_ds, h_ds, tiles_x, tile=16):
    ys, xs = np.mgrid[0:h_ds, 0:w_ds]
    return tile_flags[(ys // tile) * tiles_x + xs // tile]


# element-wise error reports of the gradient comparisons, written out at the end of
# the session when GS_PARITY_REPORT names a file (see conftest.py)
REPORT = {}


def grad_report(key, a, b):
    """max |a - b| / max |b| (the asserted per-tensor figure) beside percentiles
    of the element-wise relative error |a - b| / (|b| + 1e-3 max |b|) (the floor
    keeps elements near zero from dividing by nothing); recorded under key."""
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    scale = float(np.abs(b).max()) if b.size else 0.0
    mr = max_rel(a, b)
    if scale > 0:
        el = np.abs(a - b) / (np.abs(b) + 1e-3 * scale)
        pct = {f"p{q}": float(np.percentile(el, q)) for q in (50, 90, 99, 99.9)}
    else:
        pct = {f"p{q}": 0.0 for q in (50, 90, 99, 99.9)}
    REPORT[report_key(key)] = dict(max_rel=mr, **pct, n=int(b.size))
    return mr


def report_key(key):
    """key prefixed with the running test's id."""
    import os
    test = os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0]
    return f"{test}:{key}"
