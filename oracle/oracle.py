"""FP64 CPU oracle of the Turbo-GS dilated 3DGS rasterizer hot path (numpy API).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s ``cpu_baseline`` leg (and its ``--impl reference`` arm) may
import this module. The product package never imports it; it shares no code
with the CUDA path. The arithmetic lives in ``gs_oracle.c`` (plain C, double
precision, OpenMP over independent Gaussians and tiles), which follows the
paper step by step:

* Sec. 3, Eq. 1 and the covariance R S S^T R^T; Sec. 3 Eq. 2 alpha blending;
* Sec. 3.1 (dilated rendering): EWA projection with the original focal length
  plus the low-pass term, 3-sigma radius, Eq. 3-4 centre/radius in the
  downsampled grid, Eq. 5 mapping of downsampled pixels to hr pixels;
* Sec. 3.3 densification statistics (positional and colour gradient norms);
* Sec. 4.1 Adam.

Parity pins: every function here is pinned in ``tests/test_oracle_pins.py``
against closed forms, library routines, brute force and finite differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_HDR = os.path.join(_HERE, "gs_oracle.h")
_LIB = os.path.join(_HERE, "libgs_oracle.so")

FLAG_RADIUS = 1 << 0
FLAG_RECT = 1 << 1
FLAG_NEAR = 1 << 2
FLAG_CLAMP = 1 << 3
FLAG_RGB = 1 << 4
FLAG_CULLED = 1 << 5
FLAG_AMBIGUOUS = FLAG_RADIUS | FLAG_RECT | FLAG_NEAR | FLAG_CLAMP | FLAG_RGB


def build(force: bool = False) -> str:
    """Compile gs_oracle.c into libgs_oracle.so next to it (gcc, OpenMP)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class OrcCamera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double * 9), ("T", ctypes.c_double * 3),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("z_near", ctypes.c_double)]


class OrcDilation(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("ox", ctypes.c_int32), ("oy", ctypes.c_int32),
                ("center_mode", ctypes.c_int32), ("tile", ctypes.c_int32)]


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    cam_p, dil_p = ctypes.POINTER(OrcCamera), ctypes.POINTER(OrcDilation)
    lib.orc_grid.argtypes = [cam_p, dil_p, P, P, P, P]
    lib.orc_sh_basis.argtypes = [i32, P, P]
    lib.orc_project.argtypes = [i32, i32, P, P, P, P, P, cam_p, dil_p] + [P] * 10
    lib.orc_project.restype = i64
    lib.orc_bin.argtypes = [i32, P, P, P, i32, i32, P, P, P]
    lib.orc_bin.restype = i64
    lib.orc_bin_tiles.argtypes = [i32, P, P, i32, i32, P, P, P]
    lib.orc_bin_tiles.restype = i64
    lib.orc_render_fwd.argtypes = [P, P, P, P, P, P, P, i32, P, cam_p, dil_p, P, P, P, P, P, P]
    lib.orc_render_bwd.argtypes = [P, P, P, P, P, P, i32, P, cam_p, dil_p, P, P, P, P, P, P]
    lib.orc_loss_l1.argtypes = [cam_p, dil_p, P, P, P]
    lib.orc_loss_l1.restype = f64
    lib.orc_project_bwd.argtypes = [i32, i32, P, P, P, P, P, cam_p, dil_p] + [P] * 9
    lib.orc_densify_stats.argtypes = [i32, P, P, P, P, P, P]
    lib.orc_adam.argtypes = [i64, i32, P, P, P, P, f64, f64, f64, f64, i32, P]
    _lib = lib
    return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Camera:
    """Pinhole camera: camera-space point t = R m + T; pixel (fx tx/tz + cx, fy ty/tz + cy)."""
    R: np.ndarray
    T: np.ndarray
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    z_near: float = 0.2

    def c(self) -> OrcCamera:
        cam = OrcCamera()
        cam.R[:] = [float(v) for v in np.asarray(self.R, np.float64).reshape(9)]
        cam.T[:] = [float(v) for v in np.asarray(self.T, np.float64).reshape(3)]
        cam.fx, cam.fy, cam.cx, cam.cy = float(self.fx), float(self.fy), float(self.cx), float(self.cy)
        cam.width, cam.height, cam.z_near = int(self.width), int(self.height), float(self.z_near)
        return cam


@dataclass
class Dilation:
    d: int = 1
    ox: int = 0
    oy: int = 0
    center_mode: int = 0
    tile: int = 16

    def c(self) -> OrcDilation:
        return OrcDilation(self.d, self.ox, self.oy, self.center_mode, self.tile)


def as_camera(cam) -> Camera:
    """Accept an oracle Camera or any object with the same attributes."""
    if isinstance(cam, Camera):
        return cam
    return Camera(np.asarray(cam.R, np.float64), np.asarray(cam.T, np.float64), cam.fx, cam.fy,
                  cam.cx, cam.cy, cam.width, cam.height, getattr(cam, "z_near", 0.2))


def as_dilation(dil) -> Dilation:
    if isinstance(dil, Dilation):
        return dil
    return Dilation(dil.d, dil.ox, dil.oy, getattr(dil, "center_mode", 0), getattr(dil, "tile", 16))


def grid(cam, dil):
    """(w_ds, h_ds, tiles_x, tiles_y) of the downsampled image for this offset."""
    lib = _load()
    out = [ctypes.c_int32() for _ in range(4)]
    lib.orc_grid(ctypes.byref(as_camera(cam).c()), ctypes.byref(as_dilation(dil).c()),
                 *[ctypes.byref(o) for o in out])
    return tuple(int(o.value) for o in out)


def sh_basis(deg: int, direction) -> np.ndarray:
    lib = _load()
    d = _f64(direction).reshape(3)
    out = np.zeros((deg + 1) ** 2, np.float64)
    lib.orc_sh_basis(deg, _p(d), _p(out))
    return out


def project(params: dict, cam, dil) -> dict:
    """Project every Gaussian. params: means (n,3), log_scales (n,3), quats (n,4)
    as (w,x,y,z), opacity_logits (n,), sh (n,K,3) with K=(deg+1)^2."""
    lib = _load()
    means, log_scales = _f64(params["means"]), _f64(params["log_scales"])
    quats, logits, sh = _f64(params["quats"]), _f64(params["opacity_logits"]), _f64(params["sh"])
    n = means.shape[0]
    deg = int(round(np.sqrt(sh.shape[1]))) - 1
    if deg > 3 or (deg + 1) ** 2 != sh.shape[1]:
        raise ValueError("sh must have (deg+1)^2 <= 16 coefficients")
    out = dict(xy=np.zeros((n, 2)), conic=np.zeros((n, 3)), opacity=np.zeros(n), rgb=np.zeros((n, 3)),
               depth=np.zeros(n), cov2d=np.zeros((n, 3)), radius=np.zeros(n, np.int32),
               rect=np.zeros((n, 4), np.int32), tiles_touched=np.zeros(n, np.int64),
               flags=np.zeros(n, np.uint32))
    vis = lib.orc_project(n, deg, _p(means), _p(log_scales), _p(quats), _p(logits), _p(sh),
                          ctypes.byref(as_camera(cam).c()), ctypes.byref(as_dilation(dil).c()),
                          _p(out["xy"]), _p(out["conic"]), _p(out["opacity"]), _p(out["rgb"]),
                          _p(out["depth"]), _p(out["cov2d"]), _p(out["radius"]), _p(out["rect"]),
                          _p(out["tiles_touched"]), _p(out["flags"]))
    out["visible"] = int(vis)
    return out


def depth_bits(depth) -> np.ndarray:
    """IEEE float32 bit patterns of the depths: the depth part of the sort key."""
    return np.ascontiguousarray(np.asarray(depth, np.float64).astype(np.float32).view(np.uint32))


def bin_sort(rect, tiles_touched, dbits, tiles_x: int, tiles_y: int):
    """Keys (tile<<32 | depth bits), values (Gaussian ids) sorted by (key, id), ranges (T,2)."""
    lib = _load()
    rect = np.ascontiguousarray(rect, np.int32)
    tt = np.ascontiguousarray(tiles_touched, np.int64)
    dbits = np.ascontiguousarray(dbits, np.uint32)
    k = int(tt.sum())
    keys = np.zeros(max(k, 1), np.uint64)
    vals = np.zeros(max(k, 1), np.uint32)
    ranges = np.zeros((tiles_x * tiles_y, 2), np.uint32)
    got = lib.orc_bin(rect.shape[0], _p(rect), _p(tt), _p(dbits), tiles_x, tiles_y,
                      _p(keys), _p(vals), _p(ranges))
    assert got == k
    return keys[:k], vals[:k], ranges


def bin_tiles(rect, dbits, tiles_x: int, tile_ids):
    """Depth-ordered Gaussian lists of a subset of tiles: (vals, ranges (n_tiles,2))."""
    lib = _load()
    rect = np.ascontiguousarray(rect, np.int32)
    dbits = np.ascontiguousarray(dbits, np.uint32)
    tile_ids = np.ascontiguousarray(tile_ids, np.int32)
    nt = tile_ids.shape[0]
    ranges = np.zeros((nt, 2), np.uint32)
    total = lib.orc_bin_tiles(rect.shape[0], _p(rect), _p(dbits), tiles_x, nt, _p(tile_ids), None, _p(ranges))
    vals = np.zeros(max(int(total), 1), np.uint32)
    lib.orc_bin_tiles(rect.shape[0], _p(rect), _p(dbits), tiles_x, nt, _p(tile_ids), _p(vals), _p(ranges))
    return vals[:total], ranges


def render_fwd(proj: dict, vals, ranges, cam, dil, bg=(0.0, 0.0, 0.0), tile_ids=None,
               img=None):
    """Blend the listed tiles (all tiles when tile_ids is None)."""
    lib = _load()
    w_ds, h_ds, tx, ty = grid(cam, dil)
    P = w_ds * h_ds
    if img is None:
        img = np.zeros((h_ds, w_ds, 3))
    t_final = np.ones((h_ds, w_ds))
    last = np.zeros((h_ds, w_ds), np.uint32)
    amb = np.zeros((h_ds, w_ds), np.uint8)
    counts = np.zeros(2, np.uint64)
    vals = np.ascontiguousarray(vals, np.uint32)
    ranges = np.ascontiguousarray(ranges, np.uint32)
    bg = _f64(bg)
    tid = None if tile_ids is None else np.ascontiguousarray(tile_ids, np.int32)
    nt = tx * ty if tid is None else tid.shape[0]
    assert P == img.shape[0] * img.shape[1]
    lib.orc_render_fwd(_p(_f64(proj["xy"])), _p(_f64(proj["conic"])), _p(_f64(proj["opacity"])),
                       _p(_f64(proj["rgb"])), _p(_f64(proj["depth"])), _p(vals), _p(ranges), nt, _p(tid),
                       ctypes.byref(as_camera(cam).c()), ctypes.byref(as_dilation(dil).c()), _p(bg),
                       _p(img), _p(t_final), _p(last), _p(amb), _p(counts))
    return dict(img=img, t_final=t_final, last=last, ambiguous=amb.astype(bool),
                n_eval=int(counts[0]), n_blend=int(counts[1]))


def render_bwd(proj: dict, vals, ranges, cam, dil, dl_dimg, bg=(0.0, 0.0, 0.0), tile_ids=None):
    lib = _load()
    n = proj["xy"].shape[0]
    w_ds, h_ds, tx, ty = grid(cam, dil)
    out = dict(dxy=np.zeros((n, 2)), dconic=np.zeros((n, 3)), dopacity=np.zeros(n), drgb=np.zeros((n, 3)))
    vals = np.ascontiguousarray(vals, np.uint32)
    ranges = np.ascontiguousarray(ranges, np.uint32)
    tid = None if tile_ids is None else np.ascontiguousarray(tile_ids, np.int32)
    nt = tx * ty if tid is None else tid.shape[0]
    g = _f64(dl_dimg).reshape(h_ds, w_ds, 3)
    lib.orc_render_bwd(_p(_f64(proj["xy"])), _p(_f64(proj["conic"])), _p(_f64(proj["opacity"])),
                       _p(_f64(proj["rgb"])), _p(vals), _p(ranges), nt, _p(tid),
                       ctypes.byref(as_camera(cam).c()), ctypes.byref(as_dilation(dil).c()), _p(_f64(bg)),
                       _p(g), _p(out["dxy"]), _p(out["dconic"]), _p(out["dopacity"]), _p(out["drgb"]))
    return out


def loss_l1(img, target, cam, dil):
    """L1 loss over the rendered lattice pixels; returns (L, dL/dimg)."""
    lib = _load()
    img = _f64(img)
    target = _f64(target)
    g = np.zeros_like(img)
    L = lib.orc_loss_l1(ctypes.byref(as_camera(cam).c()), ctypes.byref(as_dilation(dil).c()),
                        _p(img), _p(target), _p(g))
    return float(L), g


def project_bwd(params: dict, cam, dil, g2d: dict) -> dict:
    lib = _load()
    means, log_scales = _f64(params["means"]), _f64(params["log_scales"])
    quats, logits, sh = _f64(params["quats"]), _f64(params["opacity_logits"]), _f64(params["sh"])
    n = means.shape[0]
    deg = int(round(np.sqrt(sh.shape[1]))) - 1
    out = dict(means=np.zeros_like(means), log_scales=np.zeros_like(log_scales), quats=np.zeros_like(quats),
               opacity_logits=np.zeros_like(logits), sh=np.zeros_like(sh))
    lib.orc_project_bwd(n, deg, _p(means), _p(log_scales), _p(quats), _p(logits), _p(sh),
                        ctypes.byref(as_camera(cam).c()), ctypes.byref(as_dilation(dil).c()),
                        _p(_f64(g2d["dxy"])), _p(_f64(g2d["dconic"])), _p(_f64(g2d["dopacity"])),
                        _p(_f64(g2d["drgb"])), _p(out["means"]), _p(out["log_scales"]), _p(out["quats"]),
                        _p(out["opacity_logits"]), _p(out["sh"]))
    return out


def densify_stats(tiles_touched, g2d: dict, pos_acc, col_acc, count):
    """Accumulate in place (arrays must be float64 / int32)."""
    lib = _load()
    tt = np.ascontiguousarray(tiles_touched, np.int64)
    lib.orc_densify_stats(tt.shape[0], _p(tt), _p(_f64(g2d["dxy"])), _p(_f64(g2d["drgb"])),
                          _p(pos_acc), _p(col_acc), _p(count))


def adam(param, grad, m, v, lr, beta1, beta2, eps, step, row_mask=None):
    """In-place Adam on float64 arrays; row_mask (per leading-dim row) optional."""
    lib = _load()
    assert param.dtype == np.float64 and m.dtype == np.float64 and v.dtype == np.float64
    row_width = int(np.prod(param.shape[1:])) if param.ndim > 1 else 1
    mask = None if row_mask is None else np.ascontiguousarray(row_mask, np.uint8)
    lib.orc_adam(param.size, row_width, _p(param), _p(_f64(grad)), _p(m), _p(v), float(lr), float(beta1),
                 float(beta2), float(eps), int(step), _p(mask))


def forward_backward(params: dict, cam, dil, target, bg=(0.0, 0.0, 0.0)):
    """The whole hot path of one view in FP64: project, bin, blend, L1 loss,
    blend backward, projection backward. Returns every intermediate."""
    proj = project(params, cam, dil)
    w_ds, h_ds, tx, ty = grid(cam, dil)
    keys, vals, ranges = bin_sort(proj["rect"], proj["tiles_touched"], depth_bits(proj["depth"]), tx, ty)
    fwd = render_fwd(proj, vals, ranges, cam, dil, bg)
    L, dl = loss_l1(fwd["img"], target, cam, dil)
    g2d = render_bwd(proj, vals, ranges, cam, dil, dl, bg)
    grads = project_bwd(params, cam, dil, g2d)
    return dict(proj=proj, keys=keys, vals=vals, ranges=ranges, fwd=fwd, loss=L, dl_dimg=dl,
                g2d=g2d, grads=grads)
