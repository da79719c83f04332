"""Thin Python binding of ``libturbogs.so`` (C ABI in ``include/turbogs.h``).

Every function here has the name of the C entry point it calls and only
marshals arguments: torch CUDA tensors become device pointers, the current
torch stream becomes the ``cudaStream_t``. All arithmetic runs in the CUDA
kernels. A missing library raises ``RuntimeError`` (no fallback).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libturbogs.so")

GS_OK, GS_ERR_ARG, GS_ERR_CAPACITY, GS_ERR_CUDA, GS_ERR_TIMEOUT = 0, 1, 2, 3, 4
GS_DTYPE_F32, GS_DTYPE_BF16, GS_DTYPE_F16 = 0, 1, 2
SPLAT_FLOATS = 16
GRAD2D_FLOATS = 12
ADAM_MAX_TENSORS = 8

MAX_VIEWS = 16

SYMBOLS = ("gs_version", "gs_last_error", "gs_grid", "gs_bin_grid", "gs_project", "gs_bin_sort_workspace_size", "gs_bin_sort",
           "gs_bin_sort_static", "gs_tile_order", "gs_render_fwd", "gs_loss_l1", "gs_render_bwd", "gs_project_bwd",
           "gs_project_bwd_adam", "gs_adam_advance", "gs_densify_stats", "gs_adam", "gs_project_batch",
           "gs_tile_order_batch", "gs_tile_order_by_last_batch", "gs_render_fwd_batch", "gs_render_fwd_l1", "gs_loss_l1_batch", "gs_render_bwd_batch",
           "gs_project_bwd_adam_batch", "gs_densify_workspace_size", "gs_densify_select", "gs_prune_select",
           "gs_gather_rows", "gs_densify_grow", "gs_ssim_workspace_size", "gs_ssim", "gs_loss_l1_dssim",
           "gs_project_bwd_adam_next")

GS_MAX_ROW_TENSORS = 24
GS_ROW_COPY, GS_ROW_MEANS, GS_ROW_LOG_SCALES, GS_ROW_QUATS, GS_ROW_STATE, GS_ROW_ZERO = range(6)


class GsError(RuntimeError):
    pass


class GsCamera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("T", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("z_near", ctypes.c_float)]


class GsDilation(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("ox", ctypes.c_int32), ("oy", ctypes.c_int32),
                ("center_mode", ctypes.c_int32), ("tile", ctypes.c_int32), ("bin_shift", ctypes.c_int32)]


class GsAdamTensor(ctypes.Structure):
    _fields_ = [("param", ctypes.c_void_p), ("grad", ctypes.c_void_p), ("m", ctypes.c_void_p),
                ("v", ctypes.c_void_p), ("shadow", ctypes.c_void_p), ("numel", ctypes.c_int64),
                ("row_width", ctypes.c_int32), ("shadow_dtype", ctypes.c_int32), ("lr", ctypes.c_float),
                ("sr_seed", ctypes.c_uint32)]


class GsAdamParams(ctypes.Structure):
    _fields_ = [("param", ctypes.c_void_p * 5), ("m", ctypes.c_void_p * 5), ("v", ctypes.c_void_p * 5),
                ("lr", ctypes.c_float * 5), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("step", ctypes.c_int32), ("sparse", ctypes.c_int32),
                ("sh_shadow", ctypes.c_void_p), ("sh_shadow_dtype", ctypes.c_int32), ("bias_dev", ctypes.c_void_p),
                ("step_dev", ctypes.c_void_p), ("sr_seed", ctypes.c_uint32)]


_VIEW_BUFFERS = ("splats", "radii", "rects", "tiles_touched", "sorted_ids", "ranges", "img", "t_final", "last",
                 "target", "dl_dimg", "grad2d", "loss", "depth_keys")


class GsRowTensor(ctypes.Structure):
    _fields_ = [("src", ctypes.c_void_p), ("dst", ctypes.c_void_p), ("row_bytes", ctypes.c_int32),
                ("role", ctypes.c_int32)]


class GsView(ctypes.Structure):
    _fields_ = [("cam", GsCamera), ("dil", GsDilation)] + [(k, ctypes.c_void_p) for k in _VIEW_BUFFERS] + \
        [("target_dtype", ctypes.c_int32)]


TARGET_F32, TARGET_U8 = 0, 1  # GS_TARGET_F32, GS_TARGET_U8


def target_dtype(t) -> int:
    """The C ABI's code for a target image tensor: FP32 values, or 8-bit values
    the kernels read as t * (1/255)."""
    if t is None or t.dtype == torch.float32:
        return TARGET_F32
    if t.dtype == torch.uint8:
        return TARGET_U8
    raise ValueError(f"target: float32 or uint8 expected, got {t.dtype}")


@dataclass(frozen=True)
class Dilation:
    """Sec. 3.1: render the lattice (d*u + ox, d*v + oy) of the hr image.
    tile: blend tile edge; bin_shift: bin with tiles of tile << bin_shift."""
    d: int = 1
    ox: int = 0
    oy: int = 0
    center_mode: int = 0
    tile: int = 16
    bin_shift: int = 0

    def c(self) -> GsDilation:
        return GsDilation(self.d, self.ox, self.oy, self.center_mode, self.tile, self.bin_shift)


@dataclass
class View:
    """One view of a batch: its camera, dilation and the device buffers of
    that view (any may be None when the call at hand does not use it)."""
    cam: object
    dil: Dilation
    splats: torch.Tensor | None = None
    radii: torch.Tensor | None = None
    rects: torch.Tensor | None = None
    tiles_touched: torch.Tensor | None = None
    sorted_ids: torch.Tensor | None = None
    ranges: torch.Tensor | None = None
    img: torch.Tensor | None = None
    t_final: torch.Tensor | None = None
    last: torch.Tensor | None = None
    target: torch.Tensor | None = None
    dl_dimg: torch.Tensor | None = None
    grad2d: torch.Tensor | None = None
    loss: torch.Tensor | None = None
    depth_keys: torch.Tensor | None = None


class ViewTable:
    """The GsView array of a batch, built once and reused by every batched
    call (it holds only pointers, so refilled buffers need no rebuild)."""

    def __init__(self, views):
        views = list(views)
        if not 1 <= len(views) <= MAX_VIEWS:
            raise ValueError(f"a batch holds 1..{MAX_VIEWS} views")
        self.views = views
        self.n = len(views)
        self.arr = (GsView * self.n)()
        for i, v in enumerate(views):
            self.arr[i].cam = camera(v.cam)
            self.arr[i].dil = v.dil.c()
            for k in _VIEW_BUFFERS:
                t = getattr(v, k)
                setattr(self.arr[i], k, None if t is None else _ptr(t).value)
            self.arr[i].target_dtype = target_dtype(v.target)


def _table(views) -> ViewTable:
    return views if isinstance(views, ViewTable) else ViewTable(views)


def camera(cam) -> GsCamera:
    """GsCamera from any object with R (3x3), T (3), fx, fy, cx, cy, width, height[, z_near]."""
    c = GsCamera()
    R = [float(x) for row in cam.R for x in row] if not hasattr(cam.R, "reshape") else \
        [float(x) for x in cam.R.reshape(9)]
    c.R[:] = R
    c.T[:] = [float(x) for x in (cam.T.reshape(3) if hasattr(cam.T, "reshape") else cam.T)]
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.z_near = float(getattr(cam, "z_near", 0.2))
    return c


_lib = None


def load():
    """Load libturbogs.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libturbogs.so is missing: build it with `python -m paper_2412_13547_b300.build_native`"
                           " (there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
    cam_p, dil_p = ctypes.POINTER(GsCamera), ctypes.POINTER(GsDilation)
    lib.gs_version.restype = i32
    lib.gs_last_error.restype = ctypes.c_char_p
    lib.gs_grid.argtypes = [cam_p, dil_p, P, P, P, P]
    lib.gs_bin_grid.argtypes = [cam_p, dil_p, P, P]
    lib.gs_project.argtypes = [i32, i32, i32, P, P, P, P, P, cam_p, dil_p, P, P, P, P, P, P]
    lib.gs_bin_sort_workspace_size.argtypes = [i32, i64, i32, i32]
    lib.gs_bin_sort_workspace_size.restype = ctypes.c_size_t
    lib.gs_bin_sort.argtypes = [i32, P, P, P, P, i32, i32, P, ctypes.c_size_t, i64, P, P, P, P, P]
    lib.gs_bin_sort_static.argtypes = [i32, P, P, P, P, i32, i32, i64, P, P, P, P, P]
    lib.gs_tile_order.argtypes = [P, i32, P, P]
    lib.gs_render_fwd.argtypes = [i32, P, P, P, cam_p, dil_p, P, P, P, P, P, i32, P, P]
    lib.gs_loss_l1.argtypes = [cam_p, dil_p, P, P, i32, P, P, P]
    lib.gs_render_bwd.argtypes = [i32, P, P, P, cam_p, dil_p, P, P, P, P, P, i32, i32, P, P]
    lib.gs_project_bwd.argtypes = [i32, i32, i32, P, P, P, P, P, cam_p, dil_p, P, P, P, P, P, P, P, P, P, P, P]
    lib.gs_densify_stats.argtypes = [i32, P, P, P, P, P, P]
    lib.gs_project_bwd_adam.argtypes = [i32, i32, i32, P, cam_p, dil_p, P, P, ctypes.POINTER(GsAdamParams), P, P,
                                        P, P, P]
    lib.gs_adam.argtypes = [ctypes.POINTER(GsAdamTensor), i32, f32, f32, f32, i32, P, P]
    lib.gs_project_bwd_adam_next.argtypes = [i32, i32, i32, P, cam_p, dil_p, P, P, ctypes.POINTER(GsAdamParams),
                                             P, P, P, P, ctypes.POINTER(GsView), P]
    lib.gs_adam_advance.argtypes = [P, f32, f32, P, P]
    view_p = ctypes.POINTER(GsView)
    lib.gs_project_batch.argtypes = [i32, i32, i32, P, P, P, P, P, view_p, i32, P]
    lib.gs_tile_order_batch.argtypes = [view_p, i32, P, P]
    lib.gs_tile_order_by_last_batch.argtypes = [view_p, i32, P, P]
    lib.gs_render_fwd_batch.argtypes = [i32, view_p, i32, P, P, P, i32, i32, P]
    lib.gs_render_fwd_l1.argtypes = [i32, P, P, P, cam_p, dil_p, P, P, P, P, P, i32, P, P, P, P, i32, P, P]
    lib.gs_loss_l1_batch.argtypes = [view_p, i32, P]
    lib.gs_render_bwd_batch.argtypes = [i32, view_p, i32, P, P, i32, i32, P]
    lib.gs_project_bwd_adam_batch.argtypes = [i32, i32, i32, P, view_p, i32, ctypes.POINTER(GsAdamParams), P, P, P,
                                              P, P]
    lib.gs_densify_workspace_size.argtypes = [i32]
    lib.gs_densify_workspace_size.restype = ctypes.c_size_t
    lib.gs_densify_select.argtypes = [i32, P, P, P, f32, f32, i32, i32, P, ctypes.c_size_t, P, P, P]
    lib.gs_prune_select.argtypes = [i32, P, f32, P, f32, P, ctypes.c_size_t, P, P, P]
    rows_p = ctypes.POINTER(GsRowTensor)
    lib.gs_gather_rows.argtypes = [i32, P, rows_p, i32, P]
    lib.gs_densify_grow.argtypes = [i32, i32, P, P, f32, rows_p, i32, P]
    lib.gs_ssim_workspace_size.argtypes = [cam_p, dil_p]
    lib.gs_ssim_workspace_size.restype = ctypes.c_size_t
    lib.gs_ssim.argtypes = [cam_p, dil_p, P, P, i32, i32, P, P, P, ctypes.c_size_t, P]
    lib.gs_loss_l1_dssim.argtypes = [cam_p, dil_p, P, P, i32, f32, i32, P, P, P, ctypes.c_size_t, P]
    for name in SYMBOLS:
        if name not in ("gs_last_error", "gs_bin_sort_workspace_size", "gs_densify_workspace_size",
                        "gs_ssim_workspace_size"):
            getattr(lib, name).restype = i32
    _lib = lib
    return lib


def _check(rc: int, name: str):
    if rc != GS_OK:
        msg = load().gs_last_error().decode(errors="replace")
        raise GsError(f"{name} failed ({rc}): {msg}")


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


_SH_DTYPE = {torch.float32: GS_DTYPE_F32, torch.bfloat16: GS_DTYPE_BF16, torch.float16: GS_DTYPE_F16}


def sh_degree_of(sh: torch.Tensor) -> int:
    k = sh.shape[1]
    deg = int(round(k ** 0.5)) - 1
    if (deg + 1) ** 2 != k or sh.shape[2] != 3:
        raise ValueError("sh must be n x (deg+1)^2 x 3")
    return deg


def gs_version() -> int:
    return int(load().gs_version())


def gs_grid(cam, dil: Dilation):
    out = [ctypes.c_int32() for _ in range(4)]
    _check(load().gs_grid(ctypes.byref(camera(cam)), ctypes.byref(dil.c()), *[ctypes.byref(o) for o in out]),
           "gs_grid")
    return tuple(int(o.value) for o in out)


def gs_bin_grid(cam, dil: Dilation):
    """(bin_tiles_x, bin_tiles_y): the grid gs_bin_sort and the ranges use."""
    out = [ctypes.c_int32() for _ in range(2)]
    _check(load().gs_bin_grid(ctypes.byref(camera(cam)), ctypes.byref(dil.c()), *[ctypes.byref(o) for o in out]),
           "gs_bin_grid")
    return tuple(int(o.value) for o in out)


def _need(t, numel, what):
    """The C ABI takes plain pointers: check here that a buffer holds what the call writes."""
    if t is not None and t.numel() < numel:
        raise ValueError(f"{what}: {t.numel()} elements, the call needs {numel}")


def _need_image(dil, cam, img=None, t_final=None, last=None, dl=None):
    w_ds, h_ds, _, _ = gs_grid(cam, dil)
    P = w_ds * h_ds
    _need(img, 3 * P, "img")
    _need(t_final, P, "t_final")
    _need(last, P, "last")
    _need(dl, 3 * P, "dl_dimg")


def gs_project(means, log_scales, quats, opacity_logits, sh, cam, dil: Dilation, splats, radii, rects,
               tiles_touched, stream=None, depth_keys=None):
    """depth_keys (optional, n uint32/int32): the depth sort keys for gs_bin_sort."""
    n = means.shape[0]
    deg = sh_degree_of(sh)
    for t, w, name in ((splats, SPLAT_FLOATS, "splats"), (radii, 1, "radii"), (rects, 4, "rects"),
                       (tiles_touched, 1, "tiles_touched"), (depth_keys, 1, "depth_keys")):
        _need(t, n * w, name)
    _check(load().gs_project(n, deg, _SH_DTYPE[sh.dtype], _ptr(means), _ptr(log_scales), _ptr(quats),
                             _ptr(opacity_logits), _ptr(sh), ctypes.byref(camera(cam)), ctypes.byref(dil.c()),
                             _ptr(splats), _ptr(radii), _ptr(rects), _ptr(tiles_touched), _ptr(depth_keys),
                             _stream(stream)),
           "gs_project")


def gs_bin_sort_workspace_size(n: int, capacity: int, tiles_x: int, tiles_y: int) -> int:
    return int(load().gs_bin_sort_workspace_size(int(n), int(capacity), int(tiles_x), int(tiles_y)))


def gs_bin_sort(n, rects, tiles_touched, splats, tiles_x, tiles_y, workspace, capacity, sorted_ids, ranges,
                num_pairs, stream=None, depth_keys=None, num_pairs_max=None):
    """depth_keys (optional): gs_project's keys of the same call (saves the pass over splats);
    num_pairs_max (optional int64[1]): high-water mark of the pair count across calls."""
    _need(ranges, 2 * int(tiles_x) * int(tiles_y), "ranges")
    _need(sorted_ids, int(capacity), "sorted_ids")
    _need(depth_keys, int(n), "depth_keys")
    _check(load().gs_bin_sort(int(n), _ptr(rects), _ptr(tiles_touched), _ptr(splats), _ptr(depth_keys),
                              int(tiles_x), int(tiles_y), _ptr(workspace), workspace.numel() * workspace.element_size(),
                              int(capacity), _ptr(sorted_ids), _ptr(ranges), _ptr(num_pairs), _ptr(num_pairs_max),
                              _stream(stream)),
           "gs_bin_sort")


BIN_SORT_STATIC_SCRATCH_BYTES = 32 << 20


def gs_bin_sort_static(n, rects, tiles_touched, splats, tiles_x, tiles_y, capacity, sorted_ids, ranges, num_pairs,
                       stream=None, depth_keys=None):
    """gs_bin_sort without a workspace argument: for callers that cannot allocate device memory."""
    _need(depth_keys, int(n), "depth_keys")
    _check(load().gs_bin_sort_static(int(n), _ptr(rects), _ptr(tiles_touched), _ptr(splats), _ptr(depth_keys),
                                     int(tiles_x), int(tiles_y), int(capacity), _ptr(sorted_ids), _ptr(ranges),
                                     _ptr(num_pairs), None, _stream(stream)), "gs_bin_sort_static")


def _bg(bg):
    arr = (ctypes.c_float * 3)(*[float(x) for x in bg])
    return arr


def gs_tile_order(ranges, num_tiles, order, stream=None):
    _check(load().gs_tile_order(_ptr(ranges), int(num_tiles), _ptr(order), _stream(stream)), "gs_tile_order")


def gs_render_fwd(n, splats, sorted_ids, ranges, cam, dil: Dilation, bg, img, t_final, last, counts=None,
                  pixels_per_thread=0, tile_order=None, stream=None):
    _need_image(dil, cam, img, t_final, last)
    _need(counts, 3, "counts")
    _check(load().gs_render_fwd(int(n), _ptr(splats), _ptr(sorted_ids), _ptr(ranges), ctypes.byref(camera(cam)),
                                ctypes.byref(dil.c()), _bg(bg), _ptr(img), _ptr(t_final), _ptr(last), _ptr(counts),
                                int(pixels_per_thread), _ptr(tile_order), _stream(stream)), "gs_render_fwd")


FWD_L1, FWD_ZERO_GRAD2D = 1, 2  # GS_FWD_L1, GS_FWD_ZERO_GRAD2D


def gs_render_fwd_l1(n, splats, sorted_ids, ranges, cam, dil: Dilation, bg, img, t_final, last, target, dl_dimg,
                     loss, grad2d_zero=None, counts=None, pixels_per_thread=0, tile_order=None, stream=None):
    """gs_render_fwd and gs_loss_l1 in one launch; grad2d_zero (optional) is zeroed by it."""
    _need_image(dil, cam, img, t_final, last, dl=dl_dimg)
    _need(target, 3 * int(cam.width) * int(cam.height), "target")
    _need(counts, 3, "counts")
    _need(grad2d_zero, int(n) * GRAD2D_FLOATS, "grad2d")
    _check(load().gs_render_fwd_l1(int(n), _ptr(splats), _ptr(sorted_ids), _ptr(ranges), ctypes.byref(camera(cam)),
                                   ctypes.byref(dil.c()), _bg(bg), _ptr(img), _ptr(t_final), _ptr(last),
                                   _ptr(target), target_dtype(target), _ptr(dl_dimg), _ptr(loss), _ptr(grad2d_zero),
                                   _ptr(counts), int(pixels_per_thread), _ptr(tile_order), _stream(stream)),
           "gs_render_fwd_l1")


def gs_loss_l1(cam, dil: Dilation, img, target, dl_dimg, loss, stream=None):
    _need_image(dil, cam, img=img, dl=dl_dimg)
    _need(target, 3 * int(cam.width) * int(cam.height), "target")
    _check(load().gs_loss_l1(ctypes.byref(camera(cam)), ctypes.byref(dil.c()), _ptr(img), _ptr(target),
                             target_dtype(target), _ptr(dl_dimg), _ptr(loss), _stream(stream)), "gs_loss_l1")


SSIM_VALID, SSIM_SAME = 0, 1


def gs_ssim_workspace_size(cam, dil: Dilation) -> int:
    return int(load().gs_ssim_workspace_size(ctypes.byref(camera(cam)), ctypes.byref(dil.c())))


def gs_ssim(cam, dil: Dilation, img, target, ssim_out, workspace, d_img=None, mode=SSIM_VALID, stream=None):
    """Mean SSIM of the lattice image against the sampled target into
    ssim_out (one float); d_img (optional) receives d(mean SSIM)/d img."""
    _need_image(dil, cam, img=img, dl=d_img)
    _need(target, 3 * int(cam.width) * int(cam.height), "target")
    _check(load().gs_ssim(ctypes.byref(camera(cam)), ctypes.byref(dil.c()), _ptr(img), _ptr(target),
                          target_dtype(target), int(mode), _ptr(ssim_out), _ptr(d_img), _ptr(workspace), workspace.numel() * workspace.element_size(),
                          _stream(stream)), "gs_ssim")


def gs_loss_l1_dssim(cam, dil: Dilation, img, target, lam, dl_dimg, loss, workspace, mode=SSIM_SAME, stream=None):
    """(1 - lam) L1 + lam (1 - SSIM) of the lattice image and its gradient."""
    _need_image(dil, cam, img=img, dl=dl_dimg)
    _need(target, 3 * int(cam.width) * int(cam.height), "target")
    _check(load().gs_loss_l1_dssim(ctypes.byref(camera(cam)), ctypes.byref(dil.c()), _ptr(img), _ptr(target),
                                   target_dtype(target), float(lam), int(mode), _ptr(dl_dimg), _ptr(loss), _ptr(workspace),
                                   workspace.numel() * workspace.element_size(), _stream(stream)),
           "gs_loss_l1_dssim")


def gs_render_bwd(n, splats, sorted_ids, ranges, cam, dil: Dilation, bg, t_final, last, dl_dimg, grad2d,
                  zero_grad2d=True, pixels_per_thread=0, tile_order=None, stream=None):
    _need_image(dil, cam, t_final=t_final, last=last, dl=dl_dimg)
    _need(grad2d, int(n) * GRAD2D_FLOATS, "grad2d")
    _check(load().gs_render_bwd(int(n), _ptr(splats), _ptr(sorted_ids), _ptr(ranges), ctypes.byref(camera(cam)),
                                ctypes.byref(dil.c()), _bg(bg), _ptr(t_final), _ptr(last), _ptr(dl_dimg),
                                _ptr(grad2d), int(bool(zero_grad2d)), int(pixels_per_thread), _ptr(tile_order),
                                _stream(stream)), "gs_render_bwd")


def gs_project_bwd(means, log_scales, quats, opacity_logits, sh, cam, dil: Dilation, tiles_touched, grad2d,
                   d_means, d_log_scales, d_quats, d_opacity_logits, d_sh, pos_acc=None, col_acc=None, count=None,
                   stream=None):
    n = means.shape[0]
    deg = sh_degree_of(sh)
    _check(load().gs_project_bwd(n, deg, _SH_DTYPE[sh.dtype], _ptr(means), _ptr(log_scales), _ptr(quats),
                                 _ptr(opacity_logits), _ptr(sh), ctypes.byref(camera(cam)), ctypes.byref(dil.c()),
                                 _ptr(tiles_touched), _ptr(grad2d), _ptr(d_means), _ptr(d_log_scales), _ptr(d_quats),
                                 _ptr(d_opacity_logits), _ptr(d_sh), _ptr(pos_acc), _ptr(col_acc), _ptr(count),
                                 _stream(stream)), "gs_project_bwd")


def _adam_params(params, m, v, lrs, beta1, beta2, eps, step, sparse, sh_shadow, bias_dev, step_dev=None,
                 sr_seed=0):
    """The GsAdamParams of a fused optimizer call. A BF16/FP16 params[4] is the
    SH kept only in that type (param[4] NULL: the call's sh_store, updated with
    stochastic rounding)."""
    a = GsAdamParams()
    for t in range(5):
        for k, (arr, src) in enumerate(((a.param, params), (a.m, m), (a.v, v))):
            lowp = k == 0 and t == 4 and src[t].dtype in (torch.bfloat16, torch.float16)
            if (src[t].dtype != torch.float32 and not lowp) or not src[t].is_contiguous() or not src[t].is_cuda:
                raise ValueError("parameters and moments must be contiguous FP32 CUDA tensors "
                                 "(the SH parameter may be BF16/FP16: then it is the SH storage itself)")
            arr[t] = None if lowp else src[t].data_ptr()
        a.lr[t] = float(lrs[t])
    a.beta1, a.beta2, a.eps, a.step, a.sparse = float(beta1), float(beta2), float(eps), int(step), int(bool(sparse))
    a.sh_shadow = sh_shadow.data_ptr() if sh_shadow is not None else None
    a.sh_shadow_dtype = _SH_DTYPE[sh_shadow.dtype] if sh_shadow is not None else GS_DTYPE_F32
    a.bias_dev = _ptr(bias_dev).value if bias_dev is not None else None
    a.step_dev = _ptr(step_dev).value if step_dev is not None else None
    a.sr_seed = int(sr_seed) & 0xFFFFFFFF
    return a


def _lowp_sh(params, sh_store):
    if params[4].dtype != torch.float32 and params[4].data_ptr() != sh_store.data_ptr():
        raise ValueError("a BF16/FP16 SH parameter must be the sh_store tensor itself")


def _grads_out(grads_out):
    if grads_out is None:
        return None
    return (ctypes.c_void_p * 5)(*[g.data_ptr() if g is not None else None for g in grads_out])


def gs_project_bwd_adam(params, m, v, lrs, beta1, beta2, eps, step, sh_store, cam, dil: Dilation, tiles_touched,
                        grad2d, sparse=False, sh_shadow=None, pos_acc=None, col_acc=None, count=None,
                        grads_out=None, bias_dev=None, step_dev=None, sr_seed=0, stream=None):
    """params, m, v: lists of the 5 tensors (means, log_scales, quats,
    opacity_logits, sh), updated in place; all FP32 except that the SH may be
    kept only in BF16/FP16 (params[4] is then sh_store, rounded stochastically
    with seed sr_seed). lrs: 5 learning rates. bias_dev (optional device
    float[2] from gs_adam_advance) replaces step; step_dev (optional device
    int32) gives the step of the rounding stream."""
    n = params[0].shape[0]
    deg = sh_degree_of(params[4])
    _lowp_sh(params, sh_store)
    a = _adam_params(params, m, v, lrs, beta1, beta2, eps, step, sparse, sh_shadow, bias_dev, step_dev, sr_seed)
    _check(load().gs_project_bwd_adam(n, deg, _SH_DTYPE[sh_store.dtype], _ptr(sh_store), ctypes.byref(camera(cam)),
                                      ctypes.byref(dil.c()), _ptr(tiles_touched), _ptr(grad2d), ctypes.byref(a),
                                      _ptr(pos_acc), _ptr(col_acc), _ptr(count), _grads_out(grads_out),
                                      _stream(stream)),
           "gs_project_bwd_adam")


def gs_project_bwd_adam_next(params, m, v, lrs, beta1, beta2, eps, step, sh_store, cam, dil: Dilation,
                             tiles_touched, grad2d, next_view, sh_shadow=None, pos_acc=None, col_acc=None, count=None,
                             grads_out=None, bias_dev=None, step_dev=None, sr_seed=0, stream=None):
    """gs_project_bwd_adam (dense Adam) and, in the same launch, gs_project of the updated
    parameters into next_view (a View: its cam, dil, splats, radii, rects, tiles_touched and
    depth_keys)."""
    n = params[0].shape[0]
    deg = sh_degree_of(params[4])
    _lowp_sh(params, sh_store)
    a = _adam_params(params, m, v, lrs, beta1, beta2, eps, step, False, sh_shadow, bias_dev, step_dev, sr_seed)
    nv = next_view if isinstance(next_view, ViewTable) else ViewTable([next_view])
    _check(load().gs_project_bwd_adam_next(n, deg, _SH_DTYPE[sh_store.dtype], _ptr(sh_store),
                                           ctypes.byref(camera(cam)), ctypes.byref(dil.c()), _ptr(tiles_touched),
                                           _ptr(grad2d), ctypes.byref(a), _ptr(pos_acc), _ptr(col_acc), _ptr(count),
                                           _grads_out(grads_out), nv.arr, _stream(stream)),
           "gs_project_bwd_adam_next")


def gs_adam_advance(step_dev, beta1, beta2, bias_dev, stream=None):
    """Device-side Adam step: step_dev (int32[1]) += 1, bias_dev (float[2]) =
    bias corrections of the new step."""
    _check(load().gs_adam_advance(_ptr(step_dev), float(beta1), float(beta2), _ptr(bias_dev), _stream(stream)),
           "gs_adam_advance")


# -- batched views -----------------------------------------------------------

def gs_project_batch(means, log_scales, quats, opacity_logits, sh, views, stream=None):
    t = _table(views)
    _check(load().gs_project_batch(means.shape[0], sh_degree_of(sh), _SH_DTYPE[sh.dtype], _ptr(means),
                                   _ptr(log_scales), _ptr(quats), _ptr(opacity_logits), _ptr(sh), t.arr, t.n,
                                   _stream(stream)), "gs_project_batch")


def _total_tiles(t: ViewTable) -> int:
    return sum(g[2] * g[3] for g in (gs_grid(v.cam, v.dil) for v in t.views))


def gs_tile_order_batch(views, order, stream=None):
    t = _table(views)
    _need(order, _total_tiles(t), "order")
    _check(load().gs_tile_order_batch(t.arr, t.n, _ptr(order), _stream(stream)), "gs_tile_order_batch")


def gs_tile_order_by_last_batch(views, order, stream=None):
    """Backward launch order: tiles longest-first by the largest `last` over
    their pixels (call after the forward)."""
    t = _table(views)
    _need(order, _total_tiles(t), "order")
    _check(load().gs_tile_order_by_last_batch(t.arr, t.n, _ptr(order), _stream(stream)),
           "gs_tile_order_by_last_batch")


def gs_render_fwd_batch(n, views, bg, tile_order=None, counts=None, pixels_per_thread=0, flags=0, stream=None):
    """flags: 0, or FWD_L1 (each view's L1 loss and dL/dimg from its target) and/or
    FWD_ZERO_GRAD2D (each view's grad2d zeroed), fused into the blend launch."""
    t = _table(views)
    _need(counts, 3, "counts")
    _check(load().gs_render_fwd_batch(int(n), t.arr, t.n, _bg(bg), _ptr(tile_order), _ptr(counts),
                                      int(pixels_per_thread), int(flags), _stream(stream)), "gs_render_fwd_batch")


def gs_loss_l1_batch(views, stream=None):
    t = _table(views)
    _check(load().gs_loss_l1_batch(t.arr, t.n, _stream(stream)), "gs_loss_l1_batch")


def gs_render_bwd_batch(n, views, bg, tile_order=None, zero_grad2d=True, pixels_per_thread=0, stream=None):
    t = _table(views)
    _check(load().gs_render_bwd_batch(int(n), t.arr, t.n, _bg(bg), _ptr(tile_order), int(bool(zero_grad2d)),
                                      int(pixels_per_thread), _stream(stream)), "gs_render_bwd_batch")


def gs_project_bwd_adam_batch(params, m, v, lrs, beta1, beta2, eps, step, sh_store, views, sparse=False,
                              sh_shadow=None, pos_acc=None, col_acc=None, count=None, grads_out=None, bias_dev=None,
                              step_dev=None, sr_seed=0, stream=None):
    t = _table(views)
    n = params[0].shape[0]
    _lowp_sh(params, sh_store)
    a = _adam_params(params, m, v, lrs, beta1, beta2, eps, step, sparse, sh_shadow, bias_dev, step_dev, sr_seed)
    _check(load().gs_project_bwd_adam_batch(n, sh_degree_of(params[4]), _SH_DTYPE[sh_store.dtype], _ptr(sh_store),
                                            t.arr, t.n, ctypes.byref(a), _ptr(pos_acc), _ptr(col_acc), _ptr(count),
                                            _grads_out(grads_out), _stream(stream)), "gs_project_bwd_adam_batch")


def gs_densify_stats(n, tiles_touched, grad2d, pos_acc, col_acc, count, stream=None):
    _check(load().gs_densify_stats(int(n), _ptr(tiles_touched), _ptr(grad2d), _ptr(pos_acc), _ptr(col_acc),
                                   _ptr(count), _stream(stream)), "gs_densify_stats")


def gs_adam(entries, beta1, beta2, eps, step, row_mask=None, stream=None):
    """entries: list of dicts with param, grad, m, v (float32 CUDA tensors), lr,
    and optional shadow (bf16/fp16/fp32 tensor of the same shape), row_width
    and sr_seed. A BF16/FP16 param is kept only in that type (no shadow): its
    update is rounded stochastically with seed sr_seed."""
    arr = (GsAdamTensor * max(1, len(entries)))()
    for i, e in enumerate(entries):
        p = e["param"]
        for k in ("grad", "m", "v"):
            if e[k].shape != p.shape or e[k].dtype != torch.float32:
                raise ValueError(f"adam entry {i}: {k} must match param (float32)")
        sh = e.get("shadow")
        arr[i].sr_seed = int(e.get("sr_seed", 0)) & 0xFFFFFFFF
        if p.dtype in (torch.bfloat16, torch.float16):
            if sh is not None:
                raise ValueError(f"adam entry {i}: a BF16/FP16 parameter takes no shadow")
            arr[i].param = None
            arr[i].grad = e["grad"].data_ptr()
            arr[i].m = e["m"].data_ptr()
            arr[i].v = e["v"].data_ptr()
            arr[i].shadow = p.data_ptr()
            arr[i].numel = p.numel()
            arr[i].row_width = int(e.get("row_width", p[0].numel() if p.dim() > 1 and p.shape[0] > 0 else 1))
            arr[i].shadow_dtype = _SH_DTYPE[p.dtype]
            arr[i].lr = float(e["lr"])
            continue
        arr[i].param = p.data_ptr()
        arr[i].grad = e["grad"].data_ptr()
        arr[i].m = e["m"].data_ptr()
        arr[i].v = e["v"].data_ptr()
        arr[i].shadow = sh.data_ptr() if sh is not None else None
        arr[i].numel = p.numel()
        arr[i].row_width = int(e.get("row_width", p[0].numel() if p.dim() > 1 and p.shape[0] > 0 else 1))
        arr[i].shadow_dtype = _SH_DTYPE[sh.dtype] if sh is not None else GS_DTYPE_F32
        arr[i].lr = float(e["lr"])
    _check(load().gs_adam(arr, len(entries), float(beta1), float(beta2), float(eps), int(step), _ptr(row_mask),
                          _stream(stream)), "gs_adam")


# -- densification and pruning ----------------------------------------------

def gs_densify_workspace_size(n: int) -> int:
    return int(load().gs_densify_workspace_size(int(n)))


def gs_densify_select(n, pos_acc, col_acc, count, tau_pos, tau_color, color_branch, max_new, workspace, selected,
                      num_selected, stream=None):
    _check(load().gs_densify_select(int(n), _ptr(pos_acc), _ptr(col_acc), _ptr(count), float(tau_pos),
                                    float(tau_color), int(bool(color_branch)), int(max_new), _ptr(workspace),
                                    workspace.numel() * workspace.element_size(), _ptr(selected),
                                    _ptr(num_selected), _stream(stream)), "gs_densify_select")


def gs_prune_select(n, opacity_logits, logit_min, log_scales, log_scale_max, workspace, keep, num_keep,
                    stream=None):
    _check(load().gs_prune_select(int(n), _ptr(opacity_logits), float(logit_min), _ptr(log_scales),
                                  float(log_scale_max), _ptr(workspace), workspace.numel() * workspace.element_size(),
                                  _ptr(keep), _ptr(num_keep), _stream(stream)), "gs_prune_select")


def _rows(entries):
    """entries: (src tensor or None, dst tensor, role); rows = first dimension."""
    arr = (GsRowTensor * len(entries))()
    for i, (src, dst, role) in enumerate(entries):
        rb = int(np.prod(dst.shape[1:], dtype=np.int64)) * dst.element_size()
        if src is not None and (src.dtype != dst.dtype or src.shape[1:] != dst.shape[1:]):
            raise ValueError(f"row tensor {i}: src and dst rows differ")
        arr[i].src = None if src is None else _ptr(src).value
        arr[i].dst = _ptr(dst).value
        arr[i].row_bytes = int(rb)
        arr[i].role = int(role)
    return arr


def gs_gather_rows(n_out, index, entries, stream=None):
    arr = _rows(entries)
    _check(load().gs_gather_rows(int(n_out), _ptr(index), arr, len(entries), _stream(stream)), "gs_gather_rows")


def gs_densify_grow(n_old, m, selected, noise, log_split_scale, entries, stream=None):
    arr = _rows(entries)
    _check(load().gs_densify_grow(int(n_old), int(m), _ptr(selected), _ptr(noise), float(log_split_scale), arr,
                                  len(entries), _stream(stream)), "gs_densify_grow")
