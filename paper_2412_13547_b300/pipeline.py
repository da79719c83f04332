"""The hot path of Turbo-GS fitting on the device: buffers, the autograd
wrapper and one full training step (project -> bin/sort -> blend -> L1 ->
blend backward -> projection backward + densification statistics -> Adam).

Every stage is one call into ``libturbogs.so`` through ``raster``; this module
only owns device memory and orders the calls on the current CUDA stream.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch

from . import raster as R
from .raster import Dilation


def _dev(x, device, dtype=torch.float32):
    return torch.as_tensor(x, dtype=dtype).to(device).contiguous()


@dataclass
class GaussianParams:
    """Device tensors of the Gaussians (Sec. 3): means, log-scales, quaternions
    (w,x,y,z), opacity logits and SH coefficients (n x K x 3). ``sh_store`` is the
    tensor the projection reads. Three forms of SH storage:

    * FP32: ``sh`` is ``sh_store``;
    * low precision (the precision form): ``sh`` is ``sh_store``, a BF16/FP16
      tensor and the only copy of the SH; Adam updates it in FP32 arithmetic
      and rounds stochastically (blending and accumulation stay FP32);
    * FP32 master: ``sh`` FP32 and ``sh_store`` its BF16/FP16 copy, refreshed
      by Adam after every update."""
    means: torch.Tensor
    log_scales: torch.Tensor
    quats: torch.Tensor
    opacity_logits: torch.Tensor
    sh: torch.Tensor
    sh_store: torch.Tensor

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @classmethod
    def from_arrays(cls, arrays: dict, device="cuda", sh_dtype=torch.float32, master: bool = False):
        """sh_dtype BF16/FP16 keeps the SH only in that type (rounded to nearest
        once here), or with master=True as a copy of an FP32 master."""
        p = {k: _dev(arrays[k], device) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
        p["opacity_logits"] = p["opacity_logits"].reshape(-1)
        if sh_dtype == torch.float32:
            return cls(sh_store=p["sh"], **p)
        store = p["sh"].to(sh_dtype).contiguous()
        if not master:
            p["sh"] = store
        return cls(sh_store=store, **p)

    @property
    def sh_lowp(self) -> bool:
        """The SH exists only in BF16/FP16 (no FP32 master)."""
        return self.sh.dtype != torch.float32

    def tensors(self):
        return [self.means, self.log_scales, self.quats, self.opacity_logits, self.sh]


class Rasterizer:
    """Scratch of the hot path for up to ``n`` Gaussians, a pair capacity and a
    tile grid. Nothing here synchronises with the host except ``num_pairs()``
    and ``ensure_capacity``."""

    def __init__(self, n: int, capacity: int = 1 << 20, max_tiles: int = 1, device="cuda",
                 pixels_per_thread: int = 0, max_grid=None, longest_first: bool = True):
        self.device = torch.device(device)
        self.ppt = int(pixels_per_thread)
        self.longest_first = bool(longest_first)
        # the last backward's launch order and the view and grid it was made for: the next forward
        # of the same view takes it (see bin)
        self._bwd_order_for = None
        self.fwd_order_kernels = 0  # order kernels the last bin() launched (0 when it reused one)
        self.n = int(n)
        self.splats = torch.zeros(self.n, R.SPLAT_FLOATS, device=self.device)
        self.radii = torch.zeros(self.n, dtype=torch.int32, device=self.device)
        self.rects = torch.zeros(self.n, 4, dtype=torch.int32, device=self.device)
        self.tiles_touched = torch.zeros(self.n, dtype=torch.int32, device=self.device)
        self.depth_keys = torch.zeros(self.n, dtype=torch.int32, device=self.device)
        self.grad2d = torch.zeros(self.n, R.GRAD2D_FLOATS, device=self.device)
        self.num_pairs_dev = torch.zeros(1, dtype=torch.int64, device=self.device)
        self.capacity = 0
        self.max_tiles = 0
        self.grid = (1, 1) if max_grid is None else (int(max_grid[0]), int(max_grid[1]))
        self.ensure_tiles(max(max_tiles, self.grid[0] * self.grid[1]))
        self._alloc_pairs(int(capacity))

    def _alloc_pairs(self, capacity: int):
        capacity = max(1, int(capacity))
        self.sorted_ids = torch.empty(capacity, dtype=torch.int32, device=self.device)
        ws = R.gs_bin_sort_workspace_size(self.n, capacity, *self.grid)
        self.workspace = torch.empty(ws, dtype=torch.uint8, device=self.device)
        self.capacity = capacity

    def ensure_tiles(self, num_tiles: int):
        """Room for num_tiles binning tiles (ranges) and blend tiles (launch order)."""
        if num_tiles > self.max_tiles:
            self.max_tiles = int(num_tiles)
            self.ranges = torch.zeros(self.max_tiles, 2, dtype=torch.int32, device=self.device)
            self.tile_order = torch.zeros(self.max_tiles, dtype=torch.int32, device=self.device)
            self.bwd_order = torch.zeros(self.max_tiles, dtype=torch.int32, device=self.device)
            self._bwd_order_for = None  # the new buffers hold no order

    def ensure_grid(self, tiles_x: int, tiles_y: int):
        """Grow the workspace so that binning grids up to (tiles_x, tiles_y) fit."""
        self.ensure_tiles(tiles_x * tiles_y)
        need = R.gs_bin_sort_workspace_size(self.n, self.capacity, tiles_x, tiles_y)
        if tiles_x > self.grid[0] or tiles_y > self.grid[1] or need > self.workspace.numel():
            self.grid = (max(self.grid[0], tiles_x), max(self.grid[1], tiles_y))
            ws = R.gs_bin_sort_workspace_size(self.n, self.capacity, *self.grid)
            self.workspace = torch.empty(ws, dtype=torch.uint8, device=self.device)

    def ensure_capacity(self, k: int, headroom: float = 1.25):
        if k > self.capacity:
            self._alloc_pairs(int(math.ceil(k * headroom)) + 1024)

    def num_pairs(self) -> int:
        return int(self.num_pairs_dev.item())

    # -- stages ---------------------------------------------------------------
    def project(self, p: GaussianParams, cam, dil: Dilation):
        R.gs_project(p.means, p.log_scales, p.quats, p.opacity_logits, p.sh_store, cam, dil, self.splats,
                     self.radii, self.rects, self.tiles_touched, depth_keys=self.depth_keys)

    def bin(self, cam, dil: Dilation):
        w_ds, h_ds, tx, ty = R.gs_grid(cam, dil)
        btx, bty = R.gs_bin_grid(cam, dil)
        if btx > self.grid[0] or bty > self.grid[1]:
            self.ensure_grid(btx, bty)
        self.ensure_tiles(tx * ty)
        R.gs_bin_sort(self.n, self.rects, self.tiles_touched, self.splats, btx, bty, self.workspace, self.capacity,
                      self.sorted_ids, self.ranges, self.num_pairs_dev, depth_keys=self.depth_keys)
        if self.longest_first:
            if self._bwd_order_for is not None and self._bwd_order_for == _order_key(cam, dil, tx, ty):
                # The forward's launch order: the previous backward's order for the same camera and
                # tile grid (tiles by the list extent their pixels replayed, which is what the forward
                # walks; a neighbouring lattice offset changes it little). It only orders the launch:
                # results are those of any order. Measured on the 4K step, the last 15% of the
                # forward ran at under half occupancy with the list-length order.
                self.tile_order, self.bwd_order = self.bwd_order, self.tile_order
                self._bwd_order_for = None
                self.fwd_order_kernels = 0
            elif dil.bin_shift:
                R.gs_tile_order_batch([R.View(cam, dil, ranges=self.ranges)], self.tile_order)
                self.fwd_order_kernels = 1
            else:
                R.gs_tile_order(self.ranges, tx * ty, self.tile_order)
                self.fwd_order_kernels = 1
        return w_ds, h_ds, tx, ty

    def bin_checked(self, cam, dil: Dilation):
        """bin(), then read K (host sync) and redo it with grown buffers on overflow."""
        grid = self.bin(cam, dil)
        k = self.num_pairs()
        if k > self.capacity:
            self.ensure_capacity(k)
            grid = self.bin(cam, dil)
        return grid

    def render(self, cam, dil: Dilation, bg, img, t_final, last, counts=None):
        R.gs_render_fwd(self.n, self.splats, self.sorted_ids, self.ranges, cam, dil, bg, img, t_final, last, counts,
                        pixels_per_thread=self.ppt, tile_order=self.tile_order if self.longest_first else None)

    def render_l1(self, cam, dil: Dilation, bg, img, t_final, last, target, dl_dimg, loss, counts=None,
                  zero_grad2d: bool = True):
        """render() and the L1 loss (into loss and dl_dimg) in one launch, which also zeroes
        the 2D-gradient rows for a render_bwd(..., zero_grad2d=False) when asked."""
        R.gs_render_fwd_l1(self.n, self.splats, self.sorted_ids, self.ranges, cam, dil, bg, img, t_final, last,
                           target, dl_dimg, loss, grad2d_zero=self.grad2d if zero_grad2d else None, counts=counts,
                           pixels_per_thread=self.ppt, tile_order=self.tile_order if self.longest_first else None)

    def render_bwd(self, cam, dil: Dilation, bg, t_final, last, dl_dimg, zero_grad2d: bool = True):
        order = None
        if self.longest_first:
            # the backward's own launch order: tiles by the list positions they replay
            R.gs_tile_order_by_last_batch([R.View(cam, dil, ranges=self.ranges, last=last)], self.bwd_order)
            order = self.bwd_order
            w_ds, h_ds, tx, ty = R.gs_grid(cam, dil)
            self._bwd_order_for = _order_key(cam, dil, tx, ty)
        R.gs_render_bwd(self.n, self.splats, self.sorted_ids, self.ranges, cam, dil, bg, t_final, last, dl_dimg,
                        self.grad2d, zero_grad2d=zero_grad2d, pixels_per_thread=self.ppt, tile_order=order)


def _view_key(cam, dil: Dilation):
    """A camera and dilation (lattice offset included), compared byte for byte."""
    return (bytes(R.camera(cam)), bytes(dil.c()))


def _order_key(cam, dil: Dilation, tx: int, ty: int):
    """What a launch order depends on: the view's camera and the tile grid (not the lattice offset)."""
    c = R.camera(cam)
    return (bytes(c), int(dil.d), int(dil.tile), int(dil.bin_shift), int(dil.center_mode), int(tx), int(ty))


def image_buffers(h_ds: int, w_ds: int, device="cuda"):
    return (torch.empty(h_ds, w_ds, 3, device=device), torch.empty(h_ds, w_ds, device=device),
            torch.empty(h_ds, w_ds, dtype=torch.int32, device=device))


# ---------------------------------------------------------------------------
# autograd
# ---------------------------------------------------------------------------

class _RasterizeFn(torch.autograd.Function):
    """Differentiable dilated render of one view. Only (t_final, last) and the
    binned lists are kept for backward; the per-pixel blend state is replayed.
    The parameter tensors go through save_for_backward, so autograd rejects a
    backward after they were changed in place (e.g. by an optimizer step)."""

    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logits, sh, cam, dil, bg, cap_hint):
        n = means.shape[0]
        p = GaussianParams(means.contiguous(), log_scales.contiguous(), quats.contiguous(),
                           opacity_logits.contiguous(), sh.contiguous(), sh.contiguous())
        w_ds, h_ds, _, _ = R.gs_grid(cam, dil)
        rast = Rasterizer(n, capacity=cap_hint[0], device=means.device, max_grid=R.gs_bin_grid(cam, dil))
        rast.project(p, cam, dil)
        rast.bin_checked(cam, dil)
        cap_hint[0] = max(cap_hint[0], rast.capacity)
        img, t_final, last = image_buffers(h_ds, w_ds, means.device)
        rast.render(cam, dil, bg, img, t_final, last)
        ctx.rast, ctx.cam, ctx.dil, ctx.bg = rast, cam, dil, bg
        ctx.save_for_backward(means, log_scales, quats, opacity_logits, sh, t_final, last)
        ctx.mark_non_differentiable(t_final, last)
        return img, t_final, last

    @staticmethod
    def backward(ctx, dl_dimg, _g_t, _g_last):
        means, log_scales, quats, opacity_logits, sh, t_final, last = ctx.saved_tensors
        p = GaussianParams(means.contiguous(), log_scales.contiguous(), quats.contiguous(),
                           opacity_logits.contiguous(), sh.contiguous(), sh.contiguous())
        rast = ctx.rast
        rast.render_bwd(ctx.cam, ctx.dil, ctx.bg, t_final, last, dl_dimg.contiguous())
        g = [torch.empty_like(t) for t in (p.means, p.log_scales, p.quats, p.opacity_logits)]
        d_sh = torch.empty(p.sh.shape, dtype=torch.float32, device=p.sh.device)
        R.gs_project_bwd(p.means, p.log_scales, p.quats, p.opacity_logits, p.sh, ctx.cam, ctx.dil,
                         rast.tiles_touched, rast.grad2d, g[0], g[1], g[2], g[3], d_sh)
        ctx.rast = None
        return g[0], g[1], g[2], g[3], d_sh.to(p.sh.dtype), None, None, None, None


_CAP_HINT = [1 << 16]


def rasterize(means, log_scales, quats, opacity_logits, sh, cam, dil: Dilation = Dilation(), bg=(0.0, 0.0, 0.0)):
    """Render the dilated lattice of one view; differentiable in the five
    parameter tensors. Returns (img h_ds x w_ds x 3, t_final, last)."""
    return _RasterizeFn.apply(means, log_scales, quats, opacity_logits, sh, cam, dil, tuple(bg), _CAP_HINT)


# ---------------------------------------------------------------------------
# One full training step of the hot path
# ---------------------------------------------------------------------------

@dataclass
class AdamConfig:
    lr_means: float = 1.6e-4
    lr_log_scales: float = 5e-3
    lr_quats: float = 1e-3
    lr_opacity: float = 5e-2
    lr_sh: float = 2.5e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15


class TrainStep:
    """project -> bin/sort -> blend -> L1 -> blend bwd -> projection bwd with
    densification statistics -> fused Adam, all on the current stream with no
    host synchronisation (the pair capacity is fixed up front)."""

    def __init__(self, params: GaussianParams, rast: Rasterizer, adam: AdamConfig = AdamConfig(),
                 max_pixels: int = 1, bg=(0.0, 0.0, 0.0), densify: bool = True, fused: bool = True,
                 sparse: bool = False, sr_seed: int = 0x2412, dssim_lambda: float = 0.0):
        """dssim_lambda > 0 trains with (1 - lambda) L1 + lambda (1 - SSIM)
        (the 3DGS loss; the paper's is the plain L1, lambda = 0)."""
        dev = params.means.device
        self.p, self.rast, self.adam, self.bg = params, rast, adam, tuple(bg)
        self.fused, self.sparse = bool(fused), bool(sparse)
        self.sr_seed = int(sr_seed)  # stream of the stochastic rounding of low-precision SH
        self._projected_for = None  # the view the last optimizer pass projected the parameters into
        self.projected = True  # the last step ran its own projection
        self.dssim_lambda = float(dssim_lambda)
        self.ssim_ws = None
        self.grads = [torch.zeros_like(t, dtype=torch.float32) for t in params.tensors()]
        self.m = [torch.zeros_like(t, dtype=torch.float32) for t in params.tensors()]
        self.v = [torch.zeros_like(t, dtype=torch.float32) for t in params.tensors()]
        self.step_count = 0
        self.img = torch.empty(max_pixels * 3, device=dev)
        self.t_final = torch.empty(max_pixels, device=dev)
        self.last = torch.empty(max_pixels, dtype=torch.int32, device=dev)
        self.dl = torch.empty(max_pixels * 3, device=dev)
        self.loss = torch.zeros(1, device=dev)
        self.counts = torch.zeros(3, dtype=torch.int64, device=dev)
        n = params.n
        self.densify = densify
        self.pos_acc = torch.zeros(n, device=dev)
        self.col_acc = torch.zeros(n, device=dev)
        self.vis_count = torch.zeros(n, dtype=torch.int32, device=dev)

    def __call__(self, cam, dil: Dilation, target: torch.Tensor, counts: bool = False, next_view=None):
        """One training step on (cam, dil, target). next_view (optional): the (camera,
        dilation) of the next step; the optimizer pass then also projects the updated
        parameters into it, and the next step on that view skips its projection (the
        parameters cross HBM once per step). Anything that changes the parameters between
        the two steps must call forget_projection()."""
        p, rast = self.p, self.rast
        self.projected = self._projected_for is None or self._projected_for != self._proj_key(cam, dil)
        if self.projected:
            rast.project(p, cam, dil)
        self._projected_for = None
        w_ds, h_ds, tx, ty = rast.bin(cam, dil)
        P = w_ds * h_ds
        img = self.img[:3 * P].view(h_ds, w_ds, 3)
        t_final = self.t_final[:P].view(h_ds, w_ds)
        last = self.last[:P].view(h_ds, w_ds)
        dl = self.dl[:3 * P].view(h_ds, w_ds, 3)
        if self.dssim_lambda <= 0.0:
            # the blend, the L1 loss and the zeroing of the 2D-gradient rows in one launch
            rast.render_l1(cam, dil, self.bg, img, t_final, last, target, dl, self.loss,
                           self.counts if counts else None)
            rast.render_bwd(cam, dil, self.bg, t_final, last, dl, zero_grad2d=False)
        else:
            rast.render(cam, dil, self.bg, img, t_final, last, self.counts if counts else None)
            self.loss_and_grad(cam, dil, img, target, dl)
            rast.render_bwd(cam, dil, self.bg, t_final, last, dl)
        self.step_count += 1
        self.optimize(cam, dil, next_view)
        return self.loss

    def forget_projection(self):
        """The next step projects again (after the parameters changed outside the step)."""
        self._projected_for = None

    def _proj_key(self, cam, dil: Dilation):
        """What a projection the optimizer pass wrote stands for: the view, and the parameter
        and output tensors it was made from and into (a densification that reallocates them,
        or a resized rasterizer, makes the next step project again by itself; an in-place
        change of the parameters needs forget_projection())."""
        p, r = self.p, self.rast
        return _view_key(cam, dil) + (p.n, p.means.data_ptr(), p.sh_store.data_ptr(), r.splats.data_ptr(),
                                      r.depth_keys.data_ptr())

    def loss_and_grad(self, cam, dil: Dilation, img, target, dl):
        """The photometric loss into self.loss and dL/dimg into dl."""
        if self.dssim_lambda <= 0.0:
            R.gs_loss_l1(cam, dil, img, target, dl, self.loss)
            return
        need = R.gs_ssim_workspace_size(cam, dil)
        if self.ssim_ws is None or self.ssim_ws.numel() < need:
            self.ssim_ws = torch.empty(need, dtype=torch.uint8, device=img.device)
        R.gs_loss_l1_dssim(cam, dil, img, target, self.dssim_lambda, dl, self.loss, self.ssim_ws)

    def optimize(self, cam, dil: Dilation, next_view=None):
        """Projection backward + densification statistics + Adam. The fused
        path (default) is one kernel; the unfused path writes the parameter
        gradients to self.grads and runs gs_adam."""
        p, rast, a, g = self.p, self.rast, self.adam, self.grads
        lrs = [a.lr_means, a.lr_log_scales, a.lr_quats, a.lr_opacity, a.lr_sh]
        shadow = p.sh_store if p.sh_store.data_ptr() != p.sh.data_ptr() else None
        stats = (self.pos_acc, self.col_acc, self.vis_count) if self.densify else (None, None, None)
        if self.fused and next_view is not None and not self.sparse:
            ncam, ndil = next_view
            nv = R.View(ncam, ndil, splats=rast.splats, radii=rast.radii, rects=rast.rects,
                        tiles_touched=rast.tiles_touched, depth_keys=rast.depth_keys)
            R.gs_project_bwd_adam_next(p.tensors(), self.m, self.v, lrs, a.beta1, a.beta2, a.eps, self.step_count,
                                       p.sh_store, cam, dil, rast.tiles_touched, rast.grad2d, nv, sh_shadow=shadow,
                                       pos_acc=stats[0], col_acc=stats[1], count=stats[2], sr_seed=self.sr_seed)
            self._projected_for = self._proj_key(ncam, ndil)
            return
        if self.fused:
            R.gs_project_bwd_adam(p.tensors(), self.m, self.v, lrs, a.beta1, a.beta2, a.eps, self.step_count,
                                  p.sh_store, cam, dil, rast.tiles_touched, rast.grad2d, sparse=self.sparse,
                                  sh_shadow=shadow, pos_acc=stats[0], col_acc=stats[1], count=stats[2],
                                  sr_seed=self.sr_seed)
            return
        R.gs_project_bwd(p.means, p.log_scales, p.quats, p.opacity_logits, p.sh_store, cam, dil, rast.tiles_touched,
                         rast.grad2d, g[0], g[1], g[2], g[3], g[4], *stats)
        entries = []
        for i, t in enumerate(p.tensors()):
            e = dict(param=t, grad=g[i], m=self.m[i], v=self.v[i], lr=lrs[i], row_width=max(1, t[0].numel()),
                     sr_seed=self.sr_seed)
            if i == 4 and shadow is not None:
                e["shadow"] = shadow
            entries.append(e)
        mask = (rast.tiles_touched > 0).to(torch.uint8) if self.sparse else None
        R.gs_adam(entries, a.beta1, a.beta2, a.eps, self.step_count, row_mask=mask)

    def launches_per_step(self) -> int:
        """Kernels the last step launched (memsets not counted): projection (none
        when the previous optimizer pass projected into this step's view), the
        binning, the forward's tile order (none when it reused the previous
        backward's), the loss zeroing and the blend with the L1 loss fused into it
        (with D-SSIM: the blend, then the SSIM loss's three kernels), the
        backward's tile order (two kernels), blend backward, and the fused
        optimizer (or projection backward + Adam)."""
        orders = (self.rast.fwd_order_kernels + 2) if self.rast.longest_first else 0
        fwd_loss = 2 if self.dssim_lambda <= 0.0 else 1 + 3
        return int(self.projected) + BIN_SORT_KERNELS + orders + fwd_loss + 1 + (1 if self.fused else 2)


# kernels in one gs_bin_sort call given the projection's depth keys: a 4-pass radix sort
# of the depths (3 kernels a pass), 5 for the row level (the row histogram also sums the
# pair count), 6 for the tile level
BIN_SORT_KERNELS = 4 * 3 + 5 + 6


# ---------------------------------------------------------------------------
# Several views per optimizer step
# ---------------------------------------------------------------------------

class BatchTrainStep:
    """One optimizer step over a batch of views of uneven resolution: batched
    projection, binning per view, ONE blend launch over the tiles of every
    view (a work queue ordered longest list first), batched L1, ONE backward
    blend launch, and ONE fused projection backward + densification statistics
    + Adam launch whose gradient is the sum over the views.

    Dilation (Sec. 3.1): with d > 1 each step renders one lattice offset per
    view; view i at phase k takes the rotating offset of k + i, so the views
    of one step cover different lattices and d*d phases cover all of them.
    The Adam step count lives on the device, so ``capture()`` can record the
    step of every phase into a CUDA graph that ``step()`` then replays; the
    only host synchronisation is in ``overflowed()``."""

    def __init__(self, params: GaussianParams, cams, targets, d: int = 1, adam: AdamConfig = AdamConfig(),
                 bg=(0.0, 0.0, 0.0), densify: bool = True, sparse: bool = False, tile: int = 16,
                 pixels_per_thread: int = 0, center_mode: int = 0, longest_first: bool = True,
                 capacity=None, headroom: float = 1.15, optimize: bool = True, bin_shift: int = 0,
                 state=None, bwd_pixels_per_thread: int = 0, sr_seed: int = 0x2412, dssim_lambda: float = 0.0):
        """cams/targets: the views of the batch (any later batch given to
        run(table=views_table(...)) must have no larger images). state: optional
        dict of m, v (lists), pos_acc, col_acc, count and step_dev to continue
        from instead of fresh moments and statistics."""
        if not 1 <= len(cams) <= R.MAX_VIEWS:
            raise ValueError(f"1..{R.MAX_VIEWS} views per batch")
        dev = params.means.device
        self.p, self.adam, self.bg, self.d = params, adam, tuple(bg), int(d)
        self.cams, self.V = list(cams), len(cams)
        self.sparse, self.densify, self.optimize_step = bool(sparse), bool(densify), bool(optimize)
        self.tile, self.ppt, self.center_mode = int(tile), int(pixels_per_thread), int(center_mode)
        self.bwd_ppt = int(bwd_pixels_per_thread)  # 0: the library's default for the backward
        self.bin_shift = int(bin_shift)
        self.longest_first = bool(longest_first)
        self.sr_seed = int(sr_seed)  # stream of the stochastic rounding of low-precision SH
        self.dssim_lambda = float(dssim_lambda)  # > 0: (1 - lambda) L1 + lambda (1 - SSIM) per view
        n, V = params.n, self.V
        self.targets = [t.contiguous() for t in targets]
        for c, t in zip(self.cams, self.targets):
            if tuple(t.shape) != (c.height, c.width, 3) or t.dtype not in (torch.float32, torch.uint8):
                raise ValueError("each target must be an FP32 or 8-bit height x width x 3 tensor on the device")
        self.splats = torch.zeros(V, n, R.SPLAT_FLOATS, device=dev)
        self.radii = torch.zeros(V, n, dtype=torch.int32, device=dev)
        self.rects = torch.zeros(V, n, 4, dtype=torch.int32, device=dev)
        self.tiles_touched = torch.zeros(V, n, dtype=torch.int32, device=dev)
        # rows padded to 16 bytes (the binning reads the keys with 16-byte vectors when aligned)
        self.depth_keys = torch.zeros(V, (n + 3) // 4 * 4, dtype=torch.int32, device=dev)[:, :n]
        self.grad2d = torch.zeros(V, n, R.GRAD2D_FLOATS, device=dev)
        self.loss = torch.zeros(V, device=dev)
        self.num_pairs = torch.zeros(V, dtype=torch.int64, device=dev)
        self.num_pairs_max = torch.zeros(V, dtype=torch.int64, device=dev)  # high-water marks since the last check
        self.counts = torch.zeros(3, dtype=torch.int64, device=dev)
        # the largest grid of each view over the offsets (offset 0 renders the most pixels)
        self.grid0 = [R.gs_grid(c, self._dil(0, 0)) for c in self.cams]
        self.bgrid0 = [R.gs_bin_grid(c, self._dil(0, 0)) for c in self.cams]
        self.ranges = [torch.zeros(g[0] * g[1], 2, dtype=torch.int32, device=dev) for g in self.bgrid0]
        self.img = [torch.empty(g[1], g[0], 3, device=dev) for g in self.grid0]
        self.t_final = [torch.empty(g[1], g[0], device=dev) for g in self.grid0]
        self.last = [torch.empty(g[1], g[0], dtype=torch.int32, device=dev) for g in self.grid0]
        self.dl = [torch.empty(g[1], g[0], 3, device=dev) for g in self.grid0]
        self.order = torch.zeros(sum(g[2] * g[3] for g in self.grid0), dtype=torch.int32, device=dev)
        self.bwd_order = torch.zeros_like(self.order)
        # The forward launches in the previous backward's order when every view keeps its tile grid
        # over the offset phases (the global tile layout is then the same in every phase) and that
        # backward ran on this step's own views; otherwise in the list-length order.
        self.reuse_order = all(len({R.gs_grid(c, self._dil(ph, i))[2:] for ph in range(self.phases)}) == 1
                               for i, c in enumerate(self.cams))
        self._bwd_order_ok = False
        # moments, device-side Adam step and densification statistics
        st = state or {}
        self.m = st.get("m") or [torch.zeros_like(t, dtype=torch.float32) for t in params.tensors()]
        self.v = st.get("v") or [torch.zeros_like(t, dtype=torch.float32) for t in params.tensors()]
        self.step_dev = st.get("step_dev", torch.zeros(1, dtype=torch.int32, device=dev))
        self.bias_dev = torch.zeros(2, device=dev)
        self.pos_acc = st.get("pos_acc", torch.zeros(n, device=dev))
        self.col_acc = st.get("col_acc", torch.zeros(n, device=dev))
        self.vis_count = st.get("count", torch.zeros(n, dtype=torch.int32, device=dev))
        self.phase = 0
        self._tables = {}
        self.graphs = {}
        self.capacity = self._capacities(headroom) if capacity is None else \
            [int(c) for c in (capacity if hasattr(capacity, "__len__") else [capacity] * V)]
        self.sorted_ids = [torch.empty(max(1, c), dtype=torch.int32, device=dev) for c in self.capacity]
        # the views bin concurrently, each on its own stream with its own workspace: one view's
        # binning is a chain of small kernels that leaves most of the GPU idle
        self.workspaces = [torch.empty(R.gs_bin_sort_workspace_size(n, c, g[0], g[1]), dtype=torch.uint8, device=dev)
                           for c, g in zip(self.capacity, self.bgrid0)]
        self.bin_streams = [torch.cuda.Stream(device=dev) for _ in range(V)]
        self.ssim_ws = None
        if self.dssim_lambda > 0.0:
            need = max(R.gs_ssim_workspace_size(c, self._dil(0, 0)) for c in self.cams)
            self.ssim_ws = torch.empty(need, dtype=torch.uint8, device=dev)

    @property
    def phases(self) -> int:
        return self.d * self.d

    def _dil(self, phase: int, view: int) -> Dilation:
        from .scenes import rotating_offset
        ox, oy = rotating_offset(phase + view, self.d)
        return Dilation(self.d, ox, oy, self.center_mode, self.tile, self.bin_shift)

    def _capacities(self, headroom: float):
        """Pairs per view = sum of tiles touched (exact); the maximum over the
        phases, with headroom for the parameters moving during the fit."""
        best = [0] * self.V
        for ph in range(self.phases):
            self._project(self.table(ph, project_only=True))
            k = self.tiles_touched.to(torch.int64).sum(1).tolist()
            best = [max(a, b) for a, b in zip(best, k)]
        return [int(math.ceil(k * headroom)) + 1024 for k in best]

    def views_table(self, cams, targets, phase: int = 0) -> R.ViewTable:
        """A table for other views of the same count and no larger images
        (e.g. a fresh draw of training cameras), not cached."""
        if len(cams) != self.V or len(targets) != self.V:
            raise ValueError(f"{self.V} views per batch")
        return self.table(phase, cams=list(cams), targets=[t.contiguous() for t in targets])

    def table(self, phase: int, project_only: bool = False, cams=None, targets=None) -> R.ViewTable:
        key = (phase % self.phases, project_only)
        if cams is not None or key not in self._tables:
            cams = self.cams if cams is None else cams
            targets = self.targets if targets is None else targets
            views = []
            for i, c in enumerate(cams):
                dil = self._dil(key[0], i)
                w_ds, h_ds, tx, ty = R.gs_grid(c, dil)
                v = R.View(c, dil, splats=self.splats[i], radii=self.radii[i], rects=self.rects[i],
                           tiles_touched=self.tiles_touched[i], grad2d=self.grad2d[i],
                           depth_keys=self.depth_keys[i])
                if not project_only:
                    P = w_ds * h_ds
                    v.sorted_ids, v.ranges = self.sorted_ids[i], self.ranges[i]
                    v.img = self.img[i].view(-1)[:3 * P]
                    v.t_final = self.t_final[i].view(-1)[:P]
                    v.last = self.last[i].view(-1)[:P]
                    v.dl_dimg = self.dl[i].view(-1)[:3 * P]
                    v.target, v.loss = targets[i], self.loss[i:i + 1]
                views.append(v)
            t = R.ViewTable(views)
            if cams is not self.cams:
                return t
            self._tables[key] = t
        return self._tables[key]

    def _project(self, t: R.ViewTable):
        p = self.p
        R.gs_project_batch(p.means, p.log_scales, p.quats, p.opacity_logits, p.sh_store, t)

    # -- the step ---------------------------------------------------------------
    def bin_views(self, t: R.ViewTable):
        """Bins every view of the table, each on its own stream forked from and
        joined back into the current one (also inside a graph capture)."""
        main = torch.cuda.current_stream()
        for i, v in enumerate(t.views):
            tx, ty = R.gs_bin_grid(v.cam, v.dil)
            s = self.bin_streams[i]
            s.wait_stream(main)
            with torch.cuda.stream(s):
                R.gs_bin_sort(self.p.n, self.rects[i], self.tiles_touched[i], self.splats[i], tx, ty,
                              self.workspaces[i], self.capacity[i], self.sorted_ids[i], self.ranges[i],
                              self.num_pairs[i:i + 1], depth_keys=self.depth_keys[i],
                              num_pairs_max=self.num_pairs_max[i:i + 1])
        for s in self.bin_streams[:len(t.views)]:
            main.wait_stream(s)

    def render_pass(self, phase: int, counts: bool = False, table=None):
        """Everything up to the 2D gradients of every view (no parameter update)."""
        own = table is None or table is self._tables.get((phase % self.phases, False))
        t = self.table(phase) if table is None else table
        self._project(t)
        self.bin_views(t)
        order = None
        if self.longest_first:
            if own and self.reuse_order and self._bwd_order_ok:
                order = self.bwd_order  # the previous backward's (tiles by the list extent they replayed)
            else:
                R.gs_tile_order_batch(t, self.order)
                order = self.order
        # with the L1 loss, the loss and the zeroing of every view's 2D-gradient rows run in the blend launch
        l1 = self.dssim_lambda <= 0.0
        R.gs_render_fwd_batch(self.p.n, t, self.bg, tile_order=order, counts=self.counts if counts else None,
                              pixels_per_thread=self.ppt, flags=(R.FWD_L1 | R.FWD_ZERO_GRAD2D) if l1 else 0)
        if not l1:
            # the views share one workspace: their loss calls run in order on this stream
            for v in t.views:
                R.gs_loss_l1_dssim(v.cam, v.dil, v.img, v.target, self.dssim_lambda, v.dl_dimg, v.loss, self.ssim_ws)
        if self.longest_first:
            R.gs_tile_order_by_last_batch(t, self.bwd_order)
            order = self.bwd_order
            self._bwd_order_ok = own and self.reuse_order
        R.gs_render_bwd_batch(self.p.n, t, self.bg, tile_order=order, zero_grad2d=not l1,
                              pixels_per_thread=self.bwd_ppt)

    def optimize(self, phase: int, table=None):
        p, a = self.p, self.adam
        lrs = [a.lr_means, a.lr_log_scales, a.lr_quats, a.lr_opacity, a.lr_sh]
        shadow = p.sh_store if p.sh_store.data_ptr() != p.sh.data_ptr() else None
        stats = (self.pos_acc, self.col_acc, self.vis_count) if self.densify else (None, None, None)
        R.gs_adam_advance(self.step_dev, a.beta1, a.beta2, self.bias_dev)
        R.gs_project_bwd_adam_batch(p.tensors(), self.m, self.v, lrs, a.beta1, a.beta2, a.eps, 1, p.sh_store,
                                    self.table(phase) if table is None else table, sparse=self.sparse,
                                    sh_shadow=shadow, pos_acc=stats[0],
                                    col_acc=stats[1], count=stats[2], bias_dev=self.bias_dev,
                                    step_dev=self.step_dev, sr_seed=self.sr_seed)

    def run(self, phase: int, counts: bool = False, table=None):
        self.render_pass(phase, counts, table)
        if self.optimize_step:
            self.optimize(phase, table)

    def capture(self):
        """Record the step of every phase into a CUDA graph (each phase is run
        eagerly once first; that run is a real step)."""
        for ph in range(self.phases):
            self.run(ph)
        torch.cuda.synchronize()
        for ph in range(self.phases):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                self.run(ph)
            self.graphs[ph] = g
        torch.cuda.synchronize()

    def step(self, counts: bool = False):
        ph = self.phase % self.phases
        if ph in self.graphs and not counts:
            self.graphs[ph].replay()
        else:
            self.run(ph, counts)
        self.phase += 1
        return self.loss

    def overflowed(self) -> bool:
        """True when a view had more pairs than its capacity in any step since
        the last call (its lists were then left empty): a high-water mark the
        binning keeps on the device, read and reset here. Host synchronisation."""
        k = self.num_pairs_max.tolist()
        self.num_pairs_max.zero_()
        return any(ki > ci for ki, ci in zip(k, self.capacity))

    def launches_per_step(self) -> int:
        """Kernels one step launches (memsets not counted): projection, the
        binning of every view, the tile orders (the forward's, none when it
        reuses the previous backward's, and the backward's from `last`: two
        kernels), both blend launches, the loss zeroing (the L1 loss runs in
        the forward launch; D-SSIM adds three kernels a view), and the Adam
        step advance + the fused optimizer."""
        orders = (2 + (0 if self.reuse_order else 1)) if self.longest_first else 0
        fwd_loss = 2 if self.dssim_lambda <= 0.0 else 1 + 3 * self.V
        return 1 + BIN_SORT_KERNELS * self.V + orders + fwd_loss + 1 + \
            (2 if self.optimize_step else 0)


def autotune_batch(params: GaussianParams, cams, targets, d: int = 1,
                   candidates=((8, 2, 1), (16, 2, 0), (16, 4, 0), (16, 2, 1), (16, 4, 1), (16, 2, 2), (16, 4, 2),
                               (32, 4, 0), (32, 4, 1)),
                   iters: int = 3, **kw):
    """Pick the launch shape of a batch: blend tile size, pixels per thread of
    the forward blend CTAs (the backward takes the library's default for the
    tile) and binning tile shift. Times ``render_pass`` (projection,
    binning, both blend launches and the loss: everything the shape affects)
    of every candidate (tile, ppt[, bin_shift]) with CUDA events and returns
    ((tile, ppt, bin_shift), {candidate: ms})."""
    times = {}
    for cand in candidates:
        tile, ppt, shift = (tuple(cand) + (0,))[:3]
        st = BatchTrainStep(params, cams, targets, d=d, tile=tile, pixels_per_thread=ppt, bin_shift=shift,
                            optimize=False, **kw)
        for ph in range(st.phases):
            st.render_pass(ph)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(iters * st.phases):
            st.render_pass(i % st.phases)
        e1.record()
        torch.cuda.synchronize()
        times[(tile, ppt, shift)] = e0.elapsed_time(e1) / (iters * st.phases)
        del st
        torch.cuda.empty_cache()
    best = min(times, key=times.get)
    return best, times
