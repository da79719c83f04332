"""End-to-end fit of a Gaussian scene to posed target images with the hot
path: training steps (one view, or a batch of views, per optimizer step),
densification under the Gaussian budget (Sec. 3.2 Eq. 7 with Algorithm 1,
Sec. 3.3) and held-out PSNR, timed with CUDA events.

Two forms are compared on the same scene, cameras and budget:

* ``plain``: the full-resolution FP32 form, one view per step (d = 1);
* ``turbo``: dilated rendering (d = 2, Sec. 3.1, a rotating lattice offset per
  view), SH stored in BF16, several views per optimizer step.

The schedule is counted in views (images rendered and back-propagated), so
both forms densify after the same amount of data. Every stage runs in the
library's kernels; the host only draws cameras, reads two counts per
densification round and the held-out PSNR.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

from . import raster as R
from .budget import AdaptiveBudget
from .densify import DensifyConfig, GaussianState, densify_and_prune
from .pipeline import AdamConfig, BatchTrainStep, GaussianParams, Rasterizer, image_buffers


@dataclass
class FitConfig:
    form: str = "turbo"            # "plain" or "turbo"
    views: int = 20000             # views rendered and back-propagated in total
    views_per_step: int = 8        # turbo: views per optimizer step (plain: 1)
    d: int = 2                     # turbo dilation (plain: 1)
    sh_dtype: torch.dtype = torch.bfloat16  # turbo SH storage (plain: FP32)
    budget: int = 3_000_000        # M of Eq. 7
    densify_from: int = 2400       # views (the 300-step warm-up of Sec. 4.1 at 8 views per step)
    densify_until: int = 24000     # views
    densify_every: int = 800       # views
    densify: DensifyConfig = field(default_factory=lambda: DensifyConfig(tau_pos=1e-7, split_scale=0.03))
    adam: AdamConfig = field(default_factory=lambda: AdamConfig(lr_means=5e-4))
    eval_every: int = 4000         # views
    tile: int = 16
    bin_shift: int = 2
    seed: int = 0

    def resolved(self) -> "FitConfig":
        if self.form == "plain":
            return FitConfig(**{**self.__dict__, "views_per_step": 1, "d": 1, "sh_dtype": torch.float32})
        return self


def render_views(params: GaussianParams, cams, bg=(0.0, 0.0, 0.0), tile=16, bin_shift=2):
    """Full-resolution (d = 1) forward renders of the cameras: a list of
    height x width x 3 FP32 device images."""
    dil = R.Dilation(1, 0, 0, tile=tile, bin_shift=bin_shift)
    grid = max((R.gs_bin_grid(c, dil) for c in cams), key=lambda g: g[0] * g[1])
    rast = Rasterizer(params.n, capacity=1 << 20, device=params.means.device, max_grid=grid)
    out = []
    for c in cams:
        rast.project(params, c, dil)
        w, h, _, _ = rast.bin_checked(c, dil)
        img, t_final, last = image_buffers(h, w, params.means.device)
        rast.render(c, dil, bg, img, t_final, last)
        out.append(img)
    return out


def psnr(params: GaussianParams, cams, targets, **kw) -> float:
    """Mean PSNR (dB, peak 1) of the full-resolution renders against the targets."""
    vals = []
    for img, tgt in zip(render_views(params, cams, **kw), targets):
        mse = torch.mean((img.clamp(0.0, 1.0) - tgt) ** 2).item()
        vals.append(10.0 * math.log10(1.0 / max(mse, 1e-20)))
    return float(np.mean(vals))


def pair_capacity(params: GaussianParams, cams, dil_of, headroom=1.3):
    """Largest pair count K over the cameras (and the offsets dil_of yields)."""
    n = params.n
    dev = params.means.device
    splats = torch.empty(n, R.SPLAT_FLOATS, device=dev)
    radii = torch.empty(n, dtype=torch.int32, device=dev)
    rects = torch.empty(n, 4, dtype=torch.int32, device=dev)
    tiles = torch.empty(n, dtype=torch.int32, device=dev)
    kmax = 0
    for c in cams:
        for dil in dil_of(c):
            R.gs_project(params.means, params.log_scales, params.quats, params.opacity_logits, params.sh_store, c,
                         dil, splats, radii, rects, tiles)
            kmax = max(kmax, int(tiles.to(torch.int64).sum().item()))
    return int(kmax * headroom) + 4096


class Fit:
    """One fit run. ``run()`` returns the history of (views, seconds, PSNR,
    Gaussians) at every evaluation; seconds count the GPU time of the steps and
    the densification rounds only (CUDA events), not the evaluations."""

    def __init__(self, cfg: FitConfig, init: dict, train_cams, train_targets, eval_cams, eval_targets,
                 device="cuda"):
        self.cfg = cfg.resolved()
        self.dev = torch.device(device)
        self.rng = np.random.default_rng(cfg.seed)
        self.train_cams, self.train_targets = list(train_cams), list(train_targets)
        self.eval_cams, self.eval_targets = list(eval_cams), list(eval_targets)
        p = GaussianParams.from_arrays(init, self.dev, self.cfg.sh_dtype)
        self.state = GaussianState(p, [torch.zeros_like(t, dtype=torch.float32) for t in p.tensors()],
                                   [torch.zeros_like(t, dtype=torch.float32) for t in p.tensors()],
                                   torch.zeros(p.n, device=self.dev), torch.zeros(p.n, device=self.dev),
                                   torch.zeros(p.n, dtype=torch.int32, device=self.dev))
        self.step_dev = torch.zeros(1, dtype=torch.int32, device=self.dev)
        self.budget = AdaptiveBudget(p.n, self.cfg.budget, self.cfg.densify_from, self.cfg.densify_until,
                                     warmup=0)
        self.step = None
        self.history = []
        self.rounds = []
        self.headroom = 1.3
        self.overflow_steps = 0  # steps in which a view overflowed its pair buffers

    def _dils(self, cam):
        c = self.cfg
        return [R.Dilation(c.d, ox, oy, tile=c.tile, bin_shift=c.bin_shift) for ox in range(c.d) for oy in range(c.d)]

    def _build(self, capacity=None):
        """(Re)build the step for the current Gaussians (after every
        densification). capacity: pairs per view, or None to measure it over
        a sample of the training cameras."""
        c, st = self.cfg, self.state
        V = c.views_per_step
        cap = capacity or pair_capacity(st.params, self.train_cams[:: max(1, len(self.train_cams) // 24)],
                                        self._dils, headroom=self.headroom)
        shape_cams = self.train_cams[:V]
        self.step = BatchTrainStep(st.params, shape_cams, self.train_targets[:V], d=c.d, adam=c.adam, tile=c.tile,
                                   bin_shift=c.bin_shift, capacity=cap,
                                   state=dict(m=st.m, v=st.v, pos_acc=st.pos_acc, col_acc=st.col_acc,
                                              count=st.count, step_dev=self.step_dev))

    def run(self):
        c = self.cfg
        V = c.views_per_step
        self._build()
        seconds, views, k = 0.0, 0, 0
        next_densify = c.densify_from
        next_eval = 0
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        while views < c.views:
            if views >= next_eval:
                torch.cuda.synchronize()
                self.history.append(dict(views=views, seconds=seconds, psnr=psnr(self.state.params, self.eval_cams,
                                                                                self.eval_targets),
                                         n=self.state.n))
                next_eval += c.eval_every
            ev0.record()
            if c.densify_from <= views <= c.densify_until and views >= next_densify:
                total = self.budget(views)
                n_old = self.state.n
                k_seen = int(self.step.num_pairs.max().item())
                self.state, info = densify_and_prune(self.state, total, c.densify, self.rng)
                b = self.budget
                self.rounds.append(dict(views=views, budget=total, alpha=b.alpha, alpha_base=b.alpha_base,
                                        rate=b.rate, m_adaptive=b.m_adaptive, **info))
                # pairs grow about like the Gaussians; an overflow below re-measures them
                cap = int(max(k_seen, 1) * max(1.0, self.state.n / max(1, n_old)) * self.headroom) + 4096
                self._build(max(cap, self.step.capacity[0]))
                next_densify += c.densify_every
            idx = self.rng.choice(len(self.train_cams), V, replace=False)
            t = self.step.views_table([self.train_cams[i] for i in idx], [self.train_targets[i] for i in idx],
                                      phase=k)
            self.step.run(k, table=t)
            ev1.record()
            ev1.synchronize()
            seconds += ev0.elapsed_time(ev1) / 1000.0
            loss = float(self.step.loss.sum().item()) / V
            if self.step.overflowed():
                # a view had more pairs than its buffers hold: its lists were left empty, so it
                # added no gradient to this update (the step itself counts, time and views). The
                # pairs are measured again with more headroom for the following steps.
                self.overflow_steps += 1
                self.headroom *= 1.5
                self._build()
            self.budget.record(views, loss)
            views += V
            k += 1
        torch.cuda.synchronize()
        self.history.append(dict(views=views, seconds=seconds, psnr=psnr(self.state.params, self.eval_cams,
                                                                        self.eval_targets), n=self.state.n))
        return self.history


def loglog_fit(steps, ema, skip_frac: float = 0.1):
    """Fig. 3's check on a fit's smoothed loss: least-squares line of
    log(EMA loss) against log(step) after the first skip_frac of the steps
    (the initial stage). Returns (slope, intercept, R^2)."""
    x = np.log(np.asarray(steps, np.float64))
    y = np.log(np.maximum(np.asarray(ema, np.float64), 1e-30))
    k = int(len(x) * skip_frac)
    x, y = x[k:], y[k:]
    if len(x) < 3:
        return 0.0, 0.0, 0.0
    A = np.c_[x, np.ones_like(x)]
    coef, *_ = np.linalg.lstsq(A, y, rcond=None)
    res = y - A @ coef
    r2 = 1.0 - float(res @ res) / max(float(((y - y.mean()) ** 2).sum()), 1e-300)
    return float(coef[0]), float(coef[1]), r2


def time_to_psnr(history, target_db: float):
    """GPU seconds at which the history first reaches target_db (linear in
    between evaluations), or None."""
    prev = None
    for h in history:
        if h["psnr"] >= target_db:
            if prev is None or h["psnr"] == prev["psnr"]:
                return h["seconds"]
            f = (target_db - prev["psnr"]) / (h["psnr"] - prev["psnr"])
            return prev["seconds"] + f * (h["seconds"] - prev["seconds"])
        prev = h
    return None
