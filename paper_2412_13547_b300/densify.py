"""Densification and pruning under the Gaussian budget (Sec. 3.2, Sec. 3.3),
driven from the host once per densification interval.

One round: the position-appearance selection (gs_densify_select) under the
budget B(t) of Eq. 7 (``budget.AdaptiveBudget``), the baseline clone/split of
the selected Gaussians (gs_densify_grow), and the opacity prune with
order-preserving compaction (gs_prune_select + gs_gather_rows). Parameters,
optimizer moments and the densification statistics move together; new and
split Gaussians start with zero moments; the statistics restart from zero.
Two host reads per round (the selected and the kept counts) size the arrays.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from . import raster as R

TAU_COLOR_RATIO = 0.01   # Sec. 3.3: tau_color = 0.01 tau_position
COLOR_BRANCH_PROB = 0.2  # Sec. 3.3: the appearance branch is active with probability 20%


@dataclass
class DensifyConfig:
    """tau_pos: threshold of the mean positional-gradient norm (hr pixel units
    of dL/dp, as gs_densify_stats accumulates it); split_scale: world size above
    which a selected Gaussian is split rather than cloned; min_opacity: prune
    threshold; max_scale: optional prune of Gaussians larger than this."""
    tau_pos: float
    split_scale: float
    min_opacity: float = 0.005
    max_scale: float | None = None
    color_prob: float = COLOR_BRANCH_PROB


@dataclass
class GaussianState:
    """Parameters with their Adam moments and densification statistics."""
    params: "object"  # pipeline.GaussianParams
    m: list
    v: list
    pos_acc: torch.Tensor
    col_acc: torch.Tensor
    count: torch.Tensor

    @property
    def n(self) -> int:
        return self.params.n


def _like_rows(t: torch.Tensor, rows: int) -> torch.Tensor:
    return torch.empty((rows,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)


def _entries(st: GaussianState, rows: int, grow: bool):
    """(src, dst, role) for every row tensor of the state, dst of ``rows`` rows."""
    from .pipeline import GaussianParams
    p = st.params
    roles = [R.GS_ROW_MEANS, R.GS_ROW_LOG_SCALES, R.GS_ROW_QUATS, R.GS_ROW_COPY, R.GS_ROW_COPY] if grow else \
        [R.GS_ROW_COPY] * 5
    dst_p = [_like_rows(t, rows) for t in p.tensors()]
    entries = [(s, d, r) for s, d, r in zip(p.tensors(), dst_p, roles)]
    shadow = None
    if p.sh_store.data_ptr() != p.sh.data_ptr():
        shadow = _like_rows(p.sh_store, rows)
        entries.append((p.sh_store, shadow, R.GS_ROW_COPY))
    state_role = R.GS_ROW_STATE if grow else R.GS_ROW_COPY
    dm = [_like_rows(t, rows) for t in st.m]
    dv = [_like_rows(t, rows) for t in st.v]
    entries += [(s, d, state_role) for s, d in zip(st.m, dm)] + [(s, d, state_role) for s, d in zip(st.v, dv)]
    stats = [_like_rows(t, rows) for t in (st.pos_acc, st.col_acc, st.count)]
    entries += [(None, d, R.GS_ROW_ZERO) for d in stats]
    new_p = GaussianParams(*dst_p, sh_store=shadow if shadow is not None else dst_p[4])
    return entries, GaussianState(new_p, dm, dv, *stats)


def densify_and_prune(st: GaussianState, budget_total: int, cfg: DensifyConfig, rng: np.random.Generator):
    """One densification round. Returns (new state, info dict)."""
    dev = st.params.means.device
    n = st.n
    max_new = max(0, int(budget_total) - n)
    branch = bool(rng.random() < cfg.color_prob)
    info = dict(n_before=n, max_new=max_new, color_branch=branch)
    ws = torch.empty(R.gs_densify_workspace_size(n), dtype=torch.uint8, device=dev)
    sel = torch.empty(max(1, min(n, max_new)), dtype=torch.int32, device=dev)
    nsel = torch.zeros(1, dtype=torch.int32, device=dev)
    tau_c = float(np.float32(cfg.tau_pos) * np.float32(TAU_COLOR_RATIO))
    R.gs_densify_select(n, st.pos_acc, st.col_acc, st.count, cfg.tau_pos, tau_c, branch, max_new, ws, sel, nsel)
    m = int(nsel.item())
    noise = torch.tensor(rng.standard_normal((max(1, m), 2, 3)), dtype=torch.float32, device=dev)
    entries, grown = _entries(st, n + m, grow=True)
    R.gs_densify_grow(n, m, sel, noise, math.log(cfg.split_scale), entries)
    n1 = n + m
    ws1 = torch.empty(R.gs_densify_workspace_size(n1), dtype=torch.uint8, device=dev)
    keep = torch.empty(max(1, n1), dtype=torch.int32, device=dev)
    nkeep = torch.zeros(1, dtype=torch.int32, device=dev)
    o = min(max(cfg.min_opacity, 1e-7), 1.0 - 1e-7)
    logit_min = math.log(o / (1.0 - o))
    log_max = math.log(cfg.max_scale) if cfg.max_scale else 0.0
    R.gs_prune_select(n1, grown.params.opacity_logits, logit_min,
                      grown.params.log_scales if cfg.max_scale else None, log_max, ws1, keep, nkeep)
    k = int(nkeep.item())
    entries2, pruned = _entries(grown, k, grow=False)
    if k > 0:
        R.gs_gather_rows(k, keep, entries2)
    info.update(selected=m, n_grown=n1, n_after=k, pruned=n1 - k)
    return pruned, info
