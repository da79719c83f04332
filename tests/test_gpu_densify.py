"""Densification and pruning kernels against the oracle (Sec. 3.2, 3.3).

Selection and prune lists are integer results taken from FP32 decisions on
both sides: compared exactly. Copied rows are compared bit for bit; split
positions (FP32 on the device, FP64 in the oracle) within 1e-6 relative.
"""
import math

import numpy as np
import pytest
import torch

from oracle import densify as od
from paper_2412_13547_b300 import raster as R
from paper_2412_13547_b300 import scenes
from paper_2412_13547_b300.densify import DensifyConfig, GaussianState, densify_and_prune, TAU_COLOR_RATIO
from paper_2412_13547_b300.pipeline import GaussianParams

pytestmark = pytest.mark.gpu
DEV = "cuda"


def stats(n, seed, quantise=False):
    rng = np.random.default_rng(seed)
    count = rng.integers(0, 6, n).astype(np.int32)
    pos = (rng.exponential(1.0, n) * count * 2e-4).astype(np.float32)
    col = (rng.exponential(1.0, n) * count * 2e-6).astype(np.float32)
    if quantise:  # many exact ties of the score
        pos = (np.round(pos / 1e-4) * 1e-4).astype(np.float32)
        col = (np.round(col / 1e-6) * 1e-6).astype(np.float32)
    return pos, col, count


def gpu_select(pos, col, count, tau, branch, max_new):
    n = len(pos)
    t = [torch.tensor(x, device=DEV) for x in (pos, col, count)]
    ws = torch.empty(R.gs_densify_workspace_size(n), dtype=torch.uint8, device=DEV)
    sel = torch.full((max(1, min(n, max_new)),), -1, dtype=torch.int32, device=DEV)
    nsel = torch.full((1,), -1, dtype=torch.int32, device=DEV)
    tau_c = float(np.float32(tau) * np.float32(TAU_COLOR_RATIO))
    R.gs_densify_select(n, *t, tau, tau_c, branch, max_new, ws, sel, nsel)
    torch.cuda.synchronize()
    m = int(nsel.item())
    return sel[:m].cpu().numpy().astype(np.int64), tau_c


@pytest.mark.parametrize("quantise", [False, True])
@pytest.mark.parametrize("branch", [False, True])
def test_select_matches_oracle(branch, quantise):
    n = 200_003
    pos, col, count = stats(n, 1 + int(quantise), quantise)
    tau = 3e-4
    cand, _ = od.densify_scores(pos, col, count, tau, np.float32(tau) * np.float32(0.01), branch)
    nc = int(cand.sum())
    assert 1000 < nc < n
    for max_new in (0, 1, 7, nc // 3, nc - 1, nc, nc + 5, n):
        got, tau_c = gpu_select(pos, col, count, tau, branch, max_new)
        want = od.densify_select(pos, col, count, tau, tau_c, branch, max_new)
        np.testing.assert_array_equal(got, want, err_msg=f"max_new={max_new}")


def test_select_ties_at_the_cut_taken_in_index_order():
    # every candidate has the same score: the cut falls inside one key
    n = 50_000
    count = np.ones(n, np.int32)
    pos = np.full(n, 5e-4, np.float32)
    pos[::3] = 0.0
    col = np.zeros(n, np.float32)
    got, tau_c = gpu_select(pos, col, count, 3e-4, False, 1234)
    want = od.densify_select(pos, col, count, 3e-4, tau_c, False, 1234)
    np.testing.assert_array_equal(got, want)
    assert got.tolist() == [i for i in range(n) if i % 3][:1234]


def _state(n, seed=3, sh_dtype=torch.float32):
    s = scenes.cluster_scene(n, index=seed, sh_degree=1)
    p = GaussianParams.from_arrays(s.as_dict(), DEV, sh_dtype)
    rng = np.random.default_rng(seed)
    m = [torch.tensor(rng.normal(size=tuple(t.shape)), dtype=torch.float32, device=DEV) for t in p.tensors()]
    v = [torch.tensor(rng.uniform(size=tuple(t.shape)), dtype=torch.float32, device=DEV) for t in p.tensors()]
    pos, col, count = stats(n, seed + 10)
    st = GaussianState(p, m, v, torch.tensor(pos, device=DEV), torch.tensor(col, device=DEV),
                       torch.tensor(count, device=DEV))
    return st, s


def _np(p):
    return {k: getattr(p, k).float().cpu().numpy().astype(np.float64)
            for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}


def test_grow_matches_oracle():
    n = 20_000
    st, _ = _state(n)
    rng = np.random.default_rng(7)
    sel = np.sort(rng.choice(n, 3000, replace=False)).astype(np.int32)
    noise = rng.standard_normal((sel.size, 2, 3)).astype(np.float32)
    log_split = float(np.float32(math.log(0.03)))
    from paper_2412_13547_b300.densify import _entries
    entries, grown = _entries(st, n + sel.size, grow=True)
    R.gs_densify_grow(n, sel.size, torch.tensor(sel, device=DEV), torch.tensor(noise, device=DEV), log_split,
                      entries)
    torch.cuda.synchronize()
    p0 = _np(st.params)
    want, fresh = od.densify_grow(p0, sel, noise.astype(np.float64), log_split)
    got = _np(grown.params)
    split = np.zeros(n + sel.size, bool)
    ls32 = st.params.log_scales.cpu().numpy()
    for j, g in enumerate(sel):
        if ls32[g].max() > np.float32(log_split):
            split[g] = split[n + j] = True
    assert 100 < split.sum() < 2 * sel.size  # both clones and splits occur
    for k in ("quats", "opacity_logits", "sh"):
        np.testing.assert_array_equal(got[k], want[k], err_msg=k)
    for k in ("means", "log_scales"):
        np.testing.assert_array_equal(got[k][~split], want[k][~split], err_msg=k)
        err = np.abs(got[k][split] - want[k][split]).max() / np.abs(want[k]).max()
        assert err < 1e-6, (k, err)
    old_rows = ~fresh[:n]
    for src, dst in zip(st.m + st.v, grown.m + grown.v):
        a, b = dst.cpu().numpy(), src.cpu().numpy()
        np.testing.assert_array_equal(a[:n][old_rows], b[old_rows])
        assert np.all(a[fresh] == 0.0)
    for t in (grown.pos_acc, grown.col_acc, grown.count):
        assert torch.count_nonzero(t).item() == 0


def test_prune_and_gather_match_oracle():
    n = 30_000
    st, _ = _state(n, sh_dtype=torch.bfloat16)
    logits = st.params.opacity_logits.cpu().numpy()
    ls = st.params.log_scales.cpu().numpy()
    for logit_min, lmax in ((-1.0, None), (0.5, math.log(0.05))):
        ws = torch.empty(R.gs_densify_workspace_size(n), dtype=torch.uint8, device=DEV)
        keep = torch.full((n,), -1, dtype=torch.int32, device=DEV)
        nk = torch.zeros(1, dtype=torch.int32, device=DEV)
        R.gs_prune_select(n, st.params.opacity_logits, logit_min, st.params.log_scales if lmax else None,
                          lmax or 0.0, ws, keep, nk)
        torch.cuda.synchronize()
        k = int(nk.item())
        want = od.prune_keep(logits, logit_min, ls if lmax else None, lmax)
        np.testing.assert_array_equal(keep[:k].cpu().numpy(), want)
    from paper_2412_13547_b300.densify import _entries
    entries, out = _entries(st, k, grow=False)
    R.gs_gather_rows(k, keep, entries)
    torch.cuda.synchronize()
    for a, b in zip(out.params.tensors() + [out.params.sh_store] + out.m + out.v,
                    st.params.tensors() + [st.params.sh_store] + st.m + st.v):
        np.testing.assert_array_equal(a.float().cpu().numpy(), b.float().cpu().numpy()[want])


def test_densify_and_prune_round_matches_oracle():
    n = 40_000
    st, _ = _state(n)
    cfg = DensifyConfig(tau_pos=3e-4, split_scale=0.03, min_opacity=0.1)
    before = _np(st.params)
    pos, col, cnt = (t.cpu().numpy() for t in (st.pos_acc, st.col_acc, st.count))
    new, info = densify_and_prune(st, budget_total=n + 2500, cfg=cfg, rng=np.random.default_rng(11))
    torch.cuda.synchronize()
    # replay the round in the oracle with the same draws
    rng = np.random.default_rng(11)
    branch = bool(rng.random() < cfg.color_prob)
    assert branch == info["color_branch"]
    tau_c = float(np.float32(cfg.tau_pos) * np.float32(TAU_COLOR_RATIO))
    sel = od.densify_select(pos, col, cnt, cfg.tau_pos, tau_c, branch, 2500)
    assert info["selected"] == sel.size == 2500
    noise = rng.standard_normal((max(1, sel.size), 2, 3)).astype(np.float32).astype(np.float64)
    grown, fresh = od.densify_grow(before, sel, noise, float(np.float32(math.log(cfg.split_scale))))
    o = cfg.min_opacity
    keep = od.prune_keep(grown["opacity_logits"], math.log(o / (1 - o)))
    assert info["n_after"] == keep.size == new.n
    got = _np(new.params)
    for k in grown:
        w = grown[k][keep]
        err = np.abs(got[k] - w).max() / max(1e-30, np.abs(w).max())
        assert err < 1e-6, (k, err)
    assert new.params.means.shape[0] == new.m[0].shape[0] == new.pos_acc.shape[0] == keep.size
    np.testing.assert_array_equal(new.m[0].cpu().numpy()[fresh[keep]], 0.0)
