"""Oracle of densification and pruning under a Gaussian budget (Sec. 3.2,
Sec. 3.3), plain numpy.

TEST INFRASTRUCTURE. Only ``tests/`` (and ``__graft_entry__.smoke()``) may
import this module; the product package never does, and nothing here is
shared with the CUDA path.

* ``budget``: Eq. 7, B(t) = N + (t^a - 1) / (100^a - 1) (M - N).
* ``densify_select``: the position-appearance rule of Sec. 3.3 -- a Gaussian
  is densified when its mean positional-gradient norm exceeds tau_pos, or,
  when the colour branch is active (the caller draws it with probability
  0.2), its mean colour-gradient norm exceeds tau_color = 0.01 tau_pos; when
  the candidates outnumber the budget, the highest-scoring ones are kept.
* ``densify_grow``: the baseline (3DGS) clone / split of the selected
  Gaussians, with the standard-normal draws of the split given as input.
* ``prune``: drop Gaussians whose opacity is below a threshold (and,
  optionally, whose largest scale is above one), keeping the order.

The decisions (thresholds, score order, clone vs split) are taken in FP32,
the precision the device takes them in, so both sides decide identically;
the continuous values (split positions) are computed in FP64.
"""
from __future__ import annotations

import numpy as np

SPLIT_SCALE_DIVISOR = 1.6  # children of a split take the parent's scales / 1.6 (3DGS baseline)


def budget(t, n_init: float, m_final: float, alpha: float):
    """Eq. 7: the Gaussian budget at progress t in [1, 100] of the densification phase."""
    t = np.asarray(t, np.float64)
    return n_init + (t ** alpha - 1.0) / (100.0 ** alpha - 1.0) * (m_final - n_init)


def densify_scores(pos_acc, col_acc, count, tau_pos, tau_color, color_branch):
    """FP32 candidate flags and ranking scores of Sec. 3.3 (see the module doc)."""
    pos_acc = np.asarray(pos_acc, np.float32)
    col_acc = np.asarray(col_acc, np.float32)
    count = np.asarray(count, np.int64)
    tau_pos, tau_color = np.float32(tau_pos), np.float32(tau_color)
    seen = count > 0
    c = np.where(seen, count, 1).astype(np.float32)
    sp = (pos_acc / c).astype(np.float32)
    sc = (col_acc / c).astype(np.float32)
    cand = seen & ((sp > tau_pos) | (bool(color_branch) & (sc > tau_color)))
    a = (sp / tau_pos).astype(np.float32)
    b = (sc / tau_color).astype(np.float32) if color_branch else np.zeros_like(a)
    score = np.maximum(a, b).astype(np.float32)
    return cand, score


def densify_select(pos_acc, col_acc, count, tau_pos, tau_color, color_branch, max_new):
    """Indices (ascending) of the Gaussians to densify: every candidate if
    there are at most max_new, else the max_new highest scores, equal scores
    taken in index order."""
    cand, score = densify_scores(pos_acc, col_acc, count, tau_pos, tau_color, color_branch)
    idx = np.nonzero(cand)[0]
    if idx.size > max_new:
        order = sorted(idx.tolist(), key=lambda i: (-float(score[i]), i))
        idx = np.array(sorted(order[:max(0, int(max_new))]), np.int64)
    return idx.astype(np.int64)


def quat_to_rot(q):
    """Rotation matrix of the normalised quaternion (w, x, y, z)."""
    w, x, y, z = np.asarray(q, np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def densify_grow(params: dict, selected, noise, log_split_scale):
    """Clone or split every selected Gaussian (3DGS baseline design):

    * clone (largest log-scale <= log_split_scale, compared in FP32): an exact
      copy is appended;
    * split: two children at mean + R(q) diag(exp(log_scales)) z_k with the
      given standard normals z_k = noise[j, k] (k = 0, 1), log-scales reduced
      by log(1.6); child 0 replaces the parent, child 1 is appended.

    Appended rows follow the old ones in the order of ``selected``. Returns
    (new params, is_new_or_split row mask: the rows whose optimizer state
    restarts from zero)."""
    n = params["means"].shape[0]
    sel = np.asarray(selected, np.int64)
    out = {k: np.concatenate([np.asarray(v, np.float64), np.asarray(v, np.float64)[sel]], 0)
           for k, v in params.items()}
    fresh = np.zeros(n + sel.size, bool)
    fresh[n:] = True
    ls32 = np.asarray(params["log_scales"], np.float32)
    thr = np.float32(log_split_scale)
    for j, g in enumerate(sel):
        if ls32[g].max() <= thr:
            continue
        Rm = quat_to_rot(params["quats"][g])
        s = np.exp(np.asarray(params["log_scales"][g], np.float64))
        mu = np.asarray(params["means"][g], np.float64)
        for k, row in ((0, g), (1, n + j)):
            out["means"][row] = mu + Rm @ (s * np.asarray(noise[j, k], np.float64))
            out["log_scales"][row] = np.asarray(params["log_scales"][g], np.float64) - np.log(SPLIT_SCALE_DIVISOR)
        fresh[g] = True
    return out, fresh


def prune_keep(opacity_logits, logit_min, log_scales=None, log_scale_max=None):
    """Indices (ascending) kept by the prune: opacity logit >= logit_min (FP32
    compare; sigmoid is monotone, so this is opacity >= sigmoid(logit_min)),
    and, when given, largest log-scale <= log_scale_max."""
    keep = np.asarray(opacity_logits, np.float32).reshape(-1) >= np.float32(logit_min)
    if log_scales is not None and log_scale_max is not None:
        keep &= np.asarray(log_scales, np.float32).max(1) <= np.float32(log_scale_max)
    return np.nonzero(keep)[0].astype(np.int64)


def algorithm1(records, calls, n_init, m_final, start, end, window=200, history=5, warmup=100, lam=0.5,
               ema_alpha=0.1, alpha_clip=(0.1, 2.0), rate_up=0.05, rate_down=-0.05, grow=1.1, shrink=0.9,
               m_cap=1.5, m_floor=0.5):
    """Algorithm 1 (the convergence-aware budget of Sec. 3.2) replayed from a
    complete record, in the algorithm's own order.

    records: (step, loss) pairs in step order; calls: the steps at which the
    budget is asked for (each call sees the records up to and including it).
    Per call, following the algorithm's lines:
      * the losses of the first ``warmup`` steps are not recorded (Sec. 3.2),
        and with fewer than three recorded the exponent is 1 (the
        algorithm's default);
      * otherwise the recorded losses are smoothed, ema_t = ema_alpha * loss_t
        + (1 - ema_alpha) * ema_{t-1} (starting at the first loss), and
        log(ema) is fitted against log(step) by least squares (numpy.polyfit,
        degree 1) over all of them: alpha_history = -slope; alpha_base is the
        mean of the last ``history`` such fits (Eq. 6's text);
      * rate = -slope of the same fit over the last ``window`` points;
      * the final count M grows x``grow`` (at most m_cap M) when
        rate > rate_up and shrinks x``shrink`` (at least m_floor M) when
        rate < rate_down;
      * Eq. 6: epsilon = alpha_recent - alpha_history in slope terms, that is
        alpha_base - rate with both as decay exponents, and
        alpha = alpha_base + lam * tanh(epsilon), clipped to alpha_clip;
      * Eq. 7: B(t) = N + (t^alpha - 1) / (100^alpha - 1) (M - N), with
        t = 1 + 99 (step - start) / (end - start) clamped to [1, 100].
    Returns, per call, a dict of alpha, alpha_base, rate, M and B."""
    out = []
    fits = []
    m_adapt = float(m_final)
    recs = [(int(s), float(l)) for s, l in records if int(s) > warmup]
    for c in calls:
        seen = [(s, l) for s, l in recs if s <= c]
        alpha, a_base, rate = 1.0, None, 0.0
        if len(seen) > 2:
            steps = np.array([s for s, _ in seen], np.float64)
            ema = np.empty(len(seen))
            for i, (_, l) in enumerate(seen):
                ema[i] = l if i == 0 else ema_alpha * l + (1.0 - ema_alpha) * ema[i - 1]
            x, y = np.log(steps), np.log(np.maximum(ema, 1e-30))
            fits.append(-np.polyfit(x, y, 1)[0])
            a_base = float(np.mean(fits[-history:]))
            k = min(window, len(seen))
            rate = float(-np.polyfit(x[-k:], y[-k:], 1)[0])
            if rate > rate_up:
                m_adapt = min(m_adapt * grow, m_final * m_cap)
            elif rate < rate_down:
                m_adapt = max(m_adapt * shrink, m_final * m_floor)
            eps = a_base - rate
            alpha = float(np.clip(a_base + lam * np.tanh(eps), *alpha_clip))
        t = 100.0 if end <= start else 1.0 + 99.0 * min(1.0, max(0.0, (c - start) / float(end - start)))
        b = float(budget(t, n_init, m_adapt, alpha))
        out.append(dict(alpha=alpha, alpha_base=a_base, rate=rate, M=m_adapt, B=b))
    return out
