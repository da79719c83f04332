"""Convergence-aware Gaussian budget (Sec. 3.2, Eq. 6-7, Algorithm 1).

Host logic: a few scalars per densification round. The budget grows from
the initial count N to the final count M along Eq. 7,

    B(t) = N + (t^a - 1) / (100^a - 1) (M - N),   t in [1, 100],

where t is the progress through the densification phase in percent (the
100^a of Eq. 7 fixes t = 100 at its end). Algorithm 1 adapts the exponent a
and the final count to how the loss converges: the log of the EMA-smoothed
loss is fitted against the log of the step, once over the whole history and
once over the recent window.

Reading of the signs (the paper's Eq. 6 text and Algorithm 1 use the fitted
slope and its negative interchangeably): let h = -slope of the historical
fit and r = -slope of the recent fit (decay exponents, positive while the loss
falls). Then eps = h - r is Eq. 6's alpha_recent - alpha_history with the
alphas taken as slopes, and Algorithm 1's "-rate - alpha_base" with
alpha_base the historical slope; the exponent is a = h + lambda tanh(eps),
clipped to [0.1, 2]. When the loss converges more slowly than the power law
of its history predicts (r < h), a grows and densification slows down, as
Sec. 3.2 states. The final count follows Algorithm 1: x1.1 (capped at 1.5 M)
while the recent rate exceeds 0.05, x0.9 (floored at 0.5 M) when it is below
-0.05.
"""
from __future__ import annotations

import math

import numpy as np

LAMBDA = 0.5          # Eq. 6 (Sec. 3.2; the sensitivity study keeps 0.5)
EMA_ALPHA = 0.1       # Algorithm 1
ALPHA_CLIP = (0.1, 2.0)
RATE_UP, RATE_DOWN = 0.05, -0.05
GROW, SHRINK = 1.1, 0.9
M_CAP, M_FLOOR = 1.5, 0.5
WARMUP = 100          # losses recorded after 100 warm-up steps (Sec. 3.2)


def budget(t: float, n_init: float, m_final: float, alpha: float) -> float:
    """Eq. 7 at progress t in [1, 100]."""
    t = min(100.0, max(1.0, float(t)))
    return n_init + (t ** alpha - 1.0) / (100.0 ** alpha - 1.0) * (m_final - n_init)


def progress(step: int, start: int, end: int) -> float:
    """Step -> t in [1, 100] over the densification phase [start, end]."""
    if end <= start:
        return 100.0
    return 1.0 + 99.0 * min(1.0, max(0.0, (step - start) / float(end - start)))


def _slope(x, y) -> float:
    """Least-squares slope of y against x (with intercept)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    xm = x - x.mean()
    den = float((xm * xm).sum())
    return float((xm * (y - y.mean())).sum() / den) if den > 0 else 0.0


class AdaptiveBudget:
    """Algorithm 1. ``record(step, loss)`` every step; ``__call__(step)`` at
    each densification round returns the budget B(t)."""

    def __init__(self, n_init: int, m_final: int, start: int, end: int, window: int = 200, history: int = 5,
                 warmup: int = WARMUP, lam: float = LAMBDA):
        self.n, self.m = float(n_init), float(m_final)
        self.m_adaptive = float(m_final)
        self.start, self.end = int(start), int(end)
        self.window, self.history, self.warmup, self.lam = int(window), int(history), int(warmup), float(lam)
        self.steps: list[int] = []
        self.ema: list[float] = []
        self.base_fits: list[float] = []
        self.alpha = 1.0
        self.rate = 0.0
        self.alpha_base = None

    def record(self, step: int, loss: float):
        if step <= self.warmup:
            return
        e = float(loss) if not self.ema else EMA_ALPHA * float(loss) + (1.0 - EMA_ALPHA) * self.ema[-1]
        self.steps.append(int(step))
        self.ema.append(e)

    def update(self):
        """Refit the exponent and the final count from the recorded losses."""
        if len(self.ema) <= 2:
            self.alpha = 1.0
            return
        logs = np.log(np.asarray(self.steps, np.float64))
        loge = np.log(np.maximum(np.asarray(self.ema, np.float64), 1e-30))
        h = -_slope(logs, loge)
        self.base_fits.append(h)
        self.alpha_base = float(np.mean(self.base_fits[-self.history:]))
        k = min(self.window, len(self.ema))
        self.rate = -_slope(logs[-k:], loge[-k:])
        if self.rate > RATE_UP:
            self.m_adaptive = min(self.m_adaptive * GROW, self.m * M_CAP)
        elif self.rate < RATE_DOWN:
            self.m_adaptive = max(self.m_adaptive * SHRINK, self.m * M_FLOOR)
        eps = self.alpha_base - self.rate
        self.alpha = float(np.clip(self.alpha_base + self.lam * math.tanh(eps), *ALPHA_CLIP))

    def __call__(self, step: int) -> int:
        self.update()
        return int(round(budget(progress(step, self.start, self.end), self.n, self.m_adaptive, self.alpha)))
