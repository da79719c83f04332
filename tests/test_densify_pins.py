"""Pins of the densification oracle and of the host budget schedule (CPU).

* Eq. 7: B(1) = N and B(100) = M for any exponent, monotone in t, linear at
  exponent 1; the adaptive exponent and final count of Algorithm 1 on loss
  curves whose power-law exponent is known.
* The constants printed in the paper (tests/golden/budget_constants.json).
* Selection, clone/split and prune of the oracle on hand-made cases whose
  answers are written out, and the split position in closed form.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import densify as od
from paper_2412_13547_b300 import budget as B
from paper_2412_13547_b300 import densify as PD

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "budget_constants.json")))


# ---------------------------------------------------------------------------
# Eq. 7 and Algorithm 1
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("alpha", [0.1, 0.3, 1.0, 1.7, 2.0])
def test_budget_endpoints_and_monotone(alpha):
    n0, m = 100_000, 3_000_000
    for f in (od.budget, B.budget):
        assert abs(float(f(1, n0, m, alpha)) - n0) < 1e-6
        assert abs(float(f(100, n0, m, alpha)) - m) < 1e-3
        vals = [float(f(t, n0, m, alpha)) for t in np.linspace(1, 100, 200)]
        assert all(b > a for a, b in zip(vals, vals[1:]))


def test_budget_linear_at_exponent_one_and_convexity():
    n0, m = 10.0, 1000.0
    assert abs(B.budget(50.5, n0, m, 1.0) - (n0 + m) / 2) < 1e-9
    # a < 1 front-loads the growth, a > 1 back-loads it
    assert B.budget(10, n0, m, 0.5) > B.budget(10, n0, m, 1.0) > B.budget(10, n0, m, 2.0)


def test_progress_maps_the_phase_to_1_100():
    assert B.progress(300, 300, 3000) == 1.0
    assert B.progress(3000, 300, 3000) == 100.0
    assert B.progress(5000, 300, 3000) == 100.0
    assert abs(B.progress(1650, 300, 3000) - 50.5) < 1e-12


def test_constants_are_the_printed_ones():
    assert B.LAMBDA == GOLD["lambda"]["value"]
    assert B.EMA_ALPHA == GOLD["ema_alpha"]["value"]
    assert list(B.ALPHA_CLIP) == GOLD["alpha_clip"]["value"]
    assert [B.RATE_UP, B.RATE_DOWN] == GOLD["rate_thresholds"]["value"]
    assert [B.GROW, B.SHRINK] == GOLD["m_adaptive_factors"]["value"]
    assert [B.M_CAP, B.M_FLOOR] == GOLD["m_adaptive_bounds"]["value"]
    assert B.WARMUP == GOLD["warmup_steps"]["value"]
    assert PD.TAU_COLOR_RATIO == GOLD["tau_color_over_tau_pos"]["value"]
    assert PD.COLOR_BRANCH_PROB == GOLD["color_branch_probability"]["value"]
    s = B.AdaptiveBudget(10, 100, 0, 1000)
    assert s.alpha == GOLD["default_alpha"]["value"]


def _feed(sched, losses, first=101):
    for i, l in enumerate(losses):
        sched.record(first + i, l)


def test_adaptive_exponent_of_a_power_law_loss():
    # loss = c t^-p: the fitted decay exponent is p (the EMA lags a little), the
    # recent rate equals it, so the exponent stays at p and the final count grows
    p = 0.4
    s = B.AdaptiveBudget(1000, 10000, 100, 5000, window=300)
    steps = np.arange(101, 3001)
    _feed(s, 2.0 * steps.astype(np.float64) ** -p)
    s.update()
    assert abs(s.alpha_base - p) < 0.05
    assert abs(s.rate - p) < 0.05
    assert abs(s.alpha - p) < 0.05
    assert s.m_adaptive == pytest.approx(10000 * 1.1)
    for _ in range(10):
        s.update()
    assert s.m_adaptive == pytest.approx(10000 * 1.5)  # capped at 1.5 M


def test_adaptive_slows_densification_when_convergence_slows():
    # the loss follows t^-0.5 and then flattens: recent decay < historical decay
    s = B.AdaptiveBudget(1000, 10000, 100, 5000, window=200)
    steps = np.arange(101, 2001).astype(np.float64)
    loss = np.where(steps < 1600, steps ** -0.5, 1600.0 ** -0.5 * (steps / 1600.0) ** -0.02)
    _feed(s, loss)
    s.update()
    assert s.rate < s.alpha_base
    assert s.alpha > s.alpha_base  # larger exponent: a smaller budget at any t in (1, 100)
    b_slow = B.budget(30, 1000, s.m_adaptive, s.alpha)
    b_base = B.budget(30, 1000, s.m_adaptive, s.alpha_base)
    assert b_slow < b_base


def test_adaptive_rising_loss_shrinks_the_final_count_and_clips():
    s = B.AdaptiveBudget(1000, 10000, 100, 5000, window=200)
    steps = np.arange(101, 1001).astype(np.float64)
    _feed(s, steps ** 0.5)  # a diverging fit
    for _ in range(20):
        s.update()
    assert s.rate < -0.05
    assert s.m_adaptive == pytest.approx(10000 * 0.5)
    assert B.ALPHA_CLIP[0] <= s.alpha <= B.ALPHA_CLIP[1]


def test_warmup_uses_the_default_exponent():
    s = B.AdaptiveBudget(1000, 10000, 0, 1000)
    for t in range(1, 101):
        s.record(t, 1.0 / t)
    b = s(50)
    assert s.alpha == 1.0
    assert b == round(B.budget(B.progress(50, 0, 1000), 1000, 10000, 1.0))


# ---------------------------------------------------------------------------
# Oracle: selection
# ---------------------------------------------------------------------------

def _acc():
    # Gaussian:        0     1     2     3      4     5       6
    count = np.array([2,    1,    4,    0,     1,    2,      2], np.int32)
    pos = np.array([0.5,  0.3,  0.8,  9.0,   0.1,  0.42,   0.5], np.float32)
    col = np.array([0.0, 0.001, 0.0,  9.0, 0.009,  0.0,  0.005], np.float32)
    # means: pos 0.25 0.3 0.2 (unseen) 0.1 0.21 0.25; colour 0 0.001 0 (unseen) 0.009 0 0.0025
    return pos, col, count


def test_select_position_only():
    pos, col, cnt = _acc()
    # tau_pos 0.2: 0, 1, 5, 6 lie above; 2 sits exactly at 0.2 (not above); 3 was never seen
    sel = od.densify_select(pos, col, cnt, 0.2, 0.002, False, 100)
    assert sel.tolist() == [0, 1, 5, 6]


def test_select_with_colour_branch():
    pos, col, cnt = _acc()
    # tau_color 0.002 adds 4 (0.009); 1's 0.001 is below
    sel = od.densify_select(pos, col, cnt, 0.2, 0.002, True, 100)
    assert sel.tolist() == [0, 1, 4, 5, 6]


def test_select_budget_keeps_highest_scores_in_index_order():
    pos, col, cnt = _acc()
    # scores: 0 -> 1.25, 1 -> 1.5, 4 -> 4.5 (colour), 5 -> 1.05, 6 -> 1.25 (position; its colour
    # score 0.0025/0.002 rounds just below 1.25 in FP32)
    sel = od.densify_select(pos, col, cnt, 0.2, 0.002, True, 2)
    assert sel.tolist() == [1, 4]
    # 0 and 6 tie at 1.25: the lower index is taken first
    sel = od.densify_select(pos, col, cnt, 0.2, 0.002, True, 3)
    assert sel.tolist() == [0, 1, 4]
    sel = od.densify_select(pos, col, cnt, 0.2, 0.002, True, 4)
    assert sel.tolist() == [0, 1, 4, 6]
    assert od.densify_select(pos, col, cnt, 0.2, 0.002, True, 0).tolist() == []
    _, score = od.densify_scores(pos, col, cnt, 0.2, 0.002, True)
    assert score[0] == score[6] == np.float32(1.25)


# ---------------------------------------------------------------------------
# Oracle: clone / split / prune
# ---------------------------------------------------------------------------

def _params(n=4):
    rng = np.random.default_rng(0)
    return dict(means=rng.normal(size=(n, 3)), log_scales=np.log(np.array([[0.01, 0.02, 0.01],
                                                                            [0.3, 0.1, 0.2],
                                                                            [0.05, 0.05, 0.05],
                                                                            [0.2, 0.2, 0.2]])[:n]),
                quats=np.array([[1.0, 0, 0, 0], [math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)],
                                [1.0, 0, 0, 0], [1.0, 0, 0, 0]])[:n],
                opacity_logits=np.array([0.5, -1.0, 2.0, -3.0])[:n],
                sh=rng.normal(size=(n, 4, 3)))


def test_clone_copies_and_split_in_closed_form():
    p = _params()
    noise = np.zeros((2, 2, 3))
    noise[1, 0] = [1.0, 0.0, 0.0]   # child 0 of the split: +1 sigma along the local x axis
    noise[1, 1] = [0.0, -2.0, 0.0]  # child 1: -2 sigma along the local y axis
    out, fresh = od.densify_grow(p, [0, 1], noise, math.log(0.1))
    assert out["means"].shape == (6, 3)
    # Gaussian 0 (max scale 0.02 <= 0.1): cloned; row 4 is its exact copy, row 0 untouched
    for k in p:
        np.testing.assert_array_equal(out[k][4], p[k][0])
        np.testing.assert_array_equal(out[k][0], p[k][0])
    # Gaussian 1 (max scale 0.3 > 0.1), rotated 90 degrees about z: local x -> world y, local y -> -world x
    np.testing.assert_allclose(out["means"][1], p["means"][1] + [0.0, 0.3, 0.0], atol=1e-12)
    np.testing.assert_allclose(out["means"][5], p["means"][1] + [2 * 0.1, 0.0, 0.0], atol=1e-12)
    for row in (1, 5):
        np.testing.assert_allclose(out["log_scales"][row], p["log_scales"][1] - math.log(1.6), atol=1e-15)
        np.testing.assert_array_equal(out["quats"][row], p["quats"][1])
        np.testing.assert_array_equal(out["sh"][row], p["sh"][1])
        np.testing.assert_array_equal(out["opacity_logits"][row], p["opacity_logits"][1])
    assert fresh.tolist() == [False, True, False, False, True, True]


def test_split_with_zero_noise_keeps_the_mean():
    p = _params()
    out, _ = od.densify_grow(p, [3], np.zeros((1, 2, 3)), math.log(0.1))
    np.testing.assert_array_equal(out["means"][3], p["means"][3])
    np.testing.assert_array_equal(out["means"][4], p["means"][3])


def test_prune_keeps_order():
    p = _params()
    assert od.prune_keep(p["opacity_logits"], -1.5).tolist() == [0, 1, 2]
    assert od.prune_keep(p["opacity_logits"], -1.5, p["log_scales"], math.log(0.25)).tolist() == [0, 2]
    assert od.prune_keep(p["opacity_logits"], 5.0).tolist() == []


def test_time_to_psnr_interpolates_between_evaluations():
    from paper_2412_13547_b300.fit import time_to_psnr
    hist = [dict(seconds=0.0, psnr=20.0), dict(seconds=10.0, psnr=24.0), dict(seconds=20.0, psnr=26.0)]
    assert time_to_psnr(hist, 20.0) == 0.0
    assert time_to_psnr(hist, 22.0) == pytest.approx(5.0)
    assert time_to_psnr(hist, 25.0) == pytest.approx(15.0)
    assert time_to_psnr(hist, 27.0) is None


# ---------------------------------------------------------------------------
# Algorithm 1: the oracle's replay pinned by hand, then the host schedule
# against it
# ---------------------------------------------------------------------------

def _calls(records, every=400):
    last = records[-1][0]
    return list(range(every, last + 1, every))


def test_algorithm1_oracle_constant_loss():
    """A flat loss: every fitted slope is 0, so rate = alpha_base = 0, the final
    count stays, and alpha = clip(0 + 0.5 tanh(0)) = 0.1, the lower clip."""
    rec = [(s, 0.25) for s in range(1, 2001)]
    n0, m = 1000.0, 5000.0
    out = od.algorithm1(rec, [600, 1200], n0, m, start=500, end=1500)
    for o, c in zip(out, (600, 1200)):
        assert o["rate"] == pytest.approx(0.0, abs=1e-12) and o["alpha_base"] == pytest.approx(0.0, abs=1e-12)
        assert o["M"] == m and o["alpha"] == 0.1
        t = 1 + 99 * (c - 500) / 1000.0
        assert o["B"] == pytest.approx(n0 + (t ** 0.1 - 1) / (100 ** 0.1 - 1) * (m - n0), rel=1e-12)


def test_algorithm1_oracle_default_exponent_before_three_losses():
    rec = [(s, 1.0 / s) for s in range(1, 103)]  # steps 101 and 102 recorded after the 100 warm-up steps
    out = od.algorithm1(rec, [102], 100.0, 300.0, start=0, end=200)
    assert out[0]["alpha"] == 1.0 and out[0]["M"] == 300.0
    t = 1 + 99 * 102 / 200.0
    assert out[0]["B"] == pytest.approx(100.0 + (t - 1) / 99.0 * 200.0, rel=1e-12)


def test_algorithm1_oracle_exact_power_laws():
    """Without smoothing (ema_alpha = 1) a loss s^-0.4 fits slope -0.4 over any
    window: alpha_base = rate = 0.4, epsilon = 0, alpha = 0.4, and the final
    count grows x1.1 per call up to 1.5 M. A rising loss s^0.2 has rate -0.2:
    the count shrinks x0.9 per call down to 0.5 M and alpha clips to 0.1."""
    calls = [400, 800, 1200, 1600, 2000, 2400]
    fall = [(s, s ** -0.4) for s in range(1, 2401)]
    out = od.algorithm1(fall, calls, 10.0, 1000.0, start=0, end=2400, ema_alpha=1.0)
    for k, o in enumerate(out, start=1):
        assert o["rate"] == pytest.approx(0.4, rel=1e-9) and o["alpha"] == pytest.approx(0.4, rel=1e-9)
        assert o["M"] == pytest.approx(min(1000.0 * 1.1 ** k, 1500.0), rel=1e-12)
    rise = [(s, s ** 0.2) for s in range(1, 2401)]
    out = od.algorithm1(rise, calls, 10.0, 1000.0, start=0, end=2400, ema_alpha=1.0)
    for k, o in enumerate(out, start=1):
        assert o["rate"] == pytest.approx(-0.2, rel=1e-9) and o["alpha"] == 0.1
        assert o["M"] == pytest.approx(max(1000.0 * 0.9 ** k, 500.0), rel=1e-12)


@pytest.mark.parametrize("shape", ["power", "flattening", "rising", "noisy"])
def test_host_schedule_equals_algorithm1_oracle(shape):
    """budget.AdaptiveBudget (recorded every step, asked at every round) gives
    the oracle's alpha, final count and budget at every call."""
    rng = np.random.default_rng(7)
    steps = np.arange(1, 4001)
    if shape == "power":
        loss = 0.5 * steps ** -0.35
    elif shape == "flattening":
        loss = 0.5 * steps ** -0.5 + 0.02
    elif shape == "rising":
        loss = 0.1 + 1e-5 * steps
    else:
        loss = 0.5 * steps ** -0.3 * np.exp(rng.normal(0, 0.05, steps.size))
    rec = list(zip(steps.tolist(), loss.tolist()))
    calls = _calls(rec)
    n0, m, start, end = 50_000, 400_000, 300, 3000
    want = od.algorithm1(rec, calls, n0, m, start, end)
    sched = B.AdaptiveBudget(n0, m, start, end)
    got = []
    it = iter(rec)
    for c in calls:
        for s, l in it:
            sched.record(s, l)
            if s == c:
                break
        got.append((sched(c), sched.alpha, sched.m_adaptive, sched.rate))
    for (b, a, mm, r), w in zip(got, want):
        assert a == pytest.approx(w["alpha"], rel=1e-9, abs=1e-12)
        assert mm == pytest.approx(w["M"], rel=1e-12)
        assert r == pytest.approx(w["rate"], rel=1e-9, abs=1e-12)
        assert b == int(round(w["B"]))
