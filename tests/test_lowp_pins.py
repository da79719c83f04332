"""Pins of the low-precision storage oracle (oracle/lowp.py), on the CPU.

What fixes it other than itself: torch's own BF16/FP16 conversions (round to
nearest must be one of the two neighbours the oracle finds), the spacing of
the types from frexp, the definition of stochastic rounding (exact values stay;
P(away from zero) equals the position between the neighbours, checked as an
expectation over the hash stream), uniformity of the hash, and the pinned
FP64 Adam oracle (the low-precision step brackets it and follows it in
expectation).
"""
import numpy as np
import pytest
import torch

from oracle import lowp
from oracle import oracle as orc

TYPES = {"bf16": torch.bfloat16, "f16": torch.float16}


def _spacing(lo, dtype):
    """The step between lo and the next magnitude of the type, from frexp."""
    a = np.abs(lo)
    _, e = np.frexp(np.where(a > 0, a, 1.0))
    if dtype == "bf16":
        return np.ldexp(1.0, e - 8)
    return np.where(a < 2.0 ** -14, 2.0 ** -24, np.ldexp(1.0, e - 11))


def _values(rng, n, dtype):
    scale = 2.0 if dtype == "bf16" else 0.5
    x = rng.standard_normal(n) * scale * np.exp(rng.uniform(-6, 2, n))
    return x.astype(np.float32)


def test_pcg_hash_is_uniform_over_consecutive_counters():
    h = lowp.pcg_hash(np.arange(1 << 18, dtype=np.uint64))
    # every byte of the output (both 16-bit halves are used)
    for part in (h >> np.uint64(24), (h >> np.uint64(16)) & np.uint64(0xFF), (h >> np.uint64(8)) & np.uint64(0xFF),
                 h & np.uint64(0xFF)):
        counts = np.bincount(part.astype(np.int64), minlength=256)
        exp = h.size / 256.0
        chi2 = float(((counts - exp) ** 2 / exp).sum())
        assert chi2 < 350.0, chi2  # 255 degrees of freedom: P(chi2 > 350) < 1e-4
    r = lowp.sr_bits16(7, 3, np.arange(1 << 16)).astype(np.float64)
    assert r.max() < 65536 and abs(r.mean() / 65535.0 - 0.5) < 0.01
    # neighbouring counters are uncorrelated
    c = np.corrcoef(r[:-1], r[1:])[0, 1]
    assert abs(c) < 0.02
    # different steps and seeds give different streams
    assert (lowp.sr_bits16(7, 4, np.arange(64)) != lowp.sr_bits16(7, 3, np.arange(64))).mean() > 0.9
    assert (lowp.sr_bits16(8, 3, np.arange(64)) != lowp.sr_bits16(7, 3, np.arange(64))).mean() > 0.9


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_neighbours_bracket_and_match_torch(dtype):
    rng = np.random.default_rng(1)
    x = _values(rng, 20000, dtype)
    lo, hi, pos = lowp.neighbours(x, dtype)
    ax = np.abs(x.astype(np.float64))
    assert (np.abs(lo) <= ax).all() and (ax <= np.abs(hi)).all()
    assert (np.sign(lo) * np.sign(x) >= 0).all()
    np.testing.assert_array_equal(np.abs(hi) - np.abs(lo), _spacing(lo, dtype))
    # both are values of the type, and torch's round-to-nearest picks one of them
    for v in (lo, hi):
        t = torch.tensor(v.astype(np.float32)).to(TYPES[dtype]).double().numpy()
        np.testing.assert_array_equal(t, v)
    rn = torch.tensor(x).to(TYPES[dtype]).double().numpy()
    assert ((rn == lo) | (rn == hi)).all()
    assert ((pos >= 0) & (pos < 65536)).all()


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_values_of_the_type_stay_and_extremes_pick_the_neighbours(dtype):
    rng = np.random.default_rng(2)
    x = torch.tensor(_values(rng, 5000, dtype)).to(TYPES[dtype]).float().numpy()
    for r in (0, 1, 32768, 65535):
        np.testing.assert_array_equal(lowp.sr_round(x, np.full(x.shape, r), dtype), x.astype(np.float64))
    y = _values(rng, 5000, dtype)
    lo, hi, pos = lowp.neighbours(y, dtype)
    np.testing.assert_array_equal(lowp.sr_round(y, np.full(y.shape, 65535), dtype), lo)
    np.testing.assert_array_equal(lowp.sr_round(y, np.zeros(y.shape), dtype), np.where(pos > 0, hi, lo))


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("frac", [0.1, 0.37, 0.5, 0.93])
def test_rounding_is_unbiased(dtype, frac):
    """P(away from zero) = the position between the neighbours: the mean over
    2^16 elements of the hash stream recovers it (4 sigma)."""
    base = np.float64(1.0 + 2.0 ** -5 if dtype == "bf16" else -0.75)
    lo, hi, _ = lowp.neighbours(np.array([base], np.float32), dtype)
    x = np.float32(lo[0] + frac * (hi[0] - lo[0]))
    lo, hi, pos = lowp.neighbours(np.array([x]), dtype)
    n = 1 << 16
    out = lowp.sr_round(np.full(n, x), lowp.sr_bits16(11, 5, np.arange(n)), dtype)
    f = float(np.mean(out == hi[0]))
    p = pos[0] / 65536.0
    assert abs(p - frac) < 1e-3
    assert abs(f - p) < 4.0 * np.sqrt(p * (1 - p) / n), (f, p)
    assert set(np.unique(out)) <= {lo[0], hi[0]}


def test_fp16_saturates_at_the_largest_finite_value():
    x = np.array([65504.0, 65519.0, -65510.0], np.float32)
    out = lowp.sr_round(x, np.zeros(3), "f16")
    np.testing.assert_array_equal(out, [65504.0, 65504.0, -65504.0])


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_adam_lowp_brackets_and_follows_fp64_adam(dtype):
    """The low-precision step's result is one of the two neighbours of the
    FP64 Adam result (rounded to FP32), and its mean over many elements with
    the same value and gradient is that result (4 sigma)."""
    n = 1 << 15
    stored = np.full(n, torch.tensor(0.3).to(TYPES[dtype]).item())
    g = np.full(n, 0.02)
    m0, v0 = np.full(n, 0.01), np.full(n, 4e-4)
    ref = stored.copy()
    mr, vr = m0.copy(), v0.copy()
    orc.adam(ref, g, mr, vr, 1e-4, 0.9, 0.999, 1e-15, 7)
    m, v = m0.copy(), v0.copy()
    out = lowp.adam_lowp(stored, g, m, v, 1e-4, 0.9, 0.999, 1e-15, 7, dtype, seed=3)
    np.testing.assert_array_equal(m, mr)
    np.testing.assert_array_equal(v, vr)
    lo, hi, pos = lowp.neighbours(ref.astype(np.float32), dtype)
    assert ((out == lo) | (out == hi)).all()
    # the update (-1e-4 x about 1) is far below half a step at 0.3, yet moves the mean
    assert abs(ref[0] - stored[0]) < 0.25 * (abs(hi[0] - lo[0]))
    p = pos[0] / 65536.0
    sig = (hi[0] - lo[0]) * np.sqrt(p * (1 - p) / n)
    assert abs(out.mean() - ref.astype(np.float32).astype(np.float64)[0]) < 4 * sig + 1e-12
    # nearest rounding would have left every element where it was
    assert torch.tensor(ref).to(TYPES[dtype]).double().numpy()[0] == stored[0]


def test_adam_lowp_element_index_selects_the_bits():
    n = 256
    stored = np.zeros(n)
    g = np.linspace(-1, 1, n)
    a = lowp.adam_lowp(stored, g, np.zeros(n), np.zeros(n), 1e-3, 0.9, 0.999, 1e-15, 1, "bf16", seed=5,
                       index0=1000)
    b = lowp.adam_lowp(stored[:128], g[:128], np.zeros(128), np.zeros(128), 1e-3, 0.9, 0.999, 1e-15, 1, "bf16",
                       seed=5, index0=1000)
    c = lowp.adam_lowp(stored[128:], g[128:], np.zeros(128), np.zeros(128), 1e-3, 0.9, 0.999, 1e-15, 1, "bf16",
                       seed=5, index0=1128)
    np.testing.assert_array_equal(a, np.r_[b, c])
