"""Oracle of the low-precision SH storage: stochastic rounding of FP32 values
to BF16/FP16 and the Adam step of a parameter kept only in that type.

TEST INFRASTRUCTURE. Only ``tests/`` (and ``__graft_entry__.smoke()``,
``bench.py``'s CPU baseline) may import this module; the product package
never does, and nothing here is shared with the CUDA path.

The precision form stores the SH coefficients (and so the colours) in BF16 or
FP16 while the blend and every accumulation stay FP32. Kept only in 16 bits,
a parameter's Adam update is often far smaller than half a step of its type;
rounding to nearest would drop it. Stochastic rounding (Gupta et al., "Deep
Learning with Limited Numerical Precision", ICML 2015) rounds to the
neighbour away from zero with probability equal to the value's position
between its two neighbours, so the stored value follows the update in
expectation. Definitions used here, one per step:

* the two neighbours of x in the 16-bit type: lo, the largest magnitude not
  above |x| with x's sign (rounding toward zero), and hi, the next magnitude;
* the position of x between them, in units of 2^-16 of the step hi - lo:
  pos = floor(65536 (|x| - |lo|) / (|hi| - |lo|));
* the random bits: elements 2k and 2k + 1 take the low and the high 16 bits
  of pcg(base + k), with base = pcg(pcg(seed) xor t) for the optimizer
  step t, where pcg is the
  PCG hash of Jarzynski and Olano ("Hash Functions for GPU Rendering",
  JCGT 9(3), 2020): one step of PCG's 32-bit LCG followed by PCG's RXS-M-XS
  output permutation (O'Neill 2014);
* the result: hi if pos > r, else lo (so P(hi) = pos / 65536). A value of
  the type (pos = 0) stays as it is; the largest finite FP16 magnitude
  saturates.

The rounding decision is taken on the FP32 value of the update (the
precision the kernel decides it in): the oracle computes Adam in FP64 and
rounds that result to FP32 first.
"""
from __future__ import annotations

import numpy as np

from . import oracle as orc

_M32 = 0xFFFFFFFF


def pcg_hash(v):
    """PCG hash (Jarzynski & Olano 2020) of uint32 values, elementwise."""
    v = np.asarray(v, dtype=np.uint64) & np.uint64(_M32)
    state = (v * np.uint64(747796405) + np.uint64(2891336453)) & np.uint64(_M32)
    shift = (state >> np.uint64(28)) + np.uint64(4)
    word = (((state >> shift) ^ state) * np.uint64(277803737)) & np.uint64(_M32)
    return ((word >> np.uint64(22)) ^ word) & np.uint64(_M32)


def sr_bits16(seed: int, step: int, e):
    """The 16 random bits of elements e (uint32 counters) at optimizer step t."""
    base = pcg_hash(pcg_hash(np.uint64(seed & _M32)) ^ np.uint64(step & _M32))
    e = np.asarray(e, dtype=np.uint64)
    h = pcg_hash((base + (e >> np.uint64(1))) & np.uint64(_M32))
    return np.where((e & np.uint64(1)) == 1, h >> np.uint64(16), h & np.uint64(0xFFFF))


def _lo_bits(x32: np.ndarray, dtype: str) -> np.ndarray:
    """Bit patterns (uint32 for bf16 as the upper half, uint16 for fp16) of the
    neighbour toward zero."""
    if dtype == "bf16":
        return x32.view(np.uint32) >> np.uint32(16)
    h = x32.astype(np.float16)                       # nearest, may overshoot |x|
    hb = h.view(np.uint16).astype(np.int64)
    over = np.abs(h.astype(np.float64)) > np.abs(x32.astype(np.float64))
    hb = np.where(over, hb - 1, hb)                  # one magnitude down: toward zero
    return hb.astype(np.uint16)


def _value(bits, dtype: str) -> np.ndarray:
    if dtype == "bf16":
        return (np.asarray(bits, np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)
    return np.asarray(bits, np.uint16).view(np.float16).astype(np.float64)


def neighbours(x, dtype: str):
    """(lo, hi): the neighbours of the FP32 values x toward and away from zero
    in the 16-bit type, as float64, and the position of x between them in
    units of 2^-16 of the step."""
    x32 = np.ascontiguousarray(x, np.float32)
    lb = _lo_bits(x32, dtype)
    if dtype == "bf16":
        hb = lb + np.uint32(1)
    else:
        hb = (lb.astype(np.int64) + 1).astype(np.uint16)
    lo, hi = _value(lb, dtype), _value(hb, dtype)
    ax = np.abs(x32.astype(np.float64))
    with np.errstate(invalid="ignore", over="ignore"):
        pos = np.floor(65536.0 * (ax - np.abs(lo)) / (np.abs(hi) - np.abs(lo)))
    if dtype == "f16":
        sat = (lb & np.uint16(0x7FFF)) >= np.uint16(0x7BFF)
        pos = np.where(sat, 0.0, pos)
        hi = np.where(sat, lo, hi)
    return lo, hi, pos


def sr_round(x, r16, dtype: str) -> np.ndarray:
    """Stochastic rounding of FP32 values x with 16 random bits r16 each:
    float64 values of the chosen 16-bit neighbours."""
    lo, hi, pos = neighbours(x, dtype)
    return np.where(pos > np.asarray(r16, np.float64), hi, lo)


def adam_lowp(stored, grad, m, v, lr, beta1, beta2, eps, step, dtype: str, seed: int, index0: int = 0):
    """One Adam step (the pinned FP64 oracle, Kingma & Ba) of a parameter kept
    only in the 16-bit type: from the stored values, the FP64 result rounded to
    FP32, then stochastically to the type with the bits of elements index0 +
    0, 1, ... (the flat element index of the tensor). m and v (float64) are
    updated in place; returns the new stored values (float64 values of the
    type)."""
    p = np.array(stored, dtype=np.float64)
    orc.adam(p, np.asarray(grad, np.float64), m, v, lr, beta1, beta2, eps, step)
    x32 = p.astype(np.float32).reshape(-1)
    e = np.uint64(index0) + np.arange(x32.size, dtype=np.uint64)
    return sr_round(x32, sr_bits16(seed, step, e), dtype).reshape(p.shape)
