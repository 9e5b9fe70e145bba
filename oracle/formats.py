"""Round-to-nearest-even into the tile storage formats, from their definitions.

Oracle (test infrastructure; see oracle/__init__.py).

A binary format with t fraction bits and minimum normal exponent emin holds
the numbers m * 2^(e - t) with |m| < 2^(t+1) integer and e >= emin (Sec. 2,
where the paper defines x = +-m * beta^(e-t+1)).  Rounding a float64 value x
means: find the exponent e of its leading bit (clamped to emin so that
subnormals share the quantum 2^(emin - t)), divide by the quantum (exact: a
power of two), round to the nearest integer with ties to even, multiply back.

Overflow: IEEE 754 round-to-nearest sends results beyond the largest finite
value to +-inf (FP32, BF16, FP16).  The OCP FP8 E4M3 format has no infinity;
conversions use saturation to +-448 ("satfinite").

Per-tile scaling of E4M3 tiles: the tile stores codes c with value c * s,
where s = 2^ceil(log2(amax / 448)) is a power of two (exact), so that
amax / s <= 448; an all-zero tile gets s = 1.
"""
from __future__ import annotations

import numpy as np

F64, F32, BF16, F16, E4M3 = 0, 1, 2, 3, 4

# (fraction bits t, minimum normal exponent emin, largest finite, overflow rule)
_FORMATS = {
    F32: (23, -126, float((2 - 2.0 ** -23) * 2.0 ** 127), "inf"),
    BF16: (7, -126, float((2 - 2.0 ** -7) * 2.0 ** 127), "inf"),
    F16: (10, -14, 65504.0, "inf"),
    E4M3: (3, -6, 448.0, "sat"),
}

E4M3_MAX = 448.0


def round_to(x, fmt: int) -> np.ndarray:
    """Round float64 values to format `fmt` (RNE); returns float64 holding the
    rounded values exactly.  F64 is the identity."""
    x = np.asarray(x, dtype=np.float64)
    if fmt == F64:
        return x.copy()
    t, emin, vmax, ovf = _FORMATS[fmt]
    ax = np.abs(x)
    finite = np.isfinite(ax) & (ax > 0)
    safe = np.where(finite, ax, 1.0)
    _, ex = np.frexp(safe)            # safe = mant * 2^ex, mant in [0.5, 1)
    e = np.maximum(ex - 1, emin)      # exponent of the leading bit, clamped
    q = np.ldexp(1.0, e - t)          # quantum of the binade
    r = np.rint(safe / q) * q         # np.rint: round half to even
    if ovf == "inf":
        r = np.where(r > vmax, np.inf, r)
    else:
        r = np.minimum(r, vmax)
    r = np.where(finite, r, ax)       # 0, inf, nan pass through
    if ovf == "sat":
        r = np.where(np.isinf(ax), vmax, r)
    return np.copysign(r, x)


def e4m3_scale(amax: float) -> float:
    """Power-of-two scale s with amax / s <= 448 (smallest such power)."""
    amax = float(amax)
    if not amax > 0.0:
        return 1.0
    e = int(np.ceil(np.log2(amax / E4M3_MAX)))
    # log2 is called, not trusted: step the exponent until the bound holds.
    while amax / 2.0 ** e > E4M3_MAX:
        e += 1
    while e > -1074 and amax / 2.0 ** (e - 1) <= E4M3_MAX:
        e -= 1
    return float(2.0 ** e)


def quantize(x, fmt: int):
    """Store float64 block `x` in format `fmt`.

    Returns (codes, scale): for E4M3 the codes are the rounded values of x / s
    and the represented values are codes * s; for the other formats the codes
    are the rounded values themselves and scale = 1.
    """
    x = np.asarray(x, dtype=np.float64)
    if fmt == E4M3:
        s = e4m3_scale(np.max(np.abs(x)) if x.size else 0.0)
        return round_to(x / s, E4M3), s
    return round_to(x, fmt), 1.0


def level(fmt: int) -> int:
    """Precision rank used by the update rule: F64 > F32 > 16-bit > E4M3."""
    return {F64: 4, F32: 3, BF16: 2, F16: 2, E4M3: 1}[fmt]


def unit_roundoff(fmt: int) -> float:
    return {F64: 2.0 ** -53, F32: 2.0 ** -24, BF16: 2.0 ** -8, F16: 2.0 ** -11,
            E4M3: 2.0 ** -4}[fmt]
