"""CPU checks of two arithmetic claims the GPU kernels rest on.

1. Ozaki digits of W (Sec. 4.3 leaves the TRSM method open; the panel solve
   multiplies by W = L_kk^{-T} split into S = 8 signed 6-bit digits): the
   balanced base-64 digits of N = rint(v 2^48) represent exactly the value
   that S successive steps d = rint(64 r), r = 64 r - d represent, with
   |d_0| <= 64 and |d_q| <= 32 for q >= 1 -- so the integer split changes
   nothing the error bound depends on.
2. e^{-x} by Tang's table-driven method (ACM TOMS 15, 1989), as the
   generation kernel evaluates it: 2^{j/64} as a double plus its remainder,
   ln2/64 as a 37-bit head plus its remainder, degree-5 Taylor polynomial on
   |r| <= ln2/128, one final rounding: within 0.8 ulp of e^{-x}.

Both re-state the kernels' integer / floating-point steps in Python (fused
multiply-adds as exact rationals rounded once) and compare them with their
mathematical definitions.
"""
import math
import random
import struct
from fractions import Fraction as F

import numpy as np
import pytest

S = 8


def _seq_digits(v):
    d = []
    for _ in range(S):
        t = v * 64.0
        r = float(np.rint(t))
        v = t - r
        d.append(int(r))
    return d


def _int_digits(v):
    n = int(np.rint(v * 2.0 ** 48))       # round half to even, as __double2ll_rn
    d = [0] * S
    m = n
    for q in range(S - 1, 0, -1):
        dq = ((m + 32) & 63) - 32
        d[q] = dq
        m = (m - dq) >> 6
    d[0] = m
    return d, n


def _value(d):
    return sum(F(x) / F(64) ** (i + 1) for i, x in enumerate(d))


def test_integer_digit_split_represents_the_sequential_value():
    rng = random.Random(7)
    vals = [rng.uniform(-1, 1) for _ in range(20000)]
    vals += [rng.uniform(-1, 1) * 2.0 ** -rng.randint(0, 60) for _ in range(10000)]
    # ties at the last digit and the ends of the range
    vals += [1.0, -1.0, 0.0, 0.5, 2.0 ** -49, 3 * 2.0 ** -49, -(2.0 ** -49), 1 - 2.0 ** -53]
    for v in vals:
        a = _seq_digits(v)
        b, n = _int_digits(v)
        assert _value(a) == _value(b) == F(n, 2 ** 48), (v, a, b)
        assert abs(b[0]) <= 64 and all(abs(x) <= 32 for x in b[1:]), (v, b)
        assert abs(a[0]) <= 64 and all(abs(x) <= 32 for x in a[1:]), (v, a)


def _fma(a, b, c):
    return float(F(a) * F(b) + F(c))


def _tables():
    if np.finfo(np.longdouble).nmant < 60:
        pytest.skip("long double without extended precision on this host")
    ld = np.longdouble
    tab = [0.0] * 131
    for j in range(64):
        v = np.exp2(ld(j) / ld(64))
        h = float(v)
        tab[j] = h
        tab[64 + j] = float(v - ld(h))
    ln = np.log(ld(2)) / ld(64)
    head = float(ln)
    u = struct.unpack("<Q", struct.pack("<d", head))[0] & ~0xFFFF
    head = struct.unpack("<d", struct.pack("<Q", u))[0]
    tab[128] = head
    tab[129] = float(ln - ld(head))
    tab[130] = float(ld(64) / np.log(ld(2)))
    return tab


def _exp_neg(x, tab):
    shifter = 6755399441055744.0
    t = _fma(-x, tab[130], shifter)
    k = struct.unpack("<q", struct.pack("<d", t))[0] & 0xFFFFFFFF
    k = k - (1 << 32) if k >= (1 << 31) else k
    kd = t - shifter
    r = _fma(-kd, tab[129], _fma(-kd, tab[128], -x))
    q = _fma(r, _fma(r, _fma(r, 1.0 / 120.0, 1.0 / 24.0), 1.0 / 6.0), 0.5)
    p = _fma(r * r, q, r)
    m, j = k >> 6, k & 63
    th = tab[j]
    v = th + _fma(th, p, tab[64 + j])
    return math.ldexp(v, m)


def test_tang_exp_within_0p8_ulp():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    tab = _tables()
    assert _exp_neg(0.0, tab) == 1.0
    rng = random.Random(1)
    xs = [rng.uniform(0, 1) for _ in range(800)] + [rng.uniform(0, 40) for _ in range(800)]
    xs += [rng.uniform(0, 700) for _ in range(400)] + [i * math.log(2) / 128 for i in range(200)]
    worst = 0.0
    for x in xs:
        got = _exp_neg(x, tab)
        ref = mpmath.exp(-mpmath.mpf(x))
        worst = max(worst, float(abs(mpmath.mpf(got) - ref) / np.spacing(float(ref))))
    assert worst < 0.8, worst
