"""Pins of the oracle's per-step rounding in the tiled factorisation (CPU).

The tiled emulation rounds at three places (right-looking tiled Cholesky
with per-tile formats, the multi-precision extension of Sec. 7, and the
"highest input precision wins" rule of Sec. 4.3 capped by the target):
  * the panel solve X = A_ik L_kk^{-T} is done in float64 and rounded once
    to p(i, k) (E4M3: a new power-of-two scale from amax X);
  * a trailing update runs its product in kind = min(p(target), max(p(A),
    p(B))): operands stored above the kind are rounded to it, products are
    accumulated in FP32 (float64 only for the FP64 kind);
  * the result of the update is rounded once to p(target).

Every expected value below is worked out by hand from those three rules on
2 x 2 tiles, with operands chosen so that each rule changes the result: a
sum whose FP32 accumulation loses a term, an operand that its rounding to
the kind moves, a result that its rounding to the target moves.  Panel
results are checked against exact rational solves rounded by an
independent exact-rational round-to-nearest-even, itself pinned to the
library casts of numpy and torch.  The planted-mistake tests at the end
swap in the two mistakes these pins exist to catch (panel rounding dropped;
the update done as a plain float64 product without kind or target
rounding) and check that the pins fail.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import mpinputs as I
from oracle import chol as C
from oracle import matern as M

torch = pytest.importorskip("torch")

# (fraction bits, minimum normal exponent, largest finite, saturating)
FMT = {I.F32: (23, -126, (2 - Fraction(1, 2 ** 23)) * Fraction(2) ** 127, False),
       I.BF16: (7, -126, (2 - Fraction(1, 2 ** 7)) * Fraction(2) ** 127, False),
       I.F16: (10, -14, Fraction(65504), False),
       I.E4M3: (3, -6, Fraction(448), True)}


def rne(x, fmt):
    """Round a rational to format `fmt`, nearest with ties to even, by exact
    rational arithmetic (no floating point involved)."""
    x = Fraction(x)
    if fmt == I.F64 or x == 0:
        return x
    t, emin, vmax, sat = FMT[fmt]
    ax = abs(x)
    e = ax.numerator.bit_length() - ax.denominator.bit_length()
    while Fraction(2) ** e > ax:
        e -= 1
    while Fraction(2) ** (e + 1) <= ax:
        e += 1
    q = Fraction(2) ** (max(e, emin) - t)
    m = ax / q
    k = m.numerator // m.denominator
    rem = m - k
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and k % 2 == 1):
        k += 1
    r = k * q
    if r > vmax:
        r = vmax if sat else Fraction(10) ** 400     # stands for infinity
    return r if x > 0 else -r


def pow2_scale(amax):
    """Smallest power of two s with amax / s <= 448 (1 for a zero tile)."""
    amax = Fraction(amax)
    if amax == 0:
        return Fraction(1)
    e = 0
    while amax / Fraction(2) ** e > 448:
        e += 1
    while amax / Fraction(2) ** (e - 1) <= 448:
        e -= 1
    return Fraction(2) ** e


# ------------------------------------------- the test's own rounding pinned

def test_exact_rounding_helper_matches_library_casts():
    rng = np.random.default_rng(0)
    x32 = (np.exp2(rng.uniform(-20, 15, 3000)) * rng.choice([-1, 1], 3000)).astype(np.float32)
    x64 = np.exp2(rng.uniform(-130, 120, 3000)) * rng.choice([-1, 1], 3000)
    for v in x64:
        assert float(rne(float(v), I.F32)) == float(np.float32(v))
    for v in x32[np.abs(x32) < 60000]:
        assert float(rne(float(v), I.F16)) == float(np.float16(v))
    tb = torch.from_numpy(x32).to(torch.bfloat16).to(torch.float64).numpy()
    for v, w in zip(x32, tb):
        assert float(rne(float(v), I.BF16)) == w
    small = x32[np.abs(x32) <= 448]
    te = torch.from_numpy(small).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    for v, w in zip(small, te):
        assert float(rne(float(v), I.E4M3)) == w


# ------------------------------------------------------ panel solve (TRSM)

def _tiles(nt, b, pmap, vals, scales=None):
    """A tiled matrix whose tile (i, j) holds the given stored codes."""
    T = C.TiledMatrix(n=nt * b, b=b, nt=nt, pmap=np.asarray(pmap, dtype=np.uint8))
    for key, v in vals.items():
        s = (scales or {}).get(key, 1.0)
        T.tiles[key] = C.Tile(np.array(v, dtype=np.float64), int(pmap[key[0]][key[1]]), s)
    return T


PANEL_ROWS = [[1, 1], [2, -1]]


def _panel_expected(fmt):
    """A_00 = [[9, 3], [3, 10]] has L = [[3, 0], [1, 3]]; the panel rows
    solve x L^T = a exactly: x0 = a0 / 3, x1 = (a1 - x0) / 3."""
    X = []
    for a0, a1 in PANEL_ROWS:
        x0 = Fraction(a0, 3)
        X.append([x0, (a1 - x0) / 3])
    if fmt == I.E4M3:
        s = pow2_scale(max(abs(v) for row in X for v in row))
        return [[rne(v / s, fmt) for v in row] for row in X], s
    return [[rne(v, fmt) for v in row] for row in X], Fraction(1)


@pytest.mark.parametrize("fmt", [I.F32, I.BF16, I.F16, I.E4M3])
def test_panel_solve_is_rounded_once_to_the_tile_format(fmt):
    pmap = [[I.F64, 255], [fmt, I.F64]]
    T = _tiles(2, 2, pmap, {(0, 0): [[9, 0], [3, 10]], (1, 0): PANEL_ROWS,
                            (1, 1): [[1, 0], [0, 1]]})
    C.step_potrf(T, 0)
    assert np.array_equal(T.tiles[(0, 0)].codes, [[3, 0], [1, 3]])
    C.step_trsm(T, 0)
    codes, s = _panel_expected(fmt)
    got = T.tiles[(1, 0)]
    assert got.fmt == fmt
    assert got.scale == float(s)
    assert np.array_equal(got.codes, np.array([[float(v) for v in r] for r in codes]))
    # the rounding is not vacuous: the exact solve is not representable
    assert float(codes[0][0] * s) != 1.0 / 3.0


# --------------------------------------------------- trailing update cases

def _update(pmap, vals, scales=None):
    T = _tiles(3, 2, pmap, vals, scales)
    C.step_update(T, 0)
    return T


def _assert_tile(T, key, codes, scale=1.0):
    t = T.tiles[key]
    assert t.scale == scale, (key, t.scale, scale)
    assert np.array_equal(t.codes, np.array(codes, dtype=np.float64)), (key, t.codes, codes)


Z = [[0, 0], [0, 0]]


def test_update_accumulates_in_fp32():
    """BF16 operands, FP32 target: kind BF16.  1*1 + 2^-15 * 2^-15 =
    1 + 2^-30 is 1 in FP32, so the target 1 + 2^-20 becomes 2^-20 (not
    2^-20 - 2^-30, which FP32 would hold).  The SYRK into the FP64
    diagonal runs at the operand's kind too: 3 - 1 = 2 exactly."""
    pmap = [[I.F64, 255, 255], [I.BF16, I.F64, 255], [I.BF16, I.F32, I.F64]]
    row = [[1, 2.0 ** -15], [0, 0]]
    T = _update(pmap, {(1, 0): row, (2, 0): row, (1, 1): [[3, 0], [0, 2]],
                       (2, 1): [[1 + 2.0 ** -20, 0], [0, 0]], (2, 2): [[5, 0], [0, 1]]})
    _assert_tile(T, (2, 1), [[2.0 ** -20, 0], [0, 0]])
    _assert_tile(T, (1, 1), [[2, 0], [0, 2]])
    _assert_tile(T, (2, 2), [[4, 0], [0, 1]])


def test_update_rounds_operands_stored_above_the_kind():
    """FP32 operand against a BF16 one into a BF16 target: kind BF16, so
    1 + 2^-10 enters as BF16(1 + 2^-10) = 1 and 1 + 2^-6 - 1 = 2^-6 (not
    2^-6 - 2^-10, which BF16 would hold).  SYRK of the FP32 tile into FP64:
    kind FP32, (1 + 2^-10)^2 = 1 + 2^-9 + 2^-20 is exact in FP32."""
    pmap = [[I.F64, 255, 255], [I.F32, I.F64, 255], [I.BF16, I.BF16, I.F64]]
    T = _update(pmap, {(1, 0): [[1 + 2.0 ** -10, 0], [0, 0]], (2, 0): [[1, 0], [0, 0]],
                       (1, 1): [[4, 0], [0, 1]], (2, 1): [[1 + 2.0 ** -6, 0], [0, 0]],
                       (2, 2): [[2, 0], [0, 1]]})
    _assert_tile(T, (2, 1), [[2.0 ** -6, 0], [0, 0]])
    _assert_tile(T, (1, 1), [[3 - 2.0 ** -9 - 2.0 ** -20, 0], [0, 1]])
    _assert_tile(T, (2, 2), [[1, 0], [0, 1]])


def test_update_rounds_the_result_to_the_target():
    """FP32 operands, FP32 target: (1 + 2^-12)^2 = 1 + 2^-11 + 2^-24 lies
    half-way between two FP32 numbers and rounds to even, 1 + 2^-11; the
    target 2 becomes 1 - 2^-11 (exact in FP32), where a float64 product
    would leave 1 - 2^-11 - 2^-24, which FP32 cannot hold."""
    pmap = [[I.F64, 255, 255], [I.F32, I.F64, 255], [I.F32, I.F32, I.F64]]
    row = [[1 + 2.0 ** -12, 0], [0, 0]]
    T = _update(pmap, {(1, 0): row, (2, 0): row, (1, 1): [[3, 0], [0, 1]],
                       (2, 1): [[2, 0], [0, 0]], (2, 2): [[3, 0], [0, 1]]})
    _assert_tile(T, (2, 1), [[1 - 2.0 ** -11, 0], [0, 0]])
    _assert_tile(T, (1, 1), [[2 - 2.0 ** -11, 0], [0, 1]])
    _assert_tile(T, (2, 2), [[2 - 2.0 ** -11, 0], [0, 1]])


def test_update_mixed_16bit_operands_run_in_fp32():
    """BF16 against FP16 below an FP32 target: the two 16-bit formats do not
    contain each other, so both are upcast and the kind is FP32.
    1 + 2^-15 * 2^-14 = 1 + 2^-29 is 1 in FP32: 1 + 2^-21 becomes 2^-21.
    SYRK of each into FP64 at its own kind: the cross terms 2^-28 and 2^-30
    vanish in FP32 as well."""
    pmap = [[I.F64, 255, 255], [I.F16, I.F64, 255], [I.BF16, I.F32, I.F64]]
    T = _update(pmap, {(1, 0): [[1, 2.0 ** -14], [0, 0]], (2, 0): [[1, 2.0 ** -15], [0, 0]],
                       (1, 1): [[5, 0], [0, 1]], (2, 1): [[1 + 2.0 ** -21, 0], [0, 0]],
                       (2, 2): [[6, 0], [0, 1]]})
    _assert_tile(T, (2, 1), [[2.0 ** -21, 0], [0, 0]])
    _assert_tile(T, (1, 1), [[4, 0], [0, 1]])
    _assert_tile(T, (2, 2), [[5, 0], [0, 1]])


def test_update_e4m3_scaled_codes_and_new_scale():
    """E4M3 everywhere below the diagonal.  Codes (2, 3) with scale 2^-4
    and (1.5, 0.5) with 2^-3: the product of the codes is 4.5, times
    2^-7; the target 224 * 2^-6 = 3.5 becomes 3.46484375, whose new scale
    is 2^-7 (3.46484375 / 2^-8 > 448) and whose code 443.5 rounds to 448;
    the entry 2^-6 keeps code 2.  SYRKs into FP64: 1 - 13 * 2^-8 and
    1 - 2.5 * 2^-6."""
    pmap = [[I.F64, 255, 255], [I.E4M3, I.F64, 255], [I.E4M3, I.E4M3, I.F64]]
    T = _update(pmap, {(1, 0): [[2, 3], [0, 0]], (2, 0): [[1.5, 0.5], [0, 0]],
                       (1, 1): [[1, 0], [0, 1]], (2, 1): [[224, 0], [0, 1]],
                       (2, 2): [[1, 0], [0, 1]]},
                scales={(1, 0): 2.0 ** -4, (2, 0): 2.0 ** -3, (2, 1): 2.0 ** -6})
    _assert_tile(T, (2, 1), [[448, 0], [0, 2]], scale=2.0 ** -7)
    _assert_tile(T, (1, 1), [[1 - 13 * 2.0 ** -8, 0], [0, 1]])
    _assert_tile(T, (2, 2), [[1 - 2.5 * 2.0 ** -6, 0], [0, 1]])


UPDATE_PINS = [test_update_accumulates_in_fp32, test_update_rounds_operands_stored_above_the_kind,
               test_update_rounds_the_result_to_the_target,
               test_update_mixed_16bit_operands_run_in_fp32,
               test_update_e4m3_scaled_codes_and_new_scale]


# --------------------------------------------------- guarded precision map

def _matern(n=1000, b=100, seed=3):
    locs, _ = M.morton_order(I.points(n, seed))
    S = M.covariance(locs, 1.5, 0.05, 1.0, 1e-4)
    return S, C.tile_norms(S, b), n // b


@pytest.mark.parametrize("far", [I.BF16, I.E4M3])
def test_guarded_map_threshold_against_dense_norm(far):
    """A far tile (i - j > band) takes the low format exactly when
    u(far) ||A_ij||_F <= eps ||A||_F / NT, with ||A||_F the Frobenius norm of
    the whole symmetric matrix (here from the dense matrix, not from the tile
    norms): on each side of a tile's own threshold the rule must flip it."""
    S, norms, nt = _matern()
    anorm = np.linalg.norm(S)
    u = {I.BF16: 2.0 ** -8, I.E4M3: 2.0 ** -4}[far]
    lo = [(i, j) for i in range(nt) for j in range(i - 2)]
    picks = [lo[k] for k in np.linspace(0, len(lo) - 1, 9).astype(int)]
    for (i, j) in picks:
        thr = u * norms[i, j] * nt / anorm          # eps at which the tile turns low
        assert C.guarded_map(norms, 2, I.F32, far, 1.02 * thr)[i, j] == far
        assert C.guarded_map(norms, 2, I.F32, far, 0.98 * thr)[i, j] == I.F32


@pytest.mark.parametrize("far,eps", [(I.BF16, 1e-5), (I.BF16, 1e-4), (I.E4M3, 1e-3)])
def test_guarded_map_bounds_the_actual_perturbation(far, eps):
    """Rounding every tile the map puts in the low format (both triangles)
    moves Sigma by at most eps ||Sigma||_F."""
    S, norms, nt = _matern()
    b = S.shape[0] // nt
    m = C.guarded_map(norms, 2, I.F32, far, eps)
    E = np.zeros_like(S)
    for i in range(nt):
        for j in range(i):
            if m[i, j] == far:
                blk = S[i * b:(i + 1) * b, j * b:(j + 1) * b]
                if far == I.E4M3:
                    s = float(pow2_scale(Fraction(float(np.max(np.abs(blk))))))
                    q = torch.from_numpy((blk / s).astype(np.float32)).to(torch.float8_e4m3fn)
                    d = q.to(torch.float64).numpy() * s - blk
                else:
                    q = torch.from_numpy(blk.astype(np.float32)).to(torch.bfloat16)
                    d = q.to(torch.float64).numpy() - blk
                E[i * b:(i + 1) * b, j * b:(j + 1) * b] = d
                E[j * b:(j + 1) * b, i * b:(i + 1) * b] = d.T
    assert (m[np.tril_indices(nt, -3)] == far).sum() > 0
    assert np.linalg.norm(E) <= eps * np.linalg.norm(S)


# -------------------------------------------- planted mistakes are caught

def _trsm_unrounded(T, k):
    L = T.tiles[(k, k)].codes
    for i in range(k + 1, T.nt):
        t = T.tiles[(i, k)]
        X = np.linalg.solve(L, t.values().T).T
        T.tiles[(i, k)] = C.Tile(X, t.fmt, 1.0)


def _update_plain_f64(T, k):
    for j in range(k + 1, T.nt):
        for i in range(j, T.nt):
            tgt = T.tiles[(i, j)]
            V = tgt.values() - T.value(i, k) @ T.value(j, k).T
            T.tiles[(i, j)] = C.Tile(V, tgt.fmt, 1.0)


@pytest.mark.parametrize("fmt", [I.F32, I.BF16, I.F16, I.E4M3])
def test_planted_unrounded_panel_solve_is_caught(monkeypatch, fmt):
    monkeypatch.setattr(C, "step_trsm", _trsm_unrounded)
    with pytest.raises(AssertionError):
        test_panel_solve_is_rounded_once_to_the_tile_format(fmt)


@pytest.mark.parametrize("pin", UPDATE_PINS, ids=lambda f: f.__name__[len("test_update_"):])
def test_planted_float64_update_is_caught(monkeypatch, pin):
    monkeypatch.setattr(C, "step_update", _update_plain_f64)
    with pytest.raises(AssertionError):
        pin()


def test_planted_update_without_operand_rounding_is_caught(monkeypatch):
    real = C.operand_as
    monkeypatch.setattr(C, "operand_as",
                        lambda t, kind: (t.values(), 1.0) if t.fmt != kind else real(t, kind))
    with pytest.raises(AssertionError):
        test_update_rounds_operands_stored_above_the_kind()


def test_planted_float64_accumulation_is_caught(monkeypatch):
    def f64_product(a, bt, kind):
        ca, sa = C.operand_as(a, kind)
        cb, sb = C.operand_as(bt, kind)
        return ca @ cb.T * (sa * sb)
    monkeypatch.setattr(C, "product", f64_product)
    with pytest.raises(AssertionError):
        test_update_accumulates_in_fp32()


@pytest.mark.parametrize("mistake", ["no_sqrt", "no_symmetry", "no_nt"])
def test_planted_guarded_map_mistakes_are_caught(monkeypatch, mistake):
    real = C.guarded_map

    def wrong(norms, band, near, far, eps):
        nt = norms.shape[0]
        tot = sum((1.0 if i == j or mistake == "no_symmetry" else 2.0) * norms[i, j] ** 2
                  for i in range(nt) for j in range(i + 1))
        bound = eps * (tot if mistake == "no_sqrt" else math.sqrt(tot)) / (1 if mistake == "no_nt" else nt)
        m = real(norms, band, near, far, eps)
        u = {I.BF16: 2.0 ** -8, I.E4M3: 2.0 ** -4}[far]
        for i in range(nt):
            for j in range(i - band):
                m[i, j] = far if u * norms[i, j] <= bound else near
        return m
    monkeypatch.setattr(C, "guarded_map", wrong)
    with pytest.raises(AssertionError):
        test_guarded_map_threshold_against_dense_norm(I.BF16)
