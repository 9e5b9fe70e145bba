"""Pins of the oracle against things other than itself: library routines,
closed forms, brute force on tiny inputs, format specifications and
invariants.  CPU only."""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.special as sp

import mpinputs as I
from oracle import chol as C
from oracle import formats as F
from oracle import matern as M

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- formats ---

def _spread(rng, n, lo, hi):
    mag = np.exp2(rng.uniform(lo, hi, n))
    return mag * rng.choice([-1.0, 1.0], n)


def test_round_f32_matches_numpy():
    rng = np.random.default_rng(0)
    x = np.concatenate([_spread(rng, 20000, -160, 130), [0.0, -0.0, 3.4028235e38 * 1.0000001]])
    assert np.array_equal(F.round_to(x, F.F32), x.astype(np.float32).astype(np.float64))


def test_round_f16_matches_numpy():
    rng = np.random.default_rng(1)
    x = np.concatenate([_spread(rng, 20000, -30, 17), [65519.0, 65520.0, 1e-9]])
    with np.errstate(over="ignore"):
        ref = x.astype(np.float16).astype(np.float64)
    assert np.array_equal(F.round_to(x, F.F16), ref)


def test_round_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    x = _spread(rng, 20000, -140, 127).astype(np.float32).astype(np.float64)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(F.round_to(x, F.BF16), ref)


def test_round_e4m3_matches_torch_in_range():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = _spread(rng, 20000, -12, 8.8).astype(np.float32).astype(np.float64)
    x = x[np.abs(x) <= 448.0]
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(F.round_to(x, F.E4M3), ref)


def test_e4m3_codes_fixed_points_and_midpoints():
    torch = pytest.importorskip("torch")
    codes = torch.arange(256, dtype=torch.uint8).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    finite = codes[np.isfinite(codes)]
    assert np.array_equal(F.round_to(finite, F.E4M3), finite)
    pos = np.unique(finite[finite >= 0])
    mids = 0.5 * (pos[:-1] + pos[1:])
    got = F.round_to(mids, F.E4M3)
    # a tie goes to the neighbour whose last fraction bit is 0 (even code)
    bits = torch.from_numpy(pos.astype(np.float32)).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    even_lo = (bits[:-1] & 1) == 0
    assert np.array_equal(got, np.where(even_lo, pos[:-1], pos[1:]))


def test_e4m3_landmarks_and_saturation():
    vals = dict(l.split() for l in open(os.path.join(GOLDEN, "e4m3_landmarks.txt"))
                if l.strip() and not l.startswith("#"))
    vals = {k: float(v) for k, v in vals.items()}
    assert F.round_to(vals["max_normal"], F.E4M3) == 448.0
    assert F.round_to(1e6, F.E4M3) == 448.0 and F.round_to(-1e6, F.E4M3) == -448.0
    assert F.round_to(464.0, F.E4M3) == 448.0          # beyond max: saturate, no inf
    assert F.round_to(vals["min_subnormal"], F.E4M3) == vals["min_subnormal"]
    assert F.round_to(vals["min_subnormal"] * 0.5, F.E4M3) == 0.0  # tie to even (zero)
    assert F.round_to(vals["min_subnormal"] * 0.51, F.E4M3) == vals["min_subnormal"]
    assert F.round_to(vals["max_subnormal"], F.E4M3) == vals["max_subnormal"]
    assert F.round_to(vals["min_normal"], F.E4M3) == vals["min_normal"]
    assert F.round_to(1.0625, F.E4M3) == 1.0                        # tie to even
    assert F.round_to(1.1875, F.E4M3) == 1.25                       # tie to even
    assert F.round_to(vals["one_plus_ulp"], F.E4M3) == 1.125


def test_overflow_to_inf_for_ieee_formats():
    assert F.round_to(1e39, F.F32) == np.inf
    assert F.round_to(-1e39, F.BF16) == -np.inf
    assert F.round_to(65520.0, F.F16) == np.inf
    assert F.round_to(65519.0, F.F16) == 65504.0


@pytest.mark.parametrize("amax", [448.0, 449.0, 1.0, 1e-3, 3.7e5, 2.0 ** -30, 0.0])
def test_e4m3_scale_is_smallest_power_of_two(amax):
    s = F.e4m3_scale(amax)
    assert s == 2.0 ** round(math.log2(s))
    if amax > 0:
        assert amax / s <= 448.0 < amax / (s / 2)
    else:
        assert s == 1.0


# ----------------------------------------------------------------- matern ---

@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_matern_closed_form_matches_bessel_definition(nu):
    a, s2 = 0.07, 1.7
    x = np.array([0.01, 0.3, 1.0, 2.7, 9.5])
    ref = s2 * x ** nu * sp.kv(nu, x) / (2.0 ** (nu - 1.0) * sp.gamma(nu))
    got = M.matern_closed(x * a, nu, a, s2)
    assert np.allclose(got, ref, rtol=1e-14, atol=0)


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_matern_general_reduces_to_closed_forms(nu):
    a, s2 = 0.07, 1.7
    r = np.array([0.0, 1e-9, 0.002, 0.03, 0.2, 0.9])
    assert np.allclose(M.matern_general(r, nu, a, s2), M.matern_closed(r, nu, a, s2), rtol=1e-13, atol=0)


@pytest.mark.parametrize("nu", [0.3, 1.0, 2.2])
def test_matern_general_matches_integral_representation(nu):
    """K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt, by adaptive
    quadrature (independent of the library Bessel routine), and the r -> 0
    limit sigma^2."""
    from scipy.integrate import quad
    a, s2 = 0.05, 1.3
    for x in (0.05, 0.7, 3.0, 11.0):
        tmax = math.acosh(800.0 / x) + 1.0          # the integrand is below e^-800 beyond
        k, _ = quad(lambda t: math.exp(-x * math.cosh(t)) * math.cosh(nu * t), 0, tmax,
                    epsabs=0, epsrel=1e-13, limit=200)
        want = s2 * 2.0 ** (1.0 - nu) / math.gamma(nu) * x ** nu * k
        assert math.isclose(float(M.matern_general(x * a, nu, a, s2)), want, rel_tol=1e-10)
    assert float(M.matern_general(0.0, nu, a, s2)) == s2
    assert math.isclose(float(M.matern_general(1e-12 * a, nu, a, s2)), s2, rel_tol=1e-6)


def test_matern_landmarks():
    a, s2 = 0.05, 1.3
    e = math.exp(-1.0)
    assert M.matern_closed(0.0, 0.5, a, s2) == s2
    assert M.matern_closed(0.0, 2.5, a, s2) == s2
    assert math.isclose(M.matern_closed(a, 0.5, a, s2), s2 * e, rel_tol=1e-15)
    assert math.isclose(M.matern_closed(a, 1.5, a, s2), 2 * s2 * e, rel_tol=1e-15)
    assert math.isclose(M.matern_closed(a, 2.5, a, s2), 7.0 / 3.0 * s2 * e, rel_tol=1e-15)


def test_covariance_symmetric_with_nugget():
    locs = I.points(50, 5)
    S = M.covariance(locs, 1.5, 0.1, 2.0, 1e-4)
    assert np.array_equal(S, S.T)
    assert np.allclose(np.diag(S), 2.0 + 1e-4, rtol=0, atol=0)
    r = np.hypot(locs[3, 0] - locs[7, 0], locs[3, 1] - locs[7, 1]) / 0.1
    assert math.isclose(S[3, 7], 2.0 * (1 + r) * math.exp(-r), rel_tol=1e-14)


def test_morton_order_matches_z_curve():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "morton_4x4.txt"))
            if l.strip() and not l.startswith("#")]
    expect = [(int(x), int(y)) for x, y in rows]
    cells = list(itertools.product(range(4), range(4)))
    rng = np.random.default_rng(0)
    rng.shuffle(cells)
    locs = (np.array(cells, dtype=np.float64) + 0.5) / 4.0
    srt, perm = M.morton_order(locs)
    got = [tuple(int(v) for v in np.floor(p * 4)) for p in srt]
    assert got == expect
    assert np.array_equal(srt, locs[perm])


def test_morton_ties_keep_index_order_and_edges():
    locs = np.array([[0.5, 0.5], [0.0, 0.0], [0.5, 0.5], [1.0, 1.0], [0.5, 0.5]])
    _, perm = M.morton_order(locs)
    assert list(perm) == [1, 0, 2, 4, 3]
    assert M.morton_keys(np.array([[1.0, 1.0]]))[0] == 0xFFFFFFFF


# ------------------------------------------------------------------- chol ---

def _spd(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, n))
    return X @ X.T + n * np.eye(n)


def test_textbook_cholesky_matches_lapack():
    A = _spd(60, 4)
    L, info = C.potrf_textbook(A)
    assert info == 0
    assert np.allclose(L, np.linalg.cholesky(A), rtol=1e-13, atol=1e-13)


def test_textbook_cholesky_reports_first_bad_pivot():
    A = np.diag([4.0, 1.0, 2.0, 3.0, 5.0, -1.0, 2.0])
    _, info = C.potrf_textbook(A)
    assert info == 6
    A = _spd(8, 1)
    A[3, 3] = np.nan
    assert C.potrf_textbook(A)[1] == 4


def _det_cofactor(A):
    n = len(A)
    if n == 1:
        return A[0][0]
    return sum((-1) ** c * A[0][c] * _det_cofactor([row[:c] + row[c + 1:] for row in A[1:]])
               for c in range(n))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 6])
def test_exact_loglik_brute_force(n):
    A = _spd(n, 10 + n)
    z = np.random.default_rng(n).standard_normal(n)
    Al = A.tolist()
    det = _det_cofactor(Al)
    # explicit inverse from cofactors: inv[j][i] = (-1)^(i+j) det(minor_ij) / det
    inv = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            minor = [row[:j] + row[j + 1:] for k, row in enumerate(Al) if k != i]
            inv[j, i] = (-1) ** (i + j) * (_det_cofactor(minor) if minor else 1.0) / det
    quad = float(z @ inv @ z)
    for method in ("lapack", "textbook"):
        r = C.exact_loglik(A, z, method)
        assert math.isclose(r["logdet"], math.log(det), rel_tol=1e-12, abs_tol=1e-12)
        assert math.isclose(r["quad"][0], quad, rel_tol=1e-12)
        ll = -0.5 * n * math.log(2 * math.pi) - 0.5 * math.log(det) - 0.5 * quad
        assert math.isclose(r["loglik"][0], ll, rel_tol=1e-12)


def _ar1(n, h, a, s2, z):
    rho = math.exp(-h / a)
    logdet = n * math.log(s2) + (n - 1) * math.log(1 - rho * rho)
    quad = (z[0] ** 2 + np.sum((z[1:] - rho * z[:-1]) ** 2) / (1 - rho * rho)) / s2
    return logdet, quad


@pytest.mark.parametrize("n,b", [(200, 64), (256, 64), (130, 32)])
def test_ar1_closed_form_end_to_end(n, b):
    """nu = 1/2 Matérn on equally spaced 1-D points is AR(1): generator,
    tiled Cholesky, solve and log-likelihood pinned in closed form."""
    h, a, s2 = 1.0 / n, 0.1, 1.3
    locs = I.points_line(n, h)
    z = I.rhs(n, 1, 3)[:, 0]
    S = M.covariance(locs, 0.5, a, s2, 0.0)
    logdet, quad = _ar1(n, h, a, s2, z)
    ex = C.exact_loglik(S, z)
    assert math.isclose(ex["logdet"], logdet, rel_tol=1e-11)
    assert math.isclose(ex["quad"][0], quad, rel_tol=1e-11)
    nt = -(-n // b)
    tl = C.tiled_loglik(S, z, b, I.uniform_map(nt, I.F64))
    assert math.isclose(tl["logdet"], logdet, rel_tol=1e-11)
    assert math.isclose(tl["quad"][0], quad, rel_tol=1e-11)
    ll = -0.5 * n * math.log(2 * math.pi) - 0.5 * logdet - 0.5 * quad
    assert math.isclose(tl["loglik"][0], ll, rel_tol=1e-12)


@pytest.mark.parametrize("far", [I.F32, I.BF16, I.F16, I.E4M3])
def test_diagonal_matrix_exact_with_any_map(far):
    n, b = 100, 32
    d = np.random.default_rng(7).uniform(0.5, 3.0, n)
    z = I.rhs(n, 2, 8)
    nt = -(-n // b)
    tl = C.tiled_loglik(np.diag(d), z, b, I.band_map(nt, I.F64, I.F32, far, 1))
    assert math.isclose(tl["logdet"], float(np.sum(np.log(d))), rel_tol=1e-13)
    assert np.allclose(tl["quad"], np.sum(z * z / d[:, None], axis=0), rtol=1e-13)


def test_tiled_fp64_matches_exact_and_reconstructs():
    n, b = 300, 64     # ragged: 5 tiles, last one padded
    locs = I.points(n, 4)
    S = M.covariance(locs, 1.5, 0.1, 1.0, 1e-4)
    z = I.rhs(n, 3, 4)
    ex = C.exact_loglik(S, z)
    tl = C.tiled_loglik(S, z, b, I.uniform_map(5, I.F64))
    assert np.allclose(tl["loglik"], ex["loglik"], rtol=1e-12, atol=0)
    L = tl["T"].dense_lower()[:n, :n]
    assert np.linalg.norm(L @ L.T - S) / np.linalg.norm(S) <= 4 * n * C.U64
    assert np.allclose(L, ex["L"], rtol=0, atol=1e-10)


def test_kind_rule_table():
    k = C.kind_of
    assert k(I.F64, I.F32, I.F32) == I.F32          # SYRK into FP64 at operand precision
    assert k(I.F64, I.BF16, I.BF16) == I.BF16
    assert k(I.F32, I.F32, I.BF16) == I.F32         # highest operand wins below the target
    assert k(I.F32, I.BF16, I.BF16) == I.BF16
    assert k(I.BF16, I.F32, I.BF16) == I.BF16       # capped by the target
    assert k(I.E4M3, I.F32, I.E4M3) == I.E4M3
    assert k(I.F32, I.E4M3, I.E4M3) == I.E4M3
    assert k(I.F32, I.BF16, I.F16) == I.F32
    assert k(I.F64, I.F64, I.F64) == I.F64


def _mixed_errors(n=512, b=64, seed=9):
    # exponential kernel (nu = 1/2, range 0.1): every map below stays SPD
    locs, _ = M.morton_order(I.points(n, seed))
    S = M.covariance(locs, 0.5, 0.1, 1.0, 1e-4)
    z = I.rhs(n, 1, seed)
    ex = C.exact_loglik(S, z)
    nt = n // b
    errs = {}
    for name, pm in [("f64", I.uniform_map(nt, I.F64)),
                     ("f32", I.band_map(nt, I.F64, I.F32, I.F32, 2)),
                     ("bf16", I.band_map(nt, I.F64, I.F32, I.BF16, 2)),
                     ("e4m3", I.band_map(nt, I.F64, I.F32, I.E4M3, 2))]:
        tl = C.tiled_loglik(S, z, b, pm)
        errs[name] = abs(tl["loglik"][0] - ex["loglik"][0]) / abs(ex["loglik"][0])
    return errs


def test_mixed_maps_error_ordering():
    e = _mixed_errors()
    assert e["f64"] < 1e-12
    assert e["f64"] <= e["f32"] <= e["bf16"] <= e["e4m3"]
    assert e["f32"] < 1e-6 and e["e4m3"] < 1e-1


def test_band_bf16_map_loses_definiteness_on_smooth_kernel():
    """nu = 3/2, range 0.05, nugget 1e-4: far tiles in Morton order still hold
    correlations near 1, and rounding them to BF16 perturbs Sigma by more
    than its smallest eigenvalue; the oracle reports the failing row."""
    n, b = 1024, 128
    locs, _ = M.morton_order(I.points(n, 9))
    S = M.covariance(locs, 1.5, 0.05, 1.0, 1e-4)
    T = C.tiled_from_dense(S, b, I.band_map(n // b, I.F64, I.F32, I.BF16, 2))
    with pytest.raises(np.linalg.LinAlgError):
        C.tiled_cholesky(T)
    assert T.info > 0


def test_refinement_recovers_exact_quad():
    n, b = 384, 64
    locs, _ = M.morton_order(I.points(n, 12))
    S = M.covariance(locs, 0.5, 0.1, 1.0, 1e-4)
    z = I.rhs(n, 4, 12)
    ex = C.exact_loglik(S, z)
    nt = n // b
    T = C.tiled_cholesky(C.tiled_from_dense(S, b, I.band_map(nt, I.F64, I.F32, I.BF16, 2)))
    x, iters, rnorm = C.refine(T, S, z, 10)
    assert np.all(iters < 10)
    snorm = np.max(np.sum(np.abs(S), axis=1))
    r = z - S @ x
    # converged columns meet the stopping rule with the pre-update iterate,
    # and the final update only shrinks the residual further
    assert np.all(np.max(np.abs(r), axis=0) <= 4 * n * C.U64 * (snorm * np.max(np.abs(x), axis=0)
                                                                + np.max(np.abs(z), axis=0)))
    quad = np.sum(z * x, axis=0)
    assert np.allclose(quad, ex["quad"], rtol=1e-11)


def test_gemm_oracle_precisions():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((40, 70))
    B = rng.standard_normal((70, 30))
    ref = A @ B
    assert np.allclose(C.gemm(A, B, np.zeros((40, 30)), F.F64), ref, rtol=1e-14, atol=1e-13)
    a32, b32 = F.round_to(A, F.F32), F.round_to(B, F.F32)
    got = C.gemm(a32, b32, np.zeros((40, 30)), F.F32)
    assert np.max(np.abs(got - a32 @ b32)) <= 70 * 2 ** -23 * np.max(np.abs(a32) @ np.abs(b32))
    ab, bb = F.round_to(A, F.BF16), F.round_to(B, F.BF16)
    got = C.gemm(ab, bb, np.zeros((40, 30)), F.BF16)
    assert np.array_equal(got, F.round_to(got, F.BF16))
    assert np.max(np.abs(got - ab @ bb)) <= 2 ** -8 * np.max(np.abs(ab @ bb)) + 1e-3


# ------------------------------------------- planted mistakes are caught ---

def test_planted_sign_error_in_update_is_caught(monkeypatch):
    real = C.product
    monkeypatch.setattr(C, "product", lambda a, b, kind: -real(a, b, kind))
    with pytest.raises((AssertionError, np.linalg.LinAlgError)):
        test_tiled_fp64_matches_exact_and_reconstructs()


def test_planted_transpose_in_update_is_caught(monkeypatch):
    def transposed(a, bt, kind):
        ca, sa = C.operand_as(a, kind)
        cb, sb = C.operand_as(bt, kind)
        return (ca.T @ cb) * (sa * sb)        # A_ik^T A_jk instead of A_ik A_jk^T
    monkeypatch.setattr(C, "product", transposed)
    with pytest.raises((AssertionError, np.linalg.LinAlgError)):
        test_tiled_fp64_matches_exact_and_reconstructs()


def test_planted_dropped_nugget_is_caught(monkeypatch):
    real = M.covariance
    monkeypatch.setattr(M, "covariance", lambda l, nu, a, s2, tau: real(l, nu, a, s2, 0.0))
    with pytest.raises(AssertionError):
        test_covariance_symmetric_with_nugget()


def test_planted_round_half_away_is_caught(monkeypatch):
    monkeypatch.setattr(np, "rint", lambda v: np.sign(v) * np.floor(np.abs(v) + 0.5))
    with pytest.raises(AssertionError):
        test_e4m3_landmarks_and_saturation()


def test_planted_missing_logdet_factor_is_caught(monkeypatch):
    real = C.step_potrf
    def half(T, k):
        before = T.logdet
        real(T, k)
        T.logdet = before + 0.5 * (T.logdet - before)
    monkeypatch.setattr(C, "step_potrf", half)
    with pytest.raises(AssertionError):
        test_ar1_closed_form_end_to_end(200, 64)


def test_exact_loglik_field_matches_dense_and_ar1():
    """The row-block O-exact for large fields: the same numbers as the dense
    O-exact on a 2-D Matérn field, and the AR(1) closed form on a line."""
    n = 900
    locs, _ = M.morton_order(I.points(n, 6))
    z = I.rhs(n, 3, 6)
    S = M.covariance(locs, 2.5, 0.07, 1.4, 1e-3)
    ref = C.exact_loglik(S, z)
    got = C.exact_loglik_field(locs, 2.5, 0.07, 1.4, 1e-3, z, rows=128, keep_factor=True)
    assert math.isclose(got["logdet"], ref["logdet"], rel_tol=1e-12)
    assert np.allclose(got["loglik"], ref["loglik"], rtol=1e-12)
    assert np.allclose(np.tril(got["L"]), ref["L"], rtol=0, atol=1e-12)
    n, a, s2 = 1000, 0.05, 1.7
    h = 1.0 / n
    rho = math.exp(-h / a)
    z = I.ar1_rhs(n, 2, rho, s2, 9)
    r = C.exact_loglik_field(I.points_line(n, h), 0.5, a, s2, 0.0, z, rows=300)
    for c in range(2):
        logdet, quad = _ar1(n, h, a, s2, z[:, c])
        assert math.isclose(r["logdet"], logdet, rel_tol=1e-11)
        assert math.isclose(r["quad"][c], quad, rel_tol=1e-10)
