"""Parity of the CUDA path (through the C ABI) with the oracle.

Tolerances follow from the arithmetic:
  * integer work (Morton permutation) is bit-exact;
  * a value rounded into a storage format may differ by one unit in the last
    place of that format when the float64 inputs differ in their last bits
    (CUDA's exp vs libm's) or when the FP32 accumulation order differs (tensor
    core / CUDA core order vs BLAS order);
  * FP32 accumulations differ by at most ~K 2^-24 sum|a||b|;
  * float64 steps agree to a few units of 2^-53 times the condition growth.
"""
import math

import numpy as np
import pytest

import mpinputs as I
from oracle import chol as OC
from oracle import formats as OF
from oracle import matern as OM

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_02701_gb300 import mpchol
    return mpchol.Context(0)


DEV = "cuda:0"
T_BITS = {I.F64: 52, I.F32: 23, I.BF16: 7, I.F16: 10, I.E4M3: 3}
EMIN = {I.F64: -1022, I.F32: -126, I.BF16: -126, I.F16: -14, I.E4M3: -6}


def ulp(x, fmt):
    ax = np.maximum(np.abs(x), 1e-300)
    e = np.maximum(np.floor(np.log2(ax)), EMIN[fmt])
    return np.ldexp(1.0, (e - T_BITS[fmt]).astype(int))


def assert_close_fmt(got, ref, fmt, extra=0.0, ulps=1, frac=1.0, what=""):
    """|got - ref| <= ulps ulp_fmt + extra everywhere; and differing entries
    are at most `frac` of all."""
    d = np.abs(got - ref)
    tol = ulps * ulp(np.maximum(np.abs(got), np.abs(ref)), fmt) + extra
    bad = d > tol
    assert not bad.any(), f"{what}: {bad.sum()} entries off, max excess {(d - tol).max():.3g}"
    if frac < 1.0:
        assert (d > 0).mean() <= frac, f"{what}: {(d > 0).mean():.4f} of entries differ"


def _mk(ctx, n, b, pmap, keep_sigma=False, simt=False, ozaki=False):
    """Panel solves by FP64 substitution unless `ozaki` (the library default)."""
    from paper_2406_02701_gb300 import mpchol
    return mpchol.TiledMatrix(ctx, n, b, pmap, keep_sigma=keep_sigma, simt_updates=simt, ozaki=ozaki)


def _pow2_above(x):
    """Smallest power of two >= x (1 where x == 0)."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(np.where(x > 0, x, 1.0))
    return np.where(x > 0, np.ldexp(1.0, np.where(m == 0.5, e - 1, e)), 1.0)


def _ozaki_digits(fmt):
    """Digits per operand the integer-digit panel product uses for a tile of
    format fmt: the smallest S whose truncation bound
    1024 (1 + (S + 3) / 3) 2^(-6S) is at most 2^-11 of half a unit in the
    last place (2^-p, p significand bits)."""
    p = {I.F32: 24, I.BF16: 8, I.F16: 11, I.E4M3: 4}[fmt]
    s = 1
    while 1024 * (1 + (s + 3) / 3) * 2.0 ** (-6 * s) > 2.0 ** (-11 - p):
        s += 1
    return s


def test_ozaki_digit_rule():
    assert [_ozaki_digits(f) for f in (I.F32, I.BF16, I.F16, I.E4M3)] == [8, 6, 6, 5]


def _ozaki_bound(a, lkk, x, digits=8):
    """Error bound of X = A W, W = L^{-T}, from 6-bit digit splits: digit
    remainders and dropped levels K (1 + (S + 3) / 3) 2^(-6S) sigma_r tau_c,
    float-float level sums S^2 2^-48 |X| (sigma_r, tau_c: powers of two
    bounding row r of A and column c of W)."""
    w = np.linalg.inv(np.tril(lkk)).T
    sig = _pow2_above(np.abs(a).max(axis=1))
    tau = _pow2_above(np.abs(w).max(axis=0))
    k = a.shape[1]
    return (k * (1 + (digits + 3) / 3) * 2.0 ** (-6 * digits) * np.outer(sig, tau)
            + digits ** 2 * 2.0 ** -48 * np.abs(x))


# --------------------------------------------------------------- Morton ----

@pytest.mark.parametrize("n", [1, 5, 1000, 3000, 70000])
def test_morton_order_bit_exact(ctx, n):
    locs = I.points(n, 17)
    if n > 5:
        locs[7] = locs[3]          # a tie: keeps index order
        locs[11] = [1.0, 0.0]      # edges of the quantiser
    srt, perm = OM.morton_order(locs)
    out, dperm = ctx.morton_order(torch.from_numpy(locs).to(DEV))
    assert np.array_equal(dperm.cpu().numpy(), perm)
    assert np.array_equal(out.cpu().numpy(), srt)


# ------------------------------------------------------------ generation ---

ALL_MAP = None


def _mixed_map(nt):
    m = np.full((nt, nt), 255, dtype=np.uint8)
    cyc = [I.F32, I.BF16, I.F16, I.E4M3]
    for i in range(nt):
        m[i, i] = I.F64
        for j in range(i):
            m[i, j] = cyc[(i + 2 * j) % 4]
    return m


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5, 0.3, 1.0, 2.2])
def test_generation_matches_oracle_every_format(ctx, nu):
    n, b = 700, 128              # 6 tiles per side, ragged last tile
    nt = -(-n // b)
    pmap = _mixed_map(nt)
    locs = I.points(n, 5)
    T = _mk(ctx, n, b, pmap)
    dl = torch.from_numpy(locs).to(DEV)
    T.generate(dl, 1.3, 0.08, nu, 1e-4)
    torch.cuda.synchronize()
    ref = OC.tiled_from_dense(OM.covariance(locs, nu, 0.08, 1.3, 1e-4), b, pmap)
    for i in range(nt):
        for j in range(i + 1):
            got, codes, s = T.get_tile(i, j)
            rt = ref.tiles[(i, j)]
            fmt = int(pmap[i, j])
            if i == j:
                got, want = np.tril(got), np.tril(rt.values())
            else:
                want = rt.values()
            if fmt == I.E4M3:
                assert s == rt.scale, (i, j, s, rt.scale)
                assert_close_fmt(codes, rt.codes, fmt, frac=1e-3, what=f"tile {i},{j}")
            elif fmt == I.F64:
                # the GPU forms x = r * fl(1 / range) (one rounding more than the
                # oracle's r / range): |dx| <= 2 ulp(x), carried by exp(-x) as a
                # relative error of 2 x 2^-52, on top of a few roundings
                ri = np.arange(i * b, min((i + 1) * b, n))
                rj = np.arange(j * b, min((j + 1) * b, n))
                d = np.hypot(locs[ri, 0][:, None] - locs[rj, 0][None, :],
                             locs[ri, 1][:, None] - locs[rj, 1][None, :])
                x = np.zeros((b, b))
                x[:len(ri), :len(rj)] = d / 0.08
                tol = (4 + 4 * x) * 2.0 ** -52 * np.abs(want) + 1e-300
                if nu not in (0.5, 1.5, 2.5):
                    # the oracle's K_nu (scipy) is good to a few 1e-14; the
                    # library's table to about 1e-15 (pinned on the CPU
                    # against forty-digit values)
                    tol = tol + 1e-13 * np.abs(want)
                if i == j:
                    tol = np.tril(tol)
                assert np.all(np.abs(got - want) <= tol), (i, j, np.max(np.abs(got - want) - tol))
            else:
                assert_close_fmt(got, want, fmt, frac=1e-3, what=f"tile {i},{j}")


def _exact_entry(p, q, s2d, nu, a, sigma2):
    """sigma^2 P(x) e^{-x}, x = sqrt(s2d) / a, in 40-digit decimal arithmetic
    from the float64 squared distance s2d (the closed forms of Sec. 6.2)."""
    import decimal
    with decimal.localcontext() as dc:
        dc.prec = 40
        x = decimal.Decimal(s2d).sqrt() / decimal.Decimal(a)
        poly = {0.5: decimal.Decimal(1), 1.5: 1 + x, 2.5: 1 + x + x * x / 3}[nu]
        return decimal.Decimal(sigma2) * poly * (-x).exp()


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
@pytest.mark.parametrize("a", [0.013, 0.3])
def test_float64_entries_within_0p6_ulp(ctx, nu, a):
    """Float64 tile entries of the closed forms (evaluated in 64-bit fixed
    point from the float64 squared distance s^2 = fma(dx, dx, dy dy)) lie
    within 0.55 + x/128 units in the last place of the exact value of
    sigma^2 P(x) e^{-x} at that s^2 -- the final rounding, a few units of
    2^-63 from the products, and x's own error (at most 8 units of 2^-63
    relative) carried x-fold by e^{-x}: 3000 sampled entries, s^2 rebuilt
    exactly with rationals (the fma's one rounding), the rest in 40 digits.
    Near-duplicate points and x up to about 240 included."""
    from fractions import Fraction
    n, b = 1000, 128
    nt = -(-n // b)
    pmap = np.full((nt, nt), I.F64, dtype=np.int32)
    locs = I.points(n, 21)
    locs[5] = locs[200] + 1e-9
    locs[130] = locs[300] + np.array([3e-7, -2e-7])
    sigma2, nugget = 1.3, 1e-4
    T = _mk(ctx, n, b, pmap, keep_sigma=True)
    T.generate(torch.from_numpy(locs).to(DEV), sigma2, a, nu, nugget)
    torch.cuda.synchronize()
    tiles = {}
    rng = np.random.default_rng(5)
    pairs = [(5, 200), (200, 5), (300, 130), (7, 7)]
    while len(pairs) < 3000:
        i, j = rng.integers(0, n, 2)
        pairs.append((max(i, j), min(i, j)))
    worst = 0.0
    for i, j in pairs:
        i, j = max(i, j), min(i, j)
        key = (i // b, j // b)
        if key not in tiles:
            tiles[key] = T.get_tile(*key)[0]
        got = tiles[key][i % b, j % b]
        if i == j:
            want = Fraction(sigma2) + Fraction(nugget)
            assert got == float(want)
            continue
        dx, dy = locs[i, 0] - locs[j, 0], locs[i, 1] - locs[j, 1]
        s2 = float(Fraction(dx) * Fraction(dx) + Fraction(dy * dy))   # fma: one rounding
        ref = _exact_entry(i, j, s2, nu, a, sigma2)
        e = math.frexp(float(ref))[1]
        err = abs(Fraction(got) - Fraction(ref)) / Fraction(2) ** (e - 53)
        x = math.sqrt(s2) / a
        worst = max(worst, float(err) - x / 128)
    assert worst <= 0.55, worst


@pytest.mark.parametrize("nu,a,keep", [(0.5, 1e-3, True)])
def test_generation_far_tail_every_format(ctx, nu, a, keep):
    """A range so short that x = r / a runs to about 1400 on the unit square:
    entries leave the fixed-point path for float64 (x > 700, or a result
    below the normal range), FP32 / BF16 / FP16 values fall below their
    normal range into subnormals and zeros, E4M3 tiles take their scale from
    amaxes down to zero -- every format against the oracle's rounding."""
    n, b = 700, 128
    nt = -(-n // b)
    pmap = _mixed_map(nt)
    locs = I.points(n, 15)
    T = _mk(ctx, n, b, pmap, keep_sigma=keep)
    T.generate(torch.from_numpy(locs).to(DEV), 1.3, a, nu, 1e-4)
    torch.cuda.synchronize()
    ref = OC.tiled_from_dense(OM.covariance(locs, nu, a, 1.3, 1e-4), b, pmap)
    for i in range(nt):
        for j in range(i + 1):
            got, codes, s = T.get_tile(i, j)
            rt = ref.tiles[(i, j)]
            fmt = int(pmap[i, j])
            want = rt.values()
            if i == j:
                got, want = np.tril(got), np.tril(want)
            if fmt == I.E4M3:
                assert s == rt.scale, (i, j, s, rt.scale)
                assert_close_fmt(codes, rt.codes, fmt, frac=1e-3, what=f"tile {i},{j}")
            elif fmt == I.F64:
                ri = np.arange(i * b, min((i + 1) * b, n))
                rj = np.arange(j * b, min((j + 1) * b, n))
                d = np.hypot(locs[ri, 0][:, None] - locs[rj, 0][None, :],
                             locs[ri, 1][:, None] - locs[rj, 1][None, :])
                x = np.zeros((b, b))
                x[:len(ri), :len(rj)] = d / a
                # relative (4 + 4x) ulps as in the moderate-range test; beyond
                # x = 708 e^{-x} is subnormal before it is multiplied by
                # sigma^2 P(x) (in the oracle, and in the kernel's float64
                # evaluation past x = 700), so each carries up to
                # sigma^2 P(x) 2^-1074 of absolute error
                poly = {0.5: 1.0 + 0 * x, 1.5: 1.0 + x, 2.5: 1.0 + x + x * x / 3.0}[nu]
                tol = (4 + 4 * x) * 2.0 ** -52 * np.abs(want) + 2.0 ** -1070 + 4 * 1.3 * poly * 2.0 ** -1074
                if i == j:
                    tol = np.tril(tol)
                assert np.all(np.abs(got - want) <= tol), (i, j, np.max(np.abs(got - want) - tol))
            else:
                assert_close_fmt(got, want, fmt, frac=1e-3, what=f"tile {i},{j}")
    # the range is short enough that tiles hold values beyond the fixed-point
    # path and below FP32's normal range
    dmax = np.max(OM.distances(locs, locs))
    assert dmax / a > 700


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
@pytest.mark.parametrize("a", [0.013, 0.05, 0.3])
def test_float_float_generation(ctx, nu, a):
    """Without a float64 copy of Sigma, tiles stored in FP32, BF16 or FP16
    are evaluated in float-float on the FP32 pipe: every value within one
    unit of the oracle's rounding, at most 1e-4 of them one unit apart; and
    the same against the float64 evaluation the matrix with the copy uses.
    Near-duplicate points and long distances (x up to 80) included."""
    n, b = 900, 128
    nt = -(-n // b)
    pmap = I.band_map(nt, I.F64, I.F32, I.BF16, 2)
    pmap[nt - 1, 0] = I.F16
    locs = I.points(n, 6)
    locs[5] = locs[200] + 1e-9                   # near-duplicate pairs in FP32 tiles
    locs[130] = locs[300] + np.array([3e-7, -2e-7])   # (1, 0) and (2, 1)
    dl = torch.from_numpy(locs).to(DEV)
    T = _mk(ctx, n, b, pmap)
    T.generate(dl, 1.3, a, nu, 1e-4)
    Ts = _mk(ctx, n, b, pmap, keep_sigma=True)
    Ts.generate(dl, 1.3, a, nu, 1e-4)
    torch.cuda.synchronize()
    ref = OC.tiled_from_dense(OM.covariance(locs, nu, a, 1.3, 1e-4), b, pmap)
    for i in range(nt):
        for j in range(i):
            fmt = int(pmap[i, j])
            got = T.get_tile(i, j)[0]
            assert_close_fmt(got, ref.tiles[(i, j)].values(), fmt, frac=1e-4, what=f"tile {i},{j}")
            assert_close_fmt(got, Ts.get_tile(i, j)[0], fmt, frac=1e-4, what=f"paths {i},{j}")


def test_tile_norms_and_guarded_map(ctx):
    n, b = 1500, 128
    nt = -(-n // b)
    locs, _ = OM.morton_order(I.points(n, 14))
    dl = torch.from_numpy(locs).to(DEV)
    got = ctx.tile_norms(n, b, dl, 1.0, 0.05, 1.5, 1e-4).cpu().numpy()
    ref = OC.tile_norms(OM.covariance(locs, 1.5, 0.05, 1.0, 1e-4), b)
    assert np.allclose(got, ref, rtol=1e-12, atol=0)
    for far, eps in [(I.BF16, 1e-5), (I.E4M3, 1e-3), (I.BF16, 1e-7)]:
        m = ctx.map_guarded(got, 2, I.F32, far, eps)
        assert np.array_equal(m, OC.guarded_map(ref, 2, I.F32, far, eps))
        lo = np.tril_indices(nt, -3)
        assert 0 < (m[lo] == far).sum() < len(lo[0]) or eps == 1e-7


# ------------------------------------------------------ one step at a time --

def _load_state(T, state, nt):
    for (i, j), t in state.tiles.items():
        T.set_tile(i, j, t.codes, t.scale)


def _abs_prod(a, bmat):
    return np.abs(a) @ np.abs(bmat).T


@pytest.mark.parametrize("mode", ["tcgen05", "cudacore", "ozaki"])
@pytest.mark.parametrize("far", [I.F32, I.BF16, I.F16, I.E4M3])
def test_single_steps_match_oracle(ctx, far, mode):
    """Load the oracle's state before step k, run step k on the GPU, compare
    every tile the step writes (POTRF, panel TRSM, SYRK/GEMM updates), with
    the trailing updates on the tensor cores or on the CUDA cores.  FP32
    products on the tensor cores are three TF32 products of hi/lo splits;
    each product then carries at most 3 * 2^-22 |a||b| error (the dropped
    lo*lo term and the truncation of the lo parts), within the same
    2 K 2^-24 sum|a||b| bound as FP32 accumulation for K >= 12.  In the
    "ozaki" mode the panel tiles (stored in FP32 or below) are integer-digit
    tensor-core products A L_kk^{-T}, within the bound of _ozaki_bound of
    the float64 solve before their rounding."""
    _single_steps(ctx, 640, 128, far, mode, 0.1)


@pytest.mark.parametrize("mode", ["tcgen05", "ozaki"])
@pytest.mark.parametrize("far", [I.BF16, I.E4M3])
@pytest.mark.parametrize("n,b", [(2048, 512), (3072, 1024)], ids=["b512", "b1024"])
def test_single_steps_match_oracle_large_tiles(ctx, n, b, far, mode):
    """The same step-by-step comparison at the tile sizes of the full-size
    workloads: at b = 512 and 1024 a tensor-core target holds 16 or 64
    128 x 128 units and the products run over K = 512 or 1024 (several
    units per tile, both TMEM accumulators in turn, the wide and the narrow
    integer-digit panel kernels), and the diagonal tiles factor as task
    graphs over 16 x 16 (b = 512) or 32 x 32 (b = 1024) blocks.  Range
    0.05: at 0.1 the E4M3 far tiles of this 2048-point field are no longer
    positive definite after rounding."""
    _single_steps(ctx, n, b, far, mode, 0.05)


def _single_steps(ctx, n, b, far, mode, a):
    simt, ozaki = mode == "cudacore", mode == "ozaki"
    nt = n // b
    pmap = I.band_map(nt, I.F64, I.F32, far, 1)
    locs, _ = OM.morton_order(I.points(n, 21))
    S = OM.covariance(locs, 0.5, a, 1.0, 1e-4)
    state = OC.tiled_from_dense(S, b, pmap)
    T = _mk(ctx, n, b, pmap, simt=simt, ozaki=ozaki)
    for k in range(nt):
        before = {key: OC.Tile(t.codes.copy(), t.fmt, t.scale) for key, t in state.tiles.items()}
        _load_state(T, state, nt)
        T.chol_steps(k, k + 1)
        torch.cuda.synchronize()
        OC.step_potrf(state, k)
        OC.step_trsm(state, k)
        # diagonal factor
        got, _, _ = T.get_tile(k, k)
        want = state.tiles[(k, k)].codes
        assert np.allclose(np.tril(got), np.tril(want), rtol=1e-12, atol=1e-14), f"potrf {k}"
        # panel: float64 solve, rounded once
        for i in range(k + 1, nt):
            got, codes, s = T.get_tile(i, k)
            rt = state.tiles[(i, k)]
            fmt = rt.fmt
            if fmt == I.E4M3:
                assert s == rt.scale
                assert_close_fmt(codes, rt.codes, fmt, frac=2e-3, what=f"trsm {i},{k}")
            else:
                extra = 1e-13 * np.abs(rt.values()).max()
                frac = 2e-3
                if ozaki:
                    ob = _ozaki_bound(before[(i, k)].values(), state.tiles[(k, k)].codes, rt.values(),
                                      _ozaki_digits(fmt))
                    extra = extra + ob
                    # a rounding flips where the exact value lies within the
                    # error of a rounding boundary: at most 2 bound / ulp
                    frac += 2 * np.mean(np.minimum(ob / ulp(rt.values(), fmt), 0.5))
                assert_close_fmt(got, rt.values(), fmt, extra=extra, frac=frac, what=f"trsm {i},{k}")
        # trailing updates, from the panel the GPU wrote: a panel entry that
        # rounded one unit apart (allowed above) must not count against them
        for i in range(k + 1, nt):
            _, codes, sc = T.get_tile(i, k)
            state.tiles[(i, k)] = OC.Tile(codes, state.tiles[(i, k)].fmt, sc)
        OC.step_update(state, k)
        for j in range(k + 1, nt):
            for i in range(j, nt):
                got, codes, s = T.get_tile(i, j)
                rt = state.tiles[(i, j)]
                a, bb = state.tiles[(i, k)], state.tiles[(j, k)]
                kind = OC.kind_of(rt.fmt, a.fmt, bb.fmt)
                u_acc = 2.0 ** -53 if kind == I.F64 else 2.0 ** -24
                bound = 2 * b * u_acc * _abs_prod(a.values(), bb.values())
                want = rt.values()
                if i == j:
                    got, want, bound = np.tril(got), np.tril(want), np.tril(bound)
                if rt.fmt == I.E4M3:
                    # the new scale comes from the amax, identical unless it
                    # straddles a power of two
                    assert s == rt.scale
                assert_close_fmt(got, want, rt.fmt, extra=bound, what=f"update {i},{j} k={k}")
        del before


# ------------------------------------------------------- whole evaluations --

def _run(ctx, n, b, pmap, locs, z, nu, a, s2, tau, refine=0, ozaki=False):
    T = _mk(ctx, n, b, pmap, keep_sigma=refine > 0, ozaki=ozaki)
    dl = torch.from_numpy(locs).to(DEV)
    T.generate(dl, s2, a, nu, tau)
    info, logdet = T.chol()
    zt = torch.from_numpy(np.ascontiguousarray(z.T)).to(DEV)
    ll, quad, iters = T.loglik(zt, refine_iters=refine)
    torch.cuda.synchronize()
    return dict(info=int(info.item()), logdet=logdet.item(), ll=ll.cpu().numpy(),
                quad=quad.cpu().numpy(), iters=iters.cpu().numpy(), T=T)


def test_plain_fp64_n1024_tile128(ctx):
    """FP64 tiled Cholesky + solve + log-det, n=1024, tile 128, Matérn
    nu=1/2, range 0.1, variance 1, nugget 1e-4, uniform points, z ~ N(0,1)."""
    c = I.CONFIGS["fp64_n1024_b128"]
    n, b = c["n"], c["b"]
    for seed in range(1, 6):
        locs = I.points(n, seed)
        z = I.rhs(n, 1, seed)
        S = OM.covariance(locs, c["nu"], c["range"], c["sigma2"], c["nugget"])
        ex = OC.exact_loglik(S, z)
        r = _run(ctx, n, b, None, locs, z, c["nu"], c["range"], c["sigma2"], c["nugget"])
        assert r["info"] == 0
        assert math.isclose(r["logdet"], ex["logdet"], rel_tol=1e-11)
        assert np.allclose(r["ll"], ex["loglik"], rtol=1e-12)
    tl = OC.tiled_loglik(S, z, b, I.uniform_map(n // b, I.F64))
    assert np.allclose(r["ll"], tl["loglik"], rtol=1e-12)
    L = r["T"]
    for i in range(n // b):
        for j in range(i + 1):
            got, _, _ = L.get_tile(i, j)
            want = tl["T"].tiles[(i, j)].codes
            if i == j:
                got, want = np.tril(got), np.tril(want)
            assert np.allclose(got, want, rtol=0, atol=1e-12), (i, j)


@pytest.mark.parametrize("far,refine,ozaki", [(I.F32, 0, False), (I.BF16, 0, False), (I.F16, 0, False),
                                              (I.E4M3, 0, False), (I.BF16, 10, False),
                                              (I.E4M3, 10, False), (I.F32, 0, True), (I.E4M3, 0, True),
                                              (I.BF16, 10, True)])
def test_mixed_loglik_matches_oracle(ctx, far, refine, ozaki):
    n, b = 1000, 128             # ragged: 8 tiles, 24 padding rows
    nt = -(-n // b)
    pmap = I.band_map(nt, I.F64, I.F32, far, 2)
    # exponential kernel; short ranges (the paper's MLE example estimates
    # a ~ 0.03) keep the mixed factor a contraction for refinement
    a = 0.1 if not refine else (0.03 if far == I.BF16 else 0.02)
    locs, _ = OM.morton_order(I.points(n, 31))
    z = I.rhs(n, 3, 31)
    S = OM.covariance(locs, 0.5, a, 1.0, 1e-4)
    ex = OC.exact_loglik(S, z)
    tl = OC.tiled_loglik(S, z, b, pmap, refine_iters=refine)
    r = _run(ctx, n, b, pmap, locs, z, 0.5, a, 1.0, 1e-4, refine=refine, ozaki=ozaki)
    assert r["info"] == 0
    err_gpu = np.abs(r["ll"] - ex["loglik"]) / np.abs(ex["loglik"])
    tol = np.maximum(10 * err_gpu, 1e-9)
    assert np.all(np.abs(r["ll"] - tl["loglik"]) / np.abs(tl["loglik"]) <= tol)
    ld_err = abs(r["logdet"] - ex["logdet"]) / abs(ex["logdet"])
    assert math.isclose(r["logdet"], tl["logdet"], rel_tol=max(1e-9, 10 * ld_err))
    if refine:
        assert np.all(tl["iters"] < refine)          # the oracle converged
        assert np.all(np.abs(r["iters"] - tl["iters"]) <= 1)
        assert np.allclose(r["quad"], ex["quad"], rtol=1e-10)
        assert np.all(err_gpu < 1e-4)


@pytest.mark.parametrize("far,refine,ozaki", [(I.BF16, 10, True), (I.BF16, 10, False), (I.F32, 0, True)])
def test_mixed_loglik_matches_oracle_b384(ctx, far, refine, ozaki):
    """b = 384: the diagonal tiles factor as task graphs over 16 x 16 blocks
    (32 x 32 below b = 384); 6 tiles, 304 padding rows."""
    n, b = 2000, 384
    nt = -(-n // b)
    pmap = I.band_map(nt, I.F64, I.F32, far, 2)
    a = 0.1 if not refine else 0.03
    locs, _ = OM.morton_order(I.points(n, 37))
    z = I.rhs(n, 2, 37)
    S = OM.covariance(locs, 0.5, a, 1.0, 1e-4)
    ex = OC.exact_loglik(S, z)
    tl = OC.tiled_loglik(S, z, b, pmap, refine_iters=refine)
    r = _run(ctx, n, b, pmap, locs, z, 0.5, a, 1.0, 1e-4, refine=refine, ozaki=ozaki)
    assert r["info"] == 0
    err_gpu = np.abs(r["ll"] - ex["loglik"]) / np.abs(ex["loglik"])
    tol = np.maximum(10 * err_gpu, 1e-9)
    assert np.all(np.abs(r["ll"] - tl["loglik"]) / np.abs(tl["loglik"]) <= tol)
    ld_err = abs(r["logdet"] - ex["logdet"]) / abs(ex["logdet"])
    assert math.isclose(r["logdet"], tl["logdet"], rel_tol=max(1e-9, 10 * ld_err))
    if refine:
        assert np.all(tl["iters"] < refine)
        assert np.all(np.abs(r["iters"] - tl["iters"]) <= 1)
        assert np.allclose(r["quad"], ex["quad"], rtol=1e-10)
        assert np.all(err_gpu < 1e-4)


@pytest.mark.parametrize("b,nrhs", [(640, 1), (768, 3), (896, 2)])
def test_refined_loglik_tile_sizes_beyond_512(ctx, b, nrhs):
    """The refinement residual's column groups at tile sizes that are not a
    power of two above 512 (one right-hand side per pass: two groups of
    320 / 384 / 448 columns; two per pass: four groups; nrhs = 3 leaves a
    last pass of one): the refined quadratic forms equal the oracle's
    exact ones, and the iteration counts the oracle's tiled refinement."""
    n = 2000
    nt = -(-n // b)
    pmap = I.band_map(nt, I.F64, I.F32, I.BF16, 1)
    locs, _ = OM.morton_order(I.points(n, 41))
    z = I.rhs(n, nrhs, 41)
    S = OM.covariance(locs, 0.5, 0.03, 1.0, 1e-4)
    ex = OC.exact_loglik(S, z)
    tl = OC.tiled_loglik(S, z, b, pmap, refine_iters=10)
    r = _run(ctx, n, b, pmap, locs, z, 0.5, 0.03, 1.0, 1e-4, refine=10, ozaki=True)
    assert r["info"] == 0
    assert np.all(tl["iters"] < 10)
    assert np.all(np.abs(r["iters"] - tl["iters"]) <= 1)
    assert np.allclose(r["quad"], ex["quad"], rtol=1e-10)


@pytest.mark.parametrize("c", [2.0 ** -40, 2.0 ** 30])
def test_refinement_scale_equivariance(ctx, c):
    """Sigma and c Sigma (sigma^2 and the nugget scaled by a power of two,
    exact in every tile format) with right-hand sides z and sqrt(c) z: the
    refined quadratic forms agree and take the same number of corrections,
    the log-determinant moves by n log c.  The refinement's fixed-point copy of Sigma takes its exponent
    from sigma^2 + nugget, so its codes -- and the residual's accuracy -- do
    not depend on c."""
    n, b, nrhs = 1500, 256, 2
    nt = -(-n // b)
    pmap = I.band_map(nt, I.F64, I.F32, I.F32, 1)
    locs, _ = OM.morton_order(I.points(n, 43))
    z = I.rhs(n, nrhs, 43)
    r1 = _run(ctx, n, b, pmap, locs, z, 1.5, 0.05, 1.3, 1e-4, refine=10, ozaki=True)
    r2 = _run(ctx, n, b, pmap, locs, z * math.sqrt(c), 1.5, 0.05, 1.3 * c, 1e-4 * c, refine=10, ozaki=True)
    assert r1["info"] == 0 and r2["info"] == 0
    assert np.all(r1["iters"] < 10)
    assert np.array_equal(r1["iters"], r2["iters"])
    assert np.allclose(r2["quad"], r1["quad"], rtol=1e-12)       # (sqrt(c) z)^T (c Sigma)^{-1} (sqrt(c) z)
    assert math.isclose(r2["logdet"], r1["logdet"] + n * math.log(c), rel_tol=1e-12)


def test_trsm_forward_backward(ctx):
    """mp_trsm against the oracle's tiled solves applied to the GPU's own
    factor (downloaded tile by tile), so only the solve is compared."""
    n, b = 900, 128
    nt = -(-n // b)
    pmap = I.band_map(nt, I.F64, I.F32, I.BF16, 1)
    locs = I.points(n, 8)
    T = _mk(ctx, n, b, pmap)
    T.generate(torch.from_numpy(locs).to(DEV), 1.0, 0.05, 1.5, 1e-2)
    info, _ = T.chol()
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    state = OC.TiledMatrix(n=n, b=b, nt=nt, pmap=pmap)
    for i in range(nt):
        for j in range(i + 1):
            vals, codes, sc = T.get_tile(i, j)
            state.tiles[(i, j)] = OC.Tile(np.tril(codes) if i == j else codes, int(pmap[i, j]), sc)
    B = I.rhs(n, 4, 8)
    for trans in (0, 1):
        Bt = torch.from_numpy(np.ascontiguousarray(B.T)).to(DEV)
        T.trsm(Bt, trans)
        torch.cuda.synchronize()
        zp = np.zeros((nt * b, 4))
        zp[:n] = B
        ref = OC.forward_solve_padded(state, zp) if trans == 0 else OC.backward_solve(state, zp)
        assert np.allclose(Bt.cpu().numpy().T, ref[:n], rtol=1e-11, atol=1e-11 * np.abs(ref).max())


@pytest.mark.parametrize("n,b,bad", [(512, 128, 300), (768, 384, 401)])
def test_not_spd_reports_first_bad_row(ctx, n, b, bad):
    """b = 128: 32 x 32 blocks; b = 384: 16 x 16 blocks (row 401 is column
    1 of the second block of the second diagonal tile)."""
    T = _mk(ctx, n, b, None)
    d = np.ones(n)
    d[bad] = -2.0
    d[bad + 40] = -1.0           # a later failure must not mask the first
    for i in range(n // b):
        for j in range(i + 1):
            blk = np.zeros((b, b))
            if i == j:
                blk = np.diag(d[i * b:(i + 1) * b])
            T.set_tile(i, j, blk)
    info, _ = T.chol()
    torch.cuda.synchronize()
    assert int(info.item()) == bad + 1
    _, oinfo = OC.potrf_textbook(np.diag(d))
    assert oinfo == bad + 1


@pytest.mark.parametrize("n,b,r", [(512, 128, 300), (512, 128, 301), (512, 128, 287),
                                   (768, 384, 420), (768, 384, 421), (768, 384, 399)])
def test_not_spd_coupled_pair_reports_first_bad_row(ctx, n, b, r):
    """The diagonal block factor takes two columns per step, the second
    pivot from the pair's leading 2 x 2 minor.  A coupled block [[1, 1.5],
    [1.5, 1]] at rows (r, r+1) of an identity breaks down at row r+1: as
    the second column of a pair (r even), as the first column of the next
    pair after its update (r odd), and across a 32- or 16-block boundary
    (r = 287 = 9 * 32 - 1, r = 399 = 384 + 16 - 1)."""
    T = _mk(ctx, n, b, None)
    A = np.eye(n)
    A[r, r + 1] = A[r + 1, r] = 1.5
    A[r + 60, r + 60] = -1.0      # a later failure must not mask the first
    for i in range(n // b):
        for j in range(i + 1):
            T.set_tile(i, j, A[i * b:(i + 1) * b, j * b:(j + 1) * b])
    info, _ = T.chol()
    torch.cuda.synchronize()
    _, oinfo = OC.potrf_textbook(A)
    assert oinfo == r + 2
    assert int(info.item()) == r + 2


@pytest.mark.parametrize("dt", [I.F64, I.F32, I.BF16, I.F16, I.E4M3])
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T")])
def test_gemm_per_precision(ctx, dt, ta, tb):
    from paper_2406_02701_gb300 import mpchol
    m, n, k = 130, 77, 200
    rng = np.random.default_rng(dt * 10 + len(ta))
    A0 = rng.standard_normal((m, k) if ta == "N" else (k, m))
    B0 = rng.standard_normal((k, n) if tb == "N" else (n, k))
    C0 = rng.standard_normal((m, n))
    if dt == I.E4M3:
        A0, B0, C0 = A0 * 4, B0 * 4, C0 * 4
    A, B, Cm = (OF.round_to(x, dt) for x in (A0, B0, C0))
    ref = OC.gemm(A, B, Cm, dt, alpha=0.5, beta=-1.0, ta=ta == "T", tb=tb == "T")

    def dev(x):       # column-major storage = row-major of the transpose
        raw = mpchol.encode(np.ascontiguousarray(x.T).reshape(-1), dt)
        return torch.from_numpy(raw).to(DEV), x.shape[0]
    dA, lda = dev(A)
    dB, ldb = dev(B)
    dC, ldc = dev(Cm)
    ctx.gemm(dt, ta, tb, m, n, k, 0.5, dA, lda, dB, ldb, -1.0, dC, ldc)
    torch.cuda.synchronize()
    got = mpchol.decode(dC.cpu().numpy(), dt).reshape(n, m).T
    a = A.T if ta == "T" else A
    bb = B.T if tb == "T" else B
    bound = 0.5 * 2 * k * (2.0 ** -53 if dt == I.F64 else 2.0 ** -24) * (np.abs(a) @ np.abs(bb))
    assert_close_fmt(got, ref, dt, extra=bound + (1e-6 * np.abs(Cm) if dt not in (I.F64, I.F32) else 0),
                     what="gemm")


def test_batch_equals_single_evaluations(ctx):
    """A batch plan gives every request the bits of its single evaluation;
    a request whose mixed factor breaks down reports MP_ERR_NOT_SPD without
    disturbing the others."""
    from paper_2406_02701_gb300 import mpchol
    reqs, singles, expect_bad = [], [], []
    b = 128
    sizes = [300, 1000, 128, 777, 2048, 513]
    for r, n in enumerate(sizes):
        nt = -(-n // b)
        pmap = I.band_map(nt, I.F64, I.F32, I.BF16, 1)
        locs, _ = OM.morton_order(I.points(n, 40 + r))
        z = I.rhs(n, 1 + r % 2, 40 + r)
        nu, a = [0.5, 1.5, 2.5][r % 3], 0.02 + 0.05 * r
        dl = torch.from_numpy(locs).to(DEV)
        zt = torch.from_numpy(np.ascontiguousarray(z.T)).to(DEV)
        reqs.append(dict(n=n, map=pmap, locs=dl, zt=zt, sigma2=1.0, range=a, nu=nu, nugget=1e-2))
        s = _run(ctx, n, b, pmap, locs, z, nu, a, 1.0, 1e-2, ozaki=True)   # the batch's panel solve
        singles.append(s)
        S = OM.covariance(locs, nu, a, 1.0, 1e-2)
        try:
            tl = OC.tiled_loglik(S, z, b, pmap)
        except np.linalg.LinAlgError:
            expect_bad.append(True)
            assert s["info"] > 0
            continue
        expect_bad.append(False)
        assert s["info"] == 0
        ex = OC.exact_loglik(S, z)
        err = np.abs(s["ll"] - ex["loglik"]) / np.abs(ex["loglik"])
        assert np.all(np.abs(s["ll"] - tl["loglik"]) / np.abs(tl["loglik"]) <= np.maximum(10 * err, 1e-9))
    assert any(expect_bad) and not all(expect_bad)
    B = mpchol.Batch(ctx, reqs, b=b)
    ll, st = B.run()
    torch.cuda.synchronize()
    ll, st = ll.cpu().numpy(), st.cpu().numpy()
    o = 0
    for s, bad, stv in zip(singles, expect_bad, st):
        k = len(s["ll"])
        assert stv == (mpchol.MP_ERR_NOT_SPD if bad else mpchol.MP_OK)
        if not bad:
            assert np.array_equal(ll[o:o + k], s["ll"]), (ll[o:o + k], s["ll"])
        o += k
    # a second run of the same graph gives the same bits
    ll2, _ = B.run()
    torch.cuda.synchronize()
    ok = np.concatenate([np.full(len(s["ll"]), not bad) for s, bad in zip(singles, expect_bad)])
    assert np.array_equal(ll2.cpu().numpy()[ok], ll[ok])


@pytest.mark.parametrize("dt", [I.BF16, I.F32, I.E4M3])
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N")])
def test_gemm_tensor_cores_several_tiles_and_k_groups(ctx, dt, ta, tb):
    """Sizes that span several output tiles with ragged edges and more than
    one group of contraction tiles (K = 9000 > 4096): the tensor-core
    product against the oracle's FP32-accumulated product."""
    from paper_2406_02701_gb300 import mpchol
    m, n, k = 1100, 700, 9000
    rng = np.random.default_rng(dt * 7 + len(ta))
    A0 = rng.standard_normal((m, k) if ta == "N" else (k, m))
    B0 = rng.standard_normal((k, n))
    C0 = rng.standard_normal((m, n))
    A, B, Cm = (OF.round_to(x, dt) for x in (A0, B0, C0))
    ref = OC.gemm(A, B, Cm, dt, alpha=0.75, beta=0.5, ta=ta == "T")

    def dev(x):
        raw = mpchol.encode(np.ascontiguousarray(x.T).reshape(-1), dt)
        return torch.from_numpy(raw).to(DEV), x.shape[0]
    dA, lda = dev(A)
    dB, ldb = dev(B)
    dC, ldc = dev(Cm)
    ctx.gemm(dt, ta, tb, m, n, k, 0.75, dA, lda, dB, ldb, 0.5, dC, ldc)
    torch.cuda.synchronize()
    got = mpchol.decode(dC.cpu().numpy(), dt).reshape(n, m).T
    a = A.T if ta == "T" else A
    bound = 0.75 * 2 * k * 2.0 ** -24 * (np.abs(a) @ np.abs(B))
    assert_close_fmt(got, ref, dt, extra=bound + (1e-6 * np.abs(Cm) if dt != I.F32 else 0), what="gemm tc")


def test_solve_and_chol2inv_through_the_factor(ctx):
    """mp_solve (Sigma X = B by the factor) and mp_chol2inv ((L L^T)^-1)
    against the oracle's tiled solves and a LAPACK inverse of the GPU's own
    factor L L^T (downloaded tile by tile)."""
    n, b = 700, 128
    nt = -(-n // b)
    pmap = I.band_map(nt, I.F64, I.F32, I.BF16, 1)
    T = _mk(ctx, n, b, pmap)
    T.generate(torch.from_numpy(I.points(n, 6)).to(DEV), 1.0, 0.05, 1.5, 1e-2)
    info, _ = T.chol()
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    state = OC.TiledMatrix(n=n, b=b, nt=nt, pmap=pmap)
    for i in range(nt):
        for j in range(i + 1):
            vals, codes, sc = T.get_tile(i, j)
            state.tiles[(i, j)] = OC.Tile(np.tril(codes) if i == j else codes, int(pmap[i, j]), sc)
    L = state.dense_lower()[:n, :n]
    Sig = L @ L.T
    B = I.rhs(n, 5, 6)
    X = T.solve(torch.from_numpy(np.ascontiguousarray(B.T)).to(DEV))
    torch.cuda.synchronize()
    zp = np.zeros((nt * b, 5))
    zp[:n] = B
    ref = OC.backward_solve(state, OC.forward_solve_padded(state, zp))[:n]
    assert np.allclose(X.cpu().numpy().T, ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())
    inv = T.chol2inv()
    torch.cuda.synchronize()
    G = inv.cpu().numpy()          # column-major n x n: the transpose of this array; symmetric
    want = np.linalg.inv(Sig)
    assert np.allclose(G, G.T, rtol=1e-10, atol=1e-10 * np.abs(want).max())
    assert np.allclose(G.T, want, rtol=1e-8, atol=1e-8 * np.abs(want).max())


def test_general_nu_in_batches_norms_and_maps(ctx):
    """Requests with nu without a closed form: a batch holds one Matérn
    table per distinct nu and gives each request the bits of its single
    evaluation; the tile norms (and so the guarded map) follow the oracle's
    definition through scipy's K_nu."""
    from paper_2406_02701_gb300 import mpchol
    b = 128
    specs, singles = [], []
    for r, (n, nu) in enumerate([(600, 0.7), (900, 1.3), (500, 0.7), (700, 2.5)]):
        nt = -(-n // b)
        pmap = I.band_map(nt, I.F64, I.F32, I.BF16, 1)
        locs, _ = OM.morton_order(I.points(n, 60 + r))
        dl = torch.from_numpy(locs).to(DEV)
        zt = torch.from_numpy(np.ascontiguousarray(I.rhs(n, 1, 60 + r).T)).to(DEV)
        z = I.rhs(n, 1, 60 + r)
        specs.append(dict(n=n, map=pmap, locs=dl, zt=zt, sigma2=1.0, range=0.04, nu=nu, nugget=1e-2))
        s = _run(ctx, n, b, pmap, locs, z, nu, 0.04, 1.0, 1e-2, ozaki=True)
        assert s["info"] == 0
        S = OM.covariance(locs, nu, 0.04, 1.0, 1e-2)
        tl, ex = OC.tiled_loglik(S, z, b, pmap), OC.exact_loglik(S, z)
        err = np.abs(s["ll"] - ex["loglik"]) / np.abs(ex["loglik"])
        assert np.all(np.abs(s["ll"] - tl["loglik"]) / np.abs(tl["loglik"]) <= np.maximum(10 * err, 1e-9))
        singles.append(s["ll"])
    B = mpchol.Batch(ctx, specs, b=b)
    ll, st = B.run()
    torch.cuda.synchronize()
    assert np.all(st.cpu().numpy() == 0)
    assert np.array_equal(ll.cpu().numpy(), np.concatenate(singles))
    n = 1100
    locs, _ = OM.morton_order(I.points(n, 70))
    got = ctx.tile_norms(n, b, torch.from_numpy(locs).to(DEV), 1.0, 0.05, 1.3, 1e-4).cpu().numpy()
    ref = OC.tile_norms(OM.covariance(locs, 1.3, 0.05, 1.0, 1e-4), b)
    assert np.allclose(got, ref, rtol=1e-11, atol=0)


@pytest.mark.parametrize("flags", [0, 32, 64])
def test_chain_trace_is_ordered_and_leaves_the_factor_alone(ctx, flags):
    """MP_TMAT_TRACE stamps the diagonal tiles' chain tasks: the factor and
    log-determinant carry the same bits as without it, the stamps of every
    block are in program order, and each chain task sees the previous
    block's inverse only after that block was factored."""
    from paper_2406_02701_gb300 import mpchol
    n, b = 1500, 512
    nt = -(-n // b)
    pmap = I.band_map(nt, I.F64, I.F32, I.F32, 1)
    locs = torch.from_numpy(I.points(n, 15)).to(DEV)
    out = []
    for fl in (flags, flags | mpchol.MP_TMAT_TRACE):
        T = mpchol.TiledMatrix(ctx, n, b, pmap, flags=fl)
        T.generate(locs, 1.0, 0.05, 1.5, 1e-3)
        info, ld = T.chol()
        torch.cuda.synchronize()
        assert int(info.item()) == 0
        out.append((ld.item(), [T.get_tile(i, j)[1].copy() for i in range(nt) for j in range(i + 1)], T))
    assert out[1][0] == out[0][0]
    for a, c in zip(out[0][1], out[1][1]):
        assert np.array_equal(a, c)
    with pytest.raises(RuntimeError):
        out[0][2].chain_trace()
    ns, cyc, db = out[1][2].chain_trace()
    assert db == {0: 16, 32: 16, 64: 32}[flags]
    assert ns.shape == (nt, b // db, 8) and cyc.shape == ns.shape
    assert np.all(ns[:, :, 0] > 0)
    assert np.all(np.diff(cyc, axis=2) >= 0)
    assert np.all(np.diff(ns, axis=2) >= 0)
    assert np.all(ns[:, 1:, 2] >= ns[:, :-1, 5])
    assert np.all(ns[1:, 0, 0] >= ns[:-1, -1, 5])
