"""Host-only planning calls of the library against the oracle (CPU)."""
import numpy as np
import pytest

import mpinputs as I
from oracle import chol as OC
from oracle import matern as OM


@pytest.mark.parametrize("n,b,nu,a", [(4096, 256, 1.5, 0.05), (8192, 256, 0.5, 0.02),
                                      (1000, 128, 0.5, 0.1), (3000, 512, 2.5, 0.3)])
@pytest.mark.parametrize("far,eps", [(I.BF16, 1e-6), (I.E4M3, 1e-3), (I.BF16, 1e-2)])
def test_bound_map_matches_oracle(n, b, nu, a, far, eps):
    from paper_2406_02701_gb300 import mpchol
    locs, _ = OM.morton_order(I.points(n, 3))
    got = mpchol.map_bound(n, b, locs, (1.0, a, nu, 1e-4), 2, I.F32, far, eps)
    assert np.array_equal(got, OC.bound_map(locs, b, nu, a, 1.0, 1e-4, 2, I.F32, far, eps))


def test_bound_map_is_more_conservative_than_exact_norms():
    n, b = 2048, 128
    locs, _ = OM.morton_order(I.points(n, 5))
    S = OM.covariance(locs, 0.5, 0.02, 1.0, 1e-4)
    exact = OC.guarded_map(OC.tile_norms(S, b), 2, I.F32, I.BF16, 1e-4)
    bound = OC.bound_map(locs, b, 0.5, 0.02, 1.0, 1e-4, 2, I.F32, I.BF16, 1e-4)
    lo = np.tril_indices(n // b, -1)
    # every tile the bound puts in BF16 is also BF16 under the exact rule
    assert np.all((bound[lo] == I.BF16) <= (exact[lo] == I.BF16))
    assert (bound[lo] == I.BF16).sum() > 0


def test_bound_map_rejects_unsupported_nu():
    """nu outside (0, 16] is refused rather than bounded with some other
    covariance."""
    from paper_2406_02701_gb300 import mpchol
    locs, _ = OM.morton_order(I.points(600, 4))
    for nu in (0.0, -1.0, 17.0):
        with pytest.raises(mpchol.MPError) as e:
            mpchol.map_bound(600, 128, locs, (1.0, 0.05, nu, 1e-4), 2, I.F32, I.BF16, 1e-6)
        assert e.value.status == mpchol.MP_ERR_ARG


@pytest.mark.parametrize("nu", [0.3, 1.0, 2.2])
def test_bound_map_general_nu_matches_oracle(nu):
    """The bound map for nu without a closed form: the oracle's bound_map
    with the covariance through scipy's K_nu gives the same map (a tile
    whose bound sits within rounding of the threshold could differ; none
    does here)."""
    from paper_2406_02701_gb300 import mpchol
    n, b = 3000, 256
    locs, _ = OM.morton_order(I.points(n, 8))
    got = mpchol.map_bound(n, b, locs, (1.0, 0.04, nu, 1e-4), 2, I.F32, I.BF16, 1e-6)
    assert np.array_equal(got, OC.bound_map(locs, b, nu, 0.04, 1.0, 1e-4, 2, I.F32, I.BF16, 1e-6))


@pytest.mark.parametrize("nu", [0.05, 0.3, 1.0, 2.2, 3.7, 7.5, 16.0])
def test_general_nu_table_matches_the_oracle(nu):
    """The library's Matérn correlation for nu without a closed form (a
    Chebyshev table of x^nu K_nu(x) per half octave, nodes by the trapezoidal
    rule on K_nu's integral representation) against the oracle's definition
    through scipy's K_nu, from coincident points to far beyond the range."""
    from paper_2406_02701_gb300 import mpchol
    a, s2 = 0.05, 1.3
    rng = np.random.default_rng(int(nu * 100))
    # (scipy's x^nu K_nu(x) overflows to nan below x ~ 1e-30 for larger nu;
    # the forty-digit test below covers those distances)
    r = np.concatenate([[0.0, 1e-9], a * np.exp(rng.uniform(np.log(1e-6), np.log(60.0), 4000))])
    got = mpchol.matern_host(r, s2, a, nu)
    want = OM.matern_general(r, nu, a, s2)
    # scipy's K_nu is itself good to a few 1e-14 (2.7e-14 at nu = 0.3,
    # x = 1.6 against a 40-digit evaluation)
    assert np.allclose(got, want, rtol=1e-13, atol=1e-300)


@pytest.mark.parametrize("nu", [0.05, 0.3, 1.0, 2.2, 7.5])
def test_general_nu_table_matches_forty_digits(nu):
    """The same against K_nu evaluated with 40 significant digits (mpmath):
    the table's own error stays within a few units of 2^-52, plus x 2^-53
    from the factor e^{-x} beyond x = 1."""
    mp = pytest.importorskip("mpmath")
    from paper_2406_02701_gb300 import mpchol
    mp.mp.dps = 40
    a, s2 = 0.05, 1.3
    rng = np.random.default_rng(int(nu * 1000))
    r = a * np.concatenate([[1e-290, 1e-100, 1e-30], np.exp(rng.uniform(np.log(1e-8), np.log(40.0), 300))])
    got = mpchol.matern_host(r, s2, a, nu)
    c = mp.mpf(2) ** (1 - nu) / mp.gamma(nu) * s2
    want = np.array([float(c * (mp.mpf(v) / a) ** nu * mp.besselk(nu, mp.mpf(v) / a)) for v in r])
    # the trapezoid nodes carry about nu units of rounding (exp(-x cosh t)
    # near the peak of the integrand, where x cosh t ~ nu)
    tol = (8 + 2 * nu + r / a) * 2.0 ** -52 * want
    bad = np.abs(got - want) > tol
    assert not bad.any(), (r[bad][:5], (np.abs(got - want) / want)[bad][:5])


def test_general_nu_half_integers_agree_with_closed_forms():
    """Near the half integers the table reproduces the closed forms (the
    table is built for nu = 1.5 + 1e-12, which no closed form covers)."""
    from paper_2406_02701_gb300 import mpchol
    r = np.linspace(0.0, 1.0, 3001)
    for nu in (0.5, 1.5, 2.5):
        got = mpchol.matern_host(r, 1.0, 0.1, nu + 1e-12)
        want = OM.matern_closed(r, nu, 0.1, 1.0)
        assert np.allclose(got, want, rtol=1e-10, atol=1e-300)


@pytest.mark.parametrize("nu", [0.0, -1.0, 16.5, float("nan")])
def test_nu_outside_the_supported_range_is_rejected(nu):
    from paper_2406_02701_gb300 import mpchol
    with pytest.raises(mpchol.MPError):
        mpchol.matern_host(np.array([0.1]), 1.0, 0.1, nu)
