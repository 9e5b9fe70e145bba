"""Nelder-Mead driver (host logic on the CPU) and the Matérn MLE on the GPU
against the oracle's exact log-likelihood (Sec. 6.2's MLE workload)."""
import math

import numpy as np
import pytest

from paper_2406_02701_gb300.mle import nelder_mead


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_02701_gb300 import mpchol
    return mpchol.Context(0)


def _batch(f):
    return lambda pts: [f(p) for p in pts]


def test_nelder_mead_quadratic():
    f = lambda x: (x[0] - 1.0) ** 2 + 10.0 * (x[1] + 2.0) ** 2
    r = nelder_mead(_batch(f), [0.0, 0.0], step=0.5, max_iter=500, reltol=1e-14)
    assert np.allclose(r["x"], [1.0, -2.0], atol=1e-6)
    assert r["f"] < 1e-11


def test_nelder_mead_rosenbrock():
    f = lambda x: 100.0 * (x[1] - x[0] ** 2) ** 2 + (1.0 - x[0]) ** 2
    r = nelder_mead(_batch(f), [-1.2, 1.0], step=0.5, max_iter=2000, reltol=1e-15)
    assert np.allclose(r["x"], [1.0, 1.0], atol=1e-4)


def test_stops_on_a_noisy_objective():
    """R optim's relative rule ends the search when the values at the
    vertices agree to about 1.5e-8, above the ~1e-10 relative differences of
    two FP64-refined evaluations of a log-likelihood."""
    g = lambda x: 850.0 + 40.0 * (x[0] + 2.3) ** 2 + 25.0 * (x[1] - 0.1) ** 2 + 3.0 * x[0] * x[1]
    noisy = lambda x: g(x) * (1.0 + 1e-10 * math.sin(1e7 * (x[0] + 2 * x[1])))
    r = nelder_mead(_batch(noisy), [-3.0, -0.7], step=0.5, max_iter=200)
    assert r["iters"] < 200 and r["converged"]
    ref = nelder_mead(_batch(g), [-3.0, -0.7], step=0.5, max_iter=2000, reltol=1e-15)
    assert abs(r["f"] - ref["f"]) <= 1e-6 * abs(ref["f"])


def test_tolerance_is_fixed_from_the_starting_value_and_cap_is_reported():
    """R optim's Nelder-Mead fixes its tolerance once, reltol (|f(x0)| +
    reltol) at the starting point: started far up a steep bowl the search
    stops at a spread that a tolerance taken from the current best value
    would not accept; a search ended by the iteration cap says so."""
    f = lambda x: 1e6 * (x[0] ** 2 + x[1] ** 2) + 1.0
    r = nelder_mead(_batch(f), [3.0, 4.0], step=0.5, max_iter=500, reltol=1e-6)
    spread = r["fvals"].max() - r["fvals"].min()
    assert r["converged"]
    assert spread <= 1e-6 * (f([3.0, 4.0]) + 1e-6)
    assert spread > 1e-6 * (abs(r["f"]) + 1e-6)
    capped = nelder_mead(_batch(f), [3.0, 4.0], step=0.5, max_iter=5, reltol=1e-12)
    assert capped["iters"] == 5 and not capped["converged"]


def test_speculative_batches_take_the_same_path():
    """Evaluating the four candidates of an iteration together changes the
    number of evaluations and round trips, not a single decision."""
    calls = []
    f = lambda x: math.sin(3 * x[0]) + (x[0] - 0.3) ** 2 + 2 * (x[1] - x[0] * x[1]) ** 2 + 0.1 * x[1] ** 2

    def fb(pts):
        calls.append(len(pts))
        return [f(p) for p in pts]

    a = nelder_mead(fb, [1.0, 1.0], max_iter=150, speculative=False)
    calls.clear()
    b = nelder_mead(fb, [1.0, 1.0], max_iter=150, speculative=True)
    assert a["iters"] == b["iters"]
    assert np.array_equal(a["simplex"], b["simplex"]) and np.array_equal(a["fvals"], b["fvals"])
    assert b["rounds"] < a["rounds"] and b["evals"] > a["evals"]
    assert all(c in (3, 4, 2) for c in calls)        # initial simplex, candidates, shrink


@pytest.mark.gpu
def test_matern_mle_matches_oracle_at_the_optimum(ctx):
    import torch
    from oracle import chol as OC
    from oracle import matern as OM
    import mpinputs as I
    from paper_2406_02701_gb300.mle import MaternMLE
    n, b, nu, nugget = 1024, 128, 0.5, 1e-4
    locs = I.points(n, 41)
    # one draw of the field at (range 0.1, sigma^2 1.2)
    S0 = OM.covariance(locs, nu, 0.1, 1.2, nugget)
    z = np.linalg.cholesky(S0) @ np.random.default_rng(41).standard_normal(n)
    zc = z.reshape(n, 1)

    def exact(rng, s2):
        return float(OC.exact_loglik(OM.covariance(locs, nu, rng, s2, nugget), zc)["loglik"][0])

    # the oracle's own optimum (Nelder-Mead on the exact log-likelihood)
    ref = nelder_mead(lambda pts: [-exact(math.exp(p[0]), math.exp(p[1])) for p in pts],
                      [math.log(0.05), math.log(0.5)], max_iter=200, speculative=True)
    ll_star = -ref["f"]
    nt = -(-n // b)
    pmap = I.band_map(nt, I.F64, I.F32, I.F32, 2)
    mle = MaternMLE(ctx, locs, z, b, nu, nugget, pmap=pmap, lanes=4, refine_iters=20)
    # four lanes at four parameter vectors, each against the oracle
    thetas = [(0.07, 0.9), (0.12, 1.5), (0.05, 0.6), (0.09, 1.1)]
    got = mle.loglik(thetas)
    for (rng, s2), g in zip(thetas, got):
        want = exact(rng, s2)
        assert abs(g - want) <= 1e-6 * abs(want), (rng, s2, g, want)
    r = mle.fit(0.05, 0.5, max_iter=200)
    mle.close()
    assert r["converged"], r["iters"]
    print("gpu fit:", r["iters"], r["evals"], r["range"], r["sigma2"], r["loglik"], "oracle fit:",
          ref["iters"], math.exp(ref["x"][0]), math.exp(ref["x"][1]), ll_star)
    # the point found is as good as the oracle's optimum (the north-star
    # tolerance for the FP32 map: 1e-6 relative), and its GPU value is the
    # oracle's there
    ll_hat = exact(r["range"], r["sigma2"])
    assert ll_hat >= ll_star - 1e-6 * abs(ll_star)
    assert abs(r["loglik"] - ll_hat) <= 1e-6 * abs(ll_hat)
    assert 0.05 < r["range"] < 0.2 and 0.6 < r["sigma2"] < 2.4
    torch.cuda.synchronize()
