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


def test_bound_map_rejects_nu_without_closed_form():
    """The host bound evaluates the half-integer closed forms only; any other
    nu is refused rather than bounded with the wrong covariance."""
    from paper_2406_02701_gb300 import mpchol
    locs, _ = OM.morton_order(I.points(600, 4))
    for nu in (1.0, 0.3, 3.5):
        with pytest.raises(mpchol.MPError) as e:
            mpchol.map_bound(600, 128, locs, (1.0, 0.05, nu, 1e-4), 2, I.F32, I.BF16, 1e-6)
        assert e.value.status == mpchol.MP_ERR_ARG
