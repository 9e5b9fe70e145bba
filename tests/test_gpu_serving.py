"""Continuous-batching server: each result is the same alone and in the
mix, agrees with the oracle, and admission respects the HBM budget."""
import numpy as np
import pytest

import mpinputs as I
from oracle import chol as OC
from oracle import matern as OM

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_02701_gb300 import mpchol
    return mpchol.Context(0)


def _reqs(count, seed=71):
    from paper_2406_02701_gb300 import serving
    reqs = serving.make_requests(count, 1e6, seed=seed, sizes=(300, 1000, 2500),
                                 weights=(3, 2, 1), nrhs=2)
    for r in reqs:
        r["arrival"] = 0.0          # all at once: maximal overlap on the device
    return reqs


def test_results_are_the_same_alone_and_in_the_mix(ctx):
    from paper_2406_02701_gb300 import mpchol, serving
    reqs = _reqs(12)
    mix = mpchol.Server(ctx, hbm_budget=8 << 30, max_slots=6, eps=1e-6)
    res_mix, _ = serving.run(mix, reqs, refine_iters=3)
    mix.close()
    for i, r in enumerate(reqs):
        alone = mpchol.Server(ctx, hbm_budget=8 << 30, max_slots=1, eps=1e-6)
        one, _ = serving.run(alone, [dict(r)], refine_iters=3)
        alone.close()
        a, m = one[0], res_mix[i]
        assert a["status"] == m["status"] == 0
        assert np.array_equal(a["ll"], m["ll"])          # bit for bit
        assert a["logdet"] == m["logdet"]


def test_server_results_match_the_oracle(ctx):
    from paper_2406_02701_gb300 import mpchol, serving
    reqs = _reqs(4, seed=5)
    srv = mpchol.Server(ctx, hbm_budget=8 << 30, max_slots=4, eps=1e-6)
    res, _ = serving.run(srv, reqs, refine_iters=5)
    srv.close()
    for i, r in enumerate(reqs):
        srt, perm = OM.morton_order(r["locs"])
        z = r["z"][perm]
        b = 128 if r["n"] <= 2048 else 256
        pmap = OC.bound_map(srt, b, r["nu"], r["range"], r["sigma2"], r["nugget"], 2, I.F32,
                            I.BF16, 1e-6)
        S = OM.covariance(srt, r["nu"], r["range"], r["sigma2"], r["nugget"])
        ex = OC.exact_loglik(S, z)
        tl = OC.tiled_loglik(S, z, b, pmap, refine_iters=5)
        got = res[i]["ll"]
        err = np.abs(got - ex["loglik"]) / np.abs(ex["loglik"])
        assert np.all(err < 1e-6), err
        assert np.all(np.abs(got - tl["loglik"]) / np.abs(tl["loglik"]) <= np.maximum(10 * err, 1e-9))


def _drive(srv, reqs):
    ids = [srv.submit(r["locs"], r["z"], (r["sigma2"], r["range"], r["nu"], r["nugget"]))
           for r in reqs]
    done, peak = {}, 0
    while len(done) < len(ids):
        for res in srv.poll():
            done[res["id"]] = res
        peak = max(peak, srv.stats()["running"])
    return ids, done, peak


def test_admission_respects_the_budget_and_release_frees(ctx):
    from paper_2406_02701_gb300 import mpchol, serving
    reqs = serving.make_requests(5, 1e6, seed=9, sizes=(1000,), weights=(1,))
    # footprint of one request (n = 1000, tile 128), measured alone
    probe = mpchol.Server(ctx, hbm_budget=8 << 30, max_slots=1, eps=1e-6)
    _drive(probe, reqs[:1])
    one = probe.stats()["bytes"]
    probe.close()
    assert one > 0
    # a budget of 1.5 requests admits one at a time, evicting the previous
    # request's kept factor
    budget = int(1.5 * one)
    srv = mpchol.Server(ctx, hbm_budget=budget, max_slots=4, eps=1e-6)
    ids, done, peak = _drive(srv, reqs)
    assert peak == 1
    assert all(r["status"] == 0 for r in done.values())
    assert srv.stats()["bytes"] <= budget
    for rid in ids:
        srv.release(rid)
    assert srv.stats()["bytes"] == 0 and srv.stats()["kept"] == 0
    srv.close()
    # with room for all, requests run concurrently on their own streams
    srv = mpchol.Server(ctx, hbm_budget=8 << 30, max_slots=4, eps=1e-6)
    ids, done, peak = _drive(srv, reqs)
    assert peak >= 2 and all(r["status"] == 0 for r in done.values())
    assert srv.stats()["kept"] == len(reqs)          # factors stay on the device
    srv.close()
