"""The autotuner: it times real plans and returns a schedule that the
library then runs, caches its choice, and every schedule flag leaves the
arithmetic of the method alone (the ring depth changes no bit; the
task-graph block only the order of float64 sums inside the diagonal
tiles; the panel solve path the last bits of each panel before its
rounding)."""
import os

import numpy as np
import pytest

import mpinputs as I
from oracle import matern as OM

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_02701_gb300 import mpchol
    return mpchol.Context(0)


def _specs(ctx, count, seed=5, n_lo=256, n_hi=1500):
    reqs = I.batch_requests(count, seed=seed, n_lo=n_lo, n_hi=n_hi)
    specs = []
    for r in reqs:
        n = r["n"]
        ds, _ = ctx.morton_order(torch.from_numpy(I.points(n, r["seed"])).cuda())
        zt = torch.from_numpy(np.ascontiguousarray(I.rhs(n, 1, r["seed"]).T)).cuda()
        specs.append(dict(n=n, locs=ds, zt=zt, sigma2=r["sigma2"], range=r["range"], nu=r["nu"],
                          nugget=r["nugget"], rule=(2, I.F32, I.BF16, 1e-6)))
    return specs


def test_tuned_batch_schedule_is_measured_cached_and_runs(ctx, tmp_path):
    from paper_2406_02701_gb300 import mpchol
    specs = _specs(ctx, 24)
    cache = str(tmp_path / "tune.txt")
    t = mpchol.tune_batch(ctx, specs, cache_path=cache)
    assert t["from_cache"] == 0 and t["tried"] >= 5 and t["ms"] > 0
    assert t["b"] in (128, 256, 384, 512)
    again = mpchol.tune_batch(ctx, specs, cache_path=cache)
    assert again["from_cache"] == 1 and (again["b"], again["flags"]) == (t["b"], t["flags"])
    assert os.path.getsize(cache) > 0
    B = mpchol.Batch(ctx, specs, b=t["b"], flags=t["flags"])
    assert B.info()["b"] == t["b"] and B.info()["flags"] == t["flags"]
    ll, st = B.run()
    torch.cuda.synchronize()
    ll, st = ll.cpu().numpy(), st.cpu().numpy()
    # each request: its single evaluation with the same b, schedule flags and map rule
    for k in (0, 7, 23):
        s = specs[k]
        b = t["b"]
        pmap = mpchol.map_bound(s["n"], b, s["locs"].cpu().numpy(), (s["sigma2"], s["range"], s["nu"], s["nugget"]),
                                2, I.F32, I.BF16, 1e-6)
        T = mpchol.TiledMatrix(ctx, s["n"], b, pmap, flags=t["flags"])
        T.generate(s["locs"], s["sigma2"], s["range"], s["nu"], s["nugget"])
        info, _ = T.chol()
        one, _, _ = T.loglik(s["zt"])
        torch.cuda.synchronize()
        if st[k] == 0:
            assert int(info.item()) == 0 and one.item() == ll[k]


def test_batch_with_b0_takes_the_tuned_schedule(ctx, tmp_path, monkeypatch):
    from paper_2406_02701_gb300 import mpchol
    specs = _specs(ctx, 8, seed=9)
    cache = str(tmp_path / "tune.txt")
    t = mpchol.tune_batch(ctx, specs, cache_path=cache)
    monkeypatch.setenv("MPCHOL_TUNE_CACHE", cache)
    B = mpchol.Batch(ctx, specs, b=0)
    assert (B.info()["b"], B.info()["flags"]) == (t["b"], t["flags"])


def test_explicit_maps_cannot_be_tuned_over_b(ctx):
    from paper_2406_02701_gb300 import mpchol
    specs = _specs(ctx, 2, seed=3)
    for s in specs:
        s["map"] = mpchol.map_bound(s["n"], 128, s["locs"].cpu().numpy(),
                                    (s["sigma2"], s["range"], s["nu"], s["nugget"]), 2, I.F32, I.BF16, 1e-6)
    with pytest.raises(mpchol.MPError):
        mpchol.tune_batch(ctx, specs)


def test_schedule_flags_leave_the_arithmetic_alone(ctx):
    from paper_2406_02701_gb300 import mpchol
    n, b = 2000, 512
    nt = -(-n // b)
    pmap = I.band_map(nt, I.F64, I.F32, I.BF16, 2)
    locs, _ = OM.morton_order(I.points(n, 12))
    dl = torch.from_numpy(locs).cuda()
    zt = torch.from_numpy(np.ascontiguousarray(I.rhs(n, 2, 12).T)).cuda()

    def ll(flags):
        T = mpchol.TiledMatrix(ctx, n, b, pmap, flags=flags)
        T.generate(dl, 1.0, 0.03, 0.5, 1e-4)
        info, ld = T.chol()
        v, _, _ = T.loglik(zt)
        torch.cuda.synchronize()
        assert int(info.item()) == 0
        return v.cpu().numpy(), ld.item()

    base, ld0 = ll(0)
    ring, ld1 = ll(mpchol.MP_TMAT_LOWP_RING4)
    assert np.array_equal(ring, base) and ld1 == ld0
    direct, ldd = ll(mpchol.MP_TMAT_DIRECT)         # no graph capture: same kernels, same bits
    assert np.array_equal(direct, base) and ldd == ld0
    d32, ld2 = ll(mpchol.MP_TMAT_DAG32)
    assert np.allclose(d32, base, rtol=1e-9) and abs(ld2 - ld0) <= 1e-9 * abs(ld0)
    f64, _ = ll(mpchol.MP_TMAT_FP64_PANEL)
    assert np.allclose(f64, base, rtol=1e-5)


def test_server_tuned_sizes(ctx, tmp_path):
    from paper_2406_02701_gb300 import mpchol, serving
    srv = mpchol.Server(ctx, hbm_budget=8 << 30, max_slots=2, eps=1e-6)
    srv.tune([700, 1800], refine_iters=2, cache_path=str(tmp_path / "t.txt"))
    chosen = {n: mpchol.tune_tmat(ctx, n, mpchol.MP_BF16, 1e-6, 2, cache_path=str(tmp_path / "t.txt"))
              for n in (700, 1800)}
    assert all(c["from_cache"] == 1 for c in chosen.values())
    reqs = serving.make_requests(4, 1e6, seed=21, sizes=(700, 1800), weights=(1, 1))
    for r in reqs:
        r["arrival"] = 0.0
    res, _ = serving.run(srv, reqs, refine_iters=2)
    srv.close()
    for i, r in enumerate(reqs):
        assert res[i]["status"] == 0
        assert res[i]["b"] == chosen[r["n"]]["b"]
