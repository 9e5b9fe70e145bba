"""Failure handling on the GPU without faulting or hanging it.

* A task-graph wait that runs out: the matrix's wait budget is set to one
  poll, so the first task that has to wait for another gives up at once;
  its kernel records the failure and returns.  The factorisation reports
  -MP_ERR_TIMEOUT in d_info, the log-likelihood is NaN, and with the
  default budget restored the same matrix factors to the same bits as
  before -- the context stays usable.
* An allocation that fails while the server admits a request, made on the
  host: that request finishes with MP_ERR_OOM and its partly built state
  is freed; the requests around it finish normally, with the results they
  get when nothing fails.
"""
import math

import numpy as np
import pytest

import mpinputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_02701_gb300 import mpchol
    return mpchol.Context(0)


def test_wait_that_runs_out_reports_timeout_and_context_recovers(ctx):
    from paper_2406_02701_gb300 import mpchol
    n, b = 2048, 512                       # 32 x 32 blocks of 16 per diagonal tile
    nt = n // b
    pmap = I.band_map(nt, I.F64, I.F32, I.BF16, 1)
    dl = torch.from_numpy(I.points(n, 3)).cuda()
    zt = torch.from_numpy(np.ascontiguousarray(I.rhs(n, 2, 3).T)).cuda()
    T = mpchol.TiledMatrix(ctx, n, b, pmap, keep_sigma=True)

    def evaluate():
        T.generate(dl, 1.0, 0.05, 0.5, 1e-4)
        info, logdet = T.chol()
        ll, _, _ = T.loglik(zt, refine_iters=3)
        torch.cuda.synchronize()
        return int(info.item()), logdet.item(), ll.cpu().numpy()

    info0, ld0, ll0 = evaluate()
    assert info0 == 0 and np.all(np.isfinite(ll0))
    T.set_wait_budget(1)
    info1, _, ll1 = evaluate()
    assert info1 == -mpchol.MP_ERR_TIMEOUT
    assert np.all(np.isnan(ll1))
    T.set_wait_budget(0)
    info2, ld2, ll2 = evaluate()
    assert info2 == 0
    assert ld2 == ld0 and np.array_equal(ll2, ll0)
    # the context serves other matrices as before (one of the same kind:
    # without a float64 copy of Sigma the FP32/BF16 tiles are generated in
    # float-float, which can round a value one unit apart)
    T2 = mpchol.TiledMatrix(ctx, n, b, pmap, keep_sigma=True)
    T2.generate(dl, 1.0, 0.05, 0.5, 1e-4)
    info3, ld3 = T2.chol()
    torch.cuda.synchronize()
    assert int(info3.item()) == 0 and ld3.item() == ld0


def test_injected_allocation_failure_at_admission(ctx):
    from paper_2406_02701_gb300 import mpchol, serving
    reqs = serving.make_requests(5, 1e6, seed=13, sizes=(600, 1500), weights=(1, 1), nrhs=1)
    for r in reqs:
        r["arrival"] = 0.0
    clean = mpchol.Server(ctx, hbm_budget=8 << 30, max_slots=1, eps=1e-6)
    ref, _ = serving.run(clean, reqs, refine_iters=2)
    clean.close()
    srv = mpchol.Server(ctx, hbm_budget=8 << 30, max_slots=1, eps=1e-6)
    srv.inject_alloc_failures(1)
    res, _ = serving.run(srv, reqs, refine_iters=2)
    assert srv.stats()["bytes"] == 0 and srv.stats()["kept"] == 0
    srv.close()
    status = [res[i]["status"] for i in range(len(reqs))]
    # one slot, arrival order: the first admission is the one that fails
    assert status[0] == mpchol.MP_ERR_OOM
    assert all(s == 0 for s in status[1:])
    for i in range(1, len(reqs)):
        assert np.array_equal(res[i]["ll"], ref[i]["ll"])
        assert math.isfinite(res[i]["logdet"])
