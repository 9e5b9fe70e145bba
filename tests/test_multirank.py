"""The multi-rank path of the benchmark on CPU: two gloo ranks, each timing
an independent replica (no data-path collective); the timings are reduced by
their maximum over the ranks and the whole-job value counts every rank's
work over that maximum."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    got_ws, got_rank, got_local = bench.dist_setup(None)
    dist.barrier()
    ms = bench.max_over_ranks([10.0 + rank, 20.0 - rank], ws)
    value = bench.whole_job(ms, ws, 1e12)
    dist.barrier()
    q.put((rank, (got_ws, got_rank, got_local), ms, value))
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, env, ms, value in out:
        assert env == (2, rank, rank)
        assert ms == [11.0, 20.0]                  # the slowest rank's time, per timing
        assert value == pytest.approx([2 * 1e12 / 11e-3 / 1e12, 2 * 1e12 / 20e-3 / 1e12])


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks([3.5, 4.0], 1) == [3.5, 4.0]
    assert bench.whole_job([1000.0], 1, 1e12) == [1.0]
