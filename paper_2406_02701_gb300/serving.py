"""Serving driver: replays a stream of log-likelihood requests with given
arrival times against an mp_server and measures latency (arrival ->
result seen by the poller) and throughput.  Argument marshalling and host
timing only; the work runs in the library."""
from __future__ import annotations

import time

import numpy as np

import mpinputs as I


def make_requests(count: int, rate_hz: float, seed: int = 31, sizes=(2048, 8192, 32768),
                  weights=(8, 3, 1), nrhs: int = 1):
    reqs = I.serving_requests(count, rate_hz, seed, sizes, weights)
    for r in reqs:
        r["locs"] = I.points(r["n"], r["seed"])
        r["z"] = I.rhs(r["n"], nrhs, r["seed"])
    return reqs


def run(server, reqs, refine_iters: int = 0, release: bool = True, timeout_s: float = 600.0):
    """Submits every request at its arrival time (seconds from the start),
    polls until all finish.  Returns (results by index, wall seconds)."""
    t0 = time.perf_counter()
    ids = {}
    results = {}
    k = 0
    order = sorted(range(len(reqs)), key=lambda i: reqs[i]["arrival"])
    while len(results) < len(reqs):
        now = time.perf_counter() - t0
        while k < len(order) and reqs[order[k]]["arrival"] <= now:
            i = order[k]
            r = reqs[i]
            rid = server.submit(r["locs"], r["z"], (r["sigma2"], r["range"], r["nu"], r["nugget"]),
                                refine_iters)
            ids[rid] = i
            r["t_arrival_host"] = t0 + r["arrival"]
            k += 1
        for res in server.poll():
            i = ids[res["id"]]
            st, ll, quad = server.result(res["id"], reqs[i]["z"].shape[1])
            res["ll"], res["quad"] = ll, quad
            results[i] = res
            if release:
                server.release(res["id"])
        if time.perf_counter() - t0 > timeout_s:
            raise TimeoutError(f"{len(results)} of {len(reqs)} requests finished")
        if k < len(order) and not server.stats()["running"]:
            time.sleep(min(1e-3, max(0.0, reqs[order[k]]["arrival"] - (time.perf_counter() - t0))))
    wall = time.perf_counter() - t0
    return results, wall


def latency_stats(results):
    lat = np.array([r["t_done"] - r["t_submit"] for r in results.values()])
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "max_ms": float(lat.max() * 1e3)}
