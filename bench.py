#!/usr/bin/env python
"""Benchmark: mixed-precision tiled Cholesky log-likelihood on GB300.

One step = the whole hot path on one batch of synthetic input: Morton order
of the locations, Matérn tile generation into the per-tile formats, the
tiled Cholesky (FP64 POTRF/TRSM, lower-precision SYRK/GEMM), forward solve,
FP64 iterative refinement, log-determinant and log-likelihood.

Workload (default): n = 16384 Morton-ordered uniform points in [0,1]^2,
tile 512, Matérn nu = 3/2, range 0.05, variance 1, nugget 1e-4, one RHS
z ~ N(0,1); precision map: FP64 diagonal, FP32 for |i-j| <= 2, BF16 beyond
where the tile's norm allows it (norm guard eps = 1e-6; the plain band map
loses positive definiteness on this kernel -- its status is reported).

Metric: Cholesky TFLOP/s (useful flops n^3/3 + n^2/2 + n/6 per step, charged
whatever the precision), whole job over all ranks.  `--impl reference` times
the CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import mpinputs as I  # noqa: E402

METRIC = "Cholesky TFLOP/s vs all-FP64 GPU at matched loglik error; solves/s, p99 latency"
UNIT = "TFLOP/s"
WORKLOAD = "mixed_bf16_n16384_b512"


def chol_flops(n: int) -> float:
    return n ** 3 / 3.0 + n ** 2 / 2.0 + n / 6.0


def oracle_step_flops(nt: int, b: int, k: int) -> float:
    m = nt - k - 1
    return b ** 3 / 3.0 + m * b ** 3 + m * b * b * (b + 1) + m * (m - 1) / 2 * 2.0 * b ** 3


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--eps", type=float, default=1e-6)
    p.add_argument("--cpu-steps", type=int, default=7, help="oracle factorisation steps sampled")
    p.add_argument("--panel", default="ozaki", choices=["fp64", "ozaki"],
                   help="panel solve of tiles stored in FP32 or below: FP64 substitution, or "
                        "integer-digit products on the tensor cores")
    p.add_argument("--no-fp64-path", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--no-batch", action="store_true")
    p.add_argument("--no-sweep", action="store_true", help="skip the norm-guard eps sweep")
    p.add_argument("--no-sec5", action="store_true", help="skip the n=32768 crossprod/backsolve context")
    p.add_argument("--profile-case", default=None,
                   help="run one operation for a profiler and exit: gemm_<bf16|f16|f32|e4m3>_<n> "
                        "(crossprod through mp_gemm) or gen_nu<nu>_<n> (Matérn generation, b = 512)")
    p.add_argument("--no-fp8", action="store_true", help="skip the n=65536 E4M3 workload")
    p.add_argument("--no-trace", action="store_true", help="skip the traced factorisation (chain stamps)")
    p.add_argument("--fp8-eps", type=float, default=1e-6, help="norm guard of the E4M3 map (2-D field)")
    p.add_argument("--fp8-eps-ar1", type=float, default=1e-5, help="norm guard of the AR(1) check")
    p.add_argument("--batch-requests", type=int, default=512)
    p.add_argument("--serve-requests", type=int, default=48, help="burst that measures capacity")
    return p.parse_args()


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(values, ws, device=None):
    """Each timing's maximum over the ranks (one all-reduce; the caller
    brackets the timed region with barriers).  Identity for one rank."""
    if ws == 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def whole_job(ms_values, ws, flops_per_rank):
    """Whole-job TFLOP/s for each time in ms: every rank did flops_per_rank
    of work in (at most) that time."""
    return [ws * flops_per_rank / (ms * 1e-3) / 1e12 for ms in ms_values]


def cpu_cores():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS"):
        if os.environ.get(v):
            return int(os.environ[v])
    return os.cpu_count() or 1


def oracle_sample(cfg, pmap, steps: int, repeats: int = 1, warmup: int = 0):
    """Times the first `steps` steps of the oracle's tiled factorisation on
    the workload (generation and tile rounding excluded).  Returns a list of
    (seconds, flops) per repeat."""
    from oracle import chol as OC
    from oracle import matern as OM
    n, b = cfg["n"], cfg["b"]
    locs = I.points(n, cfg["seed"])
    if cfg["morton"]:
        locs, _ = OM.morton_order(locs)
    S = OM.covariance(locs, cfg["nu"], cfg["range"], cfg["sigma2"], cfg["nugget"])
    nt = -(-n // b)
    base = OC.tiled_from_dense(S, b, pmap)
    del S
    out = []
    for r in range(warmup + repeats):
        T = OC.TiledMatrix(n=base.n, b=b, nt=nt, pmap=base.pmap,
                           tiles={k: OC.Tile(v.codes.copy(), v.fmt, v.scale)
                                  for k, v in base.tiles.items()})
        t0 = time.perf_counter()
        for k in range(steps):
            OC.step(T, k)
        dt = time.perf_counter() - t0
        if r >= warmup:
            out.append((dt, sum(oracle_step_flops(nt, b, k) for k in range(steps))))
    return out


def measured_peaks():
    """Measured denominators (HBM copy GB/s, cuBLAS bf16 TFLOP/s)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "of measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "of fallback"


# DRAM bytes (read + write) per launch, dram__bytes_read.sum +
# dram__bytes_write.sum from one ncu capture of the kernel as it is now on
# this workload (kernel -> bytes); absent where no capture of the current
# kernel exists.
TRAFFIC_BYTES_PER_LAUNCH = {"k_potrf_dag": 1212672 + 7680}   # b = 512 diagonal tile


# digits per operand of the integer-digit panel product by the panel tile's
# format (the library's rule: FP32 8, BF16 and FP16 6, E4M3 5)
OZ_DIGITS = {I.F32: 8, I.BF16: 6, I.F16: 6, I.E4M3: 5}


def ozaki_executed_ratio(pmap):
    """MMA flops executed per TRSM flop of the integer-digit panel products
    over the map's panel tiles: s (s + 1) / 2 digit products of 2 b^3 flops
    against the b^3 of the solve, s = OZ_DIGITS of the tile (FP64 tiles take
    the FP64 substitution and are not counted)."""
    nt = pmap.shape[0]
    r = [OZ_DIGITS[int(pmap[i, k])] * (OZ_DIGITS[int(pmap[i, k])] + 1)
         for i in range(nt) for k in range(i) if int(pmap[i, k]) in OZ_DIGITS]
    return float(np.mean(r)) if r else 72.0


def tf32_sustained_tflops(seconds=1.0, n=8192):
    """TF32 tensor-core rate measured in this run: cuBLAS FP32 GEMMs with
    TF32 allowed, n^3, back to back for about `seconds` (the sustained rate
    under the power cap, the denominator for a kernel timed inside a long
    step); 2 n^3 flops per GEMM, CUDA events.  None if it cannot run."""
    import torch
    try:
        old = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = True
        a = torch.randn((n, n), device="cuda", dtype=torch.float32)
        c = torch.empty_like(a)
        for _ in range(3):
            torch.matmul(a, a, out=c)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps, t0 = 0, time.time()
        e0.record()
        while time.time() - t0 < seconds:
            for _ in range(10):
                torch.matmul(a, a, out=c)
            reps += 10
            torch.cuda.synchronize()
        e1.record()
        torch.cuda.synchronize()
        torch.backends.cuda.matmul.allow_tf32 = old
        ms = e0.elapsed_time(e1)
        del a, c
        return 2.0 * n ** 3 * reps / (ms * 1e-3) / 1e12
    except Exception:
        return None


def kernel_rooflines(prof, chol_ms, peak64, b, oz_ratio=72.0, tf32=None):
    """Roofline of the hot kernels of one factorisation; the dominant one
    (largest share of the instrumented run) first."""
    peaks, which = measured_peaks()
    bf16 = peaks["bf16_tflops_sustained"]
    # FP32-kind products are three TF32 MMAs: a third of the TF32 rate
    # measured in this run, else the nominal TF32/BF16 dense ratio 1.1/2.25
    # of the measured BF16 rate
    if tf32:
        tf32x3, tf32_src = tf32 / 3.0, "cuBLAS TF32 GEMM 8192^3 measured in this run (1 s loop) / 3"
    else:
        tf32x3, tf32_src = bf16 * (1.1 / 2.25) / 3.0, f"bf16_tflops_sustained {which} x 1.1/2.25 / 3"
    kinds = {
        "potrf_tile": ("k_potrf_dag", "alu", peak64,
                       "FP64 DFMA loop probe in this run (mp_probe_fp64_peak); achieved counts the "
                       "method's POTRF b^3/3 per diagonal tile (executed_tflops adds the b^3/3 of "
                       "the inverse W = L^-T it also forms)"),
        "panel_trsm_first": ("k_panel_trsm (chain)", "alu", peak64, "FP64 DFMA loop probe in this run"),
        "panel_trsm": ("k_panel_trsm (bulk)", "alu", peak64, "FP64 DFMA loop probe in this run"),
        "update_tc_3xtf32": ("k_update_tc_p (FP32 kind, 3 TF32 products)", "tensor", tf32x3, tf32_src),
        "update_tc_lowp": ("k_update_tc_p (BF16/FP16/E4M3 kinds)", "tensor", bf16,
                           f"bf16_tflops_sustained {which}"),
        "panel_ozaki_gemm": ("k_oz_gemm", "tensor", bf16,
                             f"bf16_tflops_sustained {which}; achieved counts the TRSM flops b^3 per tile"),
    }
    out = []
    for cls, (kname, bound, peak, src) in kinds.items():
        v = prof.get(cls)
        if not v or not v["launches"] or v["ms"] <= 0 or not peak:
            continue
        flops = v["flops"] / 2.0 if cls == "potrf_tile" else v["flops"]
        ach = flops / (v["ms"] * 1e-3) / 1e12
        r = {"bound": bound, "kernel": kname, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
             "frac": ach / peak, "peak_source": src,
             "traffic": TRAFFIC_BYTES_PER_LAUNCH.get(kname.split(" ")[0]),
             "launches": v["launches"], "ms_per_launch": v["ms"] / v["launches"],
             "flops_per_launch": flops / v["launches"],
             "share_of_chol": v["ms"] / chol_ms if chol_ms else None}
        if cls == "potrf_tile":
            r["executed_tflops"] = ach * 2.0
            r["executed_frac"] = ach * 2.0 / peak
        if cls == "panel_ozaki_gemm":
            # s (s + 1) / 2 digit products of 2 b^3 flops each per tile
            r["executed_per_algorithmic"] = oz_ratio
            r["executed_tflops"] = ach * oz_ratio
            r["executed_frac"] = ach * oz_ratio / peak
        out.append(r)
    out.sort(key=lambda r: -(r["share_of_chol"] or 0))
    if not out:
        return None
    dom = dict(out[0])
    dom["others"] = out[1:]
    return dom


def make_map(ctx, cfg, dsorted, eps):
    n, b = cfg["n"], cfg["b"]
    nt = -(-n // b)
    spec = cfg["map"]
    if spec[0] == "uniform":
        return I.uniform_map(nt, spec[1]), "uniform"
    _, diag, near, far, band = spec
    norms = ctx.tile_norms(n, b, dsorted, cfg["sigma2"], cfg["range"], cfg["nu"], cfg["nugget"])
    m = ctx.map_guarded(norms.cpu().numpy(), band, near, far, eps)
    return m, f"band{band}+guard(eps={eps:g})"


def reference_arm(args, cfg):
    ws, rank, _ = dist_setup(args)
    if rank != 0:
        return
    import torch  # noqa: F401  (the map planner runs on the GPU when one is present)
    from oracle import chol as OC
    from oracle import matern as OM
    n, b = cfg["n"], cfg["b"]
    nt = -(-n // b)
    locs = I.points(n, cfg["seed"])
    if cfg["morton"]:
        locs, _ = OM.morton_order(locs)
    spec = cfg["map"]
    if spec[0] == "uniform":
        pmap = I.uniform_map(nt, spec[1])
    else:
        S = OM.covariance(locs, cfg["nu"], cfg["range"], cfg["sigma2"], cfg["nugget"])
        pmap = OC.guarded_map(OC.tile_norms(S, b), spec[4], spec[2], spec[3], args.eps)
        del S
    # each of the K + W repeats samples 3 steps (about 5 s on 16 cores), so
    # that the whole run stays within a few minutes
    steps = max(1, min(3, args.cpu_steps, nt))
    res = oracle_sample(cfg, pmap, steps, repeats=args.steps, warmup=args.warmup)
    secs = sum(r[0] for r in res)
    fl = sum(r[1] for r in res)
    value = fl / secs / 1e12
    sample = f"first {steps} of {nt} steps of the oracle tiled factorisation per timed step"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / len(res) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "n": n, "b": b, "map": "same as ours"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


EPS_SWEEP = (1e-6, 3e-6, 1e-5, 3e-5, 1e-4)


def eps_sweep(ctx, cfg, dsorted, norms, zt, zmt, stream):
    """The norm guard's eps against the work it saves (untimed in the step):
    for each eps the map's tile counts, one factorisation graph and one full
    step timed with CUDA events, and the log-likelihoods for the bench's z
    and for a z drawn from the model (errors are taken against the FP64
    oracle by the caller)."""
    import torch
    from paper_2406_02701_gb300 import mpchol
    n, b = cfg["n"], cfg["b"]
    nt = -(-n // b)
    _, diag, near, far, band = cfg["map"]
    out = []
    for eps in EPS_SWEEP:
        m = ctx.map_guarded(norms, band, near, far, eps)
        low = int((m[np.tril_indices(nt, -1)] == far).sum())
        T = mpchol.TiledMatrix(ctx, n, b, m, keep_sigma=True)
        info = torch.zeros(1, dtype=torch.int64, device=zt.device)
        ld = torch.zeros(1, dtype=torch.float64, device=zt.device)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        for rep in range(2):
            ev[0].record(stream)
            T.generate(dsorted, cfg["sigma2"], cfg["range"], cfg["nu"], cfg["nugget"])
            ev[1].record(stream)
            ctx.check(ctx.lib.mp_chol(T.h, mpchol._ptr(info), mpchol._ptr(ld)))
            ev[2].record(stream)
            ll, _, it = T.loglik(zt, refine_iters=cfg["refine"])
            ev[3].record(stream)
        llm, _, itm = T.loglik(zmt, refine_iters=cfg["refine"]) if zmt is not None else (None, None, None)
        torch.cuda.synchronize()
        chol_ms = ev[1].elapsed_time(ev[2])
        out.append({"eps": eps, "far_tiles": low, "offdiag_tiles": nt * (nt - 1) // 2,
                    "info": int(info.item()), "chol_graph_ms": chol_ms,
                    "chol_graph_tflops": chol_flops(n) / (chol_ms * 1e-3) / 1e12,
                    "step_ms": ev[0].elapsed_time(ev[3]),
                    "refine_iters": int(it.max().item()), "logdet": float(ld.item()),
                    "loglik": ll.cpu().numpy().tolist(),
                    "loglik_model_z": llm.cpu().numpy().tolist() if llm is not None else None,
                    "refine_iters_model_z": int(itm.max().item()) if itm is not None else None})
        T.close()
        del T
    return out


def oracle_reference(cfg, sorted_locs, z):
    """O-exact for the bench workload (CPU-baseline leg: LAPACK on the host
    cores, outside every timed region): log-determinant and log-likelihood
    of the bench's z, and a z = L eps drawn from the model with its exact
    log-likelihood (quad = ||eps||^2)."""
    from oracle import chol as OC
    t0 = time.perf_counter()
    ex = OC.exact_loglik_field(sorted_locs, cfg["nu"], cfg["range"], cfg["sigma2"], cfg["nugget"],
                               z, keep_factor=True)
    eps = np.random.default_rng(99).standard_normal((sorted_locs.shape[0], 1))
    zm = np.tril(ex.pop("L")) @ eps
    llm = float(OC.loglik_value(sorted_locs.shape[0], ex["logdet"], float(eps[:, 0] @ eps[:, 0])))
    return {"logdet": ex["logdet"], "loglik": [float(v) for v in ex["loglik"]], "z_model": zm,
            "loglik_model_z": llm, "seconds": time.perf_counter() - t0, "cores": cpu_cores()}


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64))
                        / np.abs(np.asarray(b, dtype=np.float64))))


def fp8_workload(ctx, dev, eps_2d, eps_ar1, steps=3):
    """The FP8 configuration: n = 65536, tile 1024, FP64 diagonal, FP32 for
    |i - j| <= 2, E4M3 with per-tile scales beyond (where the norm guard
    allows it), 16 right-hand sides, FP64 refinement.  (a) the 2-D Matérn
    field (Morton-ordered uniform points, nu = 3/2, range 0.05, nugget 1e-4):
    one step (Morton, generation, factorisation, solves with refinement)
    timed over `steps` after a warm-up, its E4M3 tile count and refinement
    sweeps; (b) the same sizes and map rule on the nu = 1/2 field of equally
    spaced points on a line without nugget, whose covariance is AR(1): its
    log-likelihood error against the closed form."""
    import math
    import torch
    from paper_2406_02701_gb300 import mpchol
    c = I.CONFIGS["mixed_fp8_n65536_b1024"]
    n, b, nrhs = c["n"], c["b"], c["nrhs"]
    nt = n // b
    stream = torch.cuda.current_stream()
    dl = torch.from_numpy(I.points(n, c["seed"])).to(dev)
    zt = torch.from_numpy(np.ascontiguousarray(I.rhs(n, nrhs, c["seed"]).T)).to(dev)
    ds, _ = ctx.morton_order(dl)
    norms = ctx.tile_norms(n, b, ds, c["sigma2"], c["range"], c["nu"], c["nugget"]).cpu().numpy()
    m = ctx.map_guarded(norms, 2, I.F32, I.E4M3, eps_2d)
    low = int((m[np.tril_indices(nt, -1)] == I.E4M3).sum())
    T = mpchol.TiledMatrix(ctx, n, b, m, keep_sigma=True)
    info = torch.zeros(1, dtype=torch.int64, device=dev)
    ld = torch.zeros(1, dtype=torch.float64, device=dev)
    sb = torch.empty_like(dl)
    pb = torch.empty(n, dtype=torch.int64, device=dev)
    ph = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

    def step():
        ctx.check(ctx.lib.mp_morton_order(ctx.h, n, mpchol._ptr(dl), mpchol._ptr(sb), mpchol._ptr(pb),
                                          mpchol._stream(None)))
        T.generate(sb, c["sigma2"], c["range"], c["nu"], c["nugget"])
        ph[1].record(stream)
        ctx.check(ctx.lib.mp_chol(T.h, mpchol._ptr(info), mpchol._ptr(ld)))
        ph[2].record(stream)
        return T.loglik(zt, refine_iters=c["refine"])

    step()
    torch.cuda.synchronize()
    chol_ms = []
    ph[0].record(stream)
    for _ in range(steps):
        ll, q, it = step()
        torch.cuda.synchronize()
        chol_ms.append(ph[1].elapsed_time(ph[2]))
    ph[3].record(stream)
    torch.cuda.synchronize()
    # the synchronisations between steps are inside the bracket: the step
    # time is their sum, each step's own time is what the events measure
    ms = ph[0].elapsed_time(ph[3]) / steps
    res = {"workload": "mixed_fp8_n65536_b1024", "n": n, "b": b, "nrhs": nrhs, "map": f"band2+guard(eps={eps_2d:g})",
           "e4m3_tiles": low, "f32_tiles": int((m[np.tril_indices(nt, -1)] == I.F32).sum()),
           "offdiag_tiles": nt * (nt - 1) // 2, "info": int(info.item()),
           "ms_per_step": ms, "tflops_step": chol_flops(n) / (ms * 1e-3) / 1e12,
           "chol_graph_ms": float(np.median(chol_ms)),
           "chol_graph_tflops": chol_flops(n) / (float(np.median(chol_ms)) * 1e-3) / 1e12,
           "refine_iters": it.cpu().numpy().tolist()}
    T.close()
    del T
    # AR(1) closed form at the same sizes (range 0.005: rho = 0.99695, the
    # E4M3 rounding allowed by the guard stays below the smallest eigenvalue)
    a, s2 = 0.005, 1.0
    h = 1.0 / n
    rho = math.exp(-h / a)
    z = I.ar1_rhs(n, nrhs, rho, s2, c["seed"])
    dl1 = torch.from_numpy(I.points_line(n, h)).to(dev)
    norms1 = ctx.tile_norms(n, b, dl1, s2, a, 0.5, 0.0).cpu().numpy()
    m1 = ctx.map_guarded(norms1, 2, I.F32, I.E4M3, eps_ar1)
    T1 = mpchol.TiledMatrix(ctx, n, b, m1, keep_sigma=True)
    T1.generate(dl1, s2, a, 0.5, 0.0)
    info1, ld1 = T1.chol()
    ll1, _, it1 = T1.loglik(torch.from_numpy(np.ascontiguousarray(z.T)).to(dev), refine_iters=10)
    torch.cuda.synchronize()
    ldx = n * math.log(s2) + (n - 1) * math.log(1 - rho * rho)
    qx = (z[0] ** 2 + np.sum((z[1:] - rho * z[:-1]) ** 2, axis=0) / (1 - rho * rho)) / s2
    llx = -0.5 * n * math.log(2 * math.pi) - 0.5 * ldx - 0.5 * qx
    res["ar1_closed_form"] = {
        "what": "nu=1/2, range 0.005, no nugget, n equally spaced points on a line (AR(1)); 16 RHS "
                "drawn from the model; same tile size, band and E4M3 guard",
        "map": f"band2+guard(eps={eps_ar1:g})",
        "e4m3_tiles": int((m1[np.tril_indices(nt, -1)] == I.E4M3).sum()), "info": int(info1.item()),
        "loglik_rel_err_max": rel(ll1.cpu().numpy(), llx),
        "logdet_rel_err": abs(ld1.item() - ldx) / abs(ldx),
        "refine_iters": it1.cpu().numpy().tolist()}
    T1.close()
    return res


def general_nu_generation(ctx, cfg, dsorted, pmap, stream, nus=(1.0, 0.3, 2.2)):
    """Generation time of the bench workload's matrix (same points, map and
    range) for nu without a closed form (the per-nu Chebyshev table of
    x^nu K_nu(x), built on the host at the first call of a nu and uploaded)
    against the closed form nu = 3/2; CUDA events around one generation
    after a warm-up."""
    import torch
    from paper_2406_02701_gb300 import mpchol
    n, b = cfg["n"], cfg["b"]
    T = mpchol.TiledMatrix(ctx, n, b, pmap, keep_sigma=True)
    out = {}
    for nu in (1.5,) + tuple(nus):
        t0 = time.perf_counter()
        T.generate(dsorted, cfg["sigma2"], cfg["range"], nu, cfg["nugget"])
        torch.cuda.synchronize()
        first_s = time.perf_counter() - t0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        T.generate(dsorted, cfg["sigma2"], cfg["range"], nu, cfg["nugget"])
        e1.record(stream)
        torch.cuda.synchronize()
        out[f"nu={nu:g}"] = {"generate_ms": e0.elapsed_time(e1), "first_call_s": first_s}
    T.close()
    return out


def sec5_operations(ctx, dev, stream, n=32768):
    """The paper's standalone operation benchmark at its largest size
    (Sec. 5: crossprod and backsolve at n = 32768), for context: crossprod
    X^T X through mp_gemm in each lower format on the tensor cores
    (2 n^3 flops; a few entries checked against float64 dot products of
    the rounded inputs), and the triangular solve with a mixed-precision
    factor of an n = 32768 Matérn matrix (mp_trsm, FP64 arithmetic, n^2
    flops per right-hand side) for 16 and 256 right-hand sides."""
    import torch
    from paper_2406_02701_gb300 import mpchol
    out = {"n": n, "crossprod": {}, "backsolve": {}}
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    X64 = torch.randn((n, n), generator=g, dtype=torch.float32, device=dev)
    rows = [3, 1000, 32000]
    cols = [7, 20000, 32767]
    for name, dt, tdt in [("bf16", mpchol.MP_BF16, torch.bfloat16), ("f16", mpchol.MP_F16, torch.float16),
                          ("f32", mpchol.MP_F32, torch.float32), ("e4m3", mpchol.MP_E4M3, torch.float8_e4m3fn)]:
        X = X64.to(tdt)
        Cm = torch.zeros((n, n), dtype=tdt, device=dev)
        args = (dt, "T", "N", n, n, n, 1.0, X, n, X, n, 0.0, Cm, n)
        ctx.gemm(*args)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.gemm(*args)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        # storage is column-major: element (r, c) of C sits at C_t[c, r]
        Xh = X.to(torch.float64)
        err = 0.0
        for r, c in zip(rows, cols):
            exact = float(torch.dot(Xh[r], Xh[c]))        # column r of X . column c of X
            got = float(Cm[c, r].to(torch.float64))
            scale = float(torch.dot(Xh[r].abs(), Xh[c].abs()))
            err = max(err, abs(got - exact) / scale)
        out["crossprod"][name] = {"ms": ms, "tflops": 2.0 * n ** 3 / (ms * 1e-3) / 1e12,
                                  "sampled_err_rel_to_sum_abs": err}
        del X, Cm, Xh
        torch.cuda.empty_cache()
    del X64
    torch.cuda.empty_cache()
    # backsolve with a mixed-precision factor (guarded BF16 map, b = 512)
    b = 512
    ds, _ = ctx.morton_order(torch.from_numpy(I.points(n, 77)).to(dev))
    norms = ctx.tile_norms(n, b, ds, 1.0, 0.05, 1.5, 1e-4).cpu().numpy()
    pm = ctx.map_guarded(norms, 2, I.F32, I.BF16, 1e-6)
    T = mpchol.TiledMatrix(ctx, n, b, pm)
    T.generate(ds, 1.0, 0.05, 1.5, 1e-4)
    info, _ = T.chol()
    torch.cuda.synchronize()
    out["backsolve"]["factor_info"] = int(info.item())
    for nrhs in (16, 256):
        Bt = torch.randn((nrhs, n), dtype=torch.float64, device=dev)
        T.trsm(Bt, 1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        T.trsm(Bt, 1)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out["backsolve"][f"nrhs={nrhs}"] = {"ms": ms, "tflops": float(n) ** 2 * nrhs / (ms * 1e-3) / 1e12}
    T.close()
    out["paper_context"] = {"hardware": "the paper's GPU (cuBLAS/cuSOLVER), Sec. 5",
                            "crossprod_s": {"double": 10.22, "single": 5.02, "half": 0.811},
                            "backsolve_s": {"double": 5.49, "single": 2.88},
                            "chol_s": {"double": 2.81, "single": 1.05}}
    return out


def potrf_chain(ctx, cfg, g, pmap, panel):
    """The factorisation's critical chain from the diagonal tiles' stamps
    (one traced factorisation of the bench matrix, untimed): per diagonal
    block, the cycles of each phase of its chain task (medians over blocks
    k >= 1 of all tiles), the hand-off between consecutive chain tasks, the
    model sum against the measured block-to-block time, and per diagonal
    tile its span and the gap to the next tile's first chain task."""
    import torch
    from paper_2406_02701_gb300 import mpchol
    n, b = cfg["n"], cfg["b"]
    T = mpchol.TiledMatrix(ctx, n, b, pmap, ozaki=panel == "ozaki", flags=mpchol.MP_TMAT_TRACE)
    T.generate(g, cfg["sigma2"], cfg["range"], cfg["nu"], cfg["nugget"])
    T.chol()
    T.generate(g, cfg["sigma2"], cfg["range"], cfg["nu"], cfg["nugget"])
    info, _ = T.chol()
    torch.cuda.synchronize()
    ns, cyc, db = T.chain_trace()
    T.close()
    nt, nbb = ns.shape[0], ns.shape[1]
    # SM clock seen by the chain tasks: cycles per ns over whole tasks
    ghz = float(np.sum(cyc[:, :, 7] - cyc[:, :, 0]) / max(1, np.sum(ns[:, :, 7] - ns[:, :, 0])))
    d = np.diff(cyc, axis=2)[:, 1:, :]           # blocks k >= 1: phases 0-1 ... 6-7
    names = ["wait_inputs", "wait_inverse", "solve_publish", "update_block", "factor", "publish",
             "inverse_logdet_tail"]
    med = {k: float(np.median(d[:, :, i])) for i, k in enumerate(names)}
    handoff_ns = ns[:, 1:, 2] - ns[:, :-1, 5]     # previous block factored -> inverse seen
    step_ns = ns[:, 1:, 5] - ns[:, :-1, 5]        # block-to-block time on the chain
    model = med["wait_inverse"] + med["solve_publish"] + med["update_block"] + med["factor"]
    span_ns = ns[:, -1, 6] - ns[:, 0, 0]
    gap_ns = ns[1:, 0, 0] - ns[:-1, -1, 6]
    return {
        "info": int(info.item()), "block": db, "blocks_per_tile": nbb, "sm_ghz_seen": ghz,
        "phase_cycles_median": med,
        "factor_cycles_per_column": med["factor"] / db,
        "handoff_ns_median": float(np.median(handoff_ns)),
        "block_step_cycles_median": float(np.median(step_ns)) * ghz,
        "model_cycles_per_block": model,
        "tile_span_ms_median": float(np.median(span_ns)) * 1e-6,
        "tile_span_ms_sum": float(np.sum(span_ns)) * 1e-6,
        "gap_to_next_tile_ms_median": float(np.median(gap_ns)) * 1e-6 if nt > 1 else None,
        "gap_to_next_tile_ms_sum": float(np.sum(gap_ns)) * 1e-6 if nt > 1 else None,
        "chain_ms": float(ns[-1, -1, 6] - ns[0, 0, 0]) * 1e-6,
        "tile_span_ms_first_last": [float(span_ns[0]) * 1e-6, float(span_ns[-1]) * 1e-6],
    }


def cusolver_context(dev, cfg, dsorted, stream):
    """Context only: the vendor FP64 Cholesky (torch.linalg.cholesky, which
    calls cuSOLVER's potrf) of the same covariance as one dense n x n FP64
    matrix built with torch operations; timed with CUDA events after a
    warm-up."""
    import torch
    if cfg["nu"] != 1.5:
        return None
    x = torch.cdist(dsorted, dsorted) / cfg["range"]
    S = cfg["sigma2"] * (1.0 + x) * torch.exp(-x)
    del x
    S.diagonal().add_(cfg["nugget"])
    L = torch.linalg.cholesky(S)
    del L
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    L = torch.linalg.cholesky(S)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    n = S.shape[0]
    del L, S
    torch.cuda.empty_cache()
    return {"what": "torch.linalg.cholesky (cuSOLVER potrf) of the dense FP64 covariance",
            "ms": ms, "tflops": chol_flops(n) / (ms * 1e-3) / 1e12}


def batch_run(ctx, args, dev):
    """512 independent Matérn likelihoods (n ~ U{256..4096}, range ~ U[0.02,
    0.3], nu ~ U{1/2, 3/2, 5/2}), FP64 diagonal / FP32 band / BF16 where the
    norm bound allows (a map rule, rebuilt at each tile size), Morton-ordered
    points, one CUDA graph launch for all (generation, factorisation, solve,
    log-likelihood).  The autotuner picks the tile size and schedule flags
    by timing candidate plans of this batch; the tuned plan and the default
    schedule (b = 256, no flags) are each timed over 3 launches after one
    warm-up."""
    import torch
    from paper_2406_02701_gb300 import mpchol
    reqs = I.batch_requests(args.batch_requests, seed=31)
    specs = []
    flops = 0.0
    for r in reqs:
        n = r["n"]
        ds, _ = ctx.morton_order(torch.from_numpy(I.points(n, r["seed"])).to(dev))
        zt = torch.from_numpy(np.ascontiguousarray(I.rhs(n, 1, r["seed"]).T)).to(dev)
        specs.append(dict(n=n, locs=ds, zt=zt, sigma2=r["sigma2"], range=r["range"], nu=r["nu"],
                          nugget=r["nugget"], rule=(2, I.F32, I.BF16, 1e-6)))
        flops += chol_flops(n)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tuned = mpchol.tune_batch(ctx, specs)
    tune_s = time.perf_counter() - t0

    def timed(b, flags):
        t1 = time.perf_counter()
        B = mpchol.Batch(ctx, specs, b=b, flags=flags)
        plan_s = time.perf_counter() - t1
        ll, st = B.run()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            B.run(ll, st)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        info = B.info()
        ok = int((st.cpu().numpy() == 0).sum())
        B.close()
        return {"b": info["b"], "flags": info["flags"], "ok": ok, "ms_per_launch": ms,
                "solves_per_s": len(specs) / (ms * 1e-3), "chol_tflops": flops / (ms * 1e-3) / 1e12,
                "plan_build_s": plan_s, "device_bytes": info["bytes"]}

    best = timed(tuned["b"], tuned["flags"])
    default = timed(256, 0)
    return {"requests": len(specs), **best,
            "tuner": {"b": tuned["b"], "flags": tuned["flags"], "flags_names": flag_names(tuned["flags"]),
                      "candidates_timed": tuned["tried"], "tuning_s": tune_s, "tuner_ms": tuned["ms"]},
            "default_schedule": default}


def flag_names(flags):
    from paper_2406_02701_gb300 import mpchol
    names = {mpchol.MP_TMAT_SIMT_UPDATES: "simt_updates", mpchol.MP_TMAT_FP64_PANEL: "fp64_panel",
             mpchol.MP_TMAT_DAG16: "dag16", mpchol.MP_TMAT_DAG32: "dag32",
             mpchol.MP_TMAT_LOWP_RING4: "lowp_ring4"}
    return [v for k, v in names.items() if flags & k]


def serving_run(ctx, args):
    """Continuous batching of a Poisson stream of likelihood requests:
    n in {2048, 8192, 32768} at 8:3:1, Matérn parameters drawn as in an MLE
    search, 1 RHS, 3 refinement sweeps at most, far tiles BF16 where the
    norm bound allows (eps 1e-6), b and schedule per size from the
    autotuner.  Capacity: a burst of requests all arriving at once; then
    offered load swept from 0.2x to 1.2x of that capacity, p50/p99 latency
    (arrival to result seen by the poller) and throughput at each level, and
    the split of latency into admission (queueing and host planning up to
    the moment the work is enqueued) and device time."""
    from paper_2406_02701_gb300 import mpchol, serving
    srv = mpchol.Server(ctx, hbm_budget=200 << 30, max_slots=8, eps=1e-6, far=mpchol.MP_BF16)
    t0 = time.perf_counter()
    srv.tune([2048, 8192, 32768], refine_iters=3)
    tune_s = time.perf_counter() - t0
    warm = serving.make_requests(3, 1e6, seed=7, sizes=(2048,), weights=(1,))
    for r in warm:
        r["arrival"] = 0.0
    serving.run(srv, warm, refine_iters=3)
    burst = serving.make_requests(args.serve_requests, 1e6, seed=31)
    for r in burst:
        r["arrival"] = 0.0
    _, wall = serving.run(srv, burst, refine_iters=3)
    capacity = len(burst) / wall
    levels = []
    for f in (0.2, 0.5, 0.8, 1.0, 1.2):
        rate = f * capacity
        count = int(min(150, max(40, round(6.0 * rate))))
        reqs = serving.make_requests(count, rate, seed=1000 + int(100 * f))
        res, wall = serving.run(srv, reqs, refine_iters=3)
        lat = serving.latency_stats(res)
        by_n = {}
        for i, r in res.items():
            by_n.setdefault(reqs[i]["n"], []).append(r)
        split = {str(k): {"p50_ms": float(np.percentile([(r["t_done"] - r["t_submit"]) * 1e3 for r in v], 50)),
                          "admission_p50_ms": float(np.percentile([(r["t_admit"] - r["t_submit"]) * 1e3 for r in v], 50)),
                          "device_p50_ms": float(np.percentile([(r["t_done"] - r["t_admit"]) * 1e3 for r in v], 50)),
                          "b": int(v[0]["b"]), "count": len(v)} for k, v in sorted(by_n.items())}
        ok = sum(1 for r in res.values() if r["status"] == 0)
        levels.append({"load": f, "rate_hz": rate, "requests": count, "ok": ok, "wall_s": wall,
                       "solves_per_s": count / wall, **lat, "by_n": split})
    srv.close()
    return {"capacity_solves_per_s": capacity, "capacity_burst": len(burst), "tuning_s": tune_s,
            "slots": 8, "mix": "n 2048/8192/32768 at 8:3:1, Poisson arrivals", "levels": levels}


def morton_launches(n: int) -> int:
    n2 = 1024
    while n2 < n:
        n2 <<= 1
    c = 3   # keys, first local sort, gather
    k = 2048
    while k <= n2:
        j = k >> 1
        while j >= 1024:
            c += 1
            j >>= 1
        c += 1
        k <<= 1
    return c


def ours(args, cfg):
    import torch
    import torch.distributed as dist
    from paper_2406_02701_gb300 import mpchol

    ws, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    n, b, nrhs, refine = cfg["n"], cfg["b"], cfg["nrhs"], cfg["refine"]
    nt = -(-n // b)
    ctx = mpchol.Context(local)
    # replicas: every rank evaluates its own independent likelihood
    locs_h = torch.from_numpy(I.points(n, cfg["seed"] + 100 * rank)).pin_memory()
    z_h = torch.from_numpy(np.ascontiguousarray(I.rhs(n, nrhs, cfg["seed"] + 100 * rank).T)).pin_memory()
    ll_h = torch.empty(nrhs, dtype=torch.float64).pin_memory()
    dl = locs_h.to(dev)
    zt = z_h.to(dev)
    stream = torch.cuda.current_stream()
    dsorted, dperm = ctx.morton_order(dl)
    if not cfg["morton"]:
        dsorted = dl.clone()
    torch.cuda.synchronize()
    pmap, map_name = make_map(ctx, cfg, dsorted, args.eps)
    counts = {int(k): int(v) for k, v in zip(*np.unique(pmap[np.tril_indices(nt)], return_counts=True))}

    # status of the plain band map on this workload (untimed)
    band_status = None
    if cfg["map"][0] == "band" and rank == 0:
        Tb = mpchol.TiledMatrix(ctx, n, b, I.make_map(cfg["map"], nt))
        Tb.generate(dsorted, cfg["sigma2"], cfg["range"], cfg["nu"], cfg["nugget"])
        info, _ = Tb.chol()
        torch.cuda.synchronize()
        band_status = {"map": "band (no guard)", "info": int(info.item())}
        Tb.close()
        del Tb

    T = mpchol.TiledMatrix(ctx, n, b, pmap, keep_sigma=refine > 0, ozaki=args.panel == "ozaki")
    ll = torch.empty(nrhs, dtype=torch.float64, device=dev)
    quad = torch.empty(nrhs, dtype=torch.float64, device=dev)
    iters = torch.empty(nrhs, dtype=torch.int32, device=dev)
    sorted_buf = torch.empty_like(dl)
    perm_buf = torch.empty(n, dtype=torch.int64, device=dev)
    info = torch.zeros(1, dtype=torch.int64, device=dev)
    logdet = torch.zeros(1, dtype=torch.float64, device=dev)

    def step(src):
        if cfg["morton"]:
            ctx.check(ctx.lib.mp_morton_order(ctx.h, n, mpchol._ptr(src), mpchol._ptr(sorted_buf),
                                              mpchol._ptr(perm_buf), mpchol._stream(None)))
            g = sorted_buf
        else:
            g = src
        T.generate(g, cfg["sigma2"], cfg["range"], cfg["nu"], cfg["nugget"])
        ctx.check(ctx.lib.mp_chol(T.h, mpchol._ptr(info), mpchol._ptr(logdet)))
        T.loglik(zt, refine_iters=refine, ll=ll, quad=quad, iters=iters)

    for _ in range(args.warmup):
        step(dl)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(dl)
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    # e2e: host buffers in, result out, every step
    ee0 = torch.cuda.Event(enable_timing=True)
    ee1 = torch.cuda.Event(enable_timing=True)
    ee0.record(stream)
    for _ in range(args.steps):
        dl.copy_(locs_h, non_blocking=True)
        zt.copy_(z_h, non_blocking=True)
        step(dl)
        ll_h.copy_(ll, non_blocking=True)
    ee1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_e2e = ee0.elapsed_time(ee1) / args.steps
    ms, ms_e2e = max_over_ranks([ms, ms_e2e], ws, device=dev)
    F = chol_flops(n)
    value, value_e2e = whole_job([ms, ms_e2e], ws, F)
    stats = T.stats()
    launches_per_step = (morton_launches(n) if cfg["morton"] else 0) + stats["generate"] + \
        stats["chol"] + 1 + stats["loglik"]
    ll_mixed = ll.cpu().numpy().copy()
    iters_mixed = iters.cpu().numpy().copy()
    info_mixed = int(info.item())
    logdet_mixed = float(logdet.item())

    if rank != 0:
        if ws > 1:
            dist.barrier()
        return

    # phase breakdown of one step (CUDA events on the stream, graphs as timed)
    ph = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    ph[0].record(stream)
    if cfg["morton"]:
        ctx.check(ctx.lib.mp_morton_order(ctx.h, n, mpchol._ptr(dl), mpchol._ptr(sorted_buf),
                                          mpchol._ptr(perm_buf), mpchol._stream(None)))
    ph[1].record(stream)
    T.generate(sorted_buf if cfg["morton"] else dl, cfg["sigma2"], cfg["range"], cfg["nu"],
               cfg["nugget"])
    ph[2].record(stream)
    ctx.check(ctx.lib.mp_chol(T.h, mpchol._ptr(info), mpchol._ptr(logdet)))
    ph[3].record(stream)
    T.loglik(zt, refine_iters=refine, ll=ll, quad=quad, iters=iters)
    ph[4].record(stream)
    torch.cuda.synchronize()
    phases = {k: ph[i].elapsed_time(ph[i + 1]) for i, k in
              enumerate(["morton_ms", "generate_ms", "chol_graph_ms", "loglik_refine_ms"])}

    # kernel breakdown (one instrumented factorisation, CUDA events on the stream)
    prof = T.profile()
    chol_ms = sum(v["ms"] for v in prof.values())
    roofline = kernel_rooflines(prof, chol_ms, ctx.fp64_peak(), b, ozaki_executed_ratio(pmap),
                                tf32_sustained_tflops())
    breakdown = {k: {"ms": round(v["ms"], 3), "launches": v["launches"],
                     "tflops": round(v["flops"] / (v["ms"] * 1e-3) / 1e12, 3) if v["ms"] > 0 and v["flops"] > 0 else None}
                 for k, v in prof.items() if v["launches"]}

    chain = None
    if not args.no_trace:
        chain = potrf_chain(ctx, cfg, sorted_buf if cfg["morton"] else dl, pmap, args.panel)

    # CPU-baseline leg, part 1: the FP64 oracle's log-likelihood of this
    # workload (LAPACK on the host cores), and the mixed result for a z drawn
    # from the model
    ref, err = None, None
    if not args.no_cpu_baseline and cfg["map"][0] == "band":
        ref = oracle_reference(cfg, dsorted.cpu().numpy(), I.rhs(n, nrhs, cfg["seed"]))
        zmt = torch.from_numpy(np.ascontiguousarray(ref["z_model"].T)).to(dev)
        T.generate(sorted_buf if cfg["morton"] else dl, cfg["sigma2"], cfg["range"], cfg["nu"],
                   cfg["nugget"])
        ctx.check(ctx.lib.mp_chol(T.h, mpchol._ptr(info), mpchol._ptr(logdet)))
        llm, _, itm = T.loglik(zmt, refine_iters=refine)
        torch.cuda.synchronize()
        err = {"reference": f"FP64 oracle: LAPACK dpotrf on {ref['cores']} host cores "
                            f"({ref['seconds']:.1f} s, outside the timed region)",
               "loglik_rel_err": rel(ll_mixed, ref["loglik"]),
               "logdet_rel_err": abs(logdet_mixed - ref["logdet"]) / abs(ref["logdet"]),
               "loglik_rel_err_model_z": rel(llm.cpu().numpy(), ref["loglik_model_z"]),
               "refine_iters_model_z": int(itm.max().item()),
               "target": 1e-6}
        # the same map with every lower-precision update on the CUDA cores
        # (IEEE FP32 accumulation, as the method states it): the tensor
        # cores' FP32 accumulation rounds toward zero, a bias that reaches
        # the (unrefined) log-determinant
        Ts = mpchol.TiledMatrix(ctx, n, b, pmap, keep_sigma=True, simt_updates=True,
                                ozaki=args.panel == "ozaki")
        g = sorted_buf if cfg["morton"] else dl
        Ts.generate(g, cfg["sigma2"], cfg["range"], cfg["nu"], cfg["nugget"])
        ctx.check(ctx.lib.mp_chol(Ts.h, mpchol._ptr(info), mpchol._ptr(logdet)))
        torch.cuda.synchronize()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        Ts.generate(g, cfg["sigma2"], cfg["range"], cfg["nu"], cfg["nugget"])
        s0.record(stream)
        ctx.check(ctx.lib.mp_chol(Ts.h, mpchol._ptr(info), mpchol._ptr(logdet)))
        s1.record(stream)
        lls, _, _ = Ts.loglik(zt, refine_iters=refine)
        llsm, _, _ = Ts.loglik(zmt, refine_iters=refine)
        torch.cuda.synchronize()
        err["cuda_core_updates"] = {
            "chol_graph_ms": s0.elapsed_time(s1),
            "chol_graph_tflops": chol_flops(n) / (s0.elapsed_time(s1) * 1e-3) / 1e12,
            "logdet_rel_err": abs(logdet.item() - ref["logdet"]) / abs(ref["logdet"]),
            "loglik_rel_err": rel(lls.cpu().numpy(), ref["loglik"]),
            "loglik_rel_err_model_z": rel(llsm.cpu().numpy(), ref["loglik_model_z"])}
        Ts.close()
        del Ts

    # the all-FP64 GPU path on the same workload (speedup and error reference)
    fp64 = None
    if not args.no_fp64_path:
        del T
        T64 = mpchol.TiledMatrix(ctx, n, b, None, keep_sigma=False)
        g = sorted_buf if cfg["morton"] else dl
        T64.generate(g, cfg["sigma2"], cfg["range"], cfg["nu"], cfg["nugget"])
        info64 = torch.zeros(1, dtype=torch.int64, device=dev)
        ld64 = torch.zeros(1, dtype=torch.float64, device=dev)
        ctx.check(ctx.lib.mp_chol(T64.h, mpchol._ptr(info64), mpchol._ptr(ld64)))  # warm-up
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        T64.generate(g, cfg["sigma2"], cfg["range"], cfg["nu"], cfg["nugget"])
        f0.record(stream)
        ctx.check(ctx.lib.mp_chol(T64.h, mpchol._ptr(info64), mpchol._ptr(ld64)))
        f1.record(stream)
        ll64, _, _ = T64.loglik(zt, refine_iters=0)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1)
        ll64 = ll64.cpu().numpy()
        fp64 = {"chol_ms": ms64, "tflops": F / (ms64 * 1e-3) / 1e12, "info": int(info64.item()),
                "speedup_chol_only": ms64 / chol_ms if chol_ms else None,
                "speedup_chol_graph": ms64 / phases["chol_graph_ms"],
                "speedup_step": ms64 / ms,
                "loglik_rel_err_mixed_vs_fp64": (np.abs(ll_mixed - ll64) / np.abs(ll64)).tolist(),
                "loglik_rel_err_vs_oracle": rel(ll64, ref["loglik"]) if ref else None}
        T64.close()
        del T64
        fp64["cusolver_context"] = cusolver_context(dev, cfg, sorted_buf if cfg["morton"] else dl, stream)

    sweep = None
    if not args.no_sweep and cfg["map"][0] == "band":
        norms = ctx.tile_norms(n, b, sorted_buf if cfg["morton"] else dl, cfg["sigma2"], cfg["range"],
                               cfg["nu"], cfg["nugget"]).cpu().numpy()
        sweep = eps_sweep(ctx, cfg, sorted_buf if cfg["morton"] else dl, norms, zt,
                          torch.from_numpy(np.ascontiguousarray(ref["z_model"].T)).to(dev) if ref else None,
                          stream)
        if ref:
            for e in sweep:
                e["loglik_rel_err"] = rel(e["loglik"], ref["loglik"])
                e["logdet_rel_err"] = abs(e["logdet"] - ref["logdet"]) / abs(ref["logdet"])
                if e["loglik_model_z"] is not None:
                    e["loglik_rel_err_model_z"] = rel(e["loglik_model_z"], ref["loglik_model_z"])
        for e in sweep:
            e.pop("loglik", None)
            e.pop("loglik_model_z", None)

    gen_nu = None
    if not args.no_sweep:
        gen_nu = general_nu_generation(ctx, cfg, sorted_buf if cfg["morton"] else dl, pmap, stream)

    fp8 = None
    if not args.no_fp8:
        fp8 = fp8_workload(ctx, dev, args.fp8_eps, args.fp8_eps_ar1)

    sec5 = None
    if not args.no_sec5:
        sec5 = sec5_operations(ctx, dev, stream)

    batch = None
    if not args.no_batch:
        batch = batch_run(ctx, args, dev)

    serve = None
    if not args.no_serving:
        serve = serving_run(ctx, args)

    cpu = None
    if not args.no_cpu_baseline:
        steps = max(1, min(args.cpu_steps, nt))
        res = oracle_sample(cfg, pmap, steps)
        secs, fl = res[0]
        cpu = {"value": fl / secs / 1e12, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
               "sample": f"first {steps} of {nt} tiled-factorisation steps of the oracle on the "
                         f"same workload and map ({secs:.1f} s; generation excluded)"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32+bf16", "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "b": b, "nu": cfg["nu"],
                   "range": cfg["range"], "nugget": cfg["nugget"], "nrhs": nrhs,
                   "refine_iters_max": refine, "morton": cfg["morton"], "map": map_name,
                   "panel_solve": args.panel,
                   "tiles_per_format": {I.DTYPE_NAMES[k]: v for k, v in counts.items()},
                   "l2": "inputs larger than L2 (tiles + float64 Sigma copy > 1 GB)",
                   "parallelism": f"replicas x{ws}"},
        "e2e": {"value": value_e2e, "unit": UNIT, "h2d_bytes_per_step": int(locs_h.numel() * 8 + z_h.numel() * 8),
                "d2h_bytes_per_step": int(ll_h.numel() * 8), "ms_per_step": ms_e2e},
        "gpu_launches": int(launches_per_step * args.steps),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "clocks": clk,
        "result": {"info": info_mixed, "loglik": ll_mixed.tolist(), "logdet": logdet_mixed,
                   "refine_iters": iters_mixed.tolist(), "plain_band_map": band_status},
        "fp64_path": fp64,
        "error_vs_oracle": err,
        "eps_sweep": sweep,
        "fp8_workload": fp8,
        "general_nu_generation": gen_nu,
        "sec5_operations_n32768": sec5,
        "chol_graph_tflops": F / (phases["chol_graph_ms"] * 1e-3) / 1e12,
        "serving": serve,
        "batch": batch,
        "chol_breakdown_ms": breakdown,
        "potrf_chain": chain,
        "step_phases_ms": phases,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()


def profile_case(name):
    """One operation, twice (the second is the one to capture), for ncu."""
    import torch
    from paper_2406_02701_gb300 import mpchol
    dev = torch.device("cuda", 0)
    ctx = mpchol.Context(0)
    kind, _, size = name.rpartition("_")
    n = int(size)
    if kind.startswith("gemm_"):
        fmt = kind[len("gemm_"):]
        dt, tdt = {"bf16": (mpchol.MP_BF16, torch.bfloat16), "f16": (mpchol.MP_F16, torch.float16),
                   "f32": (mpchol.MP_F32, torch.float32), "e4m3": (mpchol.MP_E4M3, torch.float8_e4m3fn)}[fmt]
        X = torch.randn((n, n), dtype=torch.float32, device=dev).to(tdt)
        Cm = torch.zeros((n, n), dtype=tdt, device=dev)
        for _ in range(2):
            ctx.gemm(dt, "T", "N", n, n, n, 1.0, X, n, X, n, 0.0, Cm, n)
    elif kind.startswith("gen_nu") or kind.startswith("gen64_nu"):
        # gen64: with the copy of Sigma the log-likelihood refines
        # against, as in the bench's step (every entry float64-accurate)
        nu = float(kind[kind.index("nu") + 2:])
        ds, _ = ctx.morton_order(torch.from_numpy(I.points(n, 11)).to(dev))
        T = mpchol.TiledMatrix(ctx, n, 512, I.band_map(-(-n // 512), I.F64, I.F32, I.BF16, 2),
                               keep_sigma=kind.startswith("gen64"))
        for _ in range(2):
            T.generate(ds, 1.0, 0.05, nu, 1e-4)
    elif kind == "chol":
        # the factorisation of an n-point field, b = 512, FP64 diagonal and
        # FP32 elsewhere (the diagonal tile's task graph is the same launch
        # whatever n)
        ds, _ = ctx.morton_order(torch.from_numpy(I.points(n, 11)).to(dev))
        nt = -(-n // 512)
        T = mpchol.TiledMatrix(ctx, n, 512, I.band_map(nt, I.F64, I.F32, I.F32, 1))
        for _ in range(2):
            T.generate(ds, 1.0, 0.05, 1.5, 1e-4)
            T.chol()
    elif kind == "loglik":
        # the same factorisation, then the log-likelihood of one right-hand
        # side with FP64 refinement (forward and backward solve graphs,
        # residuals)
        ds, _ = ctx.morton_order(torch.from_numpy(I.points(n, 11)).to(dev))
        nt = -(-n // 512)
        T = mpchol.TiledMatrix(ctx, n, 512, I.band_map(nt, I.F64, I.F32, I.F32, 1), keep_sigma=True)
        T.generate(ds, 1.0, 0.05, 1.5, 1e-4)
        T.chol()
        zt = torch.from_numpy(np.ascontiguousarray(I.rhs(n, 1, 12).T)).to(dev)
        for _ in range(2):
            T.loglik(zt, refine_iters=10)
    else:
        raise SystemExit(f"unknown profile case {name}")
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": name, "ok": True}))


def main():
    args = parse()
    if args.profile_case:
        profile_case(args.profile_case)
        return
    cfg = dict(I.CONFIGS[args.workload])
    if args.impl == "reference":
        reference_arm(args, cfg)
    else:
        ours(args, cfg)


if __name__ == "__main__":
    main()
