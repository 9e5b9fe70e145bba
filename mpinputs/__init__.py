"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the method: it only draws locations,
right-hand sides and Matérn parameters from numpy's PCG64 generator, and
spells out the per-tile precision maps and workload configurations.

The workloads stand in for the paper's spatial Matérn field (Sec. 6.2: a
Gaussian random field on the unit square, evaluated through the Gaussian
log-likelihood at every optimiser iteration).  No dataset is read.
"""
from __future__ import annotations

import numpy as np

# Tile precision codes; they equal the values of `mp_dtype` in include/mpchol.h.
F64, F32, BF16, F16, E4M3 = 0, 1, 2, 3, 4
DTYPE_NAMES = {F64: "f64", F32: "f32", BF16: "bf16", F16: "f16", E4M3: "e4m3"}
DTYPE_BYTES = {F64: 8, F32: 4, BF16: 2, F16: 2, E4M3: 1}


def points(n: int, seed: int) -> np.ndarray:
    """n locations uniform in [0,1)^2, shape (n, 2), float64, row-major."""
    rng = np.random.default_rng(seed)
    return rng.random((n, 2))


def points_line(n: int, h: float) -> np.ndarray:
    """n equally spaced locations s_i = (i*h, 0), shape (n, 2), float64."""
    p = np.zeros((n, 2))
    p[:, 0] = np.arange(n, dtype=np.float64) * h
    return p


def rhs(n: int, nrhs: int, seed: int) -> np.ndarray:
    """Right-hand sides z ~ N(0,1), shape (n, nrhs), float64 (column j = RHS j)."""
    rng = np.random.default_rng(seed + 1000)
    return rng.standard_normal((n, nrhs))


def ar1_rhs(n: int, nrhs: int, rho: float, sigma2: float, seed: int) -> np.ndarray:
    """Right-hand sides drawn from the stationary AR(1) model with lag-one
    correlation rho and variance sigma2, shape (n, nrhs): z_1 = sigma e_1,
    z_i = rho z_{i-1} + sigma sqrt(1 - rho^2) e_i with e ~ N(0, 1) from
    default_rng(seed + 1000) -- a field drawn from the covariance it is
    evaluated under, as for an exponential covariance on equally spaced
    points."""
    e = np.random.default_rng(seed + 1000).standard_normal((n, nrhs))
    z = np.empty((n, nrhs))
    s = np.sqrt(sigma2)
    c = s * np.sqrt(1.0 - rho * rho)
    z[0] = s * e[0]
    for i in range(1, n):
        z[i] = rho * z[i - 1] + c * e[i]
    return z


def band_map(nt: int, diag: int, near: int, far: int, band: int) -> np.ndarray:
    """Per-tile precision map, shape (nt, nt), uint8, row-major; lower triangle used.

    Tile (i, j), i >= j, gets `diag` when i == j, `near` when i - j <= band,
    and `far` otherwise.
    """
    m = np.full((nt, nt), 255, dtype=np.uint8)
    for i in range(nt):
        for j in range(i + 1):
            d = i - j
            m[i, j] = diag if d == 0 else (near if d <= band else far)
    return m


def uniform_map(nt: int, dtype: int) -> np.ndarray:
    m = np.full((nt, nt), 255, dtype=np.uint8)
    for i in range(nt):
        m[i, : i + 1] = dtype
    return m


# The five workload configurations (sizes, kernels and maps).  `morton` says
# whether locations are put in Morton (Z-curve) order before generation.
CONFIGS = {
    "fp64_n1024_b128": dict(n=1024, b=128, nu=0.5, range=0.1, sigma2=1.0, nugget=1e-4,
                            map=("uniform", F64), nrhs=1, seed=1, morton=False, refine=0),
    "mixed_bf16_n16384_b512": dict(n=16384, b=512, nu=1.5, range=0.05, sigma2=1.0, nugget=1e-4,
                                   map=("band", F64, F32, BF16, 2), nrhs=1, seed=11,
                                   morton=True, refine=10),
    "mixed_fp8_n65536_b1024": dict(n=65536, b=1024, nu=1.5, range=0.05, sigma2=1.0, nugget=1e-4,
                                   map=("band", F64, F32, E4M3, 2), nrhs=16, seed=21,
                                   morton=True, refine=10),
}


def make_map(spec, nt: int) -> np.ndarray:
    if spec[0] == "uniform":
        return uniform_map(nt, spec[1])
    _, diag, near, far, band = spec
    return band_map(nt, diag, near, far, band)


def batch_requests(count: int, seed: int = 31, n_lo: int = 256, n_hi: int = 4096):
    """Independent likelihood requests: n ~ U{n_lo..n_hi}, range ~ U[0.02, 0.3],
    nu ~ U{1/2, 3/2, 5/2}, sigma2 = 1, nugget 1e-4; request r draws its
    locations and right-hand side from seed + r."""
    rng = np.random.default_rng(seed)
    reqs = []
    for r in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        reqs.append(dict(n=n, range=float(rng.uniform(0.02, 0.3)),
                         nu=float(rng.choice([0.5, 1.5, 2.5])), sigma2=1.0,
                         nugget=1e-4, seed=seed + r))
    return reqs


def serving_requests(count: int, rate_hz: float, seed: int = 31,
                     sizes=(2048, 8192, 32768), weights=(8, 3, 1)):
    """Poisson arrivals of likelihood requests with Matérn parameters drawn as
    an MLE search would: log a ~ U[log 0.02, log 0.3], log sigma2 ~ U[log 0.5,
    log 2], nu ~ U{1/2, 3/2, 5/2}; n from `sizes` with probabilities
    proportional to `weights`."""
    rng = np.random.default_rng(seed)
    p = np.asarray(weights, dtype=np.float64)
    p = p / p.sum()
    t = 0.0
    reqs = []
    for r in range(count):
        t += float(rng.exponential(1.0 / rate_hz))
        reqs.append(dict(arrival=t, n=int(rng.choice(sizes, p=p)),
                         range=float(np.exp(rng.uniform(np.log(0.02), np.log(0.3)))),
                         sigma2=float(np.exp(rng.uniform(np.log(0.5), np.log(2.0)))),
                         nu=float(rng.choice([0.5, 1.5, 2.5])), nugget=1e-4,
                         seed=seed + r))
    return reqs
