"""Matérn covariance matrices and Morton (Z-curve) ordering of locations.

Oracle (test infrastructure; see oracle/__init__.py).

Covariance (Sec. 6.2, the Matérn model with theta = (nu, a, sigma^2)):
    C(r) = sigma^2 / (2^(nu-1) Gamma(nu)) * M_nu(r / a),
with M_nu(x) = x^nu K_nu(x) (K_nu the modified Bessel function of the second
kind).  The printed formula leaves M_nu undefined; this reading is the one
that reduces at nu = 1/2 to the exponential model sigma^2 exp(-r/a) that the
paper uses for its experiment (Sec. 6.2).  For half-integer nu the Bessel
function has the textbook closed forms, so with x = r / a:
    nu = 1/2:  sigma^2 exp(-x)
    nu = 3/2:  sigma^2 (1 + x) exp(-x)
    nu = 5/2:  sigma^2 (1 + x + x^2/3) exp(-x)
For other nu, `matern_general` evaluates the definition with the library
Bessel function (scipy.special.kv) as a step; C(0) = sigma^2 (the limit
x^nu K_nu(x) -> 2^(nu-1) Gamma(nu)).
The range a enters as given (no sqrt(2 nu) rescaling).  A nugget tau^2 is added
on the diagonal (Sec. 6.2 adds a small diagonal term for single precision).

Morton order: each coordinate in [0, 1] is quantised to 16 bits,
q = min(floor(x * 65536), 65535), and the key interleaves the bits with x in
the even positions and y in the odd ones; locations are sorted by key, ties
by original index.
"""
from __future__ import annotations

import numpy as np


def matern_closed(r, nu: float, a: float, sigma2: float) -> np.ndarray:
    """Matérn covariance at distances r (float64), nu in {0.5, 1.5, 2.5}."""
    x = np.asarray(r, dtype=np.float64) / a
    if nu == 0.5:
        poly = np.ones_like(x)
    elif nu == 1.5:
        poly = 1.0 + x
    elif nu == 2.5:
        poly = 1.0 + x + x * x / 3.0
    else:
        raise ValueError("closed form only for nu in {0.5, 1.5, 2.5}")
    return sigma2 * poly * np.exp(-x)


def matern_general(r, nu: float, a: float, sigma2: float) -> np.ndarray:
    """Matérn covariance at distances r for any nu > 0 (the definition,
    sigma^2 2^(1-nu) / Gamma(nu) x^nu K_nu(x), x = r / a; C(0) = sigma^2)."""
    from scipy.special import gamma, kv
    x = np.asarray(r, dtype=np.float64) / a
    out = np.full(x.shape, float(sigma2))
    pos = x > 0
    xp = x[pos]
    out[pos] = sigma2 * 2.0 ** (1.0 - nu) / gamma(nu) * xp ** nu * kv(nu, xp)
    return out


def matern(r, nu: float, a: float, sigma2: float) -> np.ndarray:
    """Closed form for nu in {1/2, 3/2, 5/2}, the definition otherwise."""
    if nu in (0.5, 1.5, 2.5):
        return matern_closed(r, nu, a, sigma2)
    return matern_general(r, nu, a, sigma2)


def distances(locs_a: np.ndarray, locs_b: np.ndarray) -> np.ndarray:
    """Euclidean distances ||s_i - s_j|| between two point sets (float64)."""
    dx = locs_a[:, 0:1] - locs_b[:, 0][None, :]
    dy = locs_a[:, 1:2] - locs_b[:, 1][None, :]
    return np.sqrt(dx * dx + dy * dy)


def covariance(locs: np.ndarray, nu: float, a: float, sigma2: float,
               nugget: float) -> np.ndarray:
    """Full n x n covariance Sigma_ij = C(||s_i - s_j||) + nugget [i == j]."""
    S = matern(distances(locs, locs), nu, a, sigma2)
    S[np.diag_indices_from(S)] += nugget
    return S


def morton_keys(locs: np.ndarray) -> np.ndarray:
    """32-bit Z-curve keys of locations in [0, 1]^2 (x bits even, y bits odd)."""
    q = np.minimum(np.floor(np.asarray(locs, dtype=np.float64) * 65536.0), 65535.0)
    q = np.maximum(q, 0.0).astype(np.uint64)
    key = np.zeros(locs.shape[0], dtype=np.uint64)
    for bit in range(16):
        key |= ((q[:, 0] >> np.uint64(bit)) & np.uint64(1)) << np.uint64(2 * bit)
        key |= ((q[:, 1] >> np.uint64(bit)) & np.uint64(1)) << np.uint64(2 * bit + 1)
    return key


def morton_order(locs: np.ndarray):
    """Returns (sorted locations, permutation) with locs_sorted = locs[perm]."""
    perm = np.argsort(morton_keys(locs), kind="stable")
    return locs[perm], perm
