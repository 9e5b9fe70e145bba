"""Gaussian log-likelihood by Cholesky: the exact FP64 reference and the
per-tile-precision tiled emulation.

Oracle (test infrastructure; see oracle/__init__.py).

The quantity (Sec. 6.2, the Gaussian log-likelihood and its evaluation
recipe): with Sigma = L L^T,
    logdet = 2 sum_t log L_tt,   w = L^{-1} z,   quad = ||w||^2,
    loglik = -n/2 log(2 pi) - logdet / 2 - quad / 2
(the paper's `nll` is -loglik).  The paper factors with `chol`, takes the
log-determinant from the factor's diagonal and solves with `forwardsolve`.

O-exact: Sigma in float64, LAPACK's Cholesky (numpy) or the textbook
column Cholesky, triangular solve (scipy); the error reference.

O-tiled: the right-looking tiled Cholesky in which tile (i, j) (i >= j) is
stored in its own format p(i, j) (the multi-precision tiled approach named
as future work in Sec. 7).  For k = 0 .. NT-1:
  POTRF  L_kk = chol(A_kk) in float64 (A_kk must be FP64); a pivot that is
         not > 0 gives info = its 1-based global row.
  TRSM   for i > k: X = A_ik L_kk^{-T} in float64 from the exactly upcast
         tile, then A_ik = round_{p(i,k)}(X) (E4M3: new scale from amax X).
  SYRK   for j > k: A_jj -= A_jk A_jk^T,
  GEMM   for i > j > k: A_ij -= A_ik A_jk^T,
with the update rule "R-MMA": the product runs in the precision
kind = min(p(target), max(p(operands))) -- the paper's rule that a result
takes the highest input precision (Sec. 4.3) capped by the target tile.
Operands stored above the kind are rounded to it, lower ones upcast
exactly; products accumulate in FP32 (FP64 when the kind is FP64); the
subtraction from the upcast target is done in float64 and the result is
rounded once to p(target) (E4M3 targets take a new scale from the amax of
the float64 result).  E4M3 products use the scaled codes and multiply the
FP32 sum by s_a s_b.  Padding beyond n is the identity (log 1 = 0).

Solves use float64 arithmetic on the exactly upcast tiles.  Refinement
(the paper's "double precision for refinement", Sec. 1): x0 = L^-T L^-1 z;
then repeatedly r = z - Sigma x with Sigma in float64, stop a column when
||r||_inf <= n u64 (||Sigma||_inf ||x||_inf + ||z||_inf), else x += L^-T L^-1 r;
quad = z^T x.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from . import formats as F

U64 = 2.0 ** -53


# ----------------------------------------------------------------------------
# exact reference
# ----------------------------------------------------------------------------

def potrf_textbook(A: np.ndarray):
    """Column-oriented Cholesky A = L L^T of a float64 SPD matrix.

    Returns (L, info): info = 0, or the 1-based index of the first pivot
    that is not > 0 (L is then partial)."""
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    L = np.zeros_like(A)
    for c in range(n):
        d = A[c, c] - np.dot(L[c, :c], L[c, :c])
        if not d > 0.0:
            return L, c + 1
        L[c, c] = math.sqrt(d)
        if c + 1 < n:
            L[c + 1:, c] = (A[c + 1:, c] - L[c + 1:, :c] @ L[c, :c]) / L[c, c]
    return L, 0


def loglik_value(n: int, logdet: float, quad) -> np.ndarray:
    """-n/2 log(2 pi) - logdet/2 - quad/2 (quad may be per right-hand side)."""
    return -0.5 * n * math.log(2.0 * math.pi) - 0.5 * logdet - 0.5 * np.asarray(quad)


def exact_loglik(S: np.ndarray, z: np.ndarray, method: str = "lapack"):
    """O-exact.  Returns dict(logdet, quad[nrhs], loglik[nrhs], L)."""
    z = np.asarray(z, dtype=np.float64).reshape(S.shape[0], -1)
    if method == "lapack":
        L = np.linalg.cholesky(S)
    else:
        L, info = potrf_textbook(S)
        if info:
            raise np.linalg.LinAlgError(f"not SPD at row {info}")
    logdet = 2.0 * float(np.sum(np.log(np.diag(L))))
    w = sla.solve_triangular(L, z, lower=True)
    quad = np.sum(w * w, axis=0)
    return dict(logdet=logdet, quad=quad, loglik=loglik_value(S.shape[0], logdet, quad), L=L)


def exact_loglik_field(locs: np.ndarray, nu: float, a: float, sigma2: float, nugget: float,
                       z: np.ndarray, rows: int = 2048, keep_factor: bool = False):
    """O-exact for a Matérn field too large for `covariance` and its
    temporaries: Sigma is built row block by row block into one float64
    array, LAPACK's Cholesky (dpotrf) factors it in place and a triangular
    solve gives w = L^{-1} z.  Same quantity as exact_loglik.  Returns
    dict(logdet, quad[nrhs], loglik[nrhs]) and, with keep_factor, L (its
    upper triangle holds what is left of Sigma)."""
    from scipy.linalg import lapack
    from . import matern as M
    n = locs.shape[0]
    z = np.asarray(z, dtype=np.float64).reshape(n, -1)
    S = np.empty((n, n), order="F")
    for r0 in range(0, n, rows):
        r1 = min(n, r0 + rows)
        blk = M.matern(M.distances(locs[r0:r1], locs), nu, a, sigma2)
        blk[np.arange(r1 - r0), np.arange(r0, r1)] += nugget
        S[r0:r1] = blk
        del blk
    L, info = lapack.dpotrf(S, lower=1, clean=0, overwrite_a=1)
    if info != 0:
        raise np.linalg.LinAlgError(f"not SPD at row {info}")
    logdet = 2.0 * float(np.sum(np.log(np.diag(L))))
    w = sla.solve_triangular(L, z, lower=True, check_finite=False)
    quad = np.sum(w * w, axis=0)
    out = dict(logdet=logdet, quad=quad, loglik=loglik_value(n, logdet, quad))
    if keep_factor:
        out["L"] = L
    return out


# ----------------------------------------------------------------------------
# tiled matrix with per-tile formats
# ----------------------------------------------------------------------------

@dataclass
class Tile:
    codes: np.ndarray     # float64 array holding the stored values (E4M3: scaled codes)
    fmt: int
    scale: float = 1.0

    def values(self) -> np.ndarray:
        return self.codes * self.scale


@dataclass
class TiledMatrix:
    n: int
    b: int
    nt: int
    pmap: np.ndarray
    tiles: dict = field(default_factory=dict)
    logdet: float = 0.0
    info: int = 0

    def value(self, i: int, j: int) -> np.ndarray:
        return self.tiles[(i, j)].values()

    def dense_lower(self) -> np.ndarray:
        """Padded (nt*b)^2 matrix of the lower tiles' values (upper zero)."""
        N = self.nt * self.b
        M = np.zeros((N, N))
        for (i, j), t in self.tiles.items():
            blk = t.values()
            if i == j:
                blk = np.tril(blk)
            M[i * self.b:(i + 1) * self.b, j * self.b:(j + 1) * self.b] = blk
        return M


def pad_identity(S: np.ndarray, b: int) -> np.ndarray:
    n = S.shape[0]
    nt = -(-n // b)
    N = nt * b
    P = np.eye(N)
    P[:n, :n] = S
    return P


def tiled_from_dense(S: np.ndarray, b: int, pmap: np.ndarray) -> TiledMatrix:
    """Tile generation: each lower tile of the (identity-padded) float64
    matrix is rounded once into its format; E4M3 tiles get their scale."""
    n = S.shape[0]
    nt = -(-n // b)
    P = pad_identity(S, b)
    T = TiledMatrix(n=n, b=b, nt=nt, pmap=np.asarray(pmap, dtype=np.uint8))
    for i in range(nt):
        if T.pmap[i, i] != F.F64:
            raise ValueError("diagonal tiles must be FP64")
        for j in range(i + 1):
            blk = P[i * b:(i + 1) * b, j * b:(j + 1) * b]
            codes, s = F.quantize(blk, int(T.pmap[i, j]))
            T.tiles[(i, j)] = Tile(codes, int(T.pmap[i, j]), s)
    return T


def tile_norms(S: np.ndarray, b: int) -> np.ndarray:
    """Frobenius norms of the lower tiles of the identity-padded matrix."""
    P = pad_identity(S, b)
    nt = P.shape[0] // b
    out = np.zeros((nt, nt))
    for i in range(nt):
        for j in range(i + 1):
            out[i, j] = np.linalg.norm(P[i * b:(i + 1) * b, j * b:(j + 1) * b])
    return out


def guarded_map(norms: np.ndarray, band: int, near: int, far: int, eps: float) -> np.ndarray:
    """A precision map for the tiled extension (Sec. 7 leaves the choice of
    precisions open): diagonal FP64, |i - j| <= band in `near`, and a farther
    tile in `far` only when u(far) ||A_ij||_F <= eps ||A||_F / NT, so that
    the rounding of all far tiles perturbs A by at most eps ||A||_F in the
    Frobenius norm; otherwise `near`.  Entries above the diagonal are 255."""
    nt = norms.shape[0]
    tot = 0.0
    for i in range(nt):
        for j in range(i + 1):
            tot += (1.0 if i == j else 2.0) * norms[i, j] ** 2
    bound = eps * math.sqrt(tot) / nt
    m = np.full((nt, nt), 255, dtype=np.uint8)
    for i in range(nt):
        m[i, i] = F.F64
        for j in range(i):
            if i - j <= band:
                m[i, j] = near
            else:
                m[i, j] = far if F.unit_roundoff(far) * norms[i, j] <= bound else near
    return m


def bound_map(sorted_locs: np.ndarray, b: int, nu: float, a: float, sigma2: float,
              nugget: float, band: int, near: int, far: int, eps: float) -> np.ndarray:
    """The guarded map with ||A_ij||_F replaced by the upper bound
    sqrt(rows_i cols_j) C(d_ij), d_ij the distance between the bounding
    boxes of the two tiles' points (the Matérn covariance decreases with
    distance), and ||A||_F by its lower bound sqrt(n) (sigma2 + nugget)
    (the diagonal alone): a more conservative choice than guarded_map."""
    from .matern import matern
    n = sorted_locs.shape[0]
    nt = -(-n // b)
    boxes = []
    for t in range(nt):
        p = sorted_locs[t * b:min(n, (t + 1) * b)]
        boxes.append((p[:, 0].min(), p[:, 0].max(), p[:, 1].min(), p[:, 1].max(), p.shape[0]))
    bound = eps * math.sqrt(n) * (sigma2 + nugget) / nt
    m = np.full((nt, nt), 255, dtype=np.uint8)
    for i in range(nt):
        m[i, i] = F.F64
        for j in range(i):
            if i - j <= band:
                m[i, j] = near
                continue
            xi0, xi1, yi0, yi1, ci = boxes[i]
            xj0, xj1, yj0, yj1, cj = boxes[j]
            dx = max(0.0, max(xi0 - xj1, xj0 - xi1))
            dy = max(0.0, max(yi0 - yj1, yj0 - yi1))
            B = math.sqrt(float(ci) * float(cj)) * float(matern(math.sqrt(dx * dx + dy * dy), nu, a, sigma2))
            m[i, j] = far if F.unit_roundoff(far) * B <= bound else near
    return m


def kind_of(q: int, pa: int, pb: int) -> int:
    """R-MMA: the format in which A_ik A_jk^T runs for a target of format q."""
    lk = min(F.level(q), max(F.level(pa), F.level(pb)))
    if lk == F.level(q):
        return q
    hi = [p for p in (pa, pb) if F.level(p) == lk]
    if len(set(hi)) > 1:        # BF16 with F16 below a wider target: upcast both
        return F.F32
    return hi[0]


def operand_as(t: Tile, kind: int):
    """Operand in the kind's format: (codes, scale).  Stored above the kind
    (or in a different format of the same rank): rounded; below: exact."""
    if t.fmt == kind or F.level(t.fmt) < F.level(kind):
        if kind == F.E4M3 and t.fmt != F.E4M3:
            raise AssertionError("unreachable: nothing ranks below E4M3")
        if t.fmt == F.E4M3 and kind != F.E4M3:
            return t.values(), 1.0          # exact upcast of c * s
        return t.codes, t.scale
    return F.quantize(t.values(), kind)


def product(a: Tile, bt: Tile, kind: int) -> np.ndarray:
    """P = A B^T in the kind's arithmetic, returned as float64."""
    ca, sa = operand_as(a, kind)
    cb, sb = operand_as(bt, kind)
    if kind == F.F64:
        return ca @ cb.T * (sa * sb)
    P = np.matmul(ca.astype(np.float32), cb.astype(np.float32).T)   # FP32 accumulation
    return P.astype(np.float64) * (sa * sb)


def step_potrf(T: TiledMatrix, k: int) -> None:
    t = T.tiles[(k, k)]
    L, info = potrf_textbook(t.values())      # reads the lower triangle only
    if info:
        T.info = k * T.b + info
        raise np.linalg.LinAlgError(f"not SPD at global row {T.info}")
    T.tiles[(k, k)] = Tile(L, F.F64, 1.0)
    T.logdet += 2.0 * float(np.sum(np.log(np.diag(L))))


def step_trsm(T: TiledMatrix, k: int) -> None:
    L = T.tiles[(k, k)].codes
    for i in range(k + 1, T.nt):
        t = T.tiles[(i, k)]
        X = sla.solve_triangular(L, t.values().T, lower=True).T     # A_ik L^{-T}
        codes, s = F.quantize(X, t.fmt)
        T.tiles[(i, k)] = Tile(codes, t.fmt, s)


def step_update(T: TiledMatrix, k: int) -> None:
    for j in range(k + 1, T.nt):
        for i in range(j, T.nt):
            tgt = T.tiles[(i, j)]
            a, bt = T.tiles[(i, k)], T.tiles[(j, k)]
            kind = kind_of(tgt.fmt, a.fmt, bt.fmt)
            V = tgt.values() - product(a, bt, kind)
            codes, s = F.quantize(V, tgt.fmt)
            T.tiles[(i, j)] = Tile(codes, tgt.fmt, s)


def step(T: TiledMatrix, k: int) -> None:
    """One right-looking step: POTRF, TRSM of column k, trailing update."""
    step_potrf(T, k)
    step_trsm(T, k)
    step_update(T, k)


def tiled_cholesky(T: TiledMatrix) -> TiledMatrix:
    for k in range(T.nt):
        step(T, k)
    return T


def forward_solve(T: TiledMatrix, z: np.ndarray) -> np.ndarray:
    """w = L^{-1} z on the padded system (z padded with zeros)."""
    z = np.asarray(z, dtype=np.float64).reshape(T.n, -1)
    zp = np.zeros((T.nt * T.b, z.shape[1]))
    zp[:T.n] = z
    return forward_solve_padded(T, zp)


def forward_solve_padded(T: TiledMatrix, zp: np.ndarray) -> np.ndarray:
    b, nt = T.b, T.nt
    w = np.array(zp, dtype=np.float64)
    for i in range(nt):
        wi = w[i * b:(i + 1) * b]
        for j in range(i):
            wi -= T.value(i, j) @ w[j * b:(j + 1) * b]
        w[i * b:(i + 1) * b] = sla.solve_triangular(T.tiles[(i, i)].codes, wi, lower=True)
    return w


def backward_solve(T: TiledMatrix, w: np.ndarray) -> np.ndarray:
    """x = L^{-T} w on the padded system."""
    b, nt = T.b, T.nt
    x = np.array(w, dtype=np.float64)
    for i in range(nt - 1, -1, -1):
        xi = x[i * b:(i + 1) * b]
        for j in range(i + 1, nt):
            xi -= T.value(j, i).T @ x[j * b:(j + 1) * b]
        x[i * b:(i + 1) * b] = sla.solve_triangular(T.tiles[(i, i)].codes, xi, lower=True,
                                                    trans="T")
    return x


def refine(T: TiledMatrix, S: np.ndarray, z: np.ndarray, max_iter: int = 10):
    """FP64 iterative refinement of Sigma x = z with the mixed factor.

    Returns (x[n, nrhs], iterations[nrhs], residual_inf[nrhs])."""
    n, b, nt = T.n, T.b, T.nt
    z = np.asarray(z, dtype=np.float64).reshape(n, -1)
    pad = nt * b - n
    def solve(r):
        rp = np.vstack([r, np.zeros((pad, r.shape[1]))])
        return backward_solve(T, forward_solve_padded(T, rp))[:n]
    x = solve(z)
    snorm = float(np.max(np.sum(np.abs(S), axis=1)))
    active = np.ones(z.shape[1], dtype=bool)
    iters = np.zeros(z.shape[1], dtype=np.int64)
    rnorm = np.zeros(z.shape[1])
    for _ in range(max_iter):
        r = z - S @ x
        rnorm = np.max(np.abs(r), axis=0)
        tol = n * U64 * (snorm * np.max(np.abs(x), axis=0) + np.max(np.abs(z), axis=0))
        active &= ~(rnorm <= tol)
        if not active.any():
            break
        x[:, active] += solve(r[:, active])
        iters[active] += 1
    return x, iters, rnorm


def tiled_loglik(S: np.ndarray, z: np.ndarray, b: int, pmap: np.ndarray,
                 refine_iters: int = 0):
    """O-tiled end to end.  Returns dict(logdet, quad, loglik, T, iters)."""
    T = tiled_cholesky(tiled_from_dense(S, b, pmap))
    z = np.asarray(z, dtype=np.float64).reshape(S.shape[0], -1)
    if refine_iters > 0:
        x, iters, _ = refine(T, S, z, refine_iters)
        quad = np.sum(z * x, axis=0)
    else:
        w = forward_solve(T, z)
        quad = np.sum(w * w, axis=0)
        iters = np.zeros(z.shape[1], dtype=np.int64)
    return dict(logdet=T.logdet, quad=quad, loglik=loglik_value(S.shape[0], T.logdet, quad),
                T=T, iters=iters)


def gemm(A: np.ndarray, B: np.ndarray, C: np.ndarray, fmt: int, alpha: float = 1.0,
         beta: float = 0.0, ta: bool = False, tb: bool = False) -> np.ndarray:
    """C = alpha op(A) op(B) + beta C with A, B, C stored in `fmt` (the
    paper's %*% / crossprod per precision, Sec. 5): products accumulate in
    FP32 (FP64 for F64); alpha, beta and the sum applied in float64; the
    result rounded once to `fmt` (E4M3 codes with scale 1)."""
    a = A.T if ta else A
    b = B.T if tb else B
    if fmt == F.F64:
        P = a @ b
    else:
        P = np.matmul(a.astype(np.float32), b.astype(np.float32)).astype(np.float64)
    R = alpha * P + (beta * C if beta != 0.0 else 0.0)
    return F.round_to(R, fmt)
