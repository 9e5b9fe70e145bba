"""Plain CPU oracle of the mixed-precision tiled Cholesky log-likelihood.

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only the tests, the smoke check and the
benchmark's CPU-baseline arm may import it; the library path never does, and
nothing here shares code with the CUDA implementation.

It is written to be read against the paper (arXiv 2406.02701, "MPCR:
Multi-Precision Computations Package in R"):
  formats  -- rounding into FP32 / BF16 / FP16 / FP8-E4M3 from the format
              definitions (Sec. 2), per-tile power-of-two FP8 scales.
  matern   -- the Matérn covariance (Sec. 6.2) in its half-integer closed
              forms and, for any other nu, its definition through the
              library Bessel function; Morton ordering of locations.
  chol     -- O-exact: the float64 Gaussian log-likelihood (Sec. 6.2);
              O-tiled: the tiled Cholesky with a per-tile precision map
              (the tiled multi-precision approach of Sec. 7), its
              triangular solves, log-determinant and FP64 refinement (Sec. 1);
              the per-precision matrix product (Sec. 5).

Every function is plain numpy/scipy in float64, except where a step's
definition fixes a lower precision (FP32 accumulation of the tile products).
Library routines used as steps: numpy's matmul and LAPACK Cholesky,
scipy's triangular solve, scipy's K_nu and Gamma (general nu only).

Parity pins live in tests/test_oracle_*.py.  Parity unpinned: none of these
functions is left without a pin; the paper's own MLE numbers (Table 3) depend
on R's random stream and are context only.
"""
from . import formats, matern, chol  # noqa: F401
