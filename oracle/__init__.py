"""Reference oracle for the extended-precision Hankel smallest-eigenvalue path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything in this package.  The product path (the CUDA library and its Python
binding) never calls it and shares no code with it.

What it computes (Emmart, Weems and Chen, "Computing the smallest eigenvalue of
large ill-conditioned Hankel matrices"):

* the Hankel moment matrix ``M_ij = m_{i+j}`` with
  ``m_k = Gamma((1+k)/beta)/beta`` (Introduction, the definition of M); the
  moments are an input here, produced by the seeded input generator;
* its factorisation ``M = R^T R`` (the paper's LDL^T of section "The LDL^T
  Determinant Algorithm", written with ``R = D^{1/2} L^T``), every trailing
  dot product accumulated exactly and rounded once, round-to-nearest-even, to
  a P-bit binary floating-point number; square roots and quotients correctly
  rounded;
* inverse iteration with two triangular solves per step and the Rayleigh
  quotient of M^-1 (section "M is extremely ill-conditioned" uses the Rayleigh
  quotient to bound the spectrum), giving ``lambda_min``.

* the paper's own method (``secant.py``): the smallest root of
  ``P(x) = det(M - xI)`` by the Secant recurrence (section "The Secant
  Algorithm"), P(x) from an LDL^T of ``M - xI`` (section "The LDL^T
  Determinant Algorithm"), and the root proved by the sign of the determinant
  just below and above it (section "Interval Verification").

All arithmetic is exact Python-integer arithmetic; the only rounding is the
explicit ``rne`` of an exact value.  Every function cites the passage it follows.
"""
from .hankel import (  # noqa: F401
    NotPositiveDefinite,
    rne,
    mp_div,
    mp_sqrt,
    exact_dot,
    cholesky,
    cholesky_row,
    cholesky_factorial,
    forward_solve,
    back_solve,
    rayleigh_lambda,
    normalise,
    inverse_iteration,
    smallest_eigenvalue,
    to_fraction,
)
