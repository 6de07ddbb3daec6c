"""Pins of the oracle of the paper's own method (oracle/secant.py): the
LDL^T determinant against the beta = 1 closed form and an independent exact
determinant, the Secant root against the inverse-iteration oracle, an
independent eigensolve at 2P and the N = 4 values, the paper's no-overshoot
property, and the verification step, with a planted mistake it must catch.
No GPU is used here."""
from fractions import Fraction
from math import factorial

import pytest

from oracle import hankel as H
from oracle import secant as S
from paper_0902_0852_gb300 import inputs

mpmath = pytest.importorskip("mpmath")
sympy = pytest.importorskip("sympy")

F = H.to_fraction


def _mp_lambda_min(moments, N, prec):
    mpmath.mp.prec = prec
    M = mpmath.matrix(N, N)
    for i in range(N):
        for j in range(N):
            n, e = moments[i + j]
            M[i, j] = mpmath.ldexp(mpmath.mpf(n), e)
    return min(mpmath.eigsy(M, eigvals_only=True))


@pytest.mark.parametrize("N", [4, 8, 12])
def test_beta1_pivots_are_factorial_squares(N):
    """For m_k = k! the LDL^T pivots are D_t = (t!)^2 (from R_ki = i! C(i, k)),
    exactly representable here, and det M = prod (t!)^2 up to the rounding of
    the running product (one RNE per factor)."""
    P = 128
    m = inputs.moments(N, (1, 1), P)
    det, D = S.ldlt_det(m, N, (0, 0), P)
    assert [F(d) for d in D] == [factorial(t) ** 2 for t in range(N)]
    exact = 1
    for t in range(N):
        exact *= factorial(t) ** 2
    assert abs(F(det) - exact) <= Fraction(N, 2 ** (P - 1)) * exact


@pytest.mark.parametrize("beta,N,P,xfrac", [((7, 4), 8, 256, Fraction(1, 3)), ((3, 4), 6, 192, Fraction(2, 1)),
                                            ((1, 1), 6, 192, Fraction(5, 2)), ((1, 2), 8, 256, Fraction(1, 2)),
                                            ((1, 3), 8, 256, Fraction(3, 2))])
def test_det_and_inertia_match_an_exact_determinant(beta, N, P, xfrac):
    """det(M - xI) at a shift below lambda_1 (xfrac < 1) or above it (xfrac > 1):
    the P-bit LDL^T determinant and the exact rational one of the oracle both
    agree with sympy's exact (Bareiss) determinant of the same rational
    matrix, and the exact inertia counts the eigenvalues below x."""
    m = inputs.moments(N, beta, P)
    lam = _mp_lambda_min(m, N, 2 * P)
    x = H.rne(int(mpmath.floor(mpmath.ldexp(lam * mpmath.mpf(xfrac.numerator) / xfrac.denominator, 2 * P))), -2 * P, P)
    A = sympy.Matrix(N, N, lambda i, j: sympy.Rational(F(m[i + j]) - (F(x) if i == j else 0)))
    num, den = sympy.fraction(A.det(method="bareiss"))
    exact = Fraction(int(num), int(den))
    det, _ = S.ldlt_det(m, N, x, P)
    assert abs(F(det) - exact) <= Fraction(1, 2 ** (P - 96)) * abs(exact)
    neg, d = S.inertia(m, N, F(x))
    assert d == exact
    evs = mpmath.eigsy(mpmath.matrix([[mpmath.mpf(F(m[i + j]).numerator) / F(m[i + j]).denominator
                                       for j in range(N)] for i in range(N)]), eigvals_only=True)
    assert neg == sum(1 for ev in evs if ev < mpmath.mpf(F(x).numerator) / F(x).denominator)


CASES = [((1, 1), 4, 256), ((7, 4), 4, 256), ((1, 1), 16, 640), ((7, 4), 24, 1024), ((3, 4), 20, 1024),
         ((3, 2), 12, 512), ((1, 2), 16, 640), ((1, 3), 16, 640)]


@pytest.mark.parametrize("beta,N,P", CASES)
def test_secant_root_agrees_with_inverse_iteration_and_eigensolve(beta, N, P):
    m = inputs.moments(N, beta, P)
    root, xs, _ = S.secant(m, N, P)
    lam, _, _ = H.smallest_eigenvalue(m, N, P, 80)
    ref = _mp_lambda_min(m, N, 2 * P)
    r = F(root)
    assert abs(r - F(lam)) <= Fraction(1, 2 ** 128) * F(lam)
    rel = abs(mpmath.mpf(r.numerator) / r.denominator - ref) / ref
    assert rel <= mpmath.mpf(2) ** -128
    assert len(xs) - 2 <= 20  # superlinear: a handful of determinants


@pytest.mark.parametrize("beta,N,P", [CASES[0], CASES[1], CASES[2], CASES[5]])
def test_secant_never_overshoots(beta, N, P):
    """From x_2 = 0 the iterates increase and stay below lambda_1: M - x_i I
    has no negative pivot at any of them (section "The Secant Algorithm", a
    statement about exact arithmetic: only iterates already within 2^-128 of
    the root, where the rounding of P(x) decides, may step past it)."""
    m = inputs.moments(N, beta, P)
    root, xs, ps = S.secant(m, N, P)
    r = F(root)
    vals = [F(x) for x in xs[1:]]
    far = [x for x in vals if abs(x - r) > r / 2 ** 128]
    assert len(far) >= 3
    assert all(a < b for a, b in zip(far, far[1:]))
    for x in far[1:]:
        neg, d = S.inertia(m, N, x)
        assert neg == 0 and d > 0
    for x in vals:
        if x not in far:
            assert abs(x - r) <= r / 2 ** 128


@pytest.mark.parametrize("beta,want", [((1, 1), "0.0529002939539"), ((7, 4), "0.00318093261069")])
def test_N4_values(beta, want):
    m = inputs.moments(4, beta, 256)
    root, _, _ = S.secant(m, 4, 256)
    r = F(root)
    got = mpmath.mpf(r.numerator) / r.denominator
    assert mpmath.nstr(got, 12, strip_zeros=False).startswith(want[:12])


def test_verification_accepts_the_root_and_rejects_neighbours():
    N, beta, P = 12, (7, 4), 512
    m = inputs.moments(N, beta, P)
    root, _, _ = S.secant(m, N, P)
    assert S.verify(m, N, root)
    n, e = root
    for off in (1 << (P - 100), -(1 << (P - 100))):
        assert not S.verify(m, N, H.rne(n + off, e, P))


def test_planted_dropped_shift_is_caught(monkeypatch):
    """A determinant that ignores the shift (M instead of M - xI) has no root:
    the recurrence stops without one that verification accepts."""
    N, beta, P = 8, (7, 4), 256
    m = inputs.moments(N, beta, P)
    real = S.ldlt_det
    monkeypatch.setattr(S, "ldlt_det", lambda mom, n, x, p: real(mom, n, (0, 0), p))
    root, _, _ = S.secant(m, N, P)
    assert not S.verify(m, N, root)
