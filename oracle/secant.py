"""Plain, slow, exact oracle of the paper's own method: the smallest eigenvalue
as the smallest root of P(x) = det(M - xI), found by the Secant recurrence,
with P(x) evaluated by an LDL^T factorisation of M - xI and the root proved by
the sign of the determinant on both sides of it.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Pins:
``tests/test_oracle_secant.py``.

Sections followed: "The Secant Algorithm" (the recurrence, the start x_1 < 0,
x_2 = 0, no overshoot below lambda_1), "The LDL^T Determinant Algorithm" (the
submatrix-order factorisation of M - xI and the determinant as the product of
the pivots D), "Interval Verification" (det(M - xI) > 0 just below the root,
< 0 just above it).  Numbers are the P-bit floats of ``hankel.py``.

Readings of the paper taken here:

S1. Arithmetic: P-bit floats, round-to-nearest-even, instead of GMP fixed
    point with K and K/2 fractional bits (as in the Cholesky oracle).
S2. LDL^T in the paper's submatrix order with every accumulated entry summed
    exactly and rounded once: at column t,
      D_t      = RNE(m_2t - x - sum_{s<t} C_s[t] Q_s[t]),
      C_t[r]   = RNE(m_{t+r} - sum_{s<t} C_s[t] Q_s[r])      (r > t),
      Q_t[r]   = RNE(C_t[r] / D_t)                          (the paper's CDivDiag),
    and det = RNE(... RNE(RNE(D_0 D_1) D_2) ... D_{N-1}), the running product
    rounded after every factor.  Negative pivots are allowed (above lambda_1
    the matrix is indefinite); a zero pivot gives det = 0 and stops.
S3. The start: x_2 = 0 and x_1 = -min_t D_t(0), the smallest pivot of M itself,
    negated (a pivot of a positive definite matrix is at least lambda_1, so
    the secant through x_1 and x_2 is well resolved at P bits).
S4. The recurrence x_{i+1} = x_i - ((x_i - x_{i-1}) / (P(x_i) - P(x_{i-1}))) P(x_i)
    with each subtraction, the quotient and the product rounded (RNE).
S5. The stop: |x_{i+1} - x_i| <= 2^-136 |x_{i+1}| (the paper's "15 decimal
    digits stabilised" replaced by the tolerance of the inverse iteration),
    or P(x_i) = P(x_{i-1}), or a step no shorter than the one before it after
    the first three (the rounding noise of P near the root reached: the
    secant converges superlinearly until then).
S6. Verification: instead of fixed-point interval arithmetic, exact rational
    arithmetic at x_lo = x (1 - 2^-b) and x_hi = x (1 + 2^-b) (b = 130 by
    default): det(M - x_lo I) > 0 with no negative pivot, det(M - x_hi I) < 0
    with exactly one (Sylvester's law of inertia), so lambda_1 lies in
    (x_lo, x_hi).
"""
from fractions import Fraction

from .hankel import exact_dot, mp_div, rne, to_fraction, _sub_exact


def mp_sub(a, b, P):
    """RNE(a - b) of two P-bit floats."""
    n, e = _sub_exact(a, b)
    return rne(n, e, P)


def mp_mul(a, b, P):
    """RNE(a b) of two P-bit floats."""
    return rne(a[0] * b[0], a[1] + b[1], P)


def ldlt_det(moments, N, x, P):
    """P(x) = det(M - xI) by the LDL^T of reading S2.  Returns (det, pivots)
    with ``pivots`` the P-bit D_t (fewer than N when a zero pivot stopped it)."""
    det, D, _, _ = ldlt_factors(moments, N, x, P)
    return det, D


def ldlt_factors(moments, N, x, P):
    """The LDL^T of reading S2 with its factors: (det, D, C, Q) where C[t] and
    Q[t] map each r > t to the column entry C_t[r] and CDivDiag Q_t[r]."""
    C, Q, D = [], [], []
    det = None
    for t in range(N):
        # column t after the updates of columns s < t (exact), then rounded
        diag = exact_dot([(C[s][t], Q[s][t]) for s in range(t)])
        a = _sub_exact(_sub_exact(moments[2 * t], x), diag)
        d = rne(a[0], a[1], P)
        D.append(d)
        det = d if det is None else mp_mul(det, d, P)
        if d[0] == 0:
            return (0, 0), D, C, Q
        Ct, Qt = {}, {}
        for r in range(t + 1, N):
            acc = exact_dot([(C[s][t], Q[s][r]) for s in range(t)])
            e = _sub_exact(moments[t + r], acc)
            Ct[r] = rne(e[0], e[1], P)
            Qt[r] = mp_div(Ct[r], d, P)
        C.append(Ct)
        Q.append(Qt)
    return det, D, C, Q


def _converged(new, old):
    """|new - old| <= 2^-136 |new|, exactly (reading S5)."""
    diff = to_fraction(new) - to_fraction(old)
    return abs(diff) * 2 ** 136 <= abs(to_fraction(new))


def secant(moments, N, P, max_steps=200):
    """The Secant recurrence of reading S4 from x_1, x_2 of reading S3.
    Returns (root, iterates, determinants) with iterates[0] = x_1,
    iterates[1] = x_2 = 0."""
    zero = (0, 0)
    p2, piv0 = ldlt_det(moments, N, zero, P)
    m = min(piv0, key=to_fraction)
    x1, x2 = (-m[0], m[1]), zero
    p1, _ = ldlt_det(moments, N, x1, P)
    xs, ps = [x1, x2], [p1, p2]
    last = None
    for k in range(max_steps):
        if p2 == p1:
            break
        step = mp_mul(mp_div(mp_sub(x2, x1, P), mp_sub(p2, p1, P), P), p2, P)
        x3 = mp_sub(x2, step, P)
        size = abs(to_fraction(step))
        if k >= 3 and last is not None and size >= last:
            break  # no progress: keep x2
        p3, _ = ldlt_det(moments, N, x3, P)
        xs.append(x3)
        ps.append(p3)
        done = _converged(x3, x2)
        x1, p1, x2, p2 = x2, p2, x3, p3
        last = size
        if done:
            break
    return x2, xs, ps


def inertia(moments, N, x):
    """(negative pivots, det) of the exact rational LDL^T of M - xI for a
    rational x (Sylvester: the count equals the eigenvalues below x); None
    for the count when a zero pivot makes the elimination break down."""
    A = [[to_fraction(moments[i + j]) - (x if i == j else 0) for j in range(N)] for i in range(N)]
    neg, det = 0, Fraction(1)
    for k in range(N):
        d = A[k][k]
        det *= d
        if d == 0:
            return None, det
        neg += d < 0
        for i in range(k + 1, N):
            f = A[i][k] / d
            if f:
                for j in range(k + 1, N):
                    A[i][j] -= f * A[k][j]
    return neg, det


def verify(moments, N, x, bits=130):
    """Reading S6: True when det(M - x_lo I) > 0 with no negative pivot and
    det(M - x_hi I) < 0 with exactly one, for x_lo, x_hi = x (1 -+ 2^-bits)."""
    xv = to_fraction(x)
    lo, hi = xv * (1 - Fraction(1, 2 ** bits)), xv * (1 + Fraction(1, 2 ** bits))
    n_lo, d_lo = inertia(moments, N, lo)
    n_hi, d_hi = inertia(moments, N, hi)
    return n_lo == 0 and d_lo > 0 and n_hi == 1 and d_hi < 0
