"""Plain, slow, exact oracle: P-bit Cholesky of the Hankel moment matrix and
inverse iteration for its smallest eigenvalue.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Parity pins: see
``tests/test_oracle_pins.py``.

Number format.  A P-bit float is a pair ``(n, e)`` of Python ints with value
``n * 2**e``; either ``n == 0 and e == 0`` or ``2**(P-1) <= |n| < 2**P``.
Exponents are unbounded (no overflow, no subnormals).

Readings of the paper taken here:

1. The paper computes an LDL^T determinant in GMP fixed point with K and K/2
   fractional bits (section "The LDL^T Determinant Algorithm").  This oracle
   keeps the submatrix-order factorisation but in P-bit floating point:
   ``A_ij = m_{i+j} - sum_{t<i} R_ti R_tj`` exactly, ``S_ij = RNE(A_ij)``,
   ``R_ii = RNE(sqrt(S_ii))``, ``R_ij = RNE(S_ij / R_ii)``.  The relation to the
   paper's factors is ``D_i = S_ii`` and ``L_ji = S_ij / S_ii``.
2. Off-diagonal entries are rounded twice (the exact numerator, then the
   quotient of two P-bit numbers); the square root is taken of the rounded
   ``S_ii``.
3. A pivot ``S_ii <= 0`` is an error (the matrix is positive definite by the
   section "Properties of M", so this means P is too small), never a clamp.
4. Inverse iteration starts from the all-ones vector, forms
   ``y = R^-T v`` and ``w = R^-1 y`` with every dot product exact and each
   entry rounded as ``RNE(RNE(numerator) / R_ii)``, estimates
   ``lambda_t = RNE(RNE(<v,v>) / RNE(<v,w>))`` (the inverse of the Rayleigh
   quotient of M^-1) and rescales ``v = w * 2**-E`` by a power of two so the
   largest entry lies in [1/2, 1).
"""
from fractions import Fraction
from math import isqrt


class NotPositiveDefinite(ArithmeticError):
    """Raised when a rounded pivot S_ii is <= 0 (reading 3)."""

    def __init__(self, row):
        super().__init__(f"pivot S_{row}{row} <= 0")
        self.row = row


# ---------------------------------------------------------------------------
# Rounding (the once-rounded semantics of every step)
# ---------------------------------------------------------------------------

def rne(n, e, P):
    """Round the exact value ``n * 2**e`` to the nearest P-bit float, ties to
    an even mantissa.  Returns ``(m, x)`` with value ``m * 2**x``."""
    if n == 0:
        return (0, 0)
    neg = n < 0
    a = -n if neg else n
    b = a.bit_length()
    if b <= P:
        m, x = a << (P - b), e - (P - b)
    else:
        sh = b - P
        q = a >> sh
        r = a - (q << sh)
        half = 1 << (sh - 1)
        if r > half or (r == half and (q & 1)):
            q += 1
            if q == (1 << P):
                q >>= 1
                sh += 1
        m, x = q, e + sh
    return (-m if neg else m, x)


def mp_div(x, y, P):
    """Correctly rounded quotient ``RNE(x / y)`` of two P-bit floats, y != 0.
    The integer quotient keeps at least P+2 bits and the remainder is folded
    into one sticky bit below them, so a single ``rne`` is exact."""
    (nx, ex), (ny, ey) = x, y
    if ny == 0:
        raise ZeroDivisionError("mp_div by zero")
    if nx == 0:
        return (0, 0)
    neg = (nx < 0) != (ny < 0)
    ax, ay = abs(nx), abs(ny)
    k = P + 2 + max(0, ay.bit_length() - ax.bit_length())
    q, r = divmod(ax << k, ay)
    q = 2 * q + (1 if r else 0)
    return rne(-q if neg else q, ex - ey - k - 1, P)


def mp_sqrt(x, P):
    """Correctly rounded square root ``RNE(sqrt(x))`` of a P-bit float x > 0,
    through the exact integer square root and a sticky bit."""
    n, e = x
    if n <= 0:
        raise ValueError("mp_sqrt of a non-positive value")
    if e & 1:
        n, e = n << 1, e - 1
    j = (P // 2) + 2 + max(0, P - n.bit_length())
    N2 = n << (2 * j)
    s = isqrt(N2)
    s2 = 2 * s + (1 if s * s != N2 else 0)
    return rne(s2, (e - 2 * j) // 2 - 1, P)


def exact_dot(pairs):
    """Exact value of ``sum x_k * y_k`` for P-bit floats, as ``(n, e)`` with
    value ``n * 2**e`` (no rounding)."""
    terms = [(xn * yn, xe + ye) for (xn, xe), (yn, ye) in pairs if xn and yn]
    if not terms:
        return (0, 0)
    emin = min(e for _, e in terms)
    return (sum(n << (e - emin) for n, e in terms), emin)


def _sub_exact(a, b):
    """Exact ``a - b`` for exact values ``(n, e)``."""
    (na, ea), (nb, eb) = a, b
    if na == 0:
        return (-nb, eb)
    if nb == 0:
        return (na, ea)
    e = min(ea, eb)
    return ((na << (ea - e)) - (nb << (eb - e)), e)


def to_fraction(x):
    """Exact rational value of ``(n, e)``."""
    n, e = x
    return Fraction(n * 2 ** e) if e >= 0 else Fraction(n, 2 ** (-e))


# ---------------------------------------------------------------------------
# Cholesky M = R^T R in submatrix order (section "The LDL^T Determinant
# Algorithm", serial form; reading 1)
# ---------------------------------------------------------------------------

def cholesky_row(i, moments, col_i, cols_j, P):
    """Row i of R from the finished rows above it.

    ``col_i`` holds ``R_ti`` for t < i; ``cols_j`` maps each column j (>= i) to
    the list ``R_tj`` for t < i.  Returns ``{j: R_ij}`` for the requested j, or
    raises NotPositiveDefinite(i) when the rounded pivot is <= 0.
    """
    # A_ii = m_2i - sum_t R_ti^2, exact; S_ii = RNE(A_ii)
    a_ii = _sub_exact(moments[2 * i], exact_dot(list(zip(col_i, col_i))))
    s_ii = rne(a_ii[0], a_ii[1], P)
    if s_ii[0] <= 0:
        raise NotPositiveDefinite(i)
    r_ii = mp_sqrt(s_ii, P)
    out = {}
    for j, col_j in cols_j.items():
        if j == i:
            out[j] = r_ii
            continue
        a_ij = _sub_exact(moments[i + j], exact_dot(list(zip(col_i, col_j))))
        s_ij = rne(a_ij[0], a_ij[1], P)
        out[j] = mp_div(s_ij, r_ii, P)
    return out


def _row_task(args):
    i, moments, col_i, cols_j, P = args
    return cholesky_row(i, moments, col_i, cols_j, P)


def cholesky(moments, N, P, rows=None, workers=1):
    """Upper-triangular R with ``M = R^T R`` (to the rounding of reading 1).

    ``moments``: the 2N-1 P-bit moments m_0..m_{2N-2} (``M_ij = m_{i+j}``).
    Returns ``R`` as a list of rows, ``R[t][j - t] = R_tj`` for j >= t.
    ``rows`` limits the computation to the first rows (all columns).
    ``workers > 1`` spreads the columns of each row over a spawn-started
    process pool; the arithmetic is unchanged.
    """
    nrows = N if rows is None else min(rows, N)
    R = []
    pool = None
    if workers > 1:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        pool = ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
    try:
        for i in range(nrows):
            col_i = [R[t][i - t] for t in range(i)]
            js = list(range(i, N))
            if pool is None or len(js) < 2 * workers:
                row = cholesky_row(i, moments, col_i, {j: [R[t][j - t] for t in range(i)] for j in js}, P)
            else:
                chunks = [js[c::workers] for c in range(workers)]
                tasks = [(i, moments, col_i, {j: [R[t][j - t] for t in range(i)] for j in ch}, P)
                         for ch in chunks if ch]
                row = {}
                for part in pool.map(_row_task, tasks):
                    row.update(part)
            R.append([row[j] for j in js])
    finally:
        if pool is not None:
            pool.shutdown()
    return R


def cholesky_factorial(N, P, rows=None):
    """R of the beta = 1 matrix (m_k = k!, the paper's first N = 4 example)
    when P is wide enough for every step of ``cholesky`` to be exact.

    Vandermonde's identity sum_t C(i,t) C(j,t) = C(i+j, i) gives
    M = R^T R with the integer factor R_ti = i! C(i, t) (t <= i).  Then
    A_ij = R_ii R_ij = i! j! C(j, i) <= (i+j)!, R_ii = i! and R_ij = j! C(j, i):
    integers below 2^P whenever (2N-2)! < 2^P, so the square root, the
    quotient and every rounding of reading 1 are exact and ``cholesky``
    returns exactly these values.  This is that result written out (it needs
    no O(N^3) arithmetic); P too small for exactness raises ValueError.
    Same layout as ``cholesky``: ``R[t][j - t] = R_tj``; ``rows`` limits it to
    the first rows (all columns).
    """
    f = 1
    for k in range(2, 2 * N - 1):
        f *= k
    if N > 0 and f.bit_length() > P:
        raise ValueError(f"(2N-2)! has {f.bit_length()} bits > P = {P}: not exact")
    fact = [1] * max(N, 1)
    for k in range(1, N):
        fact[k] = fact[k - 1] * k
    R = []
    for t in range(N if rows is None else min(rows, N)):
        row = []
        c = 1  # C(j, t) at j = t
        for j in range(t, N):
            if j > t:
                c = c * j // (j - t)
            row.append(rne(fact[j] * c, 0, P))
        R.append(row)
    return R


# ---------------------------------------------------------------------------
# Inverse iteration (reading 4)
# ---------------------------------------------------------------------------

def forward_solve(R, v, P):
    """y with R^T y = v: ``y_i = RNE(RNE(v_i - sum_{k<i} R_ki y_k) / R_ii)``."""
    N = len(R)
    y = []
    for i in range(N):
        acc = exact_dot([(R[k][i - k], y[k]) for k in range(i)])
        num = _sub_exact(v[i], acc)
        y.append(mp_div(rne(num[0], num[1], P), R[i][0], P))
    return y


def back_solve(R, y, P):
    """w with R w = y: ``w_i = RNE(RNE(y_i - sum_{k>i} R_ik w_k) / R_ii)``."""
    N = len(R)
    w = [None] * N
    for i in range(N - 1, -1, -1):
        acc = exact_dot([(R[i][k - i], w[k]) for k in range(i + 1, N)])
        num = _sub_exact(y[i], acc)
        w[i] = mp_div(rne(num[0], num[1], P), R[i][0], P)
    return w


def rayleigh_lambda(v, w, P):
    """``lambda = RNE(RNE(<v,v>) / RNE(<v,w>))`` with w = M^-1 v: the inverse
    of the Rayleigh quotient of M^-1 at v, an upper bound on lambda_1
    (section "M is extremely ill-conditioned")."""
    vv = exact_dot(list(zip(v, v)))
    vw = exact_dot(list(zip(v, w)))
    return mp_div(rne(vv[0], vv[1], P), rne(vw[0], vw[1], P), P)


def normalise(w, P):
    """``v = w * 2**-E`` with ``E = max_i (e_i + P)`` over nonzero w_i, so the
    largest |v_i| lies in [1/2, 1).  Exact (power-of-two scaling)."""
    nz = [e + P for n, e in w if n]
    E = max(nz) if nz else 0
    return [(n, e - E) if n else (0, 0) for n, e in w]


def inverse_iteration(R, P, T, v0=None):
    """T steps of inverse iteration on M = R^T R.  Returns
    ``(lambda_T, [lambda_1..lambda_T], v_T)``; ``v0`` defaults to all ones."""
    N = len(R)
    v = list(v0) if v0 is not None else [rne(1, 0, P)] * N
    history = []
    for _ in range(T):
        y = forward_solve(R, v, P)
        w = back_solve(R, y, P)
        history.append(rayleigh_lambda(v, w, P))
        v = normalise(w, P)
    return (history[-1] if history else None), history, v


def smallest_eigenvalue(moments, N, P, T, workers=1):
    """Cholesky then T inverse-iteration steps: ``(lambda_T, history, R)``."""
    R = cholesky(moments, N, P, workers=workers)
    lam, hist, _ = inverse_iteration(R, P, T)
    return lam, hist, R
