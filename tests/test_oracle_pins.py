"""Pins of the CPU oracle to facts fixed outside it: exact rational rounding,
the beta = 1 closed form, the paper's N = 4 examples and Table 3, an
independent high-precision eigensolve, and an exact inertia certificate.

No GPU is used here.  The last tests plant mistakes in the oracle (on the CPU)
and check that the pins catch them.
"""
import math
import random
from fractions import Fraction
from math import comb, factorial

import pytest

import oracle
from oracle import hankel as H
from paper_0902_0852_gb300 import inputs

mpmath = pytest.importorskip("mpmath")


# ---------------------------------------------------------------------------
# independent rounding by exhaustive candidate comparison (Fractions only)
# ---------------------------------------------------------------------------

def _candidates(x, P):
    """The two P-bit floats around the positive rational x."""
    # a first guess from the bit lengths (a float log2 would overflow for the
    # moments of fast-growing weights, beyond 2^1024), off by at most one
    x = Fraction(x)
    e = x.numerator.bit_length() - x.denominator.bit_length() - P + 1 if x > 0 else 0
    # fix e so that x / 2**e lies in [2**(P-1), 2**P)
    while x / Fraction(2) ** e >= 2 ** P:
        e += 1
    while x / Fraction(2) ** e < 2 ** (P - 1):
        e -= 1
    lo = math.floor(x / Fraction(2) ** e)
    return lo, e


def round_fraction(x, P):
    """Nearest P-bit float to the rational x, ties to even mantissa."""
    if x == 0:
        return (0, 0)
    neg = x < 0
    x = -x if neg else x
    lo, e = _candidates(x, P)
    hi = lo + 1
    dlo, dhi = x - lo * Fraction(2) ** e, hi * Fraction(2) ** e - x
    if dlo < dhi or (dlo == dhi and lo % 2 == 0):
        m = lo
    else:
        m = hi
    if m == 2 ** P:
        m, e = 2 ** (P - 1), e + 1
    return (-m if neg else m, e)


def F(x):
    return H.to_fraction(x)


def test_rne_equals_exact_rounding():
    rng = random.Random(1)
    for _ in range(3000):
        P = rng.choice([3, 5, 8, 12, 32])
        n = rng.randrange(-(1 << 40), 1 << 40)
        e = rng.randrange(-20, 20)
        assert H.rne(n, e, P) == round_fraction(F((n, e)), P)
    # explicit ties: 0b1001.1 -> 0b1010 (odd rounds up), 0b1010.1 -> 0b1010 (even stays)
    assert H.rne(0b10011, -1, 4) == (0b1010, 0)
    assert H.rne(0b10101, -1, 4) == (0b1010, 0)
    assert H.rne(-0b10011, -1, 4) == (-0b1010, 0)
    # carry out of the mantissa renormalises
    assert H.rne(0b11111, 0, 4) == (0b1000, 2)


def _rand_mp(rng, P, lo=-30, hi=30):
    m = rng.randrange(1 << (P - 1), 1 << P)
    return (m if rng.random() < 0.5 else -m, rng.randrange(lo, hi))


def test_division_correctly_rounded():
    rng = random.Random(2)
    for _ in range(3000):
        P = rng.choice([4, 7, 16, 32, 64])
        x, y = _rand_mp(rng, P), _rand_mp(rng, P)
        assert H.mp_div(x, y, P) == round_fraction(F(x) / F(y), P)


def test_sqrt_correctly_rounded():
    rng = random.Random(3)
    for _ in range(3000):
        P = rng.choice([4, 7, 16, 32, 64])
        m = rng.randrange(1 << (P - 1), 1 << P)
        x = (m, rng.randrange(-31, 31))
        r = H.mp_sqrt(x, P)
        assert r[0] > 0 and (1 << (P - 1)) <= r[0] < (1 << P)
        ulp = Fraction(2) ** r[1]
        v = F(r)
        # the exact square root lies within half an ulp of r (no ties exist)
        assert (v - ulp / 2) ** 2 <= F(x) <= (v + ulp / 2) ** 2
        # and no other P-bit float is closer: neighbours are farther
        assert not ((v + ulp / 2) ** 2 < F(x)) and not ((v - ulp / 2) ** 2 > F(x))


def test_exact_dot_is_exact():
    rng = random.Random(4)
    for _ in range(200):
        P = 40
        pairs = [(_rand_mp(rng, P, -200, 200), _rand_mp(rng, P, -200, 200)) for _ in range(rng.randrange(0, 12))]
        assert F(H.exact_dot(pairs)) == sum((F(a) * F(b) for a, b in pairs), Fraction(0))


# ---------------------------------------------------------------------------
# the paper's beta = 1 factorial matrix (Introduction, first N = 4 example)
# ---------------------------------------------------------------------------

def test_beta1_moments_are_factorials():
    for k, m in enumerate(inputs.moments(40, (1, 1), 512)):
        assert F(m) == factorial(k)


def test_beta1_N4_factorial_example():
    P = 32
    R = H.cholesky(inputs.moments(4, (1, 1), P), 4, P)
    rows = [[F(x) for x in row] for row in R]
    assert rows == [[1, 1, 2, 6], [1, 4, 18], [2, 18], [6]]
    det = 1
    for t in range(4):
        det *= rows[t][0] ** 2
    assert det == 144  # det of the 4x4 factorial Hankel matrix, prod (k!)^2


@pytest.mark.parametrize("N,P", [(64, 2048), (96, 1024)])
def test_beta1_closed_form(N, P):
    """R_ki = i! C(i, k): Vandermonde's identity gives sum_k C(i,k) C(j,k) i! j!
    = (i+j)!, i.e. R^T R = M exactly; every entry fits in P bits so the
    once-rounded factorisation must reproduce it bit for bit."""
    R = H.cholesky(inputs.moments(N, (1, 1), P), N, P)
    for k in range(N):
        for i in range(k, N):
            assert F(R[k][i - k]) == factorial(i) * comb(i, k), (k, i)


# ---------------------------------------------------------------------------
# beta = 7/4 worked example (Introduction, second N = 4 matrix)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("beta", [(7, 4), (3, 4), (3, 2), (2, 1), (3, 1), (1, 2), (1, 3), (4, 3), (4, 5), (5, 2), (5, 8),
                                  (7, 11), (3, 5), (2, 3)])
def test_moments_match_mpmath(beta):
    """The rational-recurrence moment generator equals RNE of an independent
    mpmath evaluation of Gamma((1+k)/beta)/beta at 3P bits."""
    P = 256
    p, q = beta
    mpmath.mp.prec = 3 * P
    for k in range(0, 12):
        exact = mpmath.gamma(mpmath.mpf(q * (1 + k)) / p) * q / p
        man, exp = mpmath.frexp(exact)  # exact = man * 2**exp, man in [1/2, 1)
        n = int(mpmath.floor(man * mpmath.mpf(2) ** (3 * P)))
        want = round_fraction(Fraction(n) * Fraction(2) ** (exp - 3 * P), P)
        # the 3P-bit truncation only matters within 2^-2P of a tie; none here
        assert inputs.moment(k, beta, P) == want, (beta, k)


def _residual_ok(moments, R, P):
    """Local residuals of the once-rounded factorisation:
    off-diagonal |A_ij - R_ii R_ij| <= (2^(1-P) + 2^(-2P)) |A_ij|,
    diagonal |A_ii - R_ii^2| <= 3 2^-P |A_ii|."""
    N = len(R)
    u = Fraction(1, 2 ** P)
    for i in range(N):
        for j in range(i, N):
            A = F(moments[i + j]) - sum((F(R[t][i - t]) * F(R[t][j - t]) for t in range(i)), Fraction(0))
            rii = F(R[i][0])
            if j == i:
                if abs(A - rii * rii) > 3 * u * abs(A):
                    return False
            elif abs(A - rii * F(R[i][j - i])) > (2 * u + u * u) * abs(A):
                return False
    return True


def _audit(moments, R, P):
    """Every rounding of R checked against its definition, exactly: from the
    finished rows, the exact A_ij and S_ij = RNE(A_ij) (the exhaustive rational
    rounding above, not the oracle's); R_ii against the squaring bounds of its
    rounding interval (half an ulp above, half an ulp below -- a quarter at the
    bottom of a binade -- ties to an even mantissa); R_ij against the rational
    rounding of S_ij / R_ii."""
    N = len(R)
    for i in range(N):
        rii = R[i][0]
        for j in range(i, N):
            A = F(moments[i + j]) - sum((F(R[t][i - t]) * F(R[t][j - t]) for t in range(i)), Fraction(0))
            S = round_fraction(A, P)
            if j == i:
                assert S[0] > 0, i
                n, e = rii
                v, ulp = F(rii), Fraction(2) ** e
                below = ulp / 4 if n == 1 << (P - 1) else ulp / 2
                lo2, hi2, s = (v - below) ** 2, (v + ulp / 2) ** 2, F(S)
                assert lo2 <= s <= hi2, (i, "sqrt")
                if s in (lo2, hi2):
                    assert n % 2 == 0, (i, "sqrt tie")
            else:
                assert R[i][j - i] == round_fraction(F(S) / F(rii), P), (i, j)


@pytest.mark.parametrize("beta,N,P", [((1, 1), 24, 256), ((7, 4), 40, 384), ((3, 4), 40, 384),
                                      ((3, 2), 24, 512), ((2, 1), 17, 320), ((1, 2), 30, 384),
                                      ((1, 3), 30, 384)])
def test_every_rounding_audited(beta, N, P):
    """The oracle's R, entry by entry, is the once-rounded value its
    definition gives (the same R the device parity tests compare bit for bit)."""
    m = inputs.moments(N, beta, P)
    _audit(m, H.cholesky(m, N, P), P)


def test_audit_catches_a_one_ulp_error():
    N, P = 12, 128
    m = inputs.moments(N, (7, 4), P)
    R = H.cholesky(m, N, P)
    n, e = R[5][3]
    R[5][3] = (n + 1, e)  # one ulp off in row 5
    with pytest.raises(AssertionError):
        _audit(m, R, P)


def test_beta74_N4_worked_example():
    P = 128
    m = inputs.moments(4, (7, 4), P)
    R = H.cholesky(m, 4, P)
    assert _residual_ok(m, R, P)
    # R^T R reproduces M to within a few ulps of each entry
    for i in range(4):
        for j in range(i, 4):
            recon = sum((F(R[t][i - t]) * F(R[t][j - t]) for t in range(i + 1)), Fraction(0))
            assert abs(recon - F(m[i + j])) <= Fraction(8, 2 ** P) * F(m[i + j])


@pytest.mark.parametrize("beta,N,P", [((1, 1), 14, 96), ((7, 4), 14, 96), ((3, 4), 14, 96),
                                      ((7, 4), 40, 384), ((3, 4), 40, 384), ((3, 2), 40, 384),
                                      ((7, 4), 64, 2048)])
def test_local_residuals(beta, N, P):
    """Every entry of R is the once-rounded value of its exact defining sum
    (within the bounds of one rounding), at the sizes of the device parity
    cases with beta != 1, where no closed form is known."""
    m = inputs.moments(N, beta, P)
    R = H.cholesky(m, N, P)
    assert _residual_ok(m, R, P)


# ---------------------------------------------------------------------------
# lambda_min against independent eigensolvers and the paper's tables
# ---------------------------------------------------------------------------

def _mp_lambda_min(moments, N, prec):
    mpmath.mp.prec = prec
    M = mpmath.matrix(N, N)
    for i in range(N):
        for j in range(N):
            n, e = moments[i + j]
            M[i, j] = mpmath.ldexp(mpmath.mpf(n), e)
    ev = mpmath.eigsy(M, eigvals_only=True)
    return min(ev)


@pytest.mark.parametrize("beta,N,P,T", [((1, 1), 4, 256, 60), ((7, 4), 4, 256, 60),
                                        ((1, 1), 16, 640, 40), ((7, 4), 12, 512, 40),
                                        ((3, 4), 10, 512, 40), ((7, 4), 32, 1024, 60),
                                        ((1, 1), 32, 1536, 60), ((3, 4), 24, 1024, 60),
                                        ((1, 2), 24, 1024, 60), ((1, 3), 24, 1024, 40)])
def test_lambda_vs_2P_eigensolve(beta, N, P, T):
    """Relative error of lambda_min against an independent dense symmetric
    eigensolve of the same (rounded-moment) matrix at 2P bits is <= 2^-128."""
    m = inputs.moments(N, beta, P)
    lam, hist, _ = H.smallest_eigenvalue(m, N, P, T)
    ref = _mp_lambda_min(m, N, 2 * P)
    rel = abs(mpmath.mpf(F(lam).numerator) / F(lam).denominator - ref) / ref
    assert rel <= mpmath.mpf(2) ** -128, (beta, N, float(rel))


def test_lambda_N4_values():
    # mpmath eigsy of the exact N = 4 matrices: 0.0529002939539..., 0.00318093261069...
    lam1, _, _ = H.smallest_eigenvalue(inputs.moments(4, (1, 1), 256), 4, 256, 60)
    lam2, _, _ = H.smallest_eigenvalue(inputs.moments(4, (7, 4), 256), 4, 256, 60)
    assert abs(float(F(lam1)) - 0.0529002939539) < 1e-12
    assert abs(float(F(lam2)) - 0.00318093261069) < 1e-14


@pytest.fixture(scope="module")
def table3_N100():
    out = {}
    for beta in [(1, 1), (7, 4)]:
        P = 2048
        m = inputs.moments(100, beta, P)
        lam, hist, _ = H.smallest_eigenvalue(m, 100, P, 24)
        out[beta] = (lam, hist)
    return out


def _sig(x, digits):
    return float(f"{float(x):.{digits - 1}e}")


def test_table3_N100(table3_N100):
    """Table 3 ("The smallest eigenvalue of M"): N = 100, beta = 1 -> 2.1079e-15,
    beta = 7/4 -> 1.6976e-45 (five significant figures)."""
    assert _sig(F(table3_N100[(1, 1)][0]), 5) == 2.1079e-15
    assert _sig(F(table3_N100[(7, 4)][0]), 5) == 1.6976e-45


def test_table1_consistency(table3_N100):
    """Table 1 lower bound on cond(M) is Gamma((2N-1)/beta)/beta / lambda_1:
    N = 100 -> 9.40e384 (beta = 1), 1.94e228 (beta = 7/4)."""
    mpmath.mp.prec = 256
    for beta, want in [((1, 1), "9.40e+384"), ((7, 4), "1.94e+228")]:
        p, q = beta
        lam = F(table3_N100[beta][0])
        cond = mpmath.gamma(mpmath.mpf(q * 199) / p) * q / p / (mpmath.mpf(lam.numerator) / lam.denominator)
        e10 = int(mpmath.floor(mpmath.log10(cond)))
        digits = int(mpmath.nint(cond / mpmath.mpf(10) ** (e10 - 2)))
        wm, we = want.split("e+")
        assert (digits, e10) == (int(round(float(wm) * 100)), int(we))


def test_history_monotone(table3_N100):
    """lambda_t is the inverse Rayleigh quotient of M^-1: non-increasing in
    exact arithmetic, so only rounding-level increases are allowed."""
    for lam, hist in table3_N100.values():
        vals = [F(x) for x in hist]
        for a, b in zip(vals, vals[1:]):
            assert b <= a * (1 + Fraction(1, 2 ** 2000))


def test_P_vs_P_plus_1024():
    N = 64
    lams = []
    for P in (2048, 3072):
        lam, _, _ = H.smallest_eigenvalue(inputs.moments(N, (1, 1), P), N, P, 30)
        lams.append(F(lam))
    assert abs(lams[0] - lams[1]) <= lams[1] / 2 ** 128


def _neg_pivots(moments, N, x):
    """Exact LDL^T inertia of M - xI over the rationals (Sylvester): the number
    of negative pivots equals the number of eigenvalues below x."""
    A = [[F(moments[i + j]) - (x if i == j else 0) for j in range(N)] for i in range(N)]
    neg = 0
    for k in range(N):
        d = A[k][k]
        if d == 0:
            return None
        neg += d < 0
        for i in range(k + 1, N):
            f = A[i][k] / d
            for j in range(k + 1, N):
                A[i][j] -= f * A[k][j]
    return neg


@pytest.mark.parametrize("beta,N,P", [((1, 1), 10, 512), ((7, 4), 8, 512)])
def test_inertia_certificate(beta, N, P):
    """The interval idea of section "Interval Verification", done exactly:
    with x = lambda(1 -+ 2^-130), M - xI has 0 negative pivots below and
    exactly one above, so lambda_1 is within 2^-130 relative of lambda."""
    m = inputs.moments(N, beta, P)
    lam, _, _ = H.smallest_eigenvalue(m, N, P, 40)
    L = F(lam)
    assert _neg_pivots(m, N, L * (1 - Fraction(1, 2 ** 130))) == 0
    assert _neg_pivots(m, N, L * (1 + Fraction(1, 2 ** 130))) == 1


def test_not_positive_definite():
    P = 32
    m = [H.rne(v, 0, P) for v in (1, 2, 1)]  # [[1, 2], [2, 1]], det -3
    with pytest.raises(oracle.NotPositiveDefinite) as ei:
        H.cholesky(m, 2, P)
    assert ei.value.row == 1


def test_signed_entries_measure():
    """Moments of a discrete measure with negative support points: R has
    negative entries; local residuals still hold."""
    pts = [(-3, 2), (-1, 2), (Fraction(1, 2), 1), (2, 1), (-5, 1), (-Fraction(3, 2), 2)]
    N, P = 6, 128
    mom = []
    for k in range(2 * N - 1):
        v = sum((w * Fraction(x) ** k for x, w in pts), Fraction(0))
        mom.append(round_fraction(v, P))
    R = H.cholesky(mom, N, P)
    assert any(R[t][j][0] < 0 for t in range(N) for j in range(len(R[t])))
    assert _residual_ok(mom, R, P)


# ---------------------------------------------------------------------------
# planted mistakes: each must be caught by a pin above
# ---------------------------------------------------------------------------

def test_planted_round_half_up_is_caught(monkeypatch):
    orig = H.rne

    def half_up(n, e, P):
        r = orig(n, e, P)
        # emulate ties-away: on an exact tie with an even result, bump it
        if n:
            b = abs(n).bit_length()
            if b > P:
                sh = b - P
                if abs(n) & ((1 << sh) - 1) == 1 << (sh - 1) and (abs(r[0]) & 1) == 0:
                    return orig(n + (1 if n > 0 else -1), e, P)
        return r

    monkeypatch.setattr(H, "rne", half_up)
    with pytest.raises(AssertionError):
        test_rne_equals_exact_rounding()


def test_planted_dropped_term_is_caught(monkeypatch):
    orig = H.exact_dot
    monkeypatch.setattr(H, "exact_dot", lambda pairs: orig(pairs[1:]))
    with pytest.raises(AssertionError):
        test_beta1_N4_factorial_example()


def test_planted_wrong_sign_is_caught(monkeypatch):
    def bad_sub(a, b):
        (na, ea), (nb, eb) = a, b
        if na == 0:
            return (nb, eb)
        if nb == 0:
            return (na, ea)
        e = min(ea, eb)
        return ((na << (ea - e)) + (nb << (eb - e)), e)

    monkeypatch.setattr(H, "_sub_exact", bad_sub)
    with pytest.raises(AssertionError):
        test_beta1_closed_form(64, 2048)


def test_planted_transposed_index_is_caught(monkeypatch):
    """Using R_ik for R_ki in the forward solve changes lambda."""
    def bad_forward(R, v, P):
        N = len(R)
        y = []
        for i in range(N):
            acc = H.exact_dot([(R[k][(N - 1 - i) - k] if (N - 1 - i) >= k else (0, 0), y[k]) for k in range(i)])
            num = H._sub_exact(v[i], acc)
            y.append(H.mp_div(H.rne(num[0], num[1], P), R[i][0], P))
        return y

    monkeypatch.setattr(H, "forward_solve", bad_forward)
    with pytest.raises(AssertionError):
        test_lambda_N4_values()


def test_planted_truncating_sqrt_is_caught(monkeypatch):
    def trunc_sqrt(x, P):
        n, e = x
        if e & 1:
            n, e = n << 1, e - 1
        j = P // 2 + 2
        s = math.isqrt(n << (2 * j))
        b = s.bit_length()
        return (s >> (b - P), (e - 2 * j) // 2 + (b - P))

    monkeypatch.setattr(H, "mp_sqrt", trunc_sqrt)
    with pytest.raises(AssertionError):
        test_sqrt_correctly_rounded()


def test_golden_beta1_digest_is_the_closed_form():
    """The stored digest of the N = 256, P = 8192, beta = 1 factor (written by
    tests/golden/make_golden.py from the oracle) equals the digest of the
    closed form R_ki = i! C(i, k), rounded to P bits -- a pin of the stored
    value that does not run the oracle."""
    import importlib.util
    import json
    import os
    here = os.path.dirname(os.path.abspath(__file__))
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(here, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    with open(os.path.join(here, "golden", "config2_beta1.json")) as f:
        g = json.load(f)
    N, P = g["N"], g["P"]
    R = [[H.rne(factorial(j) * comb(j, t), 0, P) for j in range(t, N)] for t in range(N)]
    assert mg.digest_R(R, P) == g["R_sha256"]


@pytest.mark.parametrize("N,P", [(1, 32), (4, 32), (24, 256), (64, 2048)])
def test_factorial_factor_is_the_oracles_cholesky(N, P):
    """The written-out beta = 1 factor (used where the O(N^3) oracle is too
    slow, N = 1000) equals the oracle's own factorisation wherever P makes
    every step exact, and refuses a P that does not."""
    assert H.cholesky_factorial(N, P) == H.cholesky(inputs.moments(N, (1, 1), P), N, P)
    with pytest.raises(ValueError):
        H.cholesky_factorial(64, 512)  # 126! has 703 bits
