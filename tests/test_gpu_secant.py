"""The paper's own method on the device against its CPU oracle
(oracle/secant.py), bit for bit: the shifted LDL^T of M - xI (pivots D_t,
columns C_t[r], CDivDiag Q_t[r], the running determinant, the negative-pivot
count) at shifts below, at and above lambda_1; the whole Secant iterate and
determinant sequence; and the verification on both sides of the root
(section "Interval Verification"), checked against the oracle's once-rounded
LDL^T at the same points and against exact rational inertia."""
from fractions import Fraction

import pytest

import oracle
from oracle import secant as S
from paper_0902_0852_gb300 import inputs

pytestmark = pytest.mark.gpu

# the last two: moments that grow so fast (beta = 1/2, 1/3) that a shift of
# order one lies wholly below the late rows' diagonal grid, where the pivot
# kernel replaces x by a one-bit stand-in of its sign (same rounded pivot)
CASES = [((1, 1), 12, 256), ((7, 4), 16, 384), ((3, 4), 16, 384), ((7, 4), 40, 512), ((1, 1), 33, 512),
         ((1, 2), 60, 512), ((1, 3), 48, 384)]


@pytest.fixture(scope="module")
def hk():
    from paper_0902_0852_gb300 import build, hk as mod
    build.build()
    return mod


def _shifts(m, N, P):
    """0, x_1 = -min pivot, the oracle's root, and a point just above it."""
    _, piv0 = S.ldlt_det(m, N, (0, 0), P)
    mn = min(piv0, key=oracle.to_fraction)
    root, _, _ = S.secant(m, N, P)
    n, e = root
    above = oracle.rne(n * ((1 << 60) + 1), e - 60, P)
    return [(0, 0), (-mn[0], mn[1]), root, above]


@pytest.mark.parametrize("beta,N,P", CASES)
def test_ldlt_factors_bit_exact(hk, beta, N, P):
    m = inputs.moments(N, beta, P)
    with hk.Hankel(0) as h:
        h.load(N, beta, P, m)
        for x in _shifts(m, N, P):
            det, neg, zr = hk.hk_ldlt_det(h.ctx, P, x)
            D = hk.hk_get_ldlt(h.ctx, 0, N, P)
            Cd = hk.hk_get_ldlt(h.ctx, 1, N, P)
            Qd = hk.hk_get_ldlt(h.ctx, 2, N, P)
            det_o, D_o, C_o, Q_o = S.ldlt_factors(m, N, x, P)
            assert D == D_o, (beta, N, x)
            assert det == det_o
            assert neg == sum(1 for d in D_o if d[0] < 0) and zr == -1
            for t in range(N - 1):
                assert [Cd[t][r - t] for r in range(t + 1, N)] == [C_o[t][r] for r in range(t + 1, N)], t
                assert [Qd[t][r - t] for r in range(t + 1, N)] == [Q_o[t][r] for r in range(t + 1, N)], t


@pytest.mark.parametrize("beta,N,P", CASES)
def test_secant_sequence_bit_exact(hk, beta, N, P):
    m = inputs.moments(N, beta, P)
    root_o, xs_o, ps_o = S.secant(m, N, P)
    with hk.Hankel(0) as h:
        h.load(N, beta, P, m)
        root, used = hk.hk_secant(h.ctx, P)
        xs, ps = hk.hk_get_secant(h.ctx, used, P)
    assert xs == xs_o and ps == ps_o
    assert root == root_o
    # and it is the smallest eigenvalue: the inverse-iteration oracle agrees
    R = oracle.cholesky(m, N, P)
    lam, _, _ = oracle.inverse_iteration(R, P, 60)
    assert abs(oracle.to_fraction(root) - oracle.to_fraction(lam)) <= oracle.to_fraction(lam) / 2 ** 128


@pytest.mark.parametrize("beta,N,P", CASES[:4])
def test_verification_of_the_root(hk, beta, N, P):
    m = inputs.moments(N, beta, P)
    root, _, _ = S.secant(m, N, P)
    bits = 130
    P2 = (P + bits + 1 + 31) // 32 * 32
    n, e = root
    lo = oracle.rne(n * ((1 << bits) - 1), e - bits, P2)
    hi = oracle.rne(n * ((1 << bits) + 1), e - bits, P2)
    # both points are exact at P2 bits
    assert oracle.to_fraction(lo) == oracle.to_fraction(root) * (1 - Fraction(1, 2 ** bits))
    with hk.Hankel(0) as h:
        h.load(N, beta, P, m)
        out = hk.hk_secant_verify(h.ctx, P, root, bits, P2)
        away = oracle.rne(n * ((1 << 100) + 1), e - 100, P)
        out_away = hk.hk_secant_verify(h.ctx, P, away, bits, P2)
    assert out == (0, 1, 1, -1)
    # the oracle's once-rounded LDL^T at P2 bits at the same two points
    for k, x in enumerate((lo, hi)):
        det_o, D_o = S.ldlt_det(m, N, x, P2)
        assert out[k] == sum(1 for d in D_o if d[0] < 0)
        assert out[2 + k] == (0 if det_o[0] == 0 else (1 if det_o[0] > 0 else -1))
    # a point 2^-100 above the root is rejected: one eigenvalue below x_lo
    assert out_away[0] == 1
    if N <= 16:  # exact rational inertia agrees (the oracle's verification; slow beyond)
        assert S.verify(m, N, root, bits) and not S.verify(m, N, away, bits)


def test_secant_arguments(hk):
    with hk.Hankel(0) as h:
        with pytest.raises(hk.HKError) as ei:
            hk.hk_secant(h.ctx, 256)
        assert ei.value.code == hk.HK_ERR_STATE  # no moments
        N, P = 8, 128
        h.load(N, (1, 1), P, inputs.moments(N, (1, 1), P))
        with pytest.raises(hk.HKError) as ei:
            hk.hk_secant_verify(h.ctx, P, (1 << (P - 1), -P), 130, P)  # P2 too small
        assert ei.value.code == hk.HK_ERR_ARG


def _rand_val(rng, P, elo, ehi):
    m = rng.getrandbits(P) | (1 << (P - 1))
    return (m if rng.random() < 0.5 else -m, rng.randrange(elo, ehi))


def test_secant_scalar_ops_against_exact_rounding(hk):
    """The scalar kernels of the Secant step (exact subtraction rounded once,
    with a sticky unit for an operand more than P + 64 bits below the other;
    product; guard-bit division; exact comparison) against the oracle's
    rounding of the exact results, for operands from equal exponents to
    exponent gaps far beyond the precision."""
    import random
    rng = random.Random(11)
    for P in (64, 256, 1024):
        cases = []
        for gap in (0, 1, 3, 31, P - 1, P, P + 1, P + 63, P + 64, P + 65, P + 200, 5 * P):
            a = _rand_val(rng, P, -50, 50)
            b = (_rand_val(rng, P, 0, 1)[0], a[1] - gap)
            cases += [(a, b), (b, a)]
        a = _rand_val(rng, P, -20, 20)
        cases += [(a, a), (a, (-a[0], a[1])), (a, (0, 0)), ((0, 0), a)]
        # a near-cancellation: b = a - one unit in the last place
        cases.append((a, (a[0] - (1 if a[0] > 0 else -1), a[1])))
        for a, b in cases:
            assert hk.hk_selftest_scalar(0, P, a, b) == S.mp_sub(a, b, P), (P, a[1] - b[1])
            assert hk.hk_selftest_scalar(1, P, a, b) == S.mp_mul(a, b, P)
            if b[0] != 0:
                assert hk.hk_selftest_scalar(2, P, a, b) == oracle.mp_div(a, b, P)
            fa, fb = oracle.to_fraction(a), oracle.to_fraction(b)
            assert hk.hk_selftest_scalar(3, P, a, b) == (fa > fb) - (fa < fb)
