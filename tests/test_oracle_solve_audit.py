"""Pins of the oracle's inverse iteration to its definition, entry by entry.

Every value of every step is recomputed from the values before it in exact
rational arithmetic and rounded by the exhaustive candidate rounding of
``test_oracle_pins.round_fraction`` (not the oracle's ``rne``):

* forward solve  y_i = RNE(RNE(v_i - sum_{k<i} R_ki y_k) / R_ii),
* back solve     w_i = RNE(RNE(y_i - sum_{k>i} R_ik w_k) / R_ii),
* estimate       lambda_t = RNE(RNE(<v,v>) / RNE(<v,w>)),
* rescaling      v <- w 2^-E by one power of two, largest |v_i| in [1/2, 1),

the two roundings of each solve entry and of the estimate being the ones the
device kernels reproduce bit for bit (the Rayleigh quotient of M^-1 at the
pre-step vector, section "M is extremely ill-conditioned", inverted).  The
factor R under audit is the oracle's own, itself audited entry by entry in
``test_oracle_pins.py``.  Planted variants of each step (one rounding instead
of two, a rescaling that is not a power of two) must fail the audit.
"""
from fractions import Fraction

import pytest

from oracle import hankel as H
from paper_0902_0852_gb300 import inputs

from test_oracle_pins import round_fraction


def F(x):
    return H.to_fraction(x)


def _rnd(x, P):
    return F(round_fraction(x, P))


def audit_iteration(R, P, T):
    """Run T oracle steps from the all-ones vector and check every value of
    every step against its definition.  Returns the audited history."""
    N = len(R)
    Rf = [[F(x) for x in row] for row in R]  # Rf[t][j - t] = R_tj
    v = [H.rne(1, 0, P)] * N
    hist = []
    for _ in range(T):
        y = H.forward_solve(R, v, P)
        yf = [F(x) for x in y]
        for i in range(N):
            num = F(v[i]) - sum((Rf[k][i - k] * yf[k] for k in range(i)), Fraction(0))
            want = round_fraction(_rnd(num, P) / Rf[i][0], P)
            assert y[i] == want, ("forward", i)
        w = H.back_solve(R, y, P)
        wf = [F(x) for x in w]
        for i in range(N - 1, -1, -1):
            num = yf[i] - sum((Rf[i][k - i] * wf[k] for k in range(i + 1, N)), Fraction(0))
            want = round_fraction(_rnd(num, P) / Rf[i][0], P)
            assert w[i] == want, ("back", i)
        lam = H.rayleigh_lambda(v, w, P)
        vf = [F(x) for x in v]
        vv = sum((a * a for a in vf), Fraction(0))
        vw = sum((a * b for a, b in zip(vf, wf)), Fraction(0))
        assert lam == round_fraction(_rnd(vv, P) / _rnd(vw, P), P), "lambda"
        hist.append(lam)
        vn = H.normalise(w, P)
        # one exact power of two for all entries, largest magnitude in [1/2, 1)
        ratios = {wf[i] / F(vn[i]) for i in range(N) if wf[i] != 0}
        assert all(F(vn[i]) == 0 for i in range(N) if wf[i] == 0), "zero entry"
        assert len(ratios) == 1, "common scale"
        r = ratios.pop()
        assert r > 0 and (r.numerator == 1 or r.denominator == 1), "scale is a power of two"
        big = r.numerator if r.denominator == 1 else r.denominator
        assert big & (big - 1) == 0, "scale is a power of two"
        top = max(abs(F(x)) for x in vn)
        assert Fraction(1, 2) <= top < 1, "largest entry in [1/2, 1)"
        v = vn
    return hist


CASES = [((1, 1), 24, 256, 4), ((7, 4), 40, 384, 3), ((3, 4), 40, 384, 3), ((3, 2), 20, 320, 4),
         ((7, 4), 12, 96, 6), ((1, 2), 24, 320, 3), ((1, 3), 24, 320, 3)]


@pytest.mark.parametrize("beta,N,P,T", CASES)
def test_inverse_iteration_audited(beta, N, P, T):
    """The oracle's y, w, lambda and rescaled v, at every step, are the values
    their definitions give (the history the device parity tests compare)."""
    m = inputs.moments(N, beta, P)
    R = H.cholesky(m, N, P)
    hist = audit_iteration(R, P, T)
    assert hist == H.inverse_iteration(R, P, T)[1]


# ---------------------------------------------------------------------------
# planted mistakes (in the oracle, on the CPU): each must fail the audit
# ---------------------------------------------------------------------------

def _planted_cases():
    out = []
    for beta, N, P in [((7, 4), 24, 128), ((3, 4), 24, 128), ((1, 1), 16, 96)]:
        m = inputs.moments(N, beta, P)
        out.append((H.cholesky(m, N, P), P))
    return out


def _fails_audit(cases, T=3):
    for R, P in cases:
        try:
            audit_iteration(R, P, T)
        except AssertionError:
            return True
    return False


def test_planted_single_rounding_forward_solve_fails(monkeypatch):
    def once_rounded(R, v, P):
        N = len(R)
        y = []
        for i in range(N):
            acc = H.exact_dot([(R[k][i - k], y[k]) for k in range(i)])
            num = H._sub_exact(v[i], acc)
            q = H.to_fraction(num) / H.to_fraction(R[i][0])
            y.append(round_fraction(q, P))  # RNE of the exact quotient: one rounding
        return y

    cases = _planted_cases()
    monkeypatch.setattr(H, "forward_solve", once_rounded)
    assert _fails_audit(cases)


def test_planted_single_rounding_back_solve_fails(monkeypatch):
    def once_rounded(R, y, P):
        N = len(R)
        w = [None] * N
        for i in range(N - 1, -1, -1):
            acc = H.exact_dot([(R[i][k - i], w[k]) for k in range(i + 1, N)])
            num = H._sub_exact(y[i], acc)
            w[i] = round_fraction(H.to_fraction(num) / H.to_fraction(R[i][0]), P)
        return w

    cases = _planted_cases()
    monkeypatch.setattr(H, "back_solve", once_rounded)
    assert _fails_audit(cases)


def test_planted_single_rounding_rayleigh_fails(monkeypatch):
    def once_rounded(v, w, P):
        vv = H.exact_dot(list(zip(v, v)))
        vw = H.exact_dot(list(zip(v, w)))
        return round_fraction(H.to_fraction(vv) / H.to_fraction(vw), P)

    cases = _planted_cases()
    monkeypatch.setattr(H, "rayleigh_lambda", once_rounded)
    assert _fails_audit(cases, T=6)


def test_planted_rescaling_by_max_fails(monkeypatch):
    def by_max(w, P):
        top = max(abs(H.to_fraction(x)) for x in w)
        return [round_fraction(H.to_fraction(x) / top / 2, P) if x[0] else (0, 0) for x in w]

    cases = _planted_cases()
    monkeypatch.setattr(H, "normalise", by_max)
    assert _fails_audit(cases)
