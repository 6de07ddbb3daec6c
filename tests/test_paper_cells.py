"""Host logic of the Table 3 cells (no GPU): the exact five-digit rounding,
the starting precision rule, and the oracle at N = 100 for beta = 1/3 and 1/2
against Table 3 (pins the method on the two betas whose moments are pure
factorials: m_k = 3 (3k+2)! and 2 (2k+1)!)."""
from fractions import Fraction

import pytest

from oracle import hankel as H
from paper_0902_0852_gb300 import inputs
from paper_0902_0852_gb300.paper_cells import TABLE3, p_cell, sig5


def test_sig5_exact_rounding():
    assert sig5((1, 0)) == (10000, 0)
    assert sig5((-3, -1)) == (15000, 0)            # 1.5
    assert sig5((12345, 0)) == (12345, 4)
    assert sig5((123455, 0)) == (12346, 5)         # exact tie 12345.5 -> even
    assert sig5((99999 * 2 + 1, -1)) == (10000, 5)  # 99999.5 rounds up to 1.0000e5
    # a value far below the double range: 2^-1100 = 7.3...e-332
    d, k = sig5((1, -1100))
    want = Fraction(1, 2 ** 1100)
    assert k == -332 and abs(Fraction(d, 10 ** 4) * Fraction(10) ** k - want) <= Fraction(10) ** (k - 4) / 2


def test_p_cell_rule():
    assert p_cell(100) == 32 * -(-(350 + 512) // 32)
    for N in (100, 300, 500, 1000, 1500):
        P = p_cell(N)
        assert P % 32 == 0 and P >= 3.5 * N + 512 and P < 3.5 * N + 512 + 32
        assert P + 1024 <= 32768  # the verification rerun stays inside the library's range


def test_inputs_small_beta_are_factorials():
    """beta = 1/3: m_k = Gamma(3(k+1)) * 3 = 3 (3k+2)!; beta = 1/2: 2 (2k+1)!."""
    from math import factorial
    P = 4096
    for k in (0, 1, 5, 40):
        for beta, exact in (((1, 3), 3 * factorial(3 * k + 2)), ((1, 2), 2 * factorial(2 * k + 1))):
            n, e = inputs.moment(k, beta, P)
            if exact.bit_length() <= P:
                assert Fraction(n) * Fraction(2) ** e == exact


@pytest.fixture(scope="module")
def oracle_N100_small_beta():
    """The oracle's lambda_1 at N = 100 for beta = 1/3 and 1/2 (it converges in
    7 and 24 steps from the all-ones vector)."""
    out = {}
    for beta, T in (((1, 3), 12), ((1, 2), 30)):
        P = p_cell(100)
        lam, _, _ = H.smallest_eigenvalue(inputs.moments(100, beta, P), 100, P, T)
        out[beta] = lam
    return out


@pytest.mark.parametrize("beta", [(1, 3), (1, 2)])
def test_oracle_table3_N100_small_beta(oracle_N100_small_beta, beta):
    """Table 3, N = 100: beta = 1/3 -> 3.4720, beta = 1/2 -> 2.7397e-1."""
    assert sig5(oracle_N100_small_beta[beta]) == TABLE3[(100, beta)]


@pytest.mark.parametrize("beta,want", [((1, 3), (852, 1396)), ((1, 2), (736, 861))])
def test_oracle_table1_N100_small_beta(oracle_N100_small_beta, beta, want):
    """Table 1's lower bound on cond(M) is Gamma((2N-1)/beta)/beta / lambda_1:
    at N = 100 it prints 8.52e1396 (beta = 1/3) and 7.36e861 (beta = 1/2).
    With beta = 1/q the numerator is the integer q (199 q - 1)!; three
    significant figures computed exactly."""
    from math import factorial, floor, log10
    q = beta[1]
    cond = Fraction(q * factorial(199 * q - 1)) / H.to_fraction(oracle_N100_small_beta[beta])
    k = floor(log10(cond.numerator) - log10(cond.denominator))
    d = round(cond / Fraction(10) ** (k - 2))
    if d >= 1000:  # the float estimate of the exponent was one low
        k += 1
        d = round(cond / Fraction(10) ** (k - 2))
    assert (d, k) == want


def _fake_solver(value):
    def solve(N, beta, predictor=None, P=None, T=None, max_escalations=8):
        return dict(lam=value, P=P, iters=8, tried=[P, P + 1024], seconds=1.0, verified=True, T=T)
    return solve


def test_run_cell_compares_with_table3(monkeypatch):
    """run_cell passes the cell's starting precision to the verified solve and
    compares the five-figure rounding of its value with Table 3 (a stand-in
    solver here: the device runs are the GPU tests and bench.py --paper-cells)."""
    from paper_0902_0852_gb300 import paper_cells as pc
    from paper_0902_0852_gb300 import predictor as pr
    monkeypatch.setattr(pr, "solve_verified", _fake_solver(inputs._round_ratio(33763, 10000, 128)))
    r = pc.run_cell(500, (1, 3))
    assert r["P"] == p_cell(500) and r["tried"] == [p_cell(500), p_cell(500) + 1024]
    assert r["lambda"] == "3.3763e0" and r["table3"] == "3.3763e0" and r["match"] and r["verified"]
    # the N = 1500, beta = 1/2 cell: the device value against the printed one
    monkeypatch.setattr(pr, "solve_verified", _fake_solver(inputs._round_ratio(65295, 1000000, 128)))
    r = pc.run_cell(1500, (1, 2))
    assert r["lambda"] == "6.5295e-2" and r["table3"] == "6.6295e-2" and not r["match"]
    # a failed solve reports no value and no match
    monkeypatch.setattr(pr, "solve_verified", _fake_solver(None))
    r = pc.run_cell(100, (7, 4))
    assert r["lambda"] is None and not r["match"]


def test_table3_holds_every_cell():
    assert len(TABLE3) == 20
    for N in (100, 300, 500, 1000, 1500):
        for beta in ((1, 3), (1, 2), (1, 1), (7, 4)):
            d, k = TABLE3[(N, beta)]
            assert 10 ** 4 <= d < 10 ** 5
    # lambda_1 decreases with N in every column (Table 3's own monotonicity)
    for beta in ((1, 3), (1, 2), (1, 1), (7, 4)):
        vals = [Fraction(TABLE3[(N, beta)][0]) * Fraction(10) ** TABLE3[(N, beta)][1]
                for N in (100, 300, 500, 1000, 1500)]
        assert vals == sorted(vals, reverse=True)
