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


@pytest.mark.parametrize("beta,T", [((1, 3), 12), ((1, 2), 30)])
def test_oracle_table3_N100_small_beta(beta, T):
    """Table 3, N = 100: beta = 1/3 -> 3.4720, beta = 1/2 -> 2.7397e-1 (the
    oracle converges in 7 and 24 steps from the all-ones vector)."""
    P = p_cell(100)
    m = inputs.moments(100, beta, P)
    lam, hist, _ = H.smallest_eigenvalue(m, 100, P, T)
    assert sig5(lam) == TABLE3[(100, beta)]
