"""The shifted LDL^T's pivot kernel replaces a shift x that lies wholly below
the diagonal's column-sum grid 2^G by a stand-in of its sign and magnitude
2^(G-1), whenever the rest of the sum Z0 = m_2t - colsum is at least
2^(G+P+1) in magnitude.  The claim: RNE_P(Z0 2^G - x) = RNE_P(Z0 2^G -
sign(x) 2^(G-1)), the right side computed as the magnitude 2|Z0| -+ 1 on the
grid 2^(G-1) with Z0's sign.  Checked here with exact rationals and the
exhaustive rounding of test_oracle_pins (no GPU), on random operands and on
sums placed exactly on and next to rounding midpoints and representable
values."""
import random
from fractions import Fraction

from test_oracle_pins import round_fraction


def _standin_magnitude(z0, s0, sx):
    same = (s0 > 0) == (sx > 0)  # x of Z0's sign: the magnitude shrinks
    return 2 * z0 - 1 if same else 2 * z0 + 1


def test_standin_gives_the_same_rounding():
    rng = random.Random(5)
    for _ in range(6000):
        P = rng.choice([8, 16, 33, 64])
        G = rng.randrange(-50, 50)
        bits = P + 2 + rng.randrange(0, 12)  # |Z0| >= 2^(P+1)
        z0 = rng.getrandbits(bits) | (1 << (bits - 1))
        if rng.random() < 0.4:
            # Z0 2^G exactly on a representable value or a midpoint of the result
            sh = bits - P
            z0 = (z0 >> sh << sh) | rng.choice([0, 1 << (sh - 1)])
        s0 = rng.choice([1, -1])
        xm = rng.getrandbits(P) | (1 << (P - 1))
        ex = G - P - rng.randrange(0, 40)  # |x| < 2^(ex + P) <= 2^G
        sx = rng.choice([1, -1])
        exact = Fraction(s0 * z0) * Fraction(2) ** G - Fraction(sx * xm) * Fraction(2) ** ex
        standin = Fraction(s0 * _standin_magnitude(z0, s0, sx)) * Fraction(2) ** (G - 1)
        assert standin == Fraction(s0 * z0) * Fraction(2) ** G - Fraction(sx) * Fraction(2) ** (G - 1)
        assert round_fraction(exact, P) == round_fraction(standin, P), (P, G, z0, s0, xm, ex, sx)


def test_standin_needs_the_magnitude_condition():
    """Below 2^(G+P+1) the stand-in can round differently: Z0 = 2^P (a power
    of two whose predecessor grid is finer) with a positive x just below one
    grid unit."""
    P, G = 8, 0
    z0 = 1 << P
    x = Fraction((1 << P) - 1, 1 << P)  # 1 - 2^-8, below 2^G = 1
    exact = Fraction(z0) - x
    standin = Fraction(z0) - Fraction(1, 2)
    assert round_fraction(exact, P) != round_fraction(standin, P)
