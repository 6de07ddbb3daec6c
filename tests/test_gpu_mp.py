"""The device multiprecision library against exact integer arithmetic
(products, reciprocals) and against the oracle's correctly rounded sqrt,
division and rounding.  Runs one single-block device operation per call
through the C ABI self-test hook."""
import random

import pytest

from oracle import hankel as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hk():
    from paper_0902_0852_gb300 import build, hk as mod
    build.build()
    mod.lib()
    return mod


def _rand_bits(rng, bits):
    return rng.getrandbits(bits) | (1 << (bits - 1))


def test_mul_exact(hk):
    rng = random.Random(10)
    sizes = [1, 2, 3, 7, 33, 100, 257, 800]
    for nx in sizes:
        for ny in [1, 5, 64, 801]:
            for kind in range(3):
                if kind == 0:
                    x, y = _rand_bits(rng, 32 * nx), _rand_bits(rng, 32 * ny)
                elif kind == 1:  # all-ones limbs: longest carry chains
                    x, y = (1 << (32 * nx)) - 1, (1 << (32 * ny)) - 1
                else:
                    x, y = 1 << (32 * nx - 1), (1 << (32 * ny)) - 1
                assert hk.hk_selftest_mp(0, 1, x, y=y) == x * y, (nx, ny, kind)


@pytest.mark.parametrize("L", [1, 2, 3, 5, 8, 17, 64, 255, 256, 768])
def test_reciprocal_is_floor(hk, L):
    rng = random.Random(L)
    P = 32 * L
    cases = [1 << (P - 1), (1 << P) - 1, (1 << (P - 1)) + 1] + [_rand_bits(rng, P) for _ in range(4)]
    for d in cases:
        assert hk.hk_selftest_mp(1, L, d) == (1 << (2 * P + 1)) // d


@pytest.mark.parametrize("L", [1, 2, 3, 4, 64, 256, 768])
def test_sqrt_correctly_rounded(hk, L):
    rng = random.Random(100 + L)
    P = 32 * L
    cases = [(1 << (P - 1), 0), ((1 << P) - 1, 1), ((1 << (P - 1)) * 1, -5)]
    cases += [(_rand_bits(rng, P), rng.randrange(-300, 300)) for _ in range(6)]
    for m, e in cases:
        got = hk.hk_selftest_mp(2, L, m, ex=e)
        want = H.mp_sqrt((m, e), P)
        assert got == want, (L, m, e)


@pytest.mark.parametrize("L", [1, 2, 3, 64, 256, 768])
def test_division_correctly_rounded(hk, L):
    rng = random.Random(200 + L)
    P = 32 * L
    top = (1 << P) - 1
    cases = [(top, 0, 1 << (P - 1), 0), (1 << (P - 1), 3, top, -2)]
    cases += [(_rand_bits(rng, P), rng.randrange(-99, 99), _rand_bits(rng, P), rng.randrange(-99, 99))
              for _ in range(6)]
    for a, ea, b, eb in cases:
        got = hk.hk_selftest_mp(3, L, a, ex=ea, y=b, ey=eb)
        want = H.mp_div((a, ea), (b, eb), P)
        assert got == want, (L, a, b)


@pytest.mark.parametrize("L", [1, 2, 3, 64, 768])
def test_division_exact_and_near_exact_quotients(hk, L):
    """Exact quotients, which the guard-bit fast path must hand to the exact
    remainder (num = den, a power-of-two divisor), and quotients next to exact
    values (num = den * k cut back to P bits, and a unit of num either side),
    against the oracle's correctly rounded division.  (An exact tie cannot
    occur: its odd part would need P + 1 bits but divides num's odd part.)"""
    rng = random.Random(400 + L)
    P = 32 * L
    cases = []
    for _ in range(3):
        den = _rand_bits(rng, P)
        cases.append((den, den))                          # quotient exactly 1
        cases.append((_rand_bits(rng, P), 1 << (P - 1)))  # power-of-two divisor
        for k in (3, 5, 7):
            num = den * k
            num >>= num.bit_length() - P
            cases += [(num, den), (num - 1, den), (num + 1, den)]
    for a, b in cases:
        if a.bit_length() != P or b.bit_length() != P:
            continue
        ea, eb = rng.randrange(-40, 40), rng.randrange(-40, 40)
        got = hk.hk_selftest_mp(3, L, a, ex=ea, y=b, ey=eb)
        assert got == H.mp_div((a, ea), (b, eb), P), (L, a, b)


@pytest.mark.parametrize("L", [1, 2, 64, 256])
def test_rounding_rne(hk, L):
    rng = random.Random(300 + L)
    P = 32 * L
    cases = []
    for bits in [1, P - 3, P, P + 1, P + 2, 2 * P + 7, 3 * P]:
        cases.append(_rand_bits(rng, bits))
    # exact ties both ways, and a carry out of the mantissa
    cases.append(((1 << P) + 1) << 1 | 1)      # odd mantissa + exact half: rounds up
    cases.append((1 << P) << 1 | 1)            # even mantissa + exact half: stays
    cases.append(((1 << (P + 1)) - 1))         # all ones: carries to 2^P
    for x in cases:
        got = hk.hk_selftest_mp(4, L, x, ex=-17)
        want = H.rne(x, -17, P)
        assert got == want, (L, x.bit_length())
