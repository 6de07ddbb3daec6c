"""Seeded, synthetic inputs: the Hankel moments of the paper's matrices.

The matrix of the paper (Introduction) is ``M_ij = Gamma((1+i+j)/beta)/beta``,
i, j = 0..N-1, the Hankel moment matrix of the weight ``exp(-x**beta)`` on
[0, inf).  Only the 2N-1 moments ``m_k = Gamma((1+k)/beta)/beta``,
k = 0..2N-2, are distinct.  They are an INPUT of the method: this module
produces them once, rounded to P bits (round to nearest, ties to even), and the
same bits go to the CUDA library and to the oracle.  It holds none of the
factorisation's arithmetic.

For a rational beta = p/q the argument (1+k)/beta = n0 + a/p splits into an
integer part and a fraction a/p, and
``Gamma(n0 + a/p) = Gamma(a/p) * prod_{i<n0} (a + i p) / p**n0``, an exact
rational multiple of one of the constants Gamma(a/p) stored in
``data/gamma_consts.txt`` (written offline by ``data/make_gamma_consts.py``).
For beta = 1 the moments are the factorials k! (the paper's first N = 4
example), exact whenever k! fits in P bits.

A value is a pair ``(n, e)`` of Python ints meaning ``n * 2**e`` with
``2**(P-1) <= |n| < 2**P`` (or n = e = 0).
"""
import os
from fractions import Fraction
from math import factorial, gcd

_CONSTS = None


def _gamma_consts():
    global _CONSTS
    if _CONSTS is None:
        table = {}
        path = os.path.join(os.path.dirname(__file__), "data", "gamma_consts.txt")
        with open(path) as f:
            for line in f:
                if line.startswith("#") or not line.strip():
                    continue
                a, p, F, g = line.split()
                table[(int(a), int(p))] = (int(F), int(g, 16))
        _CONSTS = table
    return _CONSTS


def _round_ratio(num, den, P):
    """Nearest-even P-bit value of num/den (num, den > 0 integers)."""
    k = P + 2 + max(0, den.bit_length() - num.bit_length())
    q, r = divmod(num << k, den)
    q = 2 * q + (1 if r else 0)
    e = -k - 1
    b = q.bit_length()
    sh = b - P
    m = q >> sh
    rem = q - (m << sh)
    half = 1 << (sh - 1)
    if rem > half or (rem == half and (m & 1)):
        m += 1
        if m == (1 << P):
            m >>= 1
            sh += 1
    return (m, e + sh)


def _round_int(n, P):
    if n == 0:
        return (0, 0)
    b = n.bit_length()
    if b <= P:
        return (n << (P - b), -(P - b))
    return _round_ratio(n, 1, P)


def as_ratio(beta):
    """beta as a reduced (p, q) with beta = p/q > 0."""
    if isinstance(beta, tuple):
        p, q = beta
    else:
        fr = Fraction(beta).limit_denominator(1 << 20) if isinstance(beta, float) else Fraction(beta)
        p, q = fr.numerator, fr.denominator
    g = gcd(p, q)
    p, q = p // g, q // g
    if p <= 0 or q <= 0:
        raise ValueError("beta must be positive")
    return p, q


def moment(k, beta, P):
    """``RNE_P(Gamma((1+k)/beta)/beta)`` as ``(n, e)``."""
    p, q = as_ratio(beta)
    n0, a = divmod(q * (1 + k), p)
    if a == 0:
        # Gamma(n0) / beta = q (n0-1)! / p, an exact rational
        num, den = q * factorial(n0 - 1), p
        if den == 1:
            return _round_int(num, P)
        return _round_ratio(num, den, P)
    consts = _gamma_consts()
    g = gcd(a, p)
    if (a // g, p // g) not in consts:
        raise ValueError(f"no stored constant Gamma({a}/{p}) for beta={p}/{q}")
    F, G = consts[(a // g, p // g)]
    if F < P + 160:
        raise ValueError(f"Gamma({a}/{p}) stored to {F} bits, P={P} needs {P + 160}")
    c = q
    for i in range(n0):
        c *= a + i * p
    d = p ** (n0 + 1) << F
    lo = _round_ratio(G * c, d, P)
    hi = _round_ratio((G + 1) * c, d, P)
    if lo != hi:
        raise ArithmeticError(f"moment {k} of beta={p}/{q} too close to a rounding boundary")
    return lo


def moments(N, beta, P):
    """The 2N-1 moments m_0..m_{2N-2} of the order-N matrix, rounded to P bits."""
    return MomentSource(N, beta).at(P)


class MomentSource:
    """The exact rational parts of the 2N-1 moments of one (N, beta), built
    once with running products (O(N) big-integer products instead of O(N^2)),
    then rounded to any precision P: ``at(P)`` equals ``[moment(k, beta, P)]``.
    Meant for precision searches that need the same matrix at many P."""

    def __init__(self, N, beta):
        self.N = N
        self.p, self.q = as_ratio(beta)
        p, q = self.p, self.q
        parts = []
        run = {}          # residue a -> (n0, q * prod_{i<n0} (a + i p))
        fm, fval = 0, 1   # running factorial fm! = fval
        for k in range(2 * N - 1):
            n0, a = divmod(q * (1 + k), p)
            if a == 0:
                while fm < n0 - 1:
                    fm += 1
                    fval *= fm
                parts.append((None, q * fval, p))
            else:
                n_prev, c = run.get(a, (0, q))
                for i in range(n_prev, n0):
                    c *= a + i * p
                run[a] = (n0, c)
                g = gcd(a, p)
                parts.append(((a // g, p // g), c, n0))
        self.parts = parts

    def at(self, P):
        consts = None
        out = []
        for key, c, n in self.parts:
            if key is None:
                out.append(_round_int(c, P) if n == 1 else _round_ratio(c, n, P))
                continue
            if consts is None:
                consts = _gamma_consts()
            if key not in consts:
                raise ValueError(f"no stored constant Gamma({key[0]}/{key[1]}) for beta={self.p}/{self.q}")
            F, G = consts[key]
            if F < P + 160:
                raise ValueError(f"Gamma({key[0]}/{key[1]}) stored to {F} bits, P={P} needs {P + 160}")
            d = self.p ** (n + 1) << F
            lo = _round_ratio(G * c, d, P)
            if lo != _round_ratio((G + 1) * c, d, P):
                raise ArithmeticError(f"a moment of beta={self.p}/{self.q} is too close to a rounding boundary")
            out.append(lo)
        return out


def batched_instances(count=64, seed=0):
    """The batched sweep's instances: N uniform in [100, 600], beta drawn from
    {3/4, 1, 3/2, 2, 3}, and P = ceil((log2((2N-2)!) + 4 sqrt(N) + 256)/32)*32.
    Returns a list of ``(N, (p, q), P)``."""
    import math
    import numpy as np
    rng = np.random.default_rng(seed)
    Ns = rng.integers(100, 601, count)
    betas = [(3, 4), (1, 1), (3, 2), (2, 1), (3, 1)]
    bidx = rng.integers(0, 5, count)
    out = []
    for N, b in zip(Ns, bidx):
        N = int(N)
        bits = math.lgamma(2 * N - 1) / math.log(2)
        P = int(math.ceil((bits + 4 * math.sqrt(N) + 256) / 32.0)) * 32
        out.append((N, betas[int(b)], P))
    return out
