"""Writes gamma_consts.txt: Gamma(a/p) for the denominators p that the
rational shape parameters beta = p/q of the workloads need, as
floor(Gamma(a/p) * 2^F) in hex.  The Hankel moments for beta = p/q follow
from these constants by the exact recurrence Gamma(x + 1) = x Gamma(x)
(see inputs.py), so the run-time input generator needs no special
functions.  This script runs offline with mpmath; its output is committed.

Each value is computed at F + 128 bits and truncated, so
|Gamma(a/p) - G 2^-F| < 2^(1-F).  Only reduced fractions a/p with a < p are
stored (Gamma(2/4) is Gamma(1/2)).  Reflection Gamma(x)Gamma(1-x) =
pi/sin(pi x) gives the upper half of each denominator from the lower half;
the lower-half gamma evaluations run in parallel processes.
"""
import sys
from concurrent.futures import ProcessPoolExecutor
from math import gcd

import mpmath

# denominator -> fractional bits kept
TARGETS = {2: 33024, 3: 33024, 4: 33024, 5: 33024, 7: 33024}


def _gamma(args):
    a, p, F = args
    mpmath.mp.prec = F + 128
    v = mpmath.gamma(mpmath.mpf(a) / p)
    print(f"gamma({a}/{p}) done", file=sys.stderr, flush=True)
    return (a, p), v


def main(path):
    low = [(a, p, F) for p, F in sorted(TARGETS.items()) for a in range(1, p) if gcd(a, p) == 1 and 2 * a <= p]
    with ProcessPoolExecutor(len(low)) as ex:
        vals = dict(ex.map(_gamma, low))
    lines = []
    for p, F in sorted(TARGETS.items()):
        mpmath.mp.prec = F + 128
        for a in range(1, p):
            if gcd(a, p) != 1:
                continue
            if 2 * a <= p:
                v = vals[(a, p)]
            else:
                x = mpmath.mpf(a) / p
                v = mpmath.pi / (mpmath.sin(mpmath.pi * x) * vals[(p - a, p)])
            G = int(mpmath.floor(v * mpmath.mpf(2) ** F))
            lines.append(f"{a} {p} {F} {G:x}")
    with open(path, "w") as f:
        f.write("# a p F hex(floor(Gamma(a/p) * 2^F)); |error| < 2^(1-F)\n")
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "gamma_consts.txt")
