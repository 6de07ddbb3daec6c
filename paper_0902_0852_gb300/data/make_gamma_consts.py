"""Writes gamma_consts.txt: Gamma(a/p) for the denominators p that the
rational shape parameters beta = p/q of the paper's workloads need, as
floor(Gamma(a/p) * 2^F) in hex.  The Hankel moments for beta = p/q follow
from these constants by the exact recurrence Gamma(x + 1) = x Gamma(x)
(see inputs.py), so the run-time input generator needs no special
functions.  This script runs offline with mpmath; its output is committed.

Each value is computed at F + 64 bits and truncated, so
|Gamma(a/p) - G 2^-F| < 2^(1-F).  Reflection Gamma(x)Gamma(1-x) = pi/sin(pi x)
halves the number of gamma evaluations.
"""
import sys
import mpmath

# denominator -> fractional bits kept
TARGETS = {2: 33024, 3: 33024, 7: 8704}


def main(path):
    lines = []
    for p, F in sorted(TARGETS.items()):
        mpmath.mp.prec = F + 128
        vals = {}
        for a in range(1, p):
            b = p - a
            if b in vals and b != a:
                x = mpmath.mpf(a) / p
                vals[a] = mpmath.pi / (mpmath.sin(mpmath.pi * x) * vals[b])
            else:
                vals[a] = mpmath.gamma(mpmath.mpf(a) / p)
            G = int(mpmath.floor(vals[a] * mpmath.mpf(2) ** F))
            lines.append(f"{a} {p} {F} {G:x}")
            print(f"gamma({a}/{p}) done", file=sys.stderr, flush=True)
    with open(path, "w") as f:
        f.write("# a p F hex(floor(Gamma(a/p) * 2^F)); |error| < 2^(1-F)\n")
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "gamma_consts.txt")
