"""The smallest eigenvalue at the paper's sizes (Table 3), on the device at a
verified precision.

Table 3 lists lambda_1 of M_ij = Gamma((1+i+j)/beta)/beta for N = 100 ... 1500
and beta in {1/3, 1/2, 1, 7/4}.  In the paper's fixed-point representation
every entry carries its whole integer part, so the working width grows with
the largest entry, about log2 Gamma((2N-1)/beta) bits (some 105,000 bits at
N = 1500, beta = 1/3).  Here entries are P-bit floating-point values and each
column is accumulated exactly on its own binary grid, so P only has to cover
how much the factorisation loses after its implicit diagonal scaling: about
2-3.5 N bits for beta in [1/3, 7/4] (the oracle needs 384 / 640 bits at
N = 120 / 240 for beta = 1/3 and 448 / 704 for beta = 1/2; the predictor's
training data give about 3.4 N at beta = 1 and 3.9 N at 7/4 near N = 500).
The exponent spread inside a column (about 2.9 N bits at beta = 1/3, 1.9 N at
1/2, 0.96 N at 1, measured with the oracle at N = 60 and 120) is absorbed by
the accumulation window, which widens itself when a column does not fit.

Every cell runs at ``p_cell(N)`` = 32 ceil((3.5 N + 512) / 32) bits and is
accepted when a rerun at P + 1024 agrees with it to 2^-128 (relative); on
disagreement P grows by 1024 and the check repeats (``predictor.solve_verified``).
"""
import math
from fractions import Fraction

from . import predictor as pr

# Table 3 ("The smallest eigenvalue of M"): five significant digits as
# (d, k) meaning d.dddd x 10^k (d holds the five digits as an integer)
TABLE3 = {
    (100, (1, 3)): (34720, 0), (100, (1, 2)): (27397, -1), (100, (1, 1)): (21079, -15), (100, (7, 4)): (16976, -45),
    (300, (1, 3)): (33984, 0), (300, (1, 2)): (15837, -1), (300, (1, 1)): (55215, -28), (300, (7, 4)): (14844, -102),
    (500, (1, 3)): (33763, 0), (500, (1, 2)): (12047, -1), (500, (1, 1)): (11138, -36), (500, (7, 4)): (67121, -149),
    (1000, (1, 3)): (33544, 0), (1000, (1, 2)): (82087, -2), (1000, (1, 1)): (10892, -52),
    (1000, (7, 4)): (36209, -246),
    (1500, (1, 3)): (33447, 0), (1500, (1, 2)): (66295, -2), (1500, (1, 1)): (54593, -65),
    (1500, (7, 4)): (64232, -330),
}

# the cells the paper's fixed-point format needs the widest numbers for
# (beta = 1/3 and 1/2 at N >= 500), then the rest of the N = 1500 row
DEFAULT_CELLS = [(500, (1, 3)), (500, (1, 2)), (1000, (1, 3)), (1000, (1, 2)), (1500, (1, 3)), (1500, (1, 2)),
                 (1500, (1, 1)), (1500, (7, 4))]


ALL_CELLS = [(N, beta) for N in (100, 300, 500, 1000, 1500) for beta in ((1, 3), (1, 2), (1, 1), (7, 4))]


def p_cell(N):
    """Starting precision of a Table 3 cell: 32 ceil((3.5 N + 512) / 32) bits."""
    return 32 * ((7 * N + 1024 + 63) // 64)


def sig5(v):
    """The value n 2^e (a pair of ints, n != 0) rounded to five significant
    decimal digits, exactly: (d, k) with 10^4 <= d < 10^5 and
    |v| ~ d 10^(k-4)."""
    n, e = v
    f = abs(Fraction(n) * (Fraction(2) ** e))
    k = math.floor(math.log10(abs(n)) + e * math.log10(2))
    for _ in range(3):  # the float estimate of the decimal exponent may be one off
        q = f * Fraction(10) ** (4 - k)
        if q < 10 ** 4 - Fraction(1, 2):
            k -= 1
        elif q >= 10 ** 5 - Fraction(1, 2):
            k += 1
        else:
            break
    d = round(f * Fraction(10) ** (4 - k))
    return d, k


def run_cell(N, beta, P=None, T=pr.MAX_ITERS):
    """lambda_1 of one Table 3 cell at a verified precision, with its
    comparison against the table's five digits."""
    r = pr.solve_verified(N, beta, P=p_cell(N) if P is None else P, T=T)
    dk = sig5(r["lam"]) if r["lam"] is not None else None
    want = TABLE3.get((N, beta))
    return {"N": N, "beta": f"{beta[0]}/{beta[1]}", "P": r["P"], "tried": r["tried"], "iters": r["iters"],
            "verified": r["verified"], "seconds": round(r["seconds"], 2),
            "lambda": None if dk is None else f"{dk[0] / 1e4:.4f}e{dk[1]}",
            "table3": None if want is None else f"{want[0] / 1e4:.4f}e{want[1]}",
            "match": want is not None and dk == want,
            "largest_entry_bits": int(pr.largest_entry_bits(N, beta))}
