"""The sampled-row checker (tests/rowcheck.py) on the CPU: it accepts the
oracle's own factor and catches a one-ulp change in a sampled row or in a row
above it."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import oracle  # noqa: E402
from paper_0902_0852_gb300 import inputs  # noqa: E402
from rowcheck import check_rows  # noqa: E402


def test_accepts_the_oracle_factor_and_catches_one_ulp():
    N, beta, P = 40, (7, 4), 384
    m = inputs.moments(N, beta, P)
    R = oracle.cholesky(m, N, P)
    assert check_rows(m, R, P, [0, 1, 17, 39]) == []
    # one ulp in the sampled row 17
    R2 = [list(r) for r in R]
    n, e = R2[17][5]
    R2[17][5] = (n + 1, e)
    assert (17, 22) in check_rows(m, R2, P, [17])
    # one ulp in row 9, above the sampled row 30: row 30 recomputed from it differs
    R3 = [list(r) for r in R]
    n, e = R3[9][21]  # R_{9,30}
    R3[9][21] = (n + 1, e)
    assert check_rows(m, R3, P, [30]) != []


def test_flat_parallel_checker_on_the_packed_layout():
    """The full-width checker over the C ABI's packed arrays (spawned workers)
    accepts the oracle's factor and catches a one-ulp change."""
    from paper_0902_0852_gb300 import hk
    from rowcheck import check_rows_flat
    N, beta, P = 24, (7, 4), 256
    m = inputs.moments(N, beta, P)
    R = oracle.cholesky(m, N, P)
    flat = [x for row in R for x in row]
    sign, exp, limbs = hk.pack(flat, P)
    assert check_rows_flat(m, sign, exp, limbs, N, P, [0, 7, 16, 23], workers=3) == []
    k = 7 * N - (7 * 6) // 2 + (20 - 7)  # R_{7,20}: in row 7, and above row 16 in column 20
    n, e = flat[k]
    flat[k] = (n + 1, e)
    sign, exp, limbs = hk.pack(flat, P)
    bad = check_rows_flat(m, sign, exp, limbs, N, P, [7, 16], workers=3)
    assert (7, 20) in bad and (16, 20) in bad
