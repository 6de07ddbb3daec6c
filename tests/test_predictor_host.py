"""Host logic of the precision predictor (no GPU): the beta grid, the
conservative precision rule, target encoding, and the required-bits search
driven by a synthetic solver whose error law is known."""
import math
from fractions import Fraction

import pytest

from paper_0902_0852_gb300 import predictor as pr


def test_beta_grid():
    g = pr.beta_grid()
    vals = [p / q for p, q in g]
    assert vals == sorted(vals) and min(vals) >= 0.6 and max(vals) <= 4.0
    for b in [(3, 4), (1, 1), (3, 2), (2, 1), (3, 1), (7, 4), (3, 5), (7, 11), (4, 1), (5, 2)]:
        assert b in g
    assert (4, 7) not in g and (2, 4) not in g
    assert pr.snap_beta(0.74) == (3, 4) and pr.snap_beta(1.76) == (7, 4) and pr.snap_beta(3.9) == (4, 1)


def test_conservative_rule():
    # beta = 1: the batched sweep's formula
    for N in (100, 333, 600):
        bits = math.lgamma(2 * N - 1) / math.log(2)
        assert pr.p_conservative(N, (1, 1)) == int(math.ceil((bits + 4 * math.sqrt(N) + 256) / 32)) * 32
    # beta < 1 is sized on the largest entry Gamma((2N-1)/beta)/beta
    N = 200
    assert pr.p_conservative(N, (3, 5)) >= pr.largest_entry_bits(N, (3, 5)) + 256
    assert pr.p_conservative(N, (3, 5)) > pr.p_conservative(N, (1, 1)) >= pr.p_conservative(N, (3, 1))
    # largest entry at beta = 1 is (2N-2)!
    assert pr.largest_entry_bits(50, (1, 1)) == pytest.approx(math.log2(math.factorial(98)), rel=1e-12)


def test_target_encoding_round_trip():
    for N, bits, l2, it in [(32, 288, -20.5, 17), (512, 4100, -130.0, 60)]:
        y = pr.encode_targets(N, bits, l2, it)
        b2, l22, it2 = pr.decode_targets(N, y)
        assert b2 == pytest.approx(bits) and l22 == pytest.approx(l2) and it2 == pytest.approx(it)


def test_rel_err_bits():
    ref = (3 << 200, -250)
    v = (ref[0] + (ref[0] >> 130), ref[1])  # relative change 2^-130 (up to the shift's truncation)
    assert 129.9 < pr.rel_err_bits(v, ref) < 130.1
    assert pr.rel_err_bits(ref, ref) == math.inf


def _fake_solver(req_bits, log):
    """Relative error 0.7 * 2^-(P - req + 128); pivots fail 300 bits below req;
    the iteration converges from P >= 192."""
    def solve(jobs):
        out = []
        for N, beta, P in jobs:
            req = req_bits[(N, beta)]
            log.append((N, P))
            if P < req - 300:
                out.append((2, None, 0, False))
                continue
            lam = Fraction(1, 3) * (1 + Fraction(7, 10) * Fraction(2) ** -(P - req + 128))
            n = lam.numerator * 2 ** 200 // lam.denominator
            out.append((0, (n, -200), 40, P >= 192))
        return out
    return solve


@pytest.mark.parametrize("req", [210, 300, 777, 1400])
def test_search_finds_smallest_agreeing_precision(req):
    """Requirements below the reference precision (P_ref = 2016 and 7936 here)."""
    inst = [(64, (1, 1)), (400, (3, 2))]
    assert [pr.p_conservative(N, b) + pr.DELTA for N, b in inst] == [2016, 7936]
    req_bits = {(64, (1, 1)): req, (400, (3, 2)): req + 3001}
    log = []
    recs = pr.generate(inst, solve_fn=_fake_solver(req_bits, log))
    for r in recs:
        want = int(math.ceil(req_bits[(r["N"], tuple(r["beta"]))] / 32.0)) * 32
        assert r["ok"] and r["bits"] == max(want, 224)
        assert r["iters"] == 40 and r["log2_lambda"] == pytest.approx(math.log2(1 / 3), abs=1e-9)
        assert len(r["probes"]) <= 12
