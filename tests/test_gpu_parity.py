"""Bit-exact parity of the CUDA path with the oracle: R element by element,
the inverse-iteration history lambda_1..lambda_T, and the degenerate cases.
All inputs are the seeded moments of the paper's matrices (or of small
explicit measures); the calls go through the C ABI."""
import math
from fractions import Fraction

import pytest

import oracle
from paper_0902_0852_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hk():
    from paper_0902_0852_gb300 import build, hk as mod
    build.build()
    mod.lib()
    return mod


def gpu_run(hk, N, beta, P, T, moments=None):
    m = moments if moments is not None else inputs.moments(N, beta, P)
    with hk.Hankel(0) as h:
        h.load(N, beta, P, m)
        h.factor()
        R = h.R()
        lam, hist = None, []
        if T:
            lam, used = h.smallest_eig(T)
            assert used == T
            hist = h.history(T)
        stats = h.stats()
    return m, R, lam, hist, stats


@pytest.mark.parametrize("N,beta,P", [(1, (1, 1), 32), (2, (1, 1), 32), (3, (7, 4), 64), (4, (1, 1), 32),
                                      (4, (7, 4), 128), (5, (3, 4), 64), (12, (7, 4), 256),
                                      (17, (3, 2), 320), (20, (2, 1), 96)])
def test_factor_small(hk, N, beta, P):
    m, R, _, _, _ = gpu_run(hk, N, beta, P, 0)
    assert R == oracle.cholesky(m, N, P)


def test_factor_spans_several_blocks_and_tiles(hk):
    """N = 40 crosses two 16-row panel blocks and a ragged third one."""
    N, P = 40, 384
    for beta in [(7, 4), (3, 1)]:
        m, R, _, _, _ = gpu_run(hk, N, beta, P, 0)
        assert R == oracle.cholesky(m, N, P), beta


def test_config1_factor_and_lambda(hk):
    """N = 64, beta = 1 (moments k!), P = 2048, T = 50 from the all-ones vector:
    R equals the closed form i! C(i,k) and the oracle bit for bit, and so does
    every lambda_t."""
    N, P, T = 64, 2048, 50
    m, R, lam, hist, _ = gpu_run(hk, N, (1, 1), P, T)
    for k in range(N):
        for i in range(k, N):
            n, e = R[k][i - k]
            assert Fraction(n) * Fraction(2) ** e == math.factorial(i) * math.comb(i, k)
    Ro = oracle.cholesky(m, N, P)
    assert R == Ro
    lam_o, hist_o, _ = oracle.inverse_iteration(Ro, P, T)
    assert hist == hist_o
    assert lam == lam_o


@pytest.mark.parametrize("N,beta,P,T", [(24, (7, 4), 512, 12), (30, (3, 4), 768, 10), (33, (1, 1), 640, 9)])
def test_lambda_parity(hk, N, beta, P, T):
    m, R, lam, hist, _ = gpu_run(hk, N, beta, P, T)
    Ro = oracle.cholesky(m, N, P)
    assert R == Ro
    lam_o, hist_o, _ = oracle.inverse_iteration(Ro, P, T)
    assert hist == hist_o


def test_not_positive_definite_row(hk):
    P = 32
    m = [oracle.rne(v, 0, P) for v in (1, 2, 1)]  # [[1, 2], [2, 1]]
    with hk.Hankel(0) as h:
        h.load(2, (1, 1), P, m)
        with pytest.raises(hk.HKError) as ei:
            h.factor()
    assert ei.value.code == hk.HK_ERR_NOT_PD and ei.value.extra["bad_row"] == 1


def test_not_positive_definite_late_row(hk):
    """A PD leading block followed by a failing pivot: same row as the oracle."""
    P, N = 64, 6
    base = inputs.moments(N, (1, 1), P)
    m = list(base)
    m[8] = oracle.rne(1, 0, P)  # m_8 = 1 makes S_44 negative
    with pytest.raises(oracle.NotPositiveDefinite) as eo:
        oracle.cholesky(m, N, P)
    with hk.Hankel(0) as h:
        h.load(N, (1, 1), P, m)
        with pytest.raises(hk.HKError) as ei:
            h.factor()
    assert ei.value.extra["bad_row"] == eo.value.row


def test_signed_entries(hk):
    """Moments of a measure with negative support points: negative R entries
    exercise the subtracting branch of the update kernel."""
    pts = [(-3, 2), (-1, 2), (Fraction(1, 2), 1), (2, 1), (-5, 1), (-Fraction(3, 2), 2), (4, 1), (-7, 1)]
    N, P = 8, 192
    mom = []
    for k in range(2 * N - 1):
        v = sum((w * Fraction(x) ** k for x, w in pts), Fraction(0))
        n, d = v.numerator, v.denominator
        # round v to P bits (exact rational rounding through the oracle's division)
        mom.append(oracle.mp_div(oracle.rne(n, 0, P * 4), oracle.rne(d, 0, P * 4), P) if n else (0, 0))
    m, R, lam, hist, _ = gpu_run(hk, N, (1, 1), P, 6, moments=mom)
    Ro = oracle.cholesky(mom, N, P)
    assert any(x[0] < 0 for row in Ro for x in row)
    assert R == Ro
    _, hist_o, _ = oracle.inverse_iteration(Ro, P, 6)
    assert hist == hist_o


def _digest_flat(sign, exp, limbs):
    """SHA-256 of R in the layout of tests/golden/make_golden.py: per entry,
    sign (int32), exponent (int64), limbs (uint32), little endian, packed."""
    import hashlib
    import numpy as np
    L = limbs.shape[1]
    rec = np.zeros(len(sign), dtype=np.dtype([("s", "<i4"), ("e", "<i8"), ("l", "<u4", (L,))], align=False))
    rec["s"] = sign
    rec["e"] = exp
    rec["l"] = limbs
    return hashlib.sha256(rec.tobytes()).hexdigest()


@pytest.mark.parametrize("name", ["config2_beta1", "config2_beta7_4"])
def test_config2_against_stored_oracle(hk, name):
    """N = 256, P = 8192, beta = 1 and 7/4 (moments rounded from Gamma values
    with guard bits): R bit for bit (digest) and lambda_1..lambda_10 against
    values the oracle wrote (tests/golden/make_golden.py)."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name + ".json")
    g = json.load(open(path))
    N, P, T, beta = g["N"], g["P"], g["T"], tuple(g["beta"])
    m = inputs.moments(N, beta, P)
    with hk.Hankel(0) as h:
        h.load(N, beta, P, m)
        h.factor()
        digest = _digest_flat(*hk.hk_get_R_flat(h.ctx, N, P))
        lam, used = h.smallest_eig(T)
        hist = h.history(T)
    assert digest == g["R_sha256"]
    assert hist == [(int(n), e) for n, e in g["history"]]


@pytest.mark.parametrize("N,beta,P", [(40, (7, 4), 384), (64, (1, 1), 2048), (33, (3, 4), 512)])
def test_int8_tensor_path_bit_identical(hk, N, beta, P):
    """The INT8 tensor-core update (mma.sync u8, 64-bit drains) gives the same R,
    bit for bit, as the IMAD path and the oracle."""
    m = inputs.moments(N, beta, P)
    with hk.Hankel(0) as h:
        h.load(N, beta, P, m)
        h.factor()
        R0 = h.R()
        h.set_update_path(1)
        h.load(N, beta, P, m)
        h.factor()
        R1 = h.R()
        assert h.stats()["limbprod_per_mac"] == h.stats()["W"] ** 2
    assert R1 == R0
    assert R1 == oracle.cholesky(m, N, P)


def test_int8_tensor_path_signed_entries(hk):
    pts = [(-3, 2), (-1, 2), (Fraction(1, 2), 1), (2, 1), (-5, 1), (-Fraction(3, 2), 2), (4, 1), (-7, 1)]
    N, P = 8, 192
    mom = []
    for k in range(2 * N - 1):
        v = sum((w * Fraction(x) ** k for x, w in pts), Fraction(0))
        mom.append(oracle.mp_div(oracle.rne(v.numerator, 0, P * 4), oracle.rne(v.denominator, 0, P * 4), P))
    with hk.Hankel(0) as h:
        h.set_update_path(1)
        h.load(N, (1, 1), P, mom)
        h.factor()
        R = h.R()
    assert R == oracle.cholesky(mom, N, P)


@pytest.mark.parametrize("fuse", ["0", "1000000000"])
def test_solve_paths_bit_identical(hk, monkeypatch, fuse):
    """Blocks solved entry by entry (many-CTA in-block updates) or in one
    launch per block give the same history as the oracle (N = 40 crosses
    three 16-row solve blocks)."""
    monkeypatch.setenv("HK_FUSE_WW", fuse)
    N, beta, P, T = 40, (7, 4), 384, 6
    m, R, lam, hist, _ = gpu_run(hk, N, beta, P, T)
    Ro = oracle.cholesky(m, N, P)
    assert R == Ro
    _, hist_o, _ = oracle.inverse_iteration(Ro, P, T)
    assert hist == hist_o


@pytest.mark.parametrize("N,beta,P", [(40, (7, 4), 2048), (24, (3, 4), 8192)])
def test_karatsuba_depths_bit_identical(hk, N, beta, P):
    """The factor update contracts Karatsuba pieces of one to four levels (81
    sub-contractions at four, each added at up to sixteen offsets); the
    identity is exact, so R and the inverse-iteration history (whose solves
    expand the vector with the same split points) equal the oracle's at every
    depth, and the automatic choice (-1) is one of them."""
    m = inputs.moments(N, beta, P)
    Ro = oracle.cholesky(m, N, P)
    _, hist_o, _ = oracle.inverse_iteration(Ro, P, 4)
    seen = set()
    for lv in (-1, 0, 1, 2, 3, 4):
        with hk.Hankel(0) as h:
            h.set_option(hk.HK_OPT_KARATSUBA, lv)
            h.load(N, beta, P, m)
            h.factor()
            R = h.R()
            lam, used = h.smallest_eig(4)
            hist = h.history(4)
            st = h.stats()
        assert R == Ro, lv
        assert hist == hist_o, lv
        if lv >= 0:
            assert st["karatsuba_levels"] == lv
        seen.add(st["karatsuba_levels"])
    assert len(seen) == 5


@pytest.mark.parametrize("N,beta,P,nb", [(100, (7, 4), 1024, 16), (90, (1, 1), 768, 8), (64, (3, 4), 2048, 16)])
def test_lookahead_bit_identical(hk, N, beta, P, nb):
    """The lookahead (far updates of the next block on a low-priority stream
    while the panel chain runs on a high-priority one, two column-sum buffers
    in flight) reorders only exact integer additions: R and the history equal
    the oracle's with it on or off, with graph capture on or off."""
    m = inputs.moments(N, beta, P)
    Ro = oracle.cholesky(m, N, P)
    _, hist_o, _ = oracle.inverse_iteration(Ro, P, 3)
    for la, graph in ((1, 0), (0, 0), (1, 1)):
        with hk.Hankel(0) as h:
            h.set_option(hk.HK_OPT_LOOKAHEAD, la)
            h.set_option(hk.HK_OPT_GRAPH, graph)
            h.set_option(hk.HK_OPT_PANEL_ROWS, nb)
            h.load(N, beta, P, m)
            h.factor()
            R = h.R()
            lam, used = h.smallest_eig(3)
            hist = h.history(3)
            st = h.stats()
        assert R == Ro, (la, graph)
        assert hist == hist_o, (la, graph)
        if la:
            # the solves' prepared GEMVs were used (and any dropped ones fell back)
            assert st["solve_prepared_used"] > 0, st
        else:
            assert st["solve_prepared_used"] == 0 and st["solve_prepared_dropped"] == 0, st


@pytest.mark.parametrize("N,beta,P,fuse,margin", [(120, (7, 4), 1024, "0", "32"), (100, (1, 1), 640, None, "32"),
                                                  (96, (3, 4), 1536, "0", "4096")])
def test_solve_lookahead_fallbacks_bit_identical(hk, monkeypatch, N, beta, P, fuse, margin):
    """Solve lookahead under stress: the narrowest first-attempt margin (the
    block ranges outgrow it, so blocks retry with a wider one and drop the GEMV
    prepared for the next block) and a wide one, per-entry and fused block
    solves.  The inverse-iteration history equals the oracle's bit for bit."""
    if fuse is not None:
        monkeypatch.setenv("HK_FUSE_WW", fuse)
    monkeypatch.setenv("HK_SOLVE_MARGIN", margin)
    m = inputs.moments(N, beta, P)
    Ro = oracle.cholesky(m, N, P)
    _, hist_o, _ = oracle.inverse_iteration(Ro, P, 3)
    with hk.Hankel(0) as h:
        h.set_option(hk.HK_OPT_LOOKAHEAD, 1)
        h.load(N, beta, P, m)
        h.factor()
        lam, used = h.smallest_eig(3)
        hist = h.history(3)
        st = h.stats()
    assert hist == hist_o, st
    assert st["solve_prepared_used"] + st["solve_prepared_dropped"] > 0, st


# Slack 0 fails in the first block (a restart).  L = P/32 = 15 leaves exactly
# one limb (32 bits) of slack after W is rounded up to a multiple of 4; for
# beta = 3 and 4 the first row's entries spread less than that (at most 18 and
# 16 bits here) while the diagonal entries of later columns spread up to 68 and
# 84 bits, so the failure comes in a later block and the factorisation resumes.
@pytest.mark.parametrize("N,beta,P,slack", [(40, (7, 4), 384, "0"), (57, (3, 1), 512, "0"), (48, (3, 1), 480, "16"),
                                            (56, (4, 1), 480, "16")])
def test_window_widening_resumes_bit_identical(hk, monkeypatch, N, beta, P, slack):
    """A window too narrow for the column spread (forced by HK_WINDOW_SLACK)
    fails part-way; the factorisation widens it, re-aligns the finished rows
    and resumes at the failing block (or restarts when that is block 0).  R
    and the inverse-iteration history still equal the oracle's bit for bit."""
    monkeypatch.setenv("HK_WINDOW_SLACK", slack)
    monkeypatch.setenv("HK_NB", "8")
    m, R, lam, hist, stats = gpu_run(hk, N, beta, P, 5)
    assert stats["widenings"] >= 1
    Ro = oracle.cholesky(m, N, P)
    assert R == Ro
    _, hist_o, _ = oracle.inverse_iteration(Ro, P, 5)
    assert hist == hist_o
    RESUMES.append(stats["resumes"])


RESUMES = []


def test_some_widening_resumed():
    """Of the forced widenings above, at least one resumed at a later block
    (the path that re-aligns finished rows), not only full restarts."""
    if not RESUMES:
        pytest.skip("widening cases did not run")
    assert max(RESUMES) >= 1, RESUMES


def test_sampled_rows_beyond_the_configs(hk):
    """N = 512, beta = 7/4, P = 8192 (a shape no stored value covers): sampled
    rows of the device factor -- the first, both sides of panel-block edges,
    the middle and the last -- equal the oracle's row routine applied to the
    device's own rows above them (tests/rowcheck.py), bit for bit."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from rowcheck import check_rows
    N, beta, P = 512, (7, 4), 8192
    m = inputs.moments(N, beta, P)
    with hk.Hankel(0) as h:
        h.load(N, beta, P, m)
        h.factor()
        R = h.R()
    assert check_rows(m, R, P, [0, 1, 15, 16, 17, 255, 256, 300, 511], max_cols=64) == []


@pytest.mark.parametrize("N,beta,P", [(80, (7, 4), 1024), (130, (1, 1), 768)])
def test_caller_workspace_bit_identical(hk, N, beta, P):
    """With a caller-owned workspace of exactly hk_workspace_bytes(N, P) (no
    library allocations: factor buffers, both solve vector sets of the
    lookahead, unit tables), R and the history equal the oracle's."""
    import torch
    m = inputs.moments(N, beta, P)
    Ro = oracle.cholesky(m, N, P)
    _, hist_o, _ = oracle.inverse_iteration(Ro, P, 3)
    ws = torch.empty(hk.hk_workspace_bytes(N, P), dtype=torch.uint8, device="cuda")
    with hk.Hankel(0) as h:
        hk.hk_set_workspace(h.ctx, ws)
        h.load(N, beta, P, m)
        h.factor()
        R = h.R()
        lam, used = h.smallest_eig(3)
        hist = h.history(3)
        st = h.stats()
    torch.cuda.synchronize()
    assert R == Ro
    assert hist == hist_o
    assert st["solve_prepared_used"] > 0, st
