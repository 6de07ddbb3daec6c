"""Batched solving: the worker-pool batch gives exactly the single-instance
results (also with CUDA-graph capture and autotuned update schedules, which
cannot change any bit), escalates under-provisioned instances, and agrees with
the oracle on instances of the batched sweep."""
import pytest

import oracle
from paper_0902_0852_gb300 import inputs

pytestmark = pytest.mark.gpu

SMALL = [(12, (7, 4), 256), (20, (1, 1), 320), (33, (3, 2), 512), (17, (2, 1), 256), (40, (3, 1), 640),
         (25, (3, 4), 512)]


@pytest.fixture(scope="module")
def hk():
    from paper_0902_0852_gb300 import build, hk as mod
    build.build()
    mod.lib()
    return mod


def single(hk, N, beta, P, T, options=None):
    with hk.Hankel(0) as h:
        for o, v in (options or {}).items():
            h.set_option(o, v)
        h.load(N, beta, P, inputs.moments(N, beta, P))
        h.factor()
        lam, used = h.smallest_eig(T)
        R = h.R()
    return lam, R


def test_batch_matches_single_instances(hk):
    T = 8
    want = [single(hk, N, beta, P, T)[0] for N, beta, P in SMALL]
    ctx = hk.hk_create(0)
    try:
        batch = [(N, beta, P, inputs.moments(N, beta, P)) for N, beta, P in SMALL]
        for opts in ({}, {hk.HK_OPT_GRAPH: 1}, {hk.HK_OPT_GRAPH: 1, hk.HK_OPT_AUTOTUNE: 1}):
            for o, v in opts.items():
                hk.hk_set_option(ctx, o, v)
            res = hk.hk_batch_solve(ctx, batch, iters=T, nthreads=3)
            assert [r[0] for r in res] == [hk.HK_OK] * len(SMALL)
            assert [r[1] for r in res] == want, opts
            assert [r[2] for r in res] == [T] * len(SMALL)
    finally:
        hk.hk_destroy(ctx)


def test_graph_and_autotune_keep_R_bit_identical(hk):
    N, beta, P = 40, (7, 4), 384
    _, R0 = single(hk, N, beta, P, 2)
    _, R1 = single(hk, N, beta, P, 2, {hk.HK_OPT_GRAPH: 1, hk.HK_OPT_AUTOTUNE: 1})
    _, R2 = single(hk, N, beta, P, 2, {hk.HK_OPT_KARATSUBA: 1, hk.HK_OPT_PANEL_ROWS: 5})
    assert R1 == R0 and R2 == R0


def test_batch_escalates_too_small_precision(hk):
    from paper_0902_0852_gb300 import batch
    res = batch.solve_batch([(30, (3, 4), 64), (16, (1, 1), 256)], iters=6, nthreads=2)
    assert res[0]["escalations"] >= 1 and res[0]["status"] == hk.HK_OK
    assert res[1]["escalations"] == 0 and res[1]["status"] == hk.HK_OK
    lam, _ = single(hk, 30, (3, 4), res[0]["P"], 6)
    assert res[0]["lam"] == lam


def test_batched_sweep_subset_against_oracle(hk):
    """The four smallest instances of the batched sweep (seed 0: N = 101, 102,
    104, 108; beta = 1, 3/4, 2, 1), with the sweep's precision rule and
    escalation, against the oracle at the final precision."""
    from paper_0902_0852_gb300 import batch
    inst = sorted(inputs.batched_instances(64, 0), key=lambda x: x[0])[:4]
    T = 6
    res = batch.solve_batch(inst, iters=T, nthreads=4)
    assert len(res) == 4
    for r in res:
        assert r["status"] == hk.HK_OK
        m = inputs.moments(r["N"], r["beta"], r["P"])
        lam_o, hist_o, _ = oracle.smallest_eigenvalue(m, r["N"], r["P"], T, workers=8)
        assert r["lam"] == lam_o, (r["N"], r["beta"], r["P"])
