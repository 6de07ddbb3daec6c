"""Failure detection on the device without a fault: a bounded wait on a barrier
that nothing completes runs out, the kernel records the timeout and returns,
the host reads HK_ERR_TIMEOUT, and the same context then factors and solves
bit-exactly (the status word was cleared, nothing hung)."""
import time

import pytest

import oracle
from paper_0902_0852_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("wait_ns", [1_000_000, 50_000_000])
def test_bounded_wait_runs_out_and_context_stays_usable(wait_ns):
    from paper_0902_0852_gb300 import build, hk
    build.build()
    N, P, T = 12, 256, 6
    m = inputs.moments(N, (7, 4), P)
    with hk.Hankel(0) as h:
        h.load(N, (7, 4), P, m)
        h.set_option(hk.HK_OPT_WAIT_NS, wait_ns)
        t0 = time.perf_counter()
        rc = hk.hk_selftest_wait(h.ctx)
        dt = time.perf_counter() - t0
        assert rc == hk.HK_ERR_TIMEOUT
        # the wait ran for about its limit, not for ever
        assert dt >= wait_ns * 1e-9 * 0.9 and dt < wait_ns * 1e-9 + 5.0, dt
        # the context is still usable: a factorisation and inverse iteration
        # on it equal the oracle bit for bit
        h.factor()
        R = h.R()
        lam, used = h.smallest_eig(T)
        hist = h.history(used)
    Ro = oracle.cholesky(m, N, P)
    lam_o, hist_o, _ = oracle.inverse_iteration(Ro, P, T)
    assert R == Ro
    assert hist == hist_o and lam == lam_o


def test_wait_limit_option_range():
    from paper_0902_0852_gb300 import build, hk
    build.build()
    with hk.Hankel(0) as h:
        assert hk.hk_selftest_wait(h.ctx) == hk.HK_ERR_STATE  # no moments loaded yet
        for bad in (0, 999, 60_000_000_001):
            with pytest.raises(hk.HKError) as ei:
                h.set_option(hk.HK_OPT_WAIT_NS, bad)
            assert ei.value.code == hk.HK_ERR_ARG
