"""Parity at the largest precision the library accepts, P = 32768 bits
(L = 1024 limbs; the diagonal kernel's work area then nearly fills the 227 KB
of shared memory a block may use): R element by element and the inverse-
iteration history bit-exact with the oracle."""
import pytest

import oracle
from paper_0902_0852_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("beta,N,T", [((7, 4), 24, 4), ((1, 1), 20, 3), ((3, 4), 17, 3)])
def test_max_precision_bit_exact(beta, N, T):
    from paper_0902_0852_gb300 import build, hk
    build.build()
    P = 32768
    m = inputs.moments(N, beta, P)
    with hk.Hankel(0) as h:
        h.load(N, beta, P, m)
        h.factor()
        R = h.R()
        lam, used = h.smallest_eig(T)
        hist = h.history(used)
    Ro = oracle.cholesky(m, N, P)
    lam_o, hist_o, _ = oracle.inverse_iteration(Ro, P, T)
    assert R == Ro
    assert hist == hist_o and lam == lam_o


def test_above_max_precision_is_refused():
    from paper_0902_0852_gb300 import build, hk
    build.build()
    P = 32768 + 32
    m = [(1 << (P - 1), 0)] * 3
    with hk.Hankel(0) as h:
        with pytest.raises(hk.HKError) as ei:
            h.load(2, (1, 1), P, m)
        assert ei.value.code == hk.HK_ERR_ARG
