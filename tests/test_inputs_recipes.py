"""The seeded instance recipes (CPU): the batched sweep's instances follow
their stated rule exactly (N and beta drawn from numpy's default_rng(0), P from
log2((2N-2)!) + 4 sqrt(N) + 256 rounded up to a multiple of 32, the factorial
taken exactly), and the predictor's samples stay in their stated ranges."""
import math

import numpy as np

from paper_0902_0852_gb300 import inputs
from paper_0902_0852_gb300 import predictor as pr


def test_batched_sweep_instances_follow_the_rule():
    inst = inputs.batched_instances(64, 0)
    rng = np.random.default_rng(0)
    Ns = rng.integers(100, 601, 64)
    bs = rng.integers(0, 5, 64)
    betas = [(3, 4), (1, 1), (3, 2), (2, 1), (3, 1)]
    assert len(inst) == 64
    for (N, beta, P), n, b in zip(inst, Ns, bs):
        assert N == int(n) and beta == betas[int(b)]
        exact_bits = math.log2(math.factorial(2 * N - 2))  # exact integer, one float conversion
        assert P == 32 * math.ceil((exact_bits + 4 * math.sqrt(N) + 256) / 32)
    Ps = [P for _, _, P in inst]
    assert 1536 <= min(Ps) and max(Ps) <= 10912


def test_predictor_samples_stay_in_range():
    grid = set(pr.beta_grid())
    for seed, lo, hi in ((1, 32, 512), (2, 513, 800)):
        s = pr.sample_instances(200, seed, lo, hi)
        assert len(s) == 200
        assert all(lo <= N <= hi and beta in grid for N, beta in s)
        assert s == pr.sample_instances(200, seed, lo, hi)  # seeded: reproducible
