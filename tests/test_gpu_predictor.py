"""The precision predictor end to end on the device: training by the
library's FP32 kernels on the committed method-generated tuples, predictions
verified by the P vs P + 1024 rerun, escalation from an under-provisioned
prediction, and the gain over the method at its conservative precision on
held-out instances (N in [513, 800], outside the training range)."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

DATA = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_0902_0852_gb300", "data")


@pytest.fixture(scope="module")
def pr():
    from paper_0902_0852_gb300 import build, predictor
    build.build()
    return predictor


def test_device_training_deterministic_and_fits(pr):
    tuples = json.load(open(os.path.join(DATA, "predictor_tuples.json")))["tuples"]
    a, b = pr.Predictor(), pr.Predictor()
    ha = a.fit(tuples, steps=900)
    hb = b.fit(tuples, steps=900)
    assert np.array_equal(a.params.cpu().numpy(), b.params.cpu().numpy())
    assert np.array_equal(ha, hb)
    assert ha[-1] < ha[0] / 20
    # after the margin, no training instance is under-provisioned
    rows = [t for t in tuples if t.get("ok")]
    for t in rows[:64]:
        P, T, _ = a.predict(t["N"], tuple(t["beta"]))
        assert P >= t["bits"] or P == pr.p_conservative(t["N"], tuple(t["beta"]))


def test_heldout_prediction_verified_and_cheaper(pr):
    """The held-out instance (N in [513, 800], seed 2) with the largest
    conservative precision: the predicted solve is verified, agrees with the
    conservative solve to 2^-128, and costs less device time and fewer limb
    products (N^3 P^2 summed over the solves it ran)."""
    model = pr.load_default()
    held = pr.sample_instances(64, 2, 513, 800)
    N, beta = max(held, key=lambda x: pr.p_conservative(*x))
    c = pr.solve_conservative(N, beta)
    v = pr.solve_verified(N, beta, model)
    assert c["converged"] and v["verified"], (N, beta)
    assert pr.rel_err_bits(v["lam"], c["lam"]) >= pr.AGREE_BITS
    assert v["P"] < c["P"]
    assert sum(P * P for P in v["tried"]) < c["P"] ** 2 / 4
    assert v["seconds"] < c["seconds"], (N, beta, v["seconds"], c["seconds"])


def test_escalation_from_underprovisioned_prediction(pr):
    model = pr.load_default()
    model.margin_bits = -10 ** 6  # the prediction collapses to the minimum precision
    N, beta = 100, (3, 4)
    v = pr.solve_verified(N, beta, model)
    c = pr.solve_conservative(N, beta)
    assert v["verified"] and len(v["tried"]) > 2
    assert pr.rel_err_bits(v["lam"], c["lam"]) >= pr.AGREE_BITS


def test_c_abi_predict_matches_wrapper(pr):
    """hk_predict (the network behind the C ABI, with its feature and target
    scalings) gives the same predictions as the Python wrapper."""
    from paper_0902_0852_gb300 import hk
    model = pr.load_default()
    rows = [(40, (7, 4)), (333, (1, 1)), (600, (3, 5)), (1000, (1, 1)), (777, (4, 1))]
    want = model.predict_raw(rows)
    ctx = hk.hk_create(0)
    try:
        hk.hk_set_predictor(ctx, model.params.cpu().numpy(), model.x_mean, model.x_std, model.y_mean, model.y_std)
        got = hk.hk_predict(ctx, [N for N, _ in rows], [b[0] / b[1] for _, b in rows])
    finally:
        hk.hk_destroy(ctx)
    for (b, l2, it), g in zip(want, got):
        assert abs(g[0] - b) <= 1e-3 * abs(b) + 0.5
        assert abs(g[1] - l2) <= 1e-3 * abs(l2) + 0.05
        assert abs(g[2] - it) <= 1e-3 * it
