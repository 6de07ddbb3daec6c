"""The committed predictor artefacts (paper_0902_0852_gb300/data/) are
consistent with what they claim, checked on the CPU:

* each training tuple's required precision is the smallest probed P whose
  lambda agrees with the P + 1024 reference to 2^-128, and lies below the
  conservative rule;
* the committed network, evaluated by the float64 CPU network of oracle/mlp.py
  with the committed scalings, puts no training instance below its required
  precision once the margin is added (the margin is fitted for exactly that);
* the held-out evaluation's rows are all verified at less than the
  conservative precision and its summary equals the sums over its rows."""
import json
import math
import os

import numpy as np

from oracle import mlp
from paper_0902_0852_gb300 import predictor as pr

DATA = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_0902_0852_gb300", "data")


def _load(name):
    with open(os.path.join(DATA, name)) as f:
        return json.load(f)


def test_training_tuples_hold_the_smallest_agreeing_precision():
    d = _load("predictor_tuples.json")
    grid = set(pr.beta_grid())
    rows = [t for t in d["tuples"] if t.get("ok")]
    assert len(rows) >= 0.9 * len(d["tuples"])
    for t in rows:
        N, beta = t["N"], tuple(t["beta"])
        assert 32 <= N <= 512 and beta in grid
        assert t["P_cons"] == pr.p_conservative(N, beta) and t["P_ref"] == t["P_cons"] + 1024
        assert t["bits"] % 32 == 0 and t["bits"] <= t["P_cons"]
        agree = {P: (ok and a is not None and a >= pr.AGREE_BITS) for P, _, a, _, ok in t["probes"]}
        assert agree.get(t["bits"]) is True, t
        assert not any(ok for P, ok in agree.items() if P < t["bits"]), t


def test_committed_network_covers_every_training_instance():
    m = _load("predictor.json")
    rows = [t for t in _load("predictor_tuples.json")["tuples"] if t.get("ok")]
    theta = np.asarray(m["params"], dtype=np.float64)
    X = (np.asarray([pr.features(t["N"], tuple(t["beta"])) for t in rows]) - np.asarray(m["x_mean"])) \
        / np.asarray(m["x_std"])
    Y, _ = mlp.forward(theta, X)
    Y = Y * np.asarray(m["y_std"]) + np.asarray(m["y_mean"])
    for t, y in zip(rows, Y):
        bits, _, _ = pr.decode_targets(t["N"], y)
        P = max(pr.P_MIN, 32 * math.ceil((bits + m["margin_bits"] + m["margin_per_row"] * t["N"]) / 32))
        assert P >= t["bits"], (t["N"], t["beta"], P, t["bits"])


def test_heldout_evaluation_rows_and_summary_agree():
    e = _load("predictor_eval.json")
    rows, s = e["rows"], e["summary"]
    assert s["instances"] == len(rows) == 256
    both = [r for r in rows if "cons_seconds" in r]
    assert s["conservative_checked"] == len(both) >= len(rows) // 4
    for r in rows:
        assert 513 <= r["N"] <= 800
        P_cons = pr.p_conservative(r["N"], tuple(r["beta"]))
        assert r["verified"]
        assert r["tried"][0] == r["P_pred"] and r["P_pred"] < P_cons
    for r in both:
        assert r["P_cons"] == pr.p_conservative(r["N"], tuple(r["beta"]))
        assert r["agree_bits"] >= pr.AGREE_BITS  # verified value = conservative value to 2^-128
    assert s["all_verified"] == all(r["verified"] for r in rows)
    assert abs(s["conservative_seconds"] - sum(r["cons_seconds"] for r in both)) < 1e-2
    assert abs(s["predicted_seconds_same_instances"] - sum(r["pred_seconds"] for r in both)) < 1e-2
    assert abs(s["predicted_seconds_all"] - sum(r["pred_seconds"] for r in rows)) < 1e-2
    assert abs(s["gain"] - s["conservative_seconds"] / s["predicted_seconds_same_instances"]) < 1e-3
    assert s["escalated"] == sum(1 for r in rows if len(r["tried"]) > 2)
    assert abs(s["min_agree_bits"] - min(r["agree_bits"] for r in both)) < 1e-6


def test_training_set_size():
    """4096 training instances (seed 1), at least 90% of them with a tuple."""
    d = _load("predictor_tuples.json")
    assert d["meta"]["count"] == 4096 and len(d["tuples"]) == 4096
