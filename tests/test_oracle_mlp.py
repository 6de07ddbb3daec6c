"""Pins of the float64 predictor-network reference (oracle/mlp.py) against
facts fixed outside it: finite differences, values of the normal
distribution, the published Adam update, and degenerate networks."""
import math

import numpy as np
import pytest

from oracle import mlp


def _rand(seed=0, B=37):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0, 0.4, mlp.NPARAMS)
    X = rng.normal(0, 1.0, (B, 2))
    T = rng.normal(0, 1.0, (B, 3))
    return theta, X, T


def test_layout():
    assert mlp.NPARAMS == 64 * 2 + 64 + 64 * 64 + 64 + 3 * 64 + 3 == 4547
    p = mlp.unpack(np.arange(mlp.NPARAMS, dtype=float))
    assert p["W1"][1, 0] == 2 and p["b1"][0] == 128 and p["W2"][0, 1] == 193
    assert p["b3"][2] == mlp.NPARAMS - 1


def test_gelu_values():
    z = np.array([-30.0, -2.0, -1.0, 0.0, 0.5, 1.0, 3.0, 30.0])
    g = mlp.gelu(z)
    assert g[3] == 0.0
    assert g[0] == pytest.approx(0.0, abs=1e-150) and g[-1] == 30.0
    # Phi(1) = 0.841344746068543 (standard normal table)
    assert g[5] == pytest.approx(0.841344746068543, rel=1e-14)
    # odd-part identity of z Phi(z): gelu(z) - gelu(-z) = z
    for x in (0.3, 1.7, 4.2):
        assert mlp.gelu(np.array([x]))[0] - mlp.gelu(np.array([-x]))[0] == pytest.approx(x, rel=1e-14)
    # derivative against central differences
    for x in (-2.5, -0.4, 0.0, 0.9, 2.2):
        h = 1e-6
        fd = (mlp.gelu(np.array([x + h]))[0] - mlp.gelu(np.array([x - h]))[0]) / (2 * h)
        assert mlp.gelu_grad(np.array([x]))[0] == pytest.approx(fd, rel=1e-8, abs=1e-10)


def test_gradient_against_finite_differences():
    theta, X, T = _rand(1)
    w = (1.0, 0.5, 2.0)
    L, g = mlp.loss_grad(theta, X, T, w)
    assert L == pytest.approx(mlp.loss(theta, X, T, w), rel=1e-15)
    rng = np.random.default_rng(7)
    # every block: W1, b1, W2, b2, W3, b3
    idx = list(rng.choice(128, 8, replace=False)) + list(128 + rng.choice(64, 6, replace=False)) + \
        list(192 + rng.choice(4096, 16, replace=False)) + list(4288 + rng.choice(64, 6, replace=False)) + \
        list(4352 + rng.choice(192, 8, replace=False)) + [4544, 4545, 4546]
    fd = mlp.finite_difference_grad(theta, X, T, w, idx=idx)
    np.testing.assert_allclose(g[idx], fd, rtol=1e-5, atol=2e-8)


def test_planted_backprop_mistake_is_caught():
    """A dropped GELU derivative in the first layer fails the finite-difference pin."""
    theta, X, T = _rand(2)
    _, g = mlp.loss_grad(theta, X, T)
    p = mlp.unpack(theta)
    Y, (Xc, Z1, H1, Z2, H2) = mlp.forward(theta, X)
    dY = 2.0 * (Y - T) / len(Y)
    dZ2 = (dY @ p["W3"]) * mlp.gelu_grad(Z2)
    wrong_dW1 = ((dZ2 @ p["W2"]).T @ Xc).ravel()  # missing gelu'(Z1)
    fd = mlp.finite_difference_grad(theta, X, T, idx=range(8))
    np.testing.assert_allclose(g[:8], fd, rtol=1e-5, atol=2e-8)
    assert not np.allclose(wrong_dW1[:8], fd, rtol=1e-3)


def test_degenerate_network_outputs_bias():
    theta = np.zeros(mlp.NPARAMS)
    theta[-3:] = [1.5, -2.0, 0.25]
    theta[:128] = 3.0  # W1 nonzero but W2 = W3 = 0
    Y, _ = mlp.forward(theta, np.array([[0.2, -1.0], [5.0, 7.0]]))
    np.testing.assert_array_equal(Y, [[1.5, -2.0, 0.25]] * 2)
    # gradient of the loss in b3 alone: 2 (b3 - T) mean
    T = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    _, g = mlp.loss_grad(theta, np.array([[0.2, -1.0], [5.0, 7.0]]), T)
    np.testing.assert_allclose(g[-3:], [2 * (1.5 - 0.5), 2 * (-2.0), 2 * (0.25 - 0.5)])
    assert not g[:4352].any()  # no signal reaches the layers behind W3 = 0


def test_single_hidden_unit_closed_form():
    """One active path x0 -> unit 0 -> unit 0 -> output 0 with unit weights:
    y = gelu(gelu(x0))."""
    theta = np.zeros(mlp.NPARAMS)
    p = mlp.unpack(theta)
    p["W1"][0, 0] = 1.0
    p["W2"][0, 0] = 1.0
    p["W3"][0, 0] = 1.0
    for x in (-1.3, 0.0, 0.7, 2.0):
        Phi = lambda u: 0.5 * (1 + math.erf(u / math.sqrt(2)))
        g1 = x * Phi(x)
        want = g1 * Phi(g1)
        Y, _ = mlp.forward(theta, np.array([[x, 9.0]]))
        assert Y[0, 0] == pytest.approx(want, rel=1e-14, abs=1e-300)
        assert Y[0, 1] == 0.0 and Y[0, 2] == 0.0


def test_adam_first_steps():
    """Adam's first step moves every parameter by lr * sign(g) (bias
    corrections make mhat = g and vhat = g^2), up to eps."""
    theta = np.array([1.0, -2.0, 0.5, 0.0])
    g = np.array([0.3, -4.0, 1e-3, 0.0])
    t1, m, v = mlp.adam_step(theta, g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    np.testing.assert_allclose(t1[:3], theta[:3] - 0.01 * np.sign(g[:3]), rtol=1e-6)
    assert t1[3] == 0.0
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)
    # second step with the same gradient: again lr * sign(g)
    t2, m2, v2 = mlp.adam_step(t1, g, m, v, 2, lr=0.01)
    np.testing.assert_allclose(t2[:3], theta[:3] - 0.02 * np.sign(g[:3]), rtol=1e-6)


def test_adam_descends_quadratic():
    theta = np.array([3.0, -1.0])
    m = np.zeros(2)
    v = np.zeros(2)
    for t in range(1, 2001):
        theta, m, v = mlp.adam_step(theta, 2 * theta, m, v, t, lr=0.05)
    assert np.abs(theta).max() < 1e-3
