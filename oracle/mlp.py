"""Float64 reference of the precision predictor's network: a 2 -> 64 -> 64 -> 3
multilayer perceptron with exact (erf) GELU activations, its weighted
mean-squared-error loss, the loss gradient by back-propagation, and one Adam
step.

TEST INFRASTRUCTURE ONLY (see the package docstring).  The paper has no
learned component; this network is the predictor that picks the working
precision P and the iteration budget.  What pins this file (tests in
``tests/test_oracle_mlp.py``): central finite differences of the loss in every
parameter block (independent of the back-propagation written here), GELU at
values fixed by the normal distribution (gelu(0) = 0, gelu(x) - gelu(-x) = x,
gelu(x) -> x and -> 0 in the tails, and the closed-form Phi(1)), the Adam step
against its published definition (Kingma and Ba, "Adam", Algorithm 1) with
hand-computed first-step values, and a network whose hidden weights vanish
(output equal to b3).

Parameter layout (float32 on the device, float64 here), one flat vector:
``W1[64][2], b1[64], W2[64][64], b2[64], W3[3][64], b3[3]`` (row-major,
``W[out][in]``), 4547 values.  The loss of a batch of B samples with targets
T and per-output weights w is ``(1/B) sum_b sum_k w_k (y_bk - T_bk)^2``.
"""
import math

import numpy as np

H = 64
NIN = 2
NOUT = 3
SHAPES = [("W1", (H, NIN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (NOUT, H)), ("b3", (NOUT,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    """Flat parameter vector -> dict of float64 arrays (views)."""
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = theta[o:o + n].reshape(shape)
        o += n
    return out


def _erf(x):
    return np.vectorize(math.erf, otypes=[np.float64])(x)


def gelu(z):
    """z * Phi(z), Phi the standard normal distribution function."""
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    """d/dz [z Phi(z)] = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(theta, X):
    """Network outputs for inputs X (B x 2); returns (Y, cache)."""
    p = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    Z1 = X @ p["W1"].T + p["b1"]
    H1 = gelu(Z1)
    Z2 = H1 @ p["W2"].T + p["b2"]
    H2 = gelu(Z2)
    Y = H2 @ p["W3"].T + p["b3"]
    return Y, (X, Z1, H1, Z2, H2)


def loss(theta, X, T, w=(1.0, 1.0, 1.0)):
    Y, _ = forward(theta, X)
    w = np.asarray(w, dtype=np.float64)
    return float(np.sum(w * (Y - np.asarray(T, dtype=np.float64)) ** 2) / len(Y))


def loss_grad(theta, X, T, w=(1.0, 1.0, 1.0)):
    """(loss, gradient) by back-propagation through the three layers."""
    p = unpack(theta)
    Y, (X, Z1, H1, Z2, H2) = forward(theta, X)
    w = np.asarray(w, dtype=np.float64)
    B = len(Y)
    R = Y - np.asarray(T, dtype=np.float64)
    L = float(np.sum(w * R * R) / B)
    dY = 2.0 * w * R / B
    g = {"W3": dY.T @ H2, "b3": dY.sum(0)}
    dZ2 = (dY @ p["W3"]) * gelu_grad(Z2)
    g["W2"] = dZ2.T @ H1
    g["b2"] = dZ2.sum(0)
    dZ1 = (dZ2 @ p["W2"]) * gelu_grad(Z1)
    g["W1"] = dZ1.T @ X
    g["b1"] = dZ1.sum(0)
    return L, np.concatenate([g[name].ravel() for name, _ in SHAPES])


def adam_step(theta, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step t >= 1): new (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def finite_difference_grad(theta, X, T, w=(1.0, 1.0, 1.0), h=1e-6, idx=None):
    """Central differences of ``loss`` in the listed parameter indices."""
    theta = np.array(theta, dtype=np.float64)
    idx = range(len(theta)) if idx is None else idx
    out = []
    for i in idx:
        tp = theta.copy()
        tm = theta.copy()
        tp[i] += h
        tm[i] -= h
        out.append((loss(tp, X, T, w) - loss(tm, X, T, w)) / (2 * h))
    return np.array(out)
