"""The predictor network's CUDA kernels (forward, back-propagation, Adam)
against the float64 reference in oracle/mlp.py, through the C ABI."""
import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_0902_0852_gb300 import build, hk
    build.build()
    hk.lib()
    return torch, hk


def _case(seed, B):
    rng = np.random.default_rng(seed)
    theta = (rng.normal(0, 1.0, mlp.NPARAMS) * np.concatenate([
        np.full(128, 0.7), np.full(64, 0.3), np.full(4096, 1 / 8), np.full(64, 0.3), np.full(192, 1 / 8),
        np.full(3, 0.5)])).astype(np.float32)
    X = rng.normal(0, 1.0, (B, 2)).astype(np.float32)
    T = rng.normal(0, 1.0, (B, 3)).astype(np.float32)
    return theta, X, T


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("B", [1, 63, 64, 1000, 4096])
def test_forward_matches_float64(env, B):
    torch, hk = env
    theta, X, _ = _case(B, B)
    y = torch.zeros(B, 3, dtype=torch.float32, device="cuda")
    hk.hk_mlp_forward(_dev(torch, theta), _dev(torch, X), y)
    torch.cuda.synchronize()
    want, _ = mlp.forward(theta.astype(np.float64), X.astype(np.float64))
    np.testing.assert_allclose(y.cpu().numpy(), want, rtol=1e-5, atol=1e-5 * np.abs(want).max())


@pytest.mark.parametrize("B", [5, 64, 1000, 4096])
def test_loss_gradient_matches_float64(env, B):
    torch, hk = env
    theta, X, T = _case(100 + B, B)
    w = np.array([1.0, 0.5, 2.0], dtype=np.float32)
    grad = torch.zeros(hk.HK_MLP_NPARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    work = torch.empty(hk.hk_mlp_workspace_bytes(B), dtype=torch.uint8, device="cuda")
    args = (_dev(torch, theta), _dev(torch, X), _dev(torch, T), _dev(torch, w))
    hk.hk_mlp_loss_grad(*args, grad, loss, work)
    torch.cuda.synchronize()
    L, g = mlp.loss_grad(theta.astype(np.float64), X.astype(np.float64), T.astype(np.float64), w.astype(np.float64))
    assert loss.item() == pytest.approx(L, rel=1e-5)
    gg = grad.cpu().numpy()
    o = 0
    for name, shape in mlp.SHAPES:
        n = int(np.prod(shape))
        scale = np.abs(g[o:o + n]).max()
        np.testing.assert_allclose(gg[o:o + n], g[o:o + n], rtol=1e-4, atol=1e-4 * scale, err_msg=name)
        o += n
    # fixed summation order: a second call is bit-identical
    grad2 = torch.zeros_like(grad)
    hk.hk_mlp_loss_grad(*args, grad2, loss, work)
    assert torch.equal(grad, grad2)


def test_adam_matches_reference(env):
    torch, hk = env
    rng = np.random.default_rng(5)
    n = hk.HK_MLP_NPARAMS
    p = rng.normal(0, 1, n).astype(np.float32)
    g = rng.normal(0, 1e-2, n).astype(np.float32)
    m = rng.normal(0, 1e-3, n).astype(np.float32)
    v = np.abs(rng.normal(0, 1e-4, n)).astype(np.float32)
    P, G, Mm, V = (_dev(torch, a) for a in (p, g, m, v))
    hk.hk_mlp_adam(P, G, Mm, V, step=7, lr=3e-3)
    torch.cuda.synchronize()
    # the device takes its hyperparameters as float32: give the reference the
    # same values (1 - beta is then exact in float32 as well)
    f = lambda x: float(np.float32(x))  # noqa: E731
    pw, mw, vw = mlp.adam_step(p.astype(np.float64), g.astype(np.float64), m.astype(np.float64),
                               v.astype(np.float64), 7, f(3e-3), f(0.9), f(0.999), f(1e-8))
    # float32 rounding of b1 m + (1 - b1) g is relative to the operands, not
    # to the (possibly cancelling) sum
    scale_m = 0.9 * np.abs(m.astype(np.float64)) + 0.1 * np.abs(g.astype(np.float64))
    assert np.all(np.abs(Mm.cpu().numpy() - mw) <= 4 * 2.0 ** -24 * scale_m + 1e-30)
    np.testing.assert_allclose(V.cpu().numpy(), vw, rtol=1e-6, atol=1e-14)
    np.testing.assert_allclose(P.cpu().numpy(), pw, rtol=0, atol=1e-6)


def test_training_reduces_loss(env):
    """Full-batch Adam on the device fits a smooth map of two inputs."""
    torch, hk = env
    rng = np.random.default_rng(11)
    B = 2000
    X = rng.uniform(-1, 1, (B, 2)).astype(np.float32)
    T = np.stack([np.sin(2 * X[:, 0]) + X[:, 1], X[:, 0] * X[:, 1], np.exp(0.5 * X[:, 1])], 1).astype(np.float32)
    theta, _, _ = _case(3, 1)
    P = _dev(torch, theta)
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    grad = torch.zeros_like(P)
    w = _dev(torch, np.ones(3, dtype=np.float32))
    work = torch.empty(hk.hk_mlp_workspace_bytes(B), dtype=torch.uint8, device="cuda")
    hist = torch.zeros(1500, dtype=torch.float32, device="cuda")
    hk.hk_mlp_train(P, m, v, grad, _dev(torch, X), _dev(torch, T), w, 1500, 0, 3e-3, work, hist)
    torch.cuda.synchronize()
    h = hist.cpu().numpy()
    assert np.all(np.isfinite(h))
    assert h[-1] < h[0] / 50
    # the recorded loss is the loss of the parameters at that step
    L_last = mlp.loss(P.cpu().numpy().astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    assert L_last <= h[-1] * 1.05
