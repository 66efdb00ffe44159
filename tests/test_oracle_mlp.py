"""Pins for the oracle MLP of the learned preconditioner: its hand-written
backward pass against central finite differences and against torch autograd."""
import numpy as np
import torch

from oracle import mlp


def _setup(seed=0, n=50):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(mlp.NPARAM) * 0.3
    X = rng.standard_normal((n, mlp.NIN))
    gw = rng.standard_normal(n)
    return p, X, gw


def test_backward_finite_differences():
    p, X, gw = _setup()
    g = mlp.backward(p, X, gw)
    f = lambda q: float(np.sum(gw * mlp.forward(q, X)))  # noqa: E731
    eps = 1e-6
    for i in list(range(0, mlp.NPARAM, 17)) + [mlp.NPARAM - 1]:
        e = np.zeros_like(p)
        e[i] = eps
        fd = (f(p + e) - f(p - e)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd))


def test_backward_matches_autograd():
    p, X, gw = _setup(1)
    pt = torch.tensor(p, requires_grad=True)
    Xt = torch.tensor(X)
    o = 0
    W1 = pt[o : o + 128].reshape(16, 8); o += 128
    b1 = pt[o : o + 16]; o += 16
    W2 = pt[o : o + 256].reshape(16, 16); o += 256
    b2 = pt[o : o + 16]; o += 16
    w3 = pt[o : o + 16]; o += 16
    b3 = pt[o]
    w = torch.exp(torch.tanh(torch.tanh(Xt @ W1.T + b1) @ W2.T + b2) @ w3 + b3)
    np.testing.assert_allclose(w.detach().numpy(), mlp.forward(p, X), rtol=1e-12)
    (w * torch.tensor(gw)).sum().backward()
    np.testing.assert_allclose(pt.grad.numpy(), mlp.backward(p, X, gw), rtol=1e-10, atol=1e-12)
