"""Plain numpy MLP of the learned preconditioner (test infrastructure).

Network (per element-local dof, FP64 here): features x (8) ->
  h1 = tanh(W1 x + b1) (16) -> h2 = tanh(W2 h1 + b2) (16) -> o = w3 . h2 + b3
  weight = exp(o).
Parameters are packed [W1 (16x8 row-major), b1, W2 (16x16), b2, w3 (16), b3],
433 values.  ``forward`` returns the weights; ``backward`` returns the gradient
of sum_i gw_i * weight_i with respect to the packed parameters.
"""
from __future__ import annotations

import numpy as np

NIN, NH = 8, 16
NPARAM = NH * NIN + NH + NH * NH + NH + NH + 1


def unpack(p):
    p = np.asarray(p, dtype=float)
    o = 0
    W1 = p[o : o + NH * NIN].reshape(NH, NIN)
    o += NH * NIN
    b1 = p[o : o + NH]
    o += NH
    W2 = p[o : o + NH * NH].reshape(NH, NH)
    o += NH * NH
    b2 = p[o : o + NH]
    o += NH
    w3 = p[o : o + NH]
    o += NH
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def forward(p, X):
    W1, b1, W2, b2, w3, b3 = unpack(p)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return np.exp(h2 @ w3 + b3)


def backward(p, X, gw):
    """d/dp of sum_i gw_i * forward(p, X)_i (chain rule written out layer by layer)."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    wgt = np.exp(h2 @ w3 + b3)
    go = gw * wgt  # d/do of the weight exp(o)
    g_w3 = h2.T @ go
    g_b3 = go.sum()
    gz2 = np.outer(go, w3) * (1 - h2**2)
    g_W2 = gz2.T @ h1
    g_b2 = gz2.sum(0)
    gz1 = (gz2 @ W2) * (1 - h1**2)
    g_W1 = gz1.T @ X
    g_b1 = gz1.sum(0)
    return np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
