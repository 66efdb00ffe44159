"""Gauss-Legendre rules on [0,1] (test infrastructure; see package docstring).

The paper states no quadrature orders; the rules here are the textbook n-point
Gauss-Legendre rules, computed by Newton's method on the Legendre polynomial
P_n evaluated with its three-term recurrence.
"""
from __future__ import annotations

import functools

import numpy as np


@functools.lru_cache(maxsize=None)
def gauss_legendre01(n: int) -> tuple[np.ndarray, np.ndarray]:
    """n-point Gauss-Legendre nodes (ascending) and weights on [0,1]."""
    if n < 1:
        raise ValueError("n >= 1")
    i = np.arange(n, dtype=float)
    x = np.cos(np.pi * (i + 0.75) / (n + 0.5))  # initial guesses for the roots of P_n on [-1,1]
    for _ in range(100):
        p_prev = np.ones_like(x)
        p = x.copy()
        for k in range(2, n + 1):
            p_prev, p = p, ((2 * k - 1) * x * p - (k - 1) * p_prev) / k
        if n == 1:
            p_prev, p = np.ones_like(x), x.copy()
        dp = n * (x * p - p_prev) / (x * x - 1.0)
        dx = p / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    # recompute derivative at the converged roots for the weights
    p_prev = np.ones_like(x)
    p = x.copy()
    for k in range(2, n + 1):
        p_prev, p = p, ((2 * k - 1) * x * p - (k - 1) * p_prev) / k
    if n == 1:
        p_prev, p = np.ones_like(x), x.copy()
    dp = n * (x * p - p_prev) / (x * x - 1.0)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    t = 0.5 * (1.0 - x)  # x descending -> t ascending
    order = np.argsort(t)
    return t[order].copy(), 0.5 * w[order].copy()


def tensor2(n: int) -> tuple[np.ndarray, np.ndarray]:
    """n x n tensor Gauss rule on the unit square: points (n*n, 2), weights (n*n,).

    Point index is a1 + n*a2 with a1 along the first parameter.
    """
    t, w = gauss_legendre01(n)
    s1, s2 = np.meshgrid(t, t, indexing="xy")
    w1, w2 = np.meshgrid(w, w, indexing="xy")
    pts = np.stack([s1.ravel(), s2.ravel()], axis=1)
    return pts, (w1 * w2).ravel()
