"""B-spline basis by the recursion of App. C (test infrastructure).

Readings where App. C is silent:
* 0/0 := 0 in the recursion (repeated knots).
* The right end point x = 1 belongs to the last non-empty knot interval, so the
  basis is a partition of unity on the closed interval [0,1].
"""
from __future__ import annotations

import numpy as np


def open_knots(degree: int, n_el: int, repetition: int = 1) -> np.ndarray:
    """Open knot vector on [0,1] with n_el equal elements (App. E, equidistant knots).

    End knots appear degree+1 times, interior knots ``repetition`` times.
    """
    interior = np.repeat(np.arange(1, n_el) / n_el, repetition)
    return np.concatenate([np.zeros(degree + 1), interior, np.ones(degree + 1)])


def bspline_basis(knots: np.ndarray, degree: int, x: np.ndarray) -> np.ndarray:
    """Values b_j^degree(x) for all j, shape (len(x), len(knots)-degree-1).

    Degree 0: indicator of [xi_j, xi_{j+1}); higher degrees by the two-term
    recursion of App. C with the 0/0 := 0 convention.
    """
    x = np.atleast_1d(np.asarray(x, dtype=float))
    knots = np.asarray(knots, dtype=float)
    m = len(knots)
    # degree 0
    b = np.zeros((x.size, m - 1))
    for j in range(m - 1):
        if knots[j] < knots[j + 1]:
            b[:, j] = (x >= knots[j]) & (x < knots[j + 1])
    # x == last knot goes to the last non-empty interval
    last = max(j for j in range(m - 1) if knots[j] < knots[j + 1])
    b[x >= knots[-1], :] = 0.0
    b[x >= knots[-1], last] = 1.0
    for p in range(1, degree + 1):
        nb = np.zeros((x.size, m - 1 - p))
        for j in range(m - 1 - p):
            d1 = knots[j + p] - knots[j]
            d2 = knots[j + p + 1] - knots[j + 1]
            t1 = (x - knots[j]) / d1 * b[:, j] if d1 > 0 else 0.0
            t2 = (knots[j + p + 1] - x) / d2 * b[:, j + 1] if d2 > 0 else 0.0
            nb[:, j] = t1 + t2
        b = nb
    return b


def bspline_deriv(knots: np.ndarray, degree: int, x: np.ndarray) -> np.ndarray:
    """Derivatives d/dx b_j^degree(x) for all j, shape (len(x), len(knots)-degree-1).

    Differentiating the App. C recursion gives the standard two-term formula
    b'_{j,p} = p b_{j,p-1} / (xi_{j+p} - xi_j) - p b_{j+1,p-1} / (xi_{j+p+1} - xi_{j+1})
    on the same knot vector, with 0/0 := 0.
    """
    x = np.atleast_1d(np.asarray(x, dtype=float))
    knots = np.asarray(knots, dtype=float)
    n = len(knots) - degree - 1
    if degree == 0:
        return np.zeros((x.size, n))
    low = bspline_basis(knots, degree - 1, x)  # (len(x), n + 1)
    out = np.zeros((x.size, n))
    for j in range(n):
        d1 = knots[j + degree] - knots[j]
        d2 = knots[j + degree + 1] - knots[j + 1]
        if d1 > 0:
            out[:, j] += degree * low[:, j] / d1
        if d2 > 0:
            out[:, j] -= degree * low[:, j + 1] / d2
    return out
