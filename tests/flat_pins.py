"""Closed forms for 1/|x - y| integrals over coplanar axis-aligned rectangles.

Test helper for pinning the oracle's element-pair rules; it shares nothing with
the oracle's code.  Two independent routes:

* ``pair_integral``: int_X int_Y 1/|x-y| dy dx by second differences of a fourth
  antiderivative F with d^2/du^2 d^2/dv^2 F = 1/sqrt(u^2+v^2), extended evenly
  in u and v (F_u(0, v) = F_v(u, 0) = 0, so the even extension stays C^1):
  F(u,v) = u^2 v/2 asinh(v/u) + u v^2/2 asinh(u/v) - (u^2+v^2)^{3/2}/6.
* ``weighted_pair_integral``: int_X w(x) Phi_Y(x) dx, with the rectangle
  potential Phi_Y(x) = int_Y 1/|x-y| dy from the corner formula
  Q(a,b) = int_0^a int_0^b 1/sqrt(u^2+v^2) = a asinh(b/a) + b asinh(a/b),
  and a tensor Gauss rule geometrically graded towards the given end points.
"""
import numpy as np


def _xasinh(a, b):
    # a * asinh(b / a) with the limit 0 at a = 0
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    out = np.zeros(np.broadcast(a, b).shape)
    m = a != 0
    out[m] = (a * np.arcsinh(b / np.where(m, a, 1.0)))[m]
    return out


def F4(u, v):
    u, v = np.abs(u), np.abs(v)
    return 0.5 * u * _xasinh(u, v) * v + 0.5 * v * _xasinh(v, u) * u - (u * u + v * v) ** 1.5 / 6.0


def pair_integral(X, Y):
    """int over rectangle X = ((a1,a2),(b1,b2)) and Y = ((c1,c2),(d1,d2)) of 1/|x-y|."""
    (a, b), (c, d) = X, Y
    tot = 0.0
    for i, ai in enumerate(a):
        for k, ck in enumerate(c):
            s1 = (1 if i == 1 else -1) * (1 if k == 1 else -1)
            for j, bj in enumerate(b):
                for l, dl in enumerate(d):
                    s2 = (1 if j == 1 else -1) * (1 if l == 1 else -1)
                    tot += s1 * s2 * F4(ck - ai, dl - bj)
    return float(tot)


def Q2(a, b):
    return _xasinh(a, b) + _xasinh(b, a)


def potential(x, Y):
    """Phi_Y(x) = int_Y 1/|x-y| dy for points x (n, 2) in the plane of Y."""
    (c, d) = Y
    x = np.atleast_2d(x)
    tot = np.zeros(len(x))
    for k, ck in enumerate(c):
        for l, dl in enumerate(d):
            eps = (1 if k == 1 else -1) * (1 if l == 1 else -1)
            du, dv = ck - x[:, 0], dl - x[:, 1]
            tot += eps * np.sign(du) * np.sign(dv) * Q2(np.abs(du), np.abs(dv))
    return tot


def graded_rule(lo, hi, ends, g=14, sigma=0.12, nlev=22):
    """1-D composite Gauss on [lo, hi], geometrically graded towards the listed ends."""
    xg, wg = np.polynomial.legendre.leggauss(g)
    xg, wg = 0.5 * (xg + 1), 0.5 * wg
    L = hi - lo
    # breakpoints in [0,1] graded at 0 and/or 1
    bp = {0.0, 1.0}
    for side in ends:
        for k in range(1, nlev + 1):
            t = sigma**k * (0.5 if len(ends) == 2 else 1.0)
            bp.add(t if side == lo else 1.0 - t)
    if len(ends) == 2:
        bp.add(0.5)
    bp = np.array(sorted(bp))
    pts, wts = [], []
    for u, v in zip(bp[:-1], bp[1:]):
        pts.append(lo + L * (u + (v - u) * xg))
        wts.append(L * (v - u) * wg)
    return np.concatenate(pts), np.concatenate(wts)


def weighted_pair_integral(X, Y, w, ends1, ends2):
    """int_X w(x) Phi_Y(x) dx with a tensor rule graded towards ends1 (x1) and ends2 (x2)."""
    (a, b) = X
    p1, w1 = graded_rule(a[0], a[1], ends1)
    p2, w2 = graded_rule(b[0], b[1], ends2)
    P1, P2 = np.meshgrid(p1, p2, indexing="ij")
    W = np.outer(w1, w2)
    pts = np.stack([P1.ravel(), P2.ravel()], 1)
    return float(np.sum(W.ravel() * w(pts) * potential(pts, Y)))
