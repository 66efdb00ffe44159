"""Quadrature rules for element pairs on [0,1]^2 x [0,1]^2 (test infrastructure).

Sec. 2 of the paper says the singular Galerkin integrals are computed with the
regularisation techniques of Sauter and Schwab.  The rules below are those
Duffy-type transforms for quadrilaterals, each built from a tensor Gauss rule of
g points per variable on [0,1]^4, in canonical position:

* identical elements: s, t in the same square, singular on the diagonal s = t.
  With z = t - s the integral becomes int_{[-1,1]^2} int_{box(z)} ds dz; each of
  the 4 sign quadrants of z is split into 2 triangles and Duffy-mapped
  (a, b) = (xi, xi eta) or (xi eta, xi), Jacobian xi; s runs over the box
  s_k = max(0, -z_k) + u_k (1 - |z_k|).  8 sub-domains.
* common edge: the shared edge is {s1 = 0} = {t1 = 0} with s2 and t2 the same
  point along it.  With z = t2 - s2, the point singularity of (s1, t1, |z|) at
  the origin is removed by a 3-D Duffy map per pyramid "coordinate c is the
  largest" (3 pyramids, Jacobian xi^2) for each sign of z; s2 = max(0,-z) +
  u (1 - |z|).  6 sub-domains.
* common vertex: the shared vertex is s = t = (0,0); 4-D Duffy map per pyramid
  "coordinate c of (s1, s2, t1, t2) is the largest", Jacobian xi^3.  4 sub-domains.
* separated elements: the g x g tensor Gauss rule on each square.

Each rule returns (S, T, W): points on the first element (n,2), on the second
element (n,2) and weights (n,) so that sum_k W_k f(S_k, T_k) approximates
int_{[0,1]^2} int_{[0,1]^2} f(s, t) ds dt.  The Duffy rules take one Gauss
order g or four per-variable orders, in the order the variables are listed
above: identical (xi, eta, u1, u2), edge (xi, eta1, eta2, u), vertex
(xi, eta1, eta2, eta3).  The transformed integrands are smooth but not equally
so in every variable (the u variables run along the element and need the
fewest points), which the autotuner exploits.
"""
from __future__ import annotations

import functools
import itertools

import numpy as np

from .gauss import gauss_legendre01, tensor2


@functools.lru_cache(maxsize=None)
def rule_regular(g: int):
    p, w = tensor2(g)
    n = len(w)
    S = np.repeat(p, n, axis=0)
    T = np.tile(p, (n, 1))
    W = np.repeat(w, n) * np.tile(w, n)
    return S, T, W


def _orders(g):
    """One Gauss order for all four variables, or a tuple of four (per variable)."""
    gs = (g, g, g, g) if isinstance(g, (int, np.integer)) else tuple(int(v) for v in g)
    if len(gs) != 4:
        raise ValueError("four per-variable orders expected")
    return gs


@functools.lru_cache(maxsize=None)
def grid4(g):
    """Tensor Gauss rule on [0,1]^4; variable v gets order g[v] (or g for all).
    Points (n, 4) in the order of the rules' variables, weights (n,)."""
    rules = [gauss_legendre01(gv) for gv in _orders(g)]
    pts = np.array(list(itertools.product(*[x for x, _ in rules])))
    wts = np.array([np.prod(c) for c in itertools.product(*[w for _, w in rules])])
    return pts, wts


def _grid4(g):
    return grid4(g if isinstance(g, (int, np.integer)) else _orders(g))


@functools.lru_cache(maxsize=None)
def rule_identical(g: int):
    P, Wg = _grid4(g)
    xi, eta, u1, u2 = P.T
    S_all, T_all, W_all = [], [], []
    for sg1 in (1.0, -1.0):
        for sg2 in (1.0, -1.0):
            for tri in (0, 1):
                a = xi if tri == 0 else xi * eta
                b = xi * eta if tri == 0 else xi
                z1, z2 = sg1 * a, sg2 * b
                s1 = np.maximum(0.0, -z1) + u1 * (1.0 - np.abs(z1))
                s2 = np.maximum(0.0, -z2) + u2 * (1.0 - np.abs(z2))
                S_all.append(np.stack([s1, s2], 1))
                T_all.append(np.stack([s1 + z1, s2 + z2], 1))
                W_all.append(Wg * xi * (1.0 - np.abs(z1)) * (1.0 - np.abs(z2)))
    return np.concatenate(S_all), np.concatenate(T_all), np.concatenate(W_all)


@functools.lru_cache(maxsize=None)
def rule_edge(g: int):
    P, Wg = _grid4(g)
    xi, e1, e2, u = P.T
    S_all, T_all, W_all = [], [], []
    for sg in (1.0, -1.0):
        for c in range(3):
            v = [xi * e1, xi * e2]
            v.insert(c, xi)  # coordinate c of (s1, t1, |z|) is the largest
            s1, t1, az = v
            z = sg * az
            s2 = np.maximum(0.0, -z) + u * (1.0 - az)
            S_all.append(np.stack([s1, s2], 1))
            T_all.append(np.stack([t1, s2 + z], 1))
            W_all.append(Wg * xi**2 * (1.0 - az))
    return np.concatenate(S_all), np.concatenate(T_all), np.concatenate(W_all)


@functools.lru_cache(maxsize=None)
def rule_vertex(g: int):
    P, Wg = _grid4(g)
    xi, e1, e2, e3 = P.T
    S_all, T_all, W_all = [], [], []
    for c in range(4):
        v = [xi * e1, xi * e2, xi * e3]
        v.insert(c, xi)  # coordinate c of (s1, s2, t1, t2) is the largest
        s1, s2, t1, t2 = v
        S_all.append(np.stack([s1, s2], 1))
        T_all.append(np.stack([t1, t2], 1))
        W_all.append(Wg * xi**3)
    return np.concatenate(S_all), np.concatenate(T_all), np.concatenate(W_all)
