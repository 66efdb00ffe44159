"""The S^2 B-spline boundary element space of App. E (test infrastructure).

S^2_{p,Xi}(square) = S_{p-1,Xi'} (x) S_{p-1,Xi'}: tensor B-splines of degree
d = p-1 on the truncated open knot vector with 2^L equal elements per direction;
every interior knot is repeated r times (Sec. 4.3, ``knotRepetition``; default 1,
maximal smoothness C^(d-1); r = d + 1 gives discontinuous piecewise polynomials).
Per direction there are d + 1 + (2^L - 1) r functions, and on element i the
functions r i, ..., r i + d are non-zero.  The library's degree argument is the ansatz degree d
(d = 0 piecewise constants).  With the 2-form Piola lift
phi_i(gamma(s)) = phi_hat_i(s) / |d_s gamma x d_t gamma|, every surface measure
cancels: <S phi_j, phi_i> = int int G(gamma(s), gamma(t)) phi_hat_i(s) phi_hat_j(t) ds dt
over the parameter squares, and <g, phi_i> = int g(gamma(s)) phi_hat_i(s) ds.
S^2 needs no inter-patch continuity (it is only H^{-1/2}-conforming), so every
patch carries its own (2^L + d)^2 functions.

Global dof numbering: patch * n^2 + j2 * n + j1 with n = d + 1 + (2^L - 1) r and j1 the
B-spline index along the first parameter s.  Element numbering (oracle only):
patch * 4^L + i2 * 2^L + i1.
"""
from __future__ import annotations

import numpy as np

from .bspline import bspline_basis, open_knots


class S2Space:
    def __init__(self, geom, level: int, degree: int, knot_repetition: int = 1):
        if level < 0 or degree < 0:
            raise ValueError("level, degree >= 0")
        if not 1 <= knot_repetition <= degree + 1:
            raise ValueError("knot repetition in [1, degree + 1]")
        self.r = knot_repetition
        self.geom = geom
        self.level = level
        self.d = degree
        self.n_el = 2**level
        self.h = 1.0 / self.n_el
        self.n1 = degree + 1 + (self.n_el - 1) * knot_repetition
        self.nloc = (degree + 1) ** 2
        self.npatch = geom.npatch
        self.nelem = self.npatch * self.n_el**2
        self.ndofs = self.npatch * self.n1**2
        self.knots = open_knots(degree, self.n_el, knot_repetition)

    def element(self, e: int) -> tuple[int, int, int]:
        """(patch, i1, i2) of element e."""
        patch, r = divmod(e, self.n_el**2)
        i2, i1 = divmod(r, self.n_el)
        return patch, i1, i2

    def element_index(self, patch: int, i1: int, i2: int) -> int:
        return patch * self.n_el**2 + i2 * self.n_el + i1

    def to_patch(self, e: int, st_local: np.ndarray) -> np.ndarray:
        """Element-local [0,1]^2 coordinates -> patch parameters."""
        _, i1, i2 = self.element(e)
        st_local = np.asarray(st_local, dtype=float)
        return (np.array([i1, i2], dtype=float) + st_local) * self.h

    def element_dofs(self, e: int) -> np.ndarray:
        """Global dofs of the (d+1)^2 B-splines nonzero on element e, ordered k1 + (d+1) k2."""
        patch, i1, i2 = self.element(e)
        d, n, r = self.d, self.n1, self.r
        return np.array(
            [patch * n * n + (r * i2 + k2) * n + (r * i1 + k1) for k2 in range(d + 1) for k1 in range(d + 1)],
            dtype=np.int64,
        )

    def element_basis(self, e: int, st_local: np.ndarray) -> np.ndarray:
        """phi_hat of the element's (d+1)^2 B-splines at local points: (npts, (d+1)^2).

        Evaluated as products of 1-D B-splines b_j(s) b_j'(t) (App. C recursion),
        at patch parameters, restricted to the element's closed square.
        """
        _, i1, i2 = self.element(e)
        d = self.d
        st = self.to_patch(e, st_local)
        # keep points on the element's right edge inside this element's interval
        eps = 1e-14
        s = np.clip(st[:, 0], i1 * self.h, (i1 + 1) * self.h * (1 - eps) if i1 + 1 < self.n_el else 1.0)
        t = np.clip(st[:, 1], i2 * self.h, (i2 + 1) * self.h * (1 - eps) if i2 + 1 < self.n_el else 1.0)
        r = self.r
        bs = bspline_basis(self.knots, d, s)[:, r * i1 : r * i1 + d + 1]
        bt = bspline_basis(self.knots, d, t)[:, r * i2 : r * i2 + d + 1]
        return np.einsum("pa,pb->pba", bs, bt).reshape(len(st), (d + 1) ** 2)

    def corners(self, e: int) -> np.ndarray:
        """Physical positions of the element's corners in local order (0,0),(1,0),(0,1),(1,1)."""
        patch = self.element(e)[0]
        loc = np.array([[0, 0], [1, 0], [0, 1], [1, 1]], dtype=float)
        return self.geom.eval(patch, self.to_patch(e, loc))
