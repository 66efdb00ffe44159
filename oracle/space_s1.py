"""The divergence-conforming S^1 B-spline space of App. E (test infrastructure).

On the unit square, S^1_{p,Xi} = S_{p,Xi} (x) S_{p-1,Xi'}  x  S_{p-1,Xi'} (x) S_{p,Xi}:
the first component has degree p in s and p-1 in t, the second the reverse,
with Xi the open knot vector of degree p (2^L equal elements) and Xi' its
truncation (the open knot vector of degree p-1).  The patch fields are lifted
to Gamma by the div-conforming Piola transform
    j(gamma(s)) = D gamma(s) phi_hat(s) / |d_1 gamma x d_2 gamma|,
    div_Gamma j(gamma(s)) = div phi_hat(s) / |d_1 gamma x d_2 gamma|,
so every surface measure cancels in the Galerkin integrals (App. E).

Conformity across patches (App. E, "enforcing continuity conditions"): the
normal component must be continuous across every patch edge.  Only the
functions with i = 0 or i = n_p - 1 in their degree-p direction have a normal
trace on the edge s or t in {0, 1}; with the matching condition of App. D the
reference flux through an edge equals the physical flux, so each such function
is glued to the neighbouring patch's edge function with the same tangential
B-spline (index reversed when the edge is traversed backwards) and
coefficient -sign_A * sign_B, where sign = +1 on the edges s = 1, t = 1 and
-1 on s = 0, t = 0 (outward flux of +phi_hat).  The glued pair then carries
equal and opposite outward fluxes: the normal component is continuous.

Patch-local numbering: first component i1 + n_p j2 (i1 < n_p, j2 < n_q), then
second component n_p n_q + j1 + n_q i2 (j1 < n_q, i2 < n_p), n_q = n_p - 1.
Element-local functions (2 p (p+1)): first component k1 + (p+1) k2
(k1 <= p, k2 < p), then second component p (p+1) + k1 + p k2 (k1 < p, k2 <= p).
"""
from __future__ import annotations

import numpy as np

from .bspline import bspline_basis, bspline_deriv, open_knots


class S1Space:
    def __init__(self, geom, level: int, degree: int):
        if degree < 1:
            raise ValueError("S^1 needs degree p >= 1")
        self.geom = geom
        self.level = level
        self.p = degree
        self.n_el = 2**level
        self.h = 1.0 / self.n_el
        self.np_ = self.n_el + degree
        self.nq = self.n_el + degree - 1
        self.npatch = geom.npatch
        self.nelem = self.npatch * self.n_el**2
        self.nloc = 2 * degree * (degree + 1)
        self.kp = open_knots(degree, self.n_el)
        self.kq = open_knots(degree - 1, self.n_el)
        self.per_patch = 2 * self.np_ * self.nq
        self._glue()

    # ---- patch-local indices ---------------------------------------------------------
    def c1(self, i1: int, j2: int) -> int:
        return i1 + self.np_ * j2

    def c2(self, j1: int, i2: int) -> int:
        return self.np_ * self.nq + j1 + self.nq * i2

    def _side_functions(self, side: int):
        """Patch-local indices of the edge functions on a side, ordered along the side,
        and the outward-flux sign.  Sides: 0 s=0, 1 s=1, 2 t=0, 3 t=1."""
        if side in (0, 1):
            i1 = 0 if side == 0 else self.np_ - 1
            return [self.c1(i1, j) for j in range(self.nq)], (-1 if side == 0 else 1)
        i2 = 0 if side == 2 else self.np_ - 1
        return [self.c2(j, i2) for j in range(self.nq)], (-1 if side == 2 else 1)

    def _side_ends(self, patch: int, side: int):
        ends = {0: ([0, 0], [0, 1]), 1: ([1, 0], [1, 1]), 2: ([0, 0], [1, 0]), 3: ([0, 1], [1, 1])}[side]
        return self.geom.eval(patch, np.array(ends, dtype=float))

    def _glue(self):
        key = lambda x: tuple(np.round(x * 1e9).astype(np.int64))  # noqa: E731
        sides = {}
        for P in range(self.npatch):
            for sd in range(4):
                a, b = self._side_ends(P, sd)
                sides.setdefault(frozenset([key(a), key(b)]), []).append((P, sd, key(a)))
        # partner[(P, local)] = (Q, local', coefficient)
        partner = {}
        for lst in sides.values():
            if len(lst) != 2:
                raise ValueError("each patch edge must be shared by exactly two patches (App. D)")
            (P, sa, ka), (Q, sb, kb) = lst
            fa, sga = self._side_functions(sa)
            fb, sgb = self._side_functions(sb)
            if ka != kb:
                fb = fb[::-1]
            for la, lb in zip(fa, fb):
                partner[(P, la)] = (Q, lb, -sga * sgb)
                partner[(Q, lb)] = (P, la, -sga * sgb)
        gid = -np.ones((self.npatch, self.per_patch), dtype=np.int64)
        coef = np.zeros((self.npatch, self.per_patch))
        n = 0
        for P in range(self.npatch):
            for loc in range(self.per_patch):
                if gid[P, loc] >= 0:
                    continue
                gid[P, loc] = n
                coef[P, loc] = 1.0
                if (P, loc) in partner:
                    Q, lq, c = partner[(P, loc)]
                    gid[Q, lq] = n
                    coef[Q, lq] = c
                n += 1
        self.gid, self.coef, self.ndofs = gid, coef, n

    # ---- elements ----------------------------------------------------------------------
    def element(self, e: int) -> tuple[int, int, int]:
        patch, r = divmod(e, self.n_el**2)
        i2, i1 = divmod(r, self.n_el)
        return patch, i1, i2

    def element_index(self, patch: int, i1: int, i2: int) -> int:
        return patch * self.n_el**2 + i2 * self.n_el + i1

    def to_patch(self, e: int, st_local: np.ndarray) -> np.ndarray:
        _, i1, i2 = self.element(e)
        return (np.array([i1, i2], dtype=float) + np.asarray(st_local, dtype=float)) * self.h

    def corners(self, e: int) -> np.ndarray:
        patch = self.element(e)[0]
        loc = np.array([[0, 0], [1, 0], [0, 1], [1, 1]], dtype=float)
        return self.geom.eval(patch, self.to_patch(e, loc))

    def local_patch_indices(self, e: int) -> np.ndarray:
        _, i1, i2 = self.element(e)
        p = self.p
        idx = [self.c1(i1 + k1, i2 + k2) for k2 in range(p) for k1 in range(p + 1)]
        idx += [self.c2(i1 + k1, i2 + k2) for k2 in range(p + 1) for k1 in range(p)]
        return np.array(idx, dtype=np.int64)

    def element_dofs(self, e: int):
        """(global dof, coefficient) of each element-local function."""
        patch = self.element(e)[0]
        loc = self.local_patch_indices(e)
        return self.gid[patch, loc], self.coef[patch, loc]

    def element_basis(self, e: int, st_local: np.ndarray):
        """Reference fields of the element-local functions at local points:
        V (npts, nloc, 2) = phi_hat in patch-parameter components, and
        D (npts, nloc) = div phi_hat = d_s phi_hat^1 + d_t phi_hat^2 (patch parameters)."""
        _, i1, i2 = self.element(e)
        p, h = self.p, self.h
        st = self.to_patch(e, st_local)
        eps = 1e-14
        s = np.clip(st[:, 0], i1 * h, (i1 + 1) * h * (1 - eps) if i1 + 1 < self.n_el else 1.0)
        t = np.clip(st[:, 1], i2 * h, (i2 + 1) * h * (1 - eps) if i2 + 1 < self.n_el else 1.0)
        bps = bspline_basis(self.kp, p, s)[:, i1 : i1 + p + 1]
        dps = bspline_deriv(self.kp, p, s)[:, i1 : i1 + p + 1]
        bqs = bspline_basis(self.kq, p - 1, s)[:, i1 : i1 + p]
        bpt = bspline_basis(self.kp, p, t)[:, i2 : i2 + p + 1]
        dpt = bspline_deriv(self.kp, p, t)[:, i2 : i2 + p + 1]
        bqt = bspline_basis(self.kq, p - 1, t)[:, i2 : i2 + p]
        npts = len(st)
        V = np.zeros((npts, self.nloc, 2))
        D = np.zeros((npts, self.nloc))
        k = 0
        for k2 in range(p):
            for k1 in range(p + 1):
                V[:, k, 0] = bps[:, k1] * bqt[:, k2]
                D[:, k] = dps[:, k1] * bqt[:, k2]
                k += 1
        for k2 in range(p + 1):
            for k1 in range(p):
                V[:, k, 1] = bqs[:, k1] * bpt[:, k2]
                D[:, k] = bqs[:, k1] * dpt[:, k2]
                k += 1
        return V, D
