"""Coarse-space correction of the two-level preconditioner (test infrastructure).

Not in the paper (which solves without a preconditioner).  The S^2 spaces of one degree
on the dyadic levels are nested (App. E: the fine knot vector contains the coarse one and
the Piola lift is the same on every level), so a coarse function sum_a c_a phi^c_a equals a
fine function sum_i (P c)_i phi^f_i exactly.  P is the tensor product, per patch, of the
1-D knot-insertion matrix R from level Lc to level L.  With A_c = P^T A P the Galerkin
matrix of the coarse space, the additive coarse correction of a residual r is

    z_c = P A_c^{-1} P^T r,

and the two-level preconditioner adds it to the block-Jacobi part: M^-1 = E^T D^-1 E + P A_c^{-1} P^T.

R is built here by Boehm's algorithm (one knot at a time: the new coefficient j is
(1 - a_j) c_{j-1} + a_j c_j with a_j = (t - t_j) / (t_{j+p} - t_j), clipped to [0, 1]), not
by interpolation, and A_c is the coarse Galerkin matrix assembled directly on level Lc
(``Assembler``), which equals P^T A P up to quadrature.
"""
from __future__ import annotations

import numpy as np

from .bspline import open_knots


def boehm_insert(knots: np.ndarray, degree: int, t: float) -> tuple[np.ndarray, np.ndarray]:
    """Insert knot t once: new knot vector and the matrix Q (n+1, n) with c_new = Q c."""
    knots = np.asarray(knots, dtype=float)
    n = len(knots) - degree - 1
    k = int(np.searchsorted(knots, t, side="right")) - 1  # t in [knots[k], knots[k+1])
    Q = np.zeros((n + 1, n))
    for j in range(n + 1):
        if j <= k - degree:
            Q[j, j] = 1.0
        elif j > k:
            Q[j, j - 1] = 1.0
        else:
            a = (t - knots[j]) / (knots[j + degree] - knots[j])
            Q[j, j] = a
            Q[j, j - 1] = 1.0 - a
    return np.insert(knots, k + 1, t), Q


def refinement_1d(degree: int, coarse_level: int, level: int) -> np.ndarray:
    """R (n1_fine, n1_coarse): the coarse open-knot B-splines of level Lc as combinations of
    those of level L (both with single interior knots)."""
    if not 0 <= coarse_level <= level:
        raise ValueError("0 <= coarse level <= level")
    kn = open_knots(degree, 2**coarse_level)
    R = np.eye(len(kn) - degree - 1)
    fine = open_knots(degree, 2**level)
    for t in fine[degree + 1 : len(fine) - degree - 1]:
        if np.any(np.isclose(kn, t, rtol=0.0, atol=1e-15)):
            continue  # already a knot of the coarse vector (single interior knots)
        kn, Q = boehm_insert(kn, degree, t)
        R = Q @ R
    assert np.allclose(kn, fine)
    return R


def prolongation(space_c, space_f) -> np.ndarray:
    """P (ndofs_f, ndofs_c) for two S^2 spaces of one degree on the same patches; global
    dof patch n1^2 + j2 n1 + j1 on both sides, so per patch P = kron(R, R)."""
    if space_c.d != space_f.d or space_c.r != 1 or space_f.r != 1:
        raise ValueError("same degree, single knots")
    R = refinement_1d(space_f.d, space_c.level, space_f.level)
    Pp = np.kron(R, R)  # (j2 n1 + j1) rows from (b n1c + a) columns
    npatch = space_f.npatch
    P = np.zeros((space_f.ndofs, space_c.ndofs))
    nf, nc = space_f.n1**2, space_c.n1**2
    for p in range(npatch):
        P[p * nf : (p + 1) * nf, p * nc : (p + 1) * nc] = Pp
    return P


def coarse_correction(P: np.ndarray, Ac: np.ndarray, r: np.ndarray) -> np.ndarray:
    """z_c = P A_c^{-1} P^T r for one residual or columns of residuals (ndofs_f, ...)."""
    return P @ np.linalg.solve(Ac, P.T @ r)
