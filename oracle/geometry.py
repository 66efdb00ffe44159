"""Patch parametrisations gamma_i: [0,1]^2 -> R^3 (test infrastructure).

The paper allows arbitrary smooth parametric mappings in place of NURBS
(Sec. 4.1) provided the patches meet the boundary-representation conditions of
App. D: outward normals, patches meeting at full edges or vertices, and the
matching condition (neighbouring parametrisations coincide on a shared edge up
to an affine map of the unit square).

``Sphere6`` is the unit sphere as six patches: the cube face
c(s,t) = o + (2s-1) e1 + (2t-1) e2 projected radially, gamma = c/|c|.  With
e1 x e2 = o on every face, d_s gamma x d_t gamma points outward.  Projecting the
shared cube edge makes neighbouring faces agree on their common edge up to an
affine reparametrisation, as App. D requires.
"""
from __future__ import annotations

import numpy as np

# (o, e1, e2) per face, e1 x e2 = o (outward).  Patch order: +x, -x, +y, -y, +z, -z.
SPHERE6_FACES = np.array(
    [
        [[1, 0, 0], [0, 1, 0], [0, 0, 1]],
        [[-1, 0, 0], [0, 0, 1], [0, 1, 0]],
        [[0, 1, 0], [0, 0, 1], [1, 0, 0]],
        [[0, -1, 0], [1, 0, 0], [0, 0, 1]],
        [[0, 0, 1], [1, 0, 0], [0, 1, 0]],
        [[0, 0, -1], [0, 1, 0], [1, 0, 0]],
    ],
    dtype=float,
)


class Sphere6:
    """Unit sphere, six cube-face patches, gamma = c/|c|."""

    npatch = 6

    def _cube(self, patch: int, st: np.ndarray) -> np.ndarray:
        o, e1, e2 = SPHERE6_FACES[patch]
        st = np.asarray(st, dtype=float)
        return o + (2 * st[..., 0:1] - 1) * e1 + (2 * st[..., 1:2] - 1) * e2

    def eval(self, patch: int, st: np.ndarray) -> np.ndarray:
        """gamma_patch(s,t) for points st (..., 2) -> (..., 3)."""
        c = self._cube(patch, st)
        return c / np.linalg.norm(c, axis=-1, keepdims=True)

    def jacobian(self, patch: int, st: np.ndarray) -> np.ndarray:
        """(d_s gamma, d_t gamma) stacked as (..., 3, 2)."""
        o, e1, e2 = SPHERE6_FACES[patch]
        c = self._cube(patch, st)
        n = np.linalg.norm(c, axis=-1, keepdims=True)
        g = c / n
        cols = []
        for e in (e1, e2):
            de = 2.0 * e
            cols.append((de - g * np.sum(g * de, axis=-1, keepdims=True)) / n)
        return np.stack(cols, axis=-1)
