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


def real_harmonic(l: int, m: int, x: np.ndarray) -> np.ndarray:
    """Real orthonormal spherical harmonic Y_lm at unit vectors x (..., 3), without the
    Condon-Shortley phase: N_l|m| P_l^|m|(cos theta) {sqrt2 cos(m phi), 1, sqrt2 sin(|m| phi)}
    with N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!).  scipy's lpmv includes the phase (-1)^m,
    which is removed here."""
    from math import factorial

    from scipy.special import lpmv

    x = np.asarray(x, dtype=float)
    ct = np.clip(x[..., 2], -1.0, 1.0)
    ph = np.arctan2(x[..., 1], x[..., 0])
    am = abs(m)
    norm = np.sqrt((2 * l + 1) / (4 * np.pi) * factorial(l - am) / factorial(l + am))
    p = (-1) ** am * lpmv(am, l, ct)
    if m > 0:
        return np.sqrt(2.0) * norm * p * np.cos(am * ph)
    if m < 0:
        return np.sqrt(2.0) * norm * p * np.sin(am * ph)
    return norm * p


class PerturbedSphere(Sphere6):
    """Radially perturbed sphere r(x) = 1 + amp * sum_{1<=l<=4} a_lm Y_lm(x) on the cube-face
    patches of Sphere6: gamma = r(x_hat) x_hat with x_hat the Sphere6 point.  Coefficients are
    ordered (l, m = -l..l), 24 of them."""

    def __init__(self, coeffs, amp: float = 0.1):
        self.coeffs = np.asarray(coeffs, dtype=float)
        if self.coeffs.size != 24:
            raise ValueError("24 coefficients (l = 1..4) expected")
        self.amp = amp

    def radius(self, xhat: np.ndarray) -> np.ndarray:
        r = np.ones(xhat.shape[:-1])
        k = 0
        for l in range(1, 5):
            for m in range(-l, l + 1):
                r = r + self.amp * self.coeffs[k] * real_harmonic(l, m, xhat)
                k += 1
        return r

    def eval(self, patch: int, st: np.ndarray) -> np.ndarray:
        xh = super().eval(patch, st)
        return xh * self.radius(xh)[..., None]

    def jacobian(self, patch: int, st: np.ndarray, h: float = 1e-6) -> np.ndarray:
        """Central differences (used only for mass matrices in tests)."""
        st = np.asarray(st, dtype=float)
        cols = []
        for a in range(2):
            d = np.zeros(2)
            d[a] = h
            cols.append((self.eval(patch, st + d) - self.eval(patch, st - d)) / (2 * h))
        return np.stack(cols, axis=-1)


class NurbsSurface:
    """Patches gamma(s,t) = sum N_a(s) N_b(t) w_ab P_ab / sum N_a(s) N_b(t) w_ab (rational
    tensor B-splines, Sec. 4.1 / App. C), B-spline values from scipy's design matrix.
    ``patches``: dicts with degrees (p1, p2), knots (s, t) and ctrl[i2, i1] = (x, y, z, w)."""

    def __init__(self, patches):
        self.patches = patches
        self.npatch = len(patches)

    def eval(self, patch: int, st: np.ndarray) -> np.ndarray:
        from scipy.interpolate import BSpline

        pt = self.patches[patch]
        (p1, p2), (k1s, k2s), ctrl = pt["degrees"], pt["knots"], np.asarray(pt["ctrl"], dtype=float)
        st = np.atleast_2d(np.asarray(st, dtype=float))
        Ns = BSpline.design_matrix(np.clip(st[:, 0], 0.0, 1.0), k1s, p1).toarray()  # (n, k1)
        Nt = BSpline.design_matrix(np.clip(st[:, 1], 0.0, 1.0), k2s, p2).toarray()  # (n, k2)
        w = ctrl[..., 3]
        num = np.einsum("na,nb,ba,bac->nc", Ns, Nt, w, ctrl[..., :3])
        den = np.einsum("na,nb,ba->n", Ns, Nt, w)
        return num / den[:, None]

    def jacobian(self, patch: int, st: np.ndarray, h: float = 1e-6) -> np.ndarray:
        """Central differences, one-sided at the patch boundary."""
        st = np.atleast_2d(np.asarray(st, dtype=float))
        cols = []
        for a in range(2):
            d = np.zeros(2)
            d[a] = h
            lo = np.clip(st - d, 0.0, 1.0)
            hi = np.clip(st + d, 0.0, 1.0)
            cols.append((self.eval(patch, hi) - self.eval(patch, lo)) / (hi[:, a] - lo[:, a])[:, None])
        return np.stack(cols, axis=-1)
