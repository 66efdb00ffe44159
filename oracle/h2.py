"""Dense reconstruction of the H^2 approximant (test infrastructure).

Sec. 2: the far field is compressed by an embedded fast multipole method that
interpolates the kernel on the reference domain (the unit square) per cluster
pair.  Readings used (the paper gives no formulas):

* Clusters: per patch a quadtree on the parameter square; a level-l cluster is
  a square of side 2^-l, the element level L is the finest.
* Cluster ball: centre gamma(midpoint); radius the largest distance from the
  centre to gamma on a 9 x 9 uniform grid of the closed square (corners
  included).  dist(tau, sigma) = max(0, |c_tau - c_sigma| - r_tau - r_sigma).
* Admissibility: max(diam tau, diam sigma) <= eta * dist(tau, sigma), diam = 2r.
* Block tree: all patch pairs at level 0; an admissible pair is a far block; a
  non-admissible pair at the leaf level is a near block; otherwise all 4 x 4
  child pairs are visited.
* Interpolation: q x q tensor Chebyshev nodes of the first kind,
  x_a = (1 + cos((2a+1) pi / (2q))) / 2 mapped to the cluster square, index
  a = a1 + q a2; Lagrange polynomials L_a of degree q-1 per direction.
* Far block (tau, sigma):  G(gamma(s), gamma(t)) ~ sum_ab L_a^tau(s) K_ab L_b^sigma(t)
  with K_ab = G(gamma(x_a^tau), gamma(x_b^sigma)); on elements e in tau, f in sigma
  the Galerkin block is M_e^tau K (M_f^sigma)^T with the moments
  M_e^tau[i, a] = int_e phi_hat_i(s) L_a^tau(s) ds (parameter measure).
* Near block: the element-pair quadrature of ``oracle.galerkin``.

The moments are integrated directly on every cluster by Gauss rules that are
exact for the polynomial integrand; no nested transfer matrices are used.
Because Lagrange interpolation of degree q-1 reproduces the parent's Lagrange
polynomials exactly on a child square, this equals the nested H^2 operator up
to rounding.
"""
from __future__ import annotations

import numpy as np

from .galerkin import Assembler, green
from .gauss import tensor2


def chebyshev_nodes01(q: int) -> np.ndarray:
    a = np.arange(q)
    return 0.5 * (1.0 + np.cos((2 * a + 1) * np.pi / (2 * q)))


def lagrange(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """L_a(x) for all nodes: (len(x), q)."""
    x = np.atleast_1d(x)
    q = len(nodes)
    out = np.ones((x.size, q))
    for a in range(q):
        for b in range(q):
            if b != a:
                out[:, a] *= (x - nodes[b]) / (nodes[a] - nodes[b])
    return out


class Clusters:
    """Cluster balls on every patch and level."""

    def __init__(self, geom, max_level: int):
        self.geom = geom
        self.cache: dict[tuple, tuple] = {}
        k = np.arange(9) / 8.0
        self.grid = np.stack(np.meshgrid(k, k, indexing="xy"), -1).reshape(-1, 2)

    def ball(self, c):
        if c not in self.cache:
            patch, lev, i1, i2 = c
            H = 2.0**-lev
            mid = self.geom.eval(patch, np.array([[(i1 + 0.5) * H, (i2 + 0.5) * H]]))[0]
            pts = self.geom.eval(patch, (np.array([i1, i2]) + self.grid) * H)
            r = np.max(np.linalg.norm(pts - mid, axis=1))
            self.cache[c] = (mid, r)
        return self.cache[c]


def admissible(cl: Clusters, t, s, eta: float, kdiam: float = 0.0, kabs: float = 0.0) -> bool:
    """max(diam) <= eta dist; for Helmholtz with kdiam > 0 also |kappa| max(diam) <= kdiam
    (the kernel's oscillation over the block, App. B eq. (HS))."""
    ct, rt = cl.ball(t)
    cs, rs = cl.ball(s)
    dist = max(0.0, np.linalg.norm(ct - cs) - rt - rs)
    diam = 2.0 * max(rt, rs)
    if kdiam > 0 and kabs * diam > kdiam:
        return False
    return diam <= eta * dist


def block_tree(geom, leaf_level: int, eta: float, kdiam: float = 0.0, kabs: float = 0.0):
    """(far, near): lists of cluster pairs ((patch, lev, i1, i2), (patch, lev, i1, i2))."""
    cl = Clusters(geom, leaf_level)
    far, near = [], []
    stack = [((p, 0, 0, 0), (r, 0, 0, 0)) for p in range(geom.npatch) for r in range(geom.npatch)]
    while stack:
        t, s = stack.pop()
        if eta > 0 and admissible(cl, t, s, eta, kdiam, kabs):
            far.append((t, s))
        elif t[1] == leaf_level:
            near.append((t, s))
        else:
            for c2 in range(2):
                for c1 in range(2):
                    tc = (t[0], t[1] + 1, 2 * t[2] + c1, 2 * t[3] + c2)
                    for d2 in range(2):
                        for d1 in range(2):
                            stack.append((tc, (s[0], s[1] + 1, 2 * s[2] + d1, 2 * s[3] + d2)))
    return far, near, cl


def cluster_elements(space, c) -> list[int]:
    patch, lev, i1, i2 = c
    m = 2 ** (space.level - lev)
    return [space.element_index(patch, i1 * m + a, i2 * m + b) for b in range(m) for a in range(m)]


def cluster_of(space, e: int, lev: int):
    patch, i1, i2 = space.element(e)
    sh = space.level - lev
    return (patch, lev, i1 >> sh, i2 >> sh)


class H2Oracle:
    """Block-wise H^2 approximant on an S2Space."""

    def __init__(self, space, op, kappa=0.0, q=4, eta=1.6, leaf_level=None, g_reg=4, g_sing=6, kdiam=0.0):
        self.space = space
        self.q = q
        self.leaf = max(0, space.level - 1) if leaf_level is None else leaf_level
        if self.leaf > space.level:
            raise ValueError("leaf level above element level")
        self.asm = Assembler(space, op, kappa, g_reg, g_sing)
        kabs = abs(kappa) if op == "helmholtz" else 0.0
        self.far, self.near, self.cl = block_tree(space.geom, self.leaf, eta if q > 0 else 0.0, kdiam, kabs)
        self.nodes = chebyshev_nodes01(q) if q > 0 else None
        self._mom: dict = {}
        self._xhat: dict = {}
        self._pair: dict = {}
        self.far_by_target: dict = {}
        for t, s in self.far:
            self.far_by_target.setdefault(t, []).append(s)
        self.near_by_target: dict = {}
        for t, s in self.near:
            self.near_by_target.setdefault(t, []).append(s)

    # --- interpolation pieces -------------------------------------------------
    def cluster_nodes(self, c) -> np.ndarray:
        patch, lev, i1, i2 = c
        H = 2.0**-lev
        x1 = (i1 + self.nodes) * H
        x2 = (i2 + self.nodes) * H
        X1, X2 = np.meshgrid(x1, x2, indexing="xy")
        return np.stack([X1.ravel(), X2.ravel()], 1)  # index a1 + q a2

    def coupling(self, t, s) -> np.ndarray:
        """K_ab = G(gamma(x_a^t), gamma(x_b^s))."""
        xt = self.space.geom.eval(t[0], self.cluster_nodes(t))
        xs = self.space.geom.eval(s[0], self.cluster_nodes(s))
        return green(self.asm.op, self.asm.kappa, xt[:, None, :], xs[None, :, :])

    def moment(self, e: int, c) -> np.ndarray:
        """M_e^c[i, a] = int_e phi_hat_i L_a^c ds, ((d+1)^2, q^2)."""
        key = (e, c)
        if key not in self._mom:
            sp = self.space
            pts, w = tensor2(sp.d + self.q)
            st = sp.to_patch(e, pts)
            H = 2.0 ** -c[1]
            l1 = lagrange(self.nodes, st[:, 0] / H - c[2])
            l2 = lagrange(self.nodes, st[:, 1] / H - c[3])
            L = np.einsum("pa,pb->pba", l1, l2).reshape(len(w), -1)
            B = sp.element_basis(e, pts)
            self._mom[key] = (B * (w * sp.h**2)[:, None]).T @ L
        return self._mom[key]

    def pair(self, e: int, f: int) -> np.ndarray:
        """Near-field element block; unordered pairs are integrated from the lower index."""
        if e <= f:
            key = (e, f)
            if key not in self._pair:
                self._pair[key] = self.asm.pair_block(e, f)
            return self._pair[key]
        return self.pair(f, e).T

    # --- dense reconstruction -------------------------------------------------
    def dense(self) -> np.ndarray:
        sp = self.space
        A = np.zeros((sp.ndofs, sp.ndofs), dtype=self.asm.dtype)
        for t, s in self.near:
            for e in cluster_elements(sp, t):
                de = sp.element_dofs(e)
                for f in cluster_elements(sp, s):
                    A[np.ix_(de, sp.element_dofs(f))] += self.pair(e, f)
        for t, s in self.far:
            K = self.coupling(t, s)
            for e in cluster_elements(sp, t):
                Me = self.moment(e, t)
                de = sp.element_dofs(e)
                for f in cluster_elements(sp, s):
                    A[np.ix_(de, sp.element_dofs(f))] += Me @ K @ self.moment(f, s).T
        return A

    # --- sampled rows of A~ x -------------------------------------------------
    def xhat(self, c, x: np.ndarray) -> np.ndarray:
        """Cluster moment of x: sum_{f in c} M_f^c^T x[dofs_f], computed directly."""
        if c not in self._xhat:
            sp = self.space
            acc = 0.0
            for f in cluster_elements(sp, c):
                acc = acc + self.moment(f, c).T @ x[sp.element_dofs(f)]
            self._xhat[c] = acc
        return self._xhat[c]

    def apply_rows(self, x: np.ndarray, rows) -> np.ndarray:
        """(A~ x)[rows] without forming A~.  Clears the x-moment cache first."""
        sp = self.space
        self._xhat = {}
        out = np.zeros(len(rows), dtype=np.result_type(self.asm.dtype, x.dtype))
        n = sp.n1
        for r, i in enumerate(rows):
            patch, rem = divmod(int(i), n * n)
            j2, j1 = divmod(rem, n)
            acc = 0.0
            r_ = sp.r  # element i carries the functions r i .. r i + d
            for k2 in range(sp.d + 1):
                for k1 in range(sp.d + 1):
                    if (j1 - k1) % r_ or (j2 - k2) % r_:
                        continue
                    i1, i2 = (j1 - k1) // r_, (j2 - k2) // r_
                    if not (0 <= i1 < sp.n_el and 0 <= i2 < sp.n_el):
                        continue
                    e = sp.element_index(patch, i1, i2)
                    kloc = k1 + (sp.d + 1) * k2
                    for lev in range(self.leaf + 1):
                        t = cluster_of(sp, e, lev)
                        for s in self.far_by_target.get(t, []):
                            Me = self.moment(e, t)
                            acc = acc + Me[kloc] @ (self.coupling(t, s) @ self.xhat(s, x))
                    tl = cluster_of(sp, e, self.leaf)
                    for s in self.near_by_target.get(tl, []):
                        for f in cluster_elements(sp, s):
                            acc = acc + self.pair(e, f)[kloc] @ x[sp.element_dofs(f)]
            out[r] = acc
        return out
