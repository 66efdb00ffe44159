"""Electric field integral equation on the S^1 space (test infrastructure).

(MS) writes the scattered field of a surface current j as
    E(x) = int_Gamma G(x,y) j(y) dsigma_y + kappa^-2 grad_x int_Gamma G(x,y) div_Gamma j(y) dsigma_y,
with the Helmholtz kernel G = exp(-i kappa r) / (4 pi r) of (HS).  Testing the
tangential trace with mu and moving the surface gradient onto mu (closed
surface, int grad_Gamma f . mu = -int f div_Gamma mu) gives the Galerkin form
    a(j, mu) = int int G(x,y) [ j(y) . mu(x) - kappa^-2 div_Gamma j(y) div_Gamma mu(x) ],
and the perfectly conducting boundary condition n x (E_inc + E) = 0 of (MP)
becomes a(j, mu) = -int_Gamma E_inc . mu for all mu in S^1.

With the div-conforming Piola lift of App. E (``oracle.space_s1``) all
measures cancel:
    A_ij = sum_{e,f} h^4 sum_k W_k G(x_k, y_k) [ (Dgamma(s_k) phi_hat_i(s_k)) . (Dgamma(t_k) phi_hat_j(t_k))
                                               - kappa^-2 div phi_hat_i(s_k) div phi_hat_j(t_k) ],
    b_i  = -sum_e h^2 sum_k w_k E_inc(gamma(s_k)) . (Dgamma(s_k) phi_hat_i(s_k)),
with the same element-pair rules as the scalar operators (``oracle.quadrature``,
canonical maps from ``oracle.topology``).  A is complex symmetric.
"""
from __future__ import annotations

import numpy as np

from .galerkin import pair_rule
from .gauss import tensor2
from .topology import apply_map, canonical_maps, corner_ids


def green_h(kappa: complex, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    r = np.linalg.norm(x - y, axis=-1)
    return np.exp(-1j * kappa * r) / (4.0 * np.pi * r)


class EfieAssembler:
    def __init__(self, space, kappa: complex, g_reg: int = 4, g_sing=5):
        self.space, self.kappa = space, complex(kappa)
        self.g_reg, self.g_sing = g_reg, g_sing
        self.ids = corner_ids(space)

    def _side(self, e: int, st_loc: np.ndarray):
        sp = self.space
        patch = sp.element(e)[0]
        st = sp.to_patch(e, st_loc)
        x = sp.geom.eval(patch, st)
        J = sp.geom.jacobian(patch, st)  # (n, 3, 2)
        V, D = sp.element_basis(e, st_loc)  # (n, nloc, 2), (n, nloc)
        U = np.einsum("kca,kia->kic", J, V)  # physical (unnormalised) fields D gamma phi_hat
        return x, U, D

    def pair_block(self, e: int, f: int) -> np.ndarray:
        """nloc x nloc block of the form over elements e (test side) and f (trial side)."""
        sp = self.space
        kind, me, mf = canonical_maps(self.ids[e], self.ids[f])
        S, T, W = pair_rule(kind, self.g_reg, self.g_sing)
        x, Ue, De = self._side(e, apply_map(me, S))
        y, Uf, Df = self._side(f, apply_map(mf, T))
        Gw = green_h(self.kappa, x, y) * W * sp.h**4
        vec = np.einsum("k,kic,kjc->ij", Gw, Ue, Uf)
        div = np.einsum("k,ki,kj->ij", Gw, De, Df)
        return vec - div / self.kappa**2

    def dense(self) -> np.ndarray:
        sp = self.space
        A = np.zeros((sp.ndofs, sp.ndofs), dtype=complex)
        dofs = [sp.element_dofs(e) for e in range(sp.nelem)]
        for e in range(sp.nelem):
            ge, ce = dofs[e]
            for f in range(e, sp.nelem):
                gf, cf = dofs[f]
                blk = self.pair_block(e, f) * np.outer(ce, cf)
                np.add.at(A, (ge[:, None], gf[None, :]), blk)
                if f != e:
                    np.add.at(A, (gf[:, None], ge[None, :]), blk.T)
        return A


def efie_rhs(space, e_inc, g: int = 6) -> np.ndarray:
    """b_i = -int_Gamma E_inc . mu_i; e_inc maps points (n, 3) to complex fields (n, 3)."""
    pts, w = tensor2(g)
    b = np.zeros(space.ndofs, dtype=complex)
    for e in range(space.nelem):
        patch = space.element(e)[0]
        st = space.to_patch(e, pts)
        x = space.geom.eval(patch, st)
        J = space.geom.jacobian(patch, st)
        V, _ = space.element_basis(e, pts)
        U = np.einsum("kca,kia->kic", J, V)
        ge, ce = space.element_dofs(e)
        loc = -np.einsum("kc,kic,k->i", e_inc(x), U, w * space.h**2)
        np.add.at(b, ge, ce * loc)
    return b


def efie_field(space, rho: np.ndarray, pts: np.ndarray, kappa: complex, g: int = 6) -> np.ndarray:
    """Scattered field E(x) of (MS) at points off Gamma, (npts, 3) complex.

    grad_x G = G (-i kappa - 1/r) (x - y) / r for G = exp(-i kappa r)/(4 pi r)."""
    kappa = complex(kappa)
    qp, w = tensor2(g)
    pts = np.asarray(pts, dtype=float)
    E = np.zeros((len(pts), 3), dtype=complex)
    for e in range(space.nelem):
        patch = space.element(e)[0]
        st = space.to_patch(e, qp)
        y = space.geom.eval(patch, st)
        J = space.geom.jacobian(patch, st)
        V, D = space.element_basis(e, qp)
        ge, ce = space.element_dofs(e)
        coeff = ce * rho[ge]
        jv = np.einsum("kca,kia,i->kc", J, V, coeff) * (w * space.h**2)[:, None]  # (k, 3)
        dv = (D @ coeff) * w * space.h**2  # (k,)
        d = pts[:, None, :] - y[None, :, :]
        r = np.linalg.norm(d, axis=-1)
        G = np.exp(-1j * kappa * r) / (4.0 * np.pi * r)
        gradG = (G * (-1j * kappa - 1.0 / r) / r)[..., None] * d
        E += np.einsum("pk,kc->pc", G, jv) + np.einsum("pkc,k->pc", gradG, dv) / kappa**2
    return E


class EfieH2Oracle:
    """Dense reconstruction of the H^2-compressed EFIE (test infrastructure).

    Same block tree, Chebyshev nodes and Lagrange polynomials as ``oracle.h2``.
    On a far block (tau, sigma) the kernel is interpolated on the parameter
    squares with the Jacobian factors kept inside the interpolated functions:
      G(x,y) d_alpha gamma(s) . d_beta gamma(t) ~ sum_ab L_a(s) K^{ab}_{alpha beta} L_b(t),
      K^{ab}_{alpha beta} = G(x_a, y_b) d_alpha gamma(x_a) . d_beta gamma(y_b),
      G(x,y) ~ sum_ab L_a(s) G(x_a, y_b) L_b(t),
    so the Galerkin block of elements e in tau, f in sigma is
      sum_{alpha beta} M^alpha_e K_{alpha beta} (M^beta_f)^T - kappa^-2 M^div_e K (M^div_f)^T
    with the geometry-independent moments M^alpha_e[i, a] = int_e phi_hat_i^alpha L_a ds and
    M^div_e[i, a] = int_e div phi_hat_i L_a ds (parameter measure), integrated
    directly on every cluster (no nested transfers).  Near blocks: EfieAssembler."""

    def __init__(self, space, kappa, q=4, eta=1.6, leaf_level=None, g_reg=4, g_sing=5):
        from .h2 import block_tree, chebyshev_nodes01

        self.space, self.kappa, self.q = space, complex(kappa), q
        self.leaf = max(0, space.level - 1) if leaf_level is None else leaf_level
        self.asm = EfieAssembler(space, kappa, g_reg, g_sing)
        self.far, self.near, _ = block_tree(space.geom, self.leaf, eta)
        self.nodes = chebyshev_nodes01(q)
        self._mom: dict = {}
        self._pair: dict = {}

    def cluster_nodes(self, c):
        patch, lev, i1, i2 = c
        H = 2.0 ** -lev
        X1, X2 = np.meshgrid((i1 + self.nodes) * H, (i2 + self.nodes) * H, indexing="xy")
        return np.stack([X1.ravel(), X2.ravel()], 1)

    def couplings(self, t, s):
        """(K_{alpha beta} for alpha, beta in {1, 2} as a (2, 2, q^2, q^2) array, K_div = G)."""
        sp = self.space
        st, ss = self.cluster_nodes(t), self.cluster_nodes(s)
        xt, xs = sp.geom.eval(t[0], st), sp.geom.eval(s[0], ss)
        Jt, Js = sp.geom.jacobian(t[0], st), sp.geom.jacobian(s[0], ss)
        G = green_h(self.kappa, xt[:, None, :], xs[None, :, :])
        K = np.einsum("ab,acx,bcy->xyab", G, Jt, Js)
        return K, G

    def moments(self, e, c):
        """(M^1, M^2, M^div) of element e on cluster c, each (nloc, q^2)."""
        key = (e, c)
        if key not in self._mom:
            from .h2 import lagrange

            sp = self.space
            pts, w = tensor2(sp.p + self.q)
            st = sp.to_patch(e, pts)
            H = 2.0 ** -c[1]
            l1 = lagrange(self.nodes, st[:, 0] / H - c[2])
            l2 = lagrange(self.nodes, st[:, 1] / H - c[3])
            L = np.einsum("pa,pb->pba", l1, l2).reshape(len(w), -1)
            V, D = sp.element_basis(e, pts)
            wt = (w * sp.h**2)[:, None]
            self._mom[key] = ((V[:, :, 0] * wt).T @ L, (V[:, :, 1] * wt).T @ L, (D * wt).T @ L)
        return self._mom[key]

    def pair(self, e, f):
        if e <= f:
            if (e, f) not in self._pair:
                self._pair[(e, f)] = self.asm.pair_block(e, f)
            return self._pair[(e, f)]
        return self.pair(f, e).T

    def dense(self):
        from .h2 import cluster_elements

        sp = self.space
        A = np.zeros((sp.ndofs, sp.ndofs), dtype=complex)
        dofs = [sp.element_dofs(e) for e in range(sp.nelem)]

        def add(e, f, blk):
            ge, ce = dofs[e]
            gf, cf = dofs[f]
            np.add.at(A, (ge[:, None], gf[None, :]), blk * np.outer(ce, cf))

        for t, s in self.near:
            for e in cluster_elements(sp, t):
                for f in cluster_elements(sp, s):
                    add(e, f, self.pair(e, f))
        for t, s in self.far:
            K, G = self.couplings(t, s)
            for e in cluster_elements(sp, t):
                Me = self.moments(e, t)
                for f in cluster_elements(sp, s):
                    Mf = self.moments(f, s)
                    blk = sum(Me[a] @ K[a, b] @ Mf[b].T for a in range(2) for b in range(2))
                    add(e, f, blk - (Me[2] @ G @ Mf[2].T) / self.kappa**2)
        return A
