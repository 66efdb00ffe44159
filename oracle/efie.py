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
