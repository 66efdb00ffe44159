"""Dense Galerkin assembly, load vectors and potentials (test infrastructure).

App. B, equations (LS) and (HS): the single-layer kernels
  Laplace:   G(x, y) = 1 / (4 pi |x - y|)
  Helmholtz: G(x, y) = exp(-i kappa |x - y|) / (4 pi |x - y|), kappa complex (Sec. 4.2).
Sec. 2 (conforming Galerkin scheme) and App. E (S^2 space, Piola lift):
  A_ij = sum_{e, f} h^4 sum_k W_k G(gamma(s_k), gamma(t_k)) phi_hat_i(s_k) phi_hat_j(t_k)
with the element-pair rule (S, T, W) chosen by adjacency (``oracle.quadrature``)
and h = 2^-L the element side in the parameter square.  A is symmetric
(G(x,y) = G(y,x)), so each unordered pair e <= f is integrated once, from e's
point of view, and the transposed block is used for (f, e).
"""
from __future__ import annotations

import numpy as np

from . import quadrature as Q
from .topology import apply_map, canonical_maps, corner_ids

LAPLACE, HELMHOLTZ = "laplace", "helmholtz"


def green(op: str, kappa: complex, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Single-layer kernel of (LS) / (HS) for point arrays x, y of shape (..., 3)."""
    r = np.linalg.norm(x - y, axis=-1)
    if op == LAPLACE:
        return 1.0 / (4.0 * np.pi * r)
    if op == HELMHOLTZ:
        return np.exp(-1j * kappa * r) / (4.0 * np.pi * r)
    raise ValueError(op)


def pair_rule(kind: str, g_reg: int, g_sing):
    """Rule for a pair kind; g_sing is one order for all Duffy rules or a triple
    (identical, edge, vertex) whose entries are an order or four per-variable
    orders."""
    gi, ge, gv = (g_sing, g_sing, g_sing) if isinstance(g_sing, int) else tuple(g_sing)
    gi, ge, gv = (tuple(v) if not isinstance(v, (int, np.integer)) else v for v in (gi, ge, gv))
    if kind == "regular":
        return Q.rule_regular(g_reg)
    if kind == "identical":
        return Q.rule_identical(gi)
    if kind == "edge":
        return Q.rule_edge(ge)
    if kind == "vertex":
        return Q.rule_vertex(gv)
    raise ValueError(kind)


class Assembler:
    """Element-pair integration on an S2Space.

    g_reg: Gauss points per direction on separated pairs, or a pair
    (g_ring, g_far): g_ring for the ring next to the touching pairs (some element
    holds a corner of each), g_far for pairs farther apart."""

    def __init__(self, space, op: str, kappa: complex = 0.0, g_reg=4, g_sing: int = 6):
        self.space, self.op, self.kappa = space, op, kappa
        self.g_ring, self.g_far = (g_reg, g_reg) if isinstance(g_reg, (int, np.integer)) else tuple(g_reg)
        self.g_reg, self.g_sing = self.g_ring, g_sing
        self.ids = corner_ids(space)
        self.dtype = float if op == LAPLACE else complex
        self._tab_cache: dict[tuple, tuple] = {}
        # vertex -> elements holding it
        self._v2e: dict[int, list] = {}
        for el, c in enumerate(self.ids):
            for v in c:
                self._v2e.setdefault(int(v), []).append(el)

    def classify(self, e: int, f: int):
        return canonical_maps(self.ids[e], self.ids[f])

    def ring(self, e: int, f: int) -> bool:
        """Separated pair in the ring next to the touching pairs: some element holds
        a corner of e and a corner of f."""
        cf = set(self.ids[f].tolist())
        return any(cf & set(self.ids[g].tolist()) for v in self.ids[e] for g in self._v2e[int(v)])

    def _tab(self, e: int, g: int | None = None):
        """Regular-rule data of element e: points gamma(s_p) (g^2, 3) and weighted basis (g^2, (d+1)^2)."""
        g = self.g_ring if g is None else g
        if (e, g) not in self._tab_cache:
            from .gauss import tensor2

            sp = self.space
            pts, w = tensor2(g)
            x = sp.geom.eval(sp.element(e)[0], sp.to_patch(e, pts))
            bw = sp.element_basis(e, pts) * (w * sp.h**2)[:, None]
            self._tab_cache[(e, g)] = (x, bw)
        return self._tab_cache[(e, g)]

    def pair_block(self, e: int, f: int, kind_maps=None) -> np.ndarray:
        """(d+1)^2 x (d+1)^2 block int_e int_f G phi_hat_i phi_hat_j for the pair (e, f)."""
        sp = self.space
        kind, me, mf = kind_maps if kind_maps is not None else self.classify(e, f)
        if kind == "regular":
            # tensor Gauss on both elements: sum_pq w_p w_q G(x_p, y_q) phi_i(s_p) phi_j(t_q)
            g = self.g_ring if self.ring(e, f) else self.g_far
            xe, be = self._tab(e, g)
            xf, bf = self._tab(f, g)
            Gm = green(self.op, self.kappa, xe[:, None, :], xf[None, :, :])
            return be.T @ Gm @ bf
        S, T, W = pair_rule(kind, self.g_reg, self.g_sing)
        s_loc = apply_map(me, S)
        t_loc = apply_map(mf, T)
        pe, pf = sp.element(e)[0], sp.element(f)[0]
        x = sp.geom.eval(pe, sp.to_patch(e, s_loc))
        y = sp.geom.eval(pf, sp.to_patch(f, t_loc))
        Gv = green(self.op, self.kappa, x, y) * W * sp.h**4
        Be = sp.element_basis(e, s_loc)
        Bf = sp.element_basis(f, t_loc)
        return (Be * Gv[:, None]).T @ Bf

    def dense(self) -> np.ndarray:
        """The full Galerkin matrix over global dofs (small levels only).

        Separated pairs use the tensor rule for all targets f at once; touching
        pairs (e <= f) use the Duffy rules and are mirrored.
        """
        sp = self.space
        A = np.zeros((sp.ndofs, sp.ndofs), dtype=self.dtype)
        tabs = {}
        for g in {self.g_ring, self.g_far}:
            tabs[g] = (np.stack([self._tab(e, g)[0] for e in range(sp.nelem)]),  # (nelem, g^2, 3)
                       np.stack([self._tab(e, g)[1] for e in range(sp.nelem)]))  # (nelem, g^2, nloc)
        dofs = np.stack([sp.element_dofs(e) for e in range(sp.nelem)])
        singular: dict[tuple[int, int], np.ndarray] = {}
        for e in range(sp.nelem):
            with np.errstate(divide="ignore", invalid="ignore"):  # touching pairs are replaced below
                per_order = {}
                for g, (X, BW) in tabs.items():
                    Gm = green(self.op, self.kappa, X[e][:, None, None, :], X[None, :, :, :])  # (g2, nelem, g2)
                    per_order[g] = np.einsum("pi,pfq,fqj->fij", BW[e], Gm, BW)
            blocks = per_order[self.g_far].copy()
            if self.g_far != self.g_ring:
                near = {g for v in self.ids[e] for g in self._v2e[int(v)]}
                ring_f = np.nonzero(np.isin(self.ids, np.unique(self.ids[list(near)])).any(axis=1))[0]
                blocks[ring_f] = per_order[self.g_ring][ring_f]
            touching = np.nonzero(np.isin(self.ids, self.ids[e]).any(axis=1))[0]
            for f in touching:
                if f >= e:
                    singular[(e, f)] = blocks[f] = self.pair_block(e, f)
                else:
                    blocks[f] = singular.pop((f, e)).T
            for f in range(sp.nelem):
                A[np.ix_(dofs[e], dofs[f])] += blocks[f]
        return A

    def mass(self) -> np.ndarray:
        """L^2(Gamma) Gram matrix <phi_i, phi_j> = int phi_hat_i phi_hat_j / |d_s gamma x d_t gamma| ds."""
        from .gauss import tensor2

        sp = self.space
        pts, w = tensor2(sp.d + 4)
        M = np.zeros((sp.ndofs, sp.ndofs))
        for e in range(sp.nelem):
            st = sp.to_patch(e, pts)
            J = sp.geom.jacobian(sp.element(e)[0], st)
            area = np.linalg.norm(np.cross(J[..., 0], J[..., 1]), axis=-1)
            B = sp.element_basis(e, pts)
            de = sp.element_dofs(e)
            M[np.ix_(de, de)] += (B * (w * sp.h**2 / area)[:, None]).T @ B
        return M


def rhs(space, fun, g: int = 6, dtype=float) -> np.ndarray:
    """Load vector b_i = int_square g(gamma(s)) phi_hat_i(s) ds (Sec. 4.4, Piola lift of App. E).

    ``fun`` maps points (n, 3) to values (n,).  Tensor Gauss g x g per element.
    """
    from .gauss import tensor2

    pts, w = tensor2(g)
    b = np.zeros(space.ndofs, dtype=dtype)
    for e in range(space.nelem):
        patch = space.element(e)[0]
        x = space.geom.eval(patch, space.to_patch(e, pts))
        B = space.element_basis(e, pts)
        b[space.element_dofs(e)] += B.T @ (fun(x) * w * space.h**2)
    return b


def potential(space, rho: np.ndarray, pts: np.ndarray, op: str, kappa: complex = 0.0, g: int = 6) -> np.ndarray:
    """u(x) = sum_j rho_j int_square G(x, gamma(t)) phi_hat_j(t) dt (Sec. 4.7; (LS)/(HS)).

    Tensor Gauss g x g per element.
    """
    from .gauss import tensor2

    qp, w = tensor2(g)
    pts = np.asarray(pts, dtype=float)
    u = np.zeros(len(pts), dtype=complex if (op == HELMHOLTZ or np.iscomplexobj(rho)) else float)
    for e in range(space.nelem):
        patch = space.element(e)[0]
        y = space.geom.eval(patch, space.to_patch(e, qp))
        B = space.element_basis(e, qp)
        coeff = B @ rho[space.element_dofs(e)]  # density (pulled back) at the quadrature points
        Gv = green(op, kappa, pts[:, None, :], y[None, :, :])
        u += Gv @ (coeff * w * space.h**2)
    return u
