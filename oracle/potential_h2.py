"""Compressed potential evaluation through the cluster tree (test infrastructure).

Sec. 4.7 (``Sol::evalSolution``): u(x) = sum_j rho_j int_square G(x, gamma(t)) phi_hat_j(t) dt
at evaluation points x off the surface.  Many points are evaluated with the far-field
machinery of Sec. 2: the kernel G(x, .) is interpolated on a source cluster's parameter
square at the q x q Chebyshev points wherever the cluster is admissible for the point,

    int_sigma G(x, gamma(t)) rho(t) dt  ~  sum_b G(x, gamma(x_b^sigma)) rhohat_sigma[b],
    rhohat_sigma[b] = sum_{f in sigma} sum_j rho_j int_f phi_hat_j L_b^sigma dt,

and elements of non-admissible leaf clusters are integrated by the g x g Gauss rule of
``oracle.galerkin.potential``.  Readings (the paper gives none for the point evaluation):

* The point/cluster admissibility is that of the block tree with a point as target (a ball
  of radius 0): diam(sigma) = 2 r_sigma <= eta * max(0, |x - c_sigma| - r_sigma), same
  bounding balls (``oracle.h2.Clusters``) and eta.
* The descent starts from the six patch clusters; a non-admissible cluster above the leaf
  level passes on to its four children; a non-admissible leaf is integrated directly.

Every cluster moment is integrated directly (``H2Oracle.moment``), with no transfers.
"""
from __future__ import annotations

import numpy as np

from .galerkin import green
from .gauss import tensor2
from .h2 import H2Oracle, cluster_elements


def h2_potential(space, rho, pts, op: str, kappa: complex = 0.0, q: int = 4, eta: float = 1.6,
                 leaf_level: int | None = None, g: int = 6, kdiam: float = 0.0) -> np.ndarray:
    """u~(x) at every point of pts (n, 3) for the density rho (global S^2 coefficients).
    kdiam > 0 (Helmholtz): a cluster is admissible only if also |kappa| diam <= kdiam, the
    block tree's limit on the kernel's oscillation."""
    h2 = H2Oracle(space, op, kappa, q=q, eta=eta, leaf_level=leaf_level)
    leaf = h2.leaf
    cl = h2.cl
    pts = np.asarray(pts, dtype=float)
    cplx = op == "helmholtz" or np.iscomplexobj(rho)
    u = np.zeros(len(pts), dtype=complex if cplx else float)
    qp, w = tensor2(g)
    elem_cache: dict[int, tuple] = {}

    def elem(e):  # quadrature points of element e and the density times the weights there
        if e not in elem_cache:
            patch = space.element(e)[0]
            y = space.geom.eval(patch, space.to_patch(e, qp))
            dens = space.element_basis(e, qp) @ rho[space.element_dofs(e)]
            elem_cache[e] = (y, dens * w * space.h**2)
        return elem_cache[e]

    rhohat: dict = {}

    def moment_of(c):  # rhohat_c, length q^2
        if c not in rhohat:
            acc = 0.0
            for f in cluster_elements(space, c):
                acc = acc + h2.moment(f, c).T @ rho[space.element_dofs(f)]
            rhohat[c] = acc
        return rhohat[c]

    nodes: dict = {}

    def nodes_of(c):
        if c not in nodes:
            nodes[c] = space.geom.eval(c[0], h2.cluster_nodes(c))
        return nodes[c]

    for i, x in enumerate(pts):
        acc = 0.0
        stack = [(p, 0, 0, 0) for p in range(space.npatch)]
        while stack:
            c = stack.pop()
            ctr, r = cl.ball(c)
            dist = max(0.0, float(np.linalg.norm(x - ctr)) - r)
            osc_ok = not (op == "helmholtz" and kdiam > 0) or abs(kappa) * 2.0 * r <= kdiam
            if osc_ok and 2.0 * r <= eta * dist:
                acc = acc + green(op, kappa, x[None, :], nodes_of(c)) @ moment_of(c)
            elif c[1] == leaf:
                for f in cluster_elements(space, c):
                    y, dw = elem(f)
                    acc = acc + green(op, kappa, x[None, :], y) @ dw
            else:
                patch, lev, i1, i2 = c
                stack.extend((patch, lev + 1, 2 * i1 + a, 2 * i2 + b) for b in range(2) for a in range(2))
        u[i] = acc
    return u


def sphere_grid(radius: float, n: int) -> np.ndarray:
    """n points on each of n circles of latitude of the sphere of the given radius about the
    origin (Sec. 5, ``Util::makeSphereGrid``): polar angles pi (i + 1/2) / n, azimuths
    2 pi j / n, point i n + j."""
    th = np.pi * (np.arange(n) + 0.5) / n
    ph = 2 * np.pi * np.arange(n) / n
    T, P = np.meshgrid(th, ph, indexing="ij")
    return radius * np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)
