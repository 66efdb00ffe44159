"""Pins of the EFIE oracle: S^1 basis (derivatives, glue, div-conformity),
Galerkin form (complex symmetry), field evaluation (gradient term), and the
whole chain against the Mie series of a perfectly conducting sphere."""
import functools
import os

import numpy as np
import pytest
from scipy.interpolate import BSpline

from mie import incident_series_bh, scattered_pec
from oracle.bspline import bspline_deriv, open_knots
from oracle.efie import EfieAssembler, efie_field, efie_rhs
from oracle.geometry import Sphere6
from oracle.space_s1 import S1Space


@pytest.mark.parametrize("p,n_el", [(1, 4), (2, 4), (3, 2)])
def test_bspline_derivative(p, n_el):
    kn = open_knots(p, n_el)
    x = np.linspace(0.0, 1.0, 37)
    d = bspline_deriv(kn, p, x)
    n = len(kn) - p - 1
    for j in range(n):
        c = np.zeros(n)
        c[j] = 1.0
        ref = BSpline(kn, c, p).derivative()(x)
        # scipy evaluates x = 1 from the left, as the recursion's convention does
        np.testing.assert_allclose(d[:, j], ref, atol=1e-12)


@pytest.mark.parametrize("L,p", [(0, 1), (2, 1), (1, 2), (4, 2)])
def test_s1_dof_count(L, p):
    sp = S1Space(Sphere6(), L, p)
    n_el = 2**L
    per_edge = n_el + p - 1
    assert sp.ndofs == 6 * 2 * (n_el + p) * (n_el + p - 1) - 12 * per_edge
    if (L, p) == (4, 2):
        assert sp.ndofs == 3468


def _field_at(sp, patch, st, gdof):
    """Physical field of global function gdof on one patch at patch parameters st (n,2)."""
    J = sp.geom.jacobian(patch, st)
    det = np.linalg.norm(np.cross(J[..., 0], J[..., 1]), axis=-1)
    out = np.zeros((len(st), 3))
    for i, loc in enumerate(range(sp.per_patch)):
        if sp.gid[patch, loc] != gdof:
            continue
        # evaluate this patch-local function through any element containing each point
        for k, s in enumerate(st):
            i1 = min(int(s[0] * sp.n_el), sp.n_el - 1)
            i2 = min(int(s[1] * sp.n_el), sp.n_el - 1)
            e = patch * sp.n_el**2 + i2 * sp.n_el + i1
            locs = sp.local_patch_indices(e)
            hit = np.nonzero(locs == loc)[0]
            if len(hit) == 0:
                continue
            V, _ = sp.element_basis(e, (s / sp.h - [i1, i2])[None, :])
            out[k] += sp.coef[patch, loc] * (J[k] @ V[0, hit[0]]) / det[k]
    return out


def test_normal_flux_continuous_across_patch_edges():
    """Glued edge functions have equal normal components from both sides (div-conformity)."""
    sp = S1Space(Sphere6(), 1, 2)
    tpar = np.array([0.1, 0.37, 0.5, 0.81])
    checked = 0
    for P in range(6):
        # side s = 1 of patch P, points along t
        stA = np.stack([np.ones_like(tpar), tpar], axis=1)
        xA = sp.geom.eval(P, stA)
        JA = sp.geom.jacobian(P, stA)
        nu = JA[..., 0] / np.linalg.norm(JA[..., 0], axis=1)[:, None]  # crosses the edge
        nrm = np.cross(JA[..., 0], JA[..., 1])
        nrm /= np.linalg.norm(nrm, axis=1)[:, None]
        nu = nu - np.sum(nu * nrm, axis=1)[:, None] * nrm  # in-surface, orthogonal to... projected
        tang = JA[..., 1] / np.linalg.norm(JA[..., 1], axis=1)[:, None]
        nu = nu - np.sum(nu * tang, axis=1)[:, None] * tang
        nu /= np.linalg.norm(nu, axis=1)[:, None]
        # the neighbour patch and its parameters of the same physical points
        for Q in range(6):
            if Q == P:
                continue
            best = None
            for side in range(4):
                g = np.linspace(0, 1, 201)
                edge = {0: np.stack([0 * g, g], 1), 1: np.stack([1 + 0 * g, g], 1), 2: np.stack([g, 0 * g], 1),
                        3: np.stack([g, 1 + 0 * g], 1)}[side]
                xe = sp.geom.eval(Q, edge)
                dist = np.linalg.norm(xA[:, None, :] - xe[None, :, :], axis=2).min(axis=1)
                if dist.max() < 1e-2:
                    best = side
            if best is None:
                continue
            # refine: solve for Q's edge parameter of each point by dense search + Newton-free refinement
            g = np.linspace(0, 1, 200001)
            edge = {0: np.stack([0 * g, g], 1), 1: np.stack([1 + 0 * g, g], 1), 2: np.stack([g, 0 * g], 1),
                    3: np.stack([g, 1 + 0 * g], 1)}[best]
            xe = sp.geom.eval(Q, edge)
            stB = edge[[np.argmin(np.linalg.norm(xe - x, axis=1)) for x in xA]]
            gd = [d for d in np.unique(sp.gid[P]) if d in set(sp.gid[Q].tolist())]
            for d in gd:
                fa = _field_at(sp, P, stA, d)
                fb = _field_at(sp, Q, stB, d)
                np.testing.assert_allclose(np.sum(fa * nu, 1), np.sum(fb * nu, 1), atol=2e-4)
                checked += 1
    assert checked >= 6 * (sp.nq)


def test_divergence_theorem():
    """Every global function is a closed-surface div-conforming field: int_Gamma div_Gamma j = 0."""
    from oracle.gauss import tensor2

    sp = S1Space(Sphere6(), 1, 2)
    pts, w = tensor2(4)
    tot = np.zeros(sp.ndofs)
    for e in range(sp.nelem):
        _, D = sp.element_basis(e, pts)
        ge, ce = sp.element_dofs(e)
        np.add.at(tot, ge, ce * (D.T @ (w * sp.h**2)))
    assert np.abs(tot).max() < 1e-13


def test_efie_matrix_complex_symmetric():
    A = EfieAssembler(S1Space(Sphere6(), 1, 1), 2.0, 3, 4).dense()
    assert np.abs(A - A.T).max() < 1e-13 * np.abs(A).max()
    assert np.abs(A - A.conj().T).max() > 1e-3 * np.abs(A).max()  # not Hermitian


def test_field_gradient_term():
    """efie_field's kappa^-2 grad term matches a central difference of the scalar potential."""
    from oracle.gauss import tensor2

    sp = S1Space(Sphere6(), 0, 1)
    k = 1.7
    rho = np.random.default_rng(3).standard_normal(sp.ndofs) + 0j
    x0 = np.array([[0.3, -2.1, 1.2]])

    def scalar_pot(x):
        qp, w = tensor2(6)
        u = 0j
        for e in range(sp.nelem):
            patch = sp.element(e)[0]
            y = sp.geom.eval(patch, sp.to_patch(e, qp))
            _, D = sp.element_basis(e, qp)
            ge, ce = sp.element_dofs(e)
            r = np.linalg.norm(x - y, axis=1)
            u += np.sum(np.exp(-1j * k * r) / (4 * np.pi * r) * (D @ (ce * rho[ge])) * w * sp.h**2)
        return u

    # vector part alone: field of rho minus the gradient part computed by differences
    E = efie_field(sp, rho, x0, k)[0]
    hstep = 1e-4
    grad = np.array([(scalar_pot(x0[0] + hstep * ei) - scalar_pot(x0[0] - hstep * ei)) / (2 * hstep)
                     for ei in np.eye(3)])
    # vector part by direct quadrature
    qp, w = tensor2(6)
    vec = np.zeros(3, dtype=complex)
    for e in range(sp.nelem):
        patch = sp.element(e)[0]
        st = sp.to_patch(e, qp)
        y = sp.geom.eval(patch, st)
        J = sp.geom.jacobian(patch, st)
        V, _ = sp.element_basis(e, qp)
        ge, ce = sp.element_dofs(e)
        jv = np.einsum("kca,kia,i->kc", J, V, ce * rho[ge])
        r = np.linalg.norm(x0[0] - y, axis=1)
        vec += np.einsum("k,kc->c", np.exp(-1j * k * r) / (4 * np.pi * r) * w * sp.h**2, jv)
    np.testing.assert_allclose(E, vec + grad / k**2, rtol=1e-6)


def test_mie_helper_pins():
    """The Mie helper reproduces the incident plane wave and the PEC boundary condition."""
    rng = np.random.default_rng(0)
    pts = rng.standard_normal((20, 3))
    pts *= (1.5 / np.linalg.norm(pts, axis=1))[:, None]
    k = 2.0
    ref = np.zeros((20, 3), dtype=complex)
    ref[:, 0] = np.exp(1j * k * pts[:, 2])
    assert np.abs(incident_series_bh(pts, k) - ref).max() < 1e-8
    p1 = rng.standard_normal((30, 3))
    p1 /= np.linalg.norm(p1, axis=1)[:, None]
    tot = scattered_pec(p1, k)
    tot[:, 0] += np.exp(-1j * k * p1[:, 2])
    tang = tot - np.sum(tot * p1, axis=1)[:, None] * p1
    assert np.abs(tang).max() < 1e-10


@functools.lru_cache(maxsize=None)
def _mie_error(L, p):
    """Relative error of the oracle's scattered field (plane wave along z, x-polarised,
    k = 2) at 20 points on the sphere of radius 3 against the Mie series."""
    k = 2.0
    rng = np.random.default_rng(4)
    pts = rng.standard_normal((20, 3))
    pts *= (3.0 / np.linalg.norm(pts, axis=1))[:, None]
    ref = scattered_pec(pts, k)
    einc = lambda x: np.stack([np.exp(-1j * k * x[:, 2]), 0 * x[:, 0], 0 * x[:, 0]], axis=1)  # noqa: E731
    sp = S1Space(Sphere6(), L, p)
    rho = np.linalg.solve(EfieAssembler(sp, k, 4, 5).dense(), efie_rhs(sp, einc))
    return np.linalg.norm(efie_field(sp, rho, pts, k) - ref) / np.linalg.norm(ref)


def test_efie_converges_to_mie():
    assert _mie_error(1, 1) < 0.1 and _mie_error(0, 1) / _mie_error(1, 1) > 5.0
    assert _mie_error(1, 2) < _mie_error(1, 1)


@pytest.mark.slow
def test_efie_convergence_orders_of_the_paper():
    """Observed orders of the scattered-field error under uniform refinement against
    the orders 2P + 1 the paper prints (tests/golden/efie_convergence_orders.txt):
    P = 1 fitted over levels 0..2 (about 2.9), P = 2 from level 1 to 2 (about 4.7,
    level 0 is pre-asymptotic)."""
    table = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "efie_convergence_orders.txt"))
    order = {int(P): o for P, o in table}
    e1 = [np.log2(_mie_error(L, 1)) for L in (0, 1, 2)]
    slope1 = -np.polyfit([0, 1, 2], e1, 1)[0]
    assert abs(slope1 - order[1]) < 0.5, slope1
    slope2 = np.log2(_mie_error(1, 2) / _mie_error(2, 2))
    assert abs(slope2 - order[2]) < 1.0, slope2


def test_compressed_efie_converges_to_dense():
    """The H^2 EFIE (Jacobian factors interpolated with G) approaches the dense EFIE as q grows."""
    from oracle.efie import EfieH2Oracle

    sp = S1Space(Sphere6(), 2, 1)
    A = EfieAssembler(sp, 2.0, 3, 4).dense()
    errs = []
    for q in (3, 5):
        h2 = EfieH2Oracle(sp, 2.0, q=q, eta=1.6, leaf_level=1, g_reg=3, g_sing=4)
        assert len(h2.far) > 0
        errs.append(np.abs(h2.dense() - A).max() / np.abs(A).max())
    assert errs[1] < errs[0] / 20 and errs[1] < 1e-4, errs
