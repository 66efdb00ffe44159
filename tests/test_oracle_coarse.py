"""Pins of the coarse-space correction (nested S^2 spaces, App. E; the two-level
preconditioner itself is not in the paper).

* The knot-insertion matrix reproduces every coarse B-spline exactly as a combination of
  the fine ones (checked pointwise with scipy's B-splines, an evaluation independent of
  Boehm's algorithm).
* Nesting of the Galerkin matrices: P^T A_L P equals the matrix assembled directly on the
  coarse level, up to quadrature error (both at high orders).
* With A_c = P^T A P the correction C = P A_c^{-1} P^T makes C A a projection that keeps the
  coarse functions: C A P = P and (C A)^2 = C A; a transposed or misplaced P fails these.
"""
import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle.bspline import open_knots
from oracle.coarse import coarse_correction, prolongation, refinement_1d
from oracle.galerkin import Assembler
from oracle.geometry import Sphere6
from oracle.space import S2Space


@pytest.mark.parametrize("d,Lc,L", [(0, 1, 3), (1, 0, 2), (1, 2, 5), (2, 1, 4), (2, 3, 6), (3, 2, 4)])
def test_refinement_reproduces_coarse_splines(d, Lc, L):
    R = refinement_1d(d, Lc, L)
    assert R.shape == (d + 2**L, d + 2**Lc)
    x = np.random.default_rng(d + 10 * L).random(400)
    Bc = BSpline.design_matrix(x, open_knots(d, 2**Lc), d).toarray()
    Bf = BSpline.design_matrix(x, open_knots(d, 2**L), d).toarray()
    np.testing.assert_allclose(Bf @ R, Bc, atol=1e-14)
    assert R.min() >= 0.0  # knot insertion takes convex combinations
    # integrals: int B_j = (t_{j+d+1} - t_j) / (d + 1) on either knot vector
    kc, kf = open_knots(d, 2**Lc), open_knots(d, 2**L)
    ic, jf = (kc[d + 1 :] - kc[: -d - 1]) / (d + 1), (kf[d + 1 :] - kf[: -d - 1]) / (d + 1)
    np.testing.assert_allclose(jf @ R, ic, atol=1e-15)
    # partition of unity is kept: the coarse coefficients 1 map to fine coefficients 1
    np.testing.assert_allclose(R @ np.ones(R.shape[1]), 1.0, atol=1e-14)


def test_prolongation_blocks_and_point_values():
    sc, sf = S2Space(Sphere6(), 1, 2), S2Space(Sphere6(), 2, 2)
    P = prolongation(sc, sf)
    c = np.random.default_rng(4).standard_normal(sc.ndofs)
    f = P @ c
    st = np.random.default_rng(5).random((7, 2))
    for e_f in (0, 21, sf.nelem - 1):
        patch, i1, i2 = sf.element(e_f)
        st_patch = sf.to_patch(e_f, st)
        # the coarse element containing these points, and the points in its local frame
        e_c = sc.element_index(patch, i1 // 2, i2 // 2)
        st_c = st_patch / sc.h - np.array([i1 // 2, i2 // 2])
        v_f = sf.element_basis(e_f, st) @ f[sf.element_dofs(e_f)]
        v_c = sc.element_basis(e_c, st_c) @ c[sc.element_dofs(e_c)]
        np.testing.assert_allclose(v_f, v_c, atol=1e-13)


@pytest.mark.parametrize("op,k", [("laplace", 0.0), ("helmholtz", 2.0)])
def test_galerkin_nesting(op, k):
    sc, sf = S2Space(Sphere6(), 0, 1), S2Space(Sphere6(), 1, 1)
    P = prolongation(sc, sf)
    Af = Assembler(sf, op, k, 10, 10).dense()
    Ac = Assembler(sc, op, k, 10, 10).dense()
    rel = np.max(np.abs(P.T @ Af @ P - Ac)) / np.max(np.abs(Ac))
    assert rel < 1e-6, rel


def test_coarse_correction_is_a_projection():
    sc, sf = S2Space(Sphere6(), 0, 1), S2Space(Sphere6(), 1, 1)
    P = prolongation(sc, sf)
    A = Assembler(sf, "helmholtz", 1.5, 4, 5).dense()
    Ac = P.T @ A @ P
    CA = coarse_correction(P, Ac, A)
    np.testing.assert_allclose(CA @ P, P, atol=1e-11)
    np.testing.assert_allclose(CA @ CA, CA, atol=1e-10 * np.abs(CA).max())
    # a transposed-in-place prolongation (coarse dofs read in the other patch order) breaks it
    perm = np.arange(sc.ndofs).reshape(sc.npatch, sc.n1, sc.n1).transpose(0, 2, 1).ravel()
    Pbad = P[:, perm]
    CAb = coarse_correction(Pbad, Ac, A)
    assert np.max(np.abs(CAb @ Pbad - Pbad)) > 1e-3
