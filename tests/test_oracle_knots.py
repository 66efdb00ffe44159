"""Pins of the S^2 space with repeated interior knots (Sec. 4.3 knotRepetition; App. C, E).

Repeating every interior knot r times lowers the smoothness inside a patch to C^(d-r)
and gives d + 1 + (2^L - 1) r functions per direction; r = d + 1 gives discontinuous
piecewise polynomials.  The recursion of App. C on such knot vectors must agree with
scipy's B-splines, remain a partition of unity, and have exactly the stated
continuity; the Galerkin single-layer matrix on these spaces keeps its structure (SPD)
and its Rayleigh quotients tend to the eigenvalues 1/(2l+1) as for r = 1.
"""
import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle.bspline import bspline_basis, open_knots
from oracle.galerkin import Assembler
from oracle.geometry import Sphere6
from oracle.h2 import H2Oracle
from oracle.space import S2Space


@pytest.mark.parametrize("d,r", [(1, 2), (2, 2), (2, 3), (2, 1)])
def test_basis_matches_scipy_and_partition_of_unity(d, r):
    kn = open_knots(d, 4, r)
    assert len(kn) - d - 1 == d + 1 + 3 * r
    x = np.random.default_rng(0).random(200)
    B = bspline_basis(kn, d, x)
    ref = BSpline.design_matrix(x, kn, d).toarray()
    np.testing.assert_allclose(B, ref, atol=1e-14)
    np.testing.assert_allclose(B.sum(axis=1), 1.0, atol=1e-14)


@pytest.mark.parametrize("d,r", [(2, 1), (2, 2), (2, 3), (1, 2)])
def test_continuity_at_interior_knots(d, r):
    """C^(d-r): values continuous for r <= d, a jump for r = d + 1 (per function)."""
    kn = open_knots(d, 4, r)
    xk = np.array([0.25, 0.5, 0.75])
    eps = 1e-9
    lo, hi = bspline_basis(kn, d, xk - eps), bspline_basis(kn, d, xk + eps)
    jump = np.max(np.abs(hi - lo))
    if r <= d:
        assert jump < 1e-7
    else:
        assert jump > 0.5


def test_space_counts_and_supports():
    for d, r in ((2, 2), (2, 3), (1, 2)):
        sp = S2Space(Sphere6(), 2, d, r)
        assert sp.ndofs == 6 * (d + 1 + 3 * r) ** 2
        seen = np.zeros(sp.ndofs, int)
        for e in range(sp.nelem):
            seen[sp.element_dofs(e)] += 1
        assert seen.min() >= 1  # every function lives on some element
        if r == d + 1:  # discontinuous: every function on exactly one element
            assert seen.max() == 1
    with pytest.raises(ValueError):
        S2Space(Sphere6(), 2, 1, 3)


def test_element_basis_partition_of_unity_with_repeats():
    sp = S2Space(Sphere6(), 2, 2, 2)
    st = np.random.default_rng(1).random((30, 2))
    for e in (0, 5, sp.element_index(3, 3, 1)):
        np.testing.assert_allclose(sp.element_basis(e, st).sum(axis=1), 1.0, atol=1e-14)


def test_galerkin_repeated_knots_spd_and_eigenvalue():
    """Laplace single layer on S^2 with d = 2, r = 2 (C^0 splines), level 1: SPD, and the
    Rayleigh quotient of the l = 1 harmonic z close to 1/3."""
    sp = S2Space(Sphere6(), 1, 2, 2)
    asm = Assembler(sp, "laplace", 0.0, 5, 5)
    A = asm.dense()
    M = asm.mass()
    assert np.allclose(A, A.T, atol=1e-14 * np.abs(A).max())
    assert np.linalg.eigvalsh(A).min() > 0
    from oracle.galerkin import rhs

    c = np.linalg.solve(M, rhs(sp, lambda x: x[:, 2], g=6))
    lam = c @ A @ c / (c @ M @ c)
    assert abs(lam * 3 - 1) < 0.02


def test_h2_rows_with_repeated_knots():
    """Sampled rows of the H^2 approximant equal the rows of its dense reconstruction."""
    sp = S2Space(Sphere6(), 2, 2, 2)
    h2 = H2Oracle(sp, "laplace", q=3, eta=1.6, leaf_level=1, g_reg=3, g_sing=4)
    A = h2.dense()
    x = np.random.default_rng(2).standard_normal(sp.ndofs)
    rows = np.array([0, 7, 31, sp.ndofs - 1])
    np.testing.assert_allclose(h2.apply_rows(x, rows), (A @ x)[rows], rtol=1e-12, atol=1e-13 * np.abs(A @ x).max())
