"""Pins for the oracle's Galerkin operators on the unit sphere (App. B).

* Laplace single layer: S Y_lm = Y_lm / (2l + 1) on the unit sphere.
* Helmholtz single layer with the paper's kernel exp(-i kappa r)/(4 pi r):
  S Y_lm = -i k j_l(k) h_l^(2)(k) Y_lm.
Rayleigh quotients of the L^2-projected harmonics converge to these at the
projection-error rate h^(2(d+1)).
* Interior Dirichlet problem with u = 1/|x - x0|, x0 = (0,0,2) (LP, Remark in
  App. B): the single-layer potential reproduces u inside the ball.
* Exterior Helmholtz problem with a point source inside (HP): reproduces the
  source's field outside.
* Symmetry of the bilinear form: the block of (f, e) integrated from f's side
  equals the transposed block of (e, f); the Laplace matrix is SPD.
"""
import numpy as np
import pytest

from inputs import ball_points, sphere_points
from oracle.galerkin import Assembler, potential, rhs
from oracle.geometry import Sphere6
from oracle.space import S2Space
from sph import helmholtz_sl_eig, real_ylm

_cache = {}


def system(L, d, op, k=0.0, g_reg=4, g_sing=6):
    key = (L, d, op, k, g_reg, g_sing)
    if key not in _cache:
        sp = S2Space(Sphere6(), L, d)
        asm = Assembler(sp, op, k, g_reg, g_sing)
        _cache[key] = (sp, asm, asm.dense(), asm.mass())
    return _cache[key]


def rayleigh(L, d, op, k, l, m):
    sp, asm, A, M = system(L, d, op, k)
    c = np.linalg.solve(M, rhs(sp, lambda x: real_ylm(l, m, x)))
    return (c @ A @ c) / (c @ M @ c)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_laplace_eigenvalues(d):
    for l in range(4):
        lam = rayleigh(2, d, "laplace", 0.0, l, min(l, 1))
        err = abs(lam - 1.0 / (2 * l + 1)) * (2 * l + 1)
        assert err < [0.15, 0.02, 0.006][d], (l, err)


def test_laplace_eigenvalue_convergence_p0():
    for l in range(3):
        e2 = abs(rayleigh(2, 0, "laplace", 0.0, l, 0) * (2 * l + 1) - 1)
        e3 = abs(rayleigh(3, 0, "laplace", 0.0, l, 0) * (2 * l + 1) - 1)
        assert e3 < e2 / 3.0 and e3 < 0.04


@pytest.mark.parametrize("k", [1.0, 2.5])
def test_helmholtz_eigenvalues(k):
    for l in range(4):
        lam = rayleigh(2, 1, "helmholtz", k, l, 0)
        ex = helmholtz_sl_eig(l, k)
        assert abs(lam - ex) / abs(ex) < 0.02, (l, lam, ex)
        # the kernel sign fixes the sign of the imaginary part (exp(+ikr) would conjugate it)
        if l <= 1:
            assert abs(lam.imag - ex.imag) < 0.1 * abs(ex.imag), (l, lam, ex)


def test_laplace_spd_and_pair_symmetry():
    sp, asm, A, M = system(2, 1, "laplace")
    assert np.max(np.abs(A - A.T)) < 1e-15
    assert np.linalg.eigvalsh(A).min() > 0
    for e, f in [(0, 1), (0, 4), (0, 5), (3, 17), (10, 40), (5, 77)]:
        a = asm.pair_block(e, f)
        b = asm.pair_block(f, e).T
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-13 * np.abs(a).max())


def test_point_charge_interior_ball():
    """Interior Dirichlet problem of the dense Laplace workload (level 3, degree 0)."""
    x0 = np.array([0.0, 0.0, 2.0])
    pts = ball_points(100, 0.5, 1)
    exact = 1.0 / np.linalg.norm(pts - x0, axis=1)
    errs = []
    for L in (2, 3):
        sp, asm, A, M = system(L, 0, "laplace")
        b = rhs(sp, lambda x: 1.0 / np.linalg.norm(x - x0, axis=1))
        rho = np.linalg.solve(A, b)
        u = potential(sp, rho, pts, "laplace")
        errs.append(np.max(np.abs(u - exact) / exact))
    assert errs[1] < 5e-4 and errs[1] < errs[0] / 5, errs


def test_helmholtz_exterior_point_source():
    k = 2.0
    src = np.array([0.1, -0.2, 0.15])
    G = lambda x: np.exp(-1j * k * np.linalg.norm(x - src, axis=1)) / (4 * np.pi * np.linalg.norm(x - src, axis=1))  # noqa: E731
    pts = sphere_points(20, 3.0, 7)
    sp, asm, A, M = system(2, 1, "helmholtz", k)
    b = rhs(sp, G, dtype=complex)
    rho = np.linalg.solve(A, b)
    u = potential(sp, rho, pts, "helmholtz", k)
    assert np.max(np.abs(u - G(pts)) / np.abs(G(pts))) < 2e-3


def test_ring_classification_matches_index_distance():
    """Inside one patch (away from its boundary) a separated pair lies in the ring
    next to the touching pairs exactly when the elements are two steps apart in
    the index grid (Chebyshev distance 2)."""
    from oracle.galerkin import Assembler
    from oracle.geometry import Sphere6
    from oracle.space import S2Space

    sp = S2Space(Sphere6(), 3, 0)
    asm = Assembler(sp, "laplace", 0.0, (4, 3), 4)
    n = sp.n_el
    for e in range(sp.nelem):
        pe, i1, i2 = sp.element(e)
        if pe != 0 or not (2 <= i1 < n - 2 and 2 <= i2 < n - 2):
            continue
        for f in range(sp.nelem):
            pf, j1, j2 = sp.element(f)
            if pf != 0:
                continue
            dist = max(abs(i1 - j1), abs(i2 - j2))
            if dist >= 2:
                assert asm.ring(e, f) == (dist == 2)


def test_graded_separated_orders_dense_matches_pairwise():
    """The vectorised dense assembly picks the ring order for ring pairs and the far order
    for the others, as the pair-by-pair blocks do."""
    from oracle.galerkin import Assembler
    from oracle.geometry import Sphere6
    from oracle.space import S2Space

    sp = S2Space(Sphere6(), 2, 1)
    asm = Assembler(sp, "laplace", 0.0, (5, 2), 4)
    A = asm.dense()
    rng = np.random.default_rng(0)
    checked = {True: 0, False: 0}
    for _ in range(400):
        e, f = rng.integers(0, sp.nelem, 2)
        if asm.classify(e, f)[0] != "regular":
            continue
        blk = asm.pair_block(e, f)
        ring = asm.ring(e, f)
        g = 5 if ring else 2
        ref = Assembler(sp, "laplace", 0.0, g, 4).pair_block(e, f)
        assert np.abs(blk - ref).max() < 1e-15 * np.abs(ref).max() + 1e-300
        checked[ring] += 1
    assert checked[True] > 0 and checked[False] > 0
    # dense = sum of pair blocks (spot check one row against the pairwise sum)
    row = 7
    acc = np.zeros(sp.ndofs)
    for e in range(sp.nelem):
        de = sp.element_dofs(e)
        if row not in de:
            continue
        i = int(np.nonzero(de == row)[0][0])
        for f in range(sp.nelem):
            acc[sp.element_dofs(f)] += asm.pair_block(e, f)[i]
    assert np.abs(acc - A[row]).max() < 1e-13 * np.abs(A[row]).max()
