"""Pins for the oracle's building blocks: Gauss rules, B-splines (App. C), the
6-patch sphere and its topology (App. D)."""
import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle.bspline import bspline_basis, open_knots
from oracle.gauss import gauss_legendre01
from oracle.geometry import Sphere6
from oracle.space import S2Space
from oracle.topology import canonical_maps, corner_ids


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 13, 20])
def test_gauss_matches_library(n):
    x, w = gauss_legendre01(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, 0.5 * (xr + 1), atol=1e-15)
    np.testing.assert_allclose(w, 0.5 * wr, atol=1e-15)
    # exact for degree 2n-1 on [0,1]
    for k in range(2 * n):
        assert abs(np.sum(w * x**k) - 1.0 / (k + 1)) < 1e-14


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
@pytest.mark.parametrize("nel", [1, 4, 8])
def test_bspline_matches_library_and_partition(deg, nel):
    kn = open_knots(deg, nel)
    x = np.linspace(0, 1, 97)
    B = bspline_basis(kn, deg, x)
    assert B.shape == (97, nel + deg)
    np.testing.assert_allclose(B.sum(1), 1.0, atol=1e-14)  # partition of unity incl. x = 1
    for j in range(nel + deg):
        c = np.zeros(nel + deg)
        c[j] = 1
        ref = BSpline(kn, c, deg, extrapolate=False)(x[:-1])
        np.testing.assert_allclose(B[:-1, j], np.nan_to_num(ref), atol=1e-14)


def test_sphere6_geometry():
    g = Sphere6()
    rng = np.random.default_rng(0)
    st = rng.random((50, 2))
    for p in range(6):
        x = g.eval(p, st)
        np.testing.assert_allclose(np.linalg.norm(x, axis=1), 1.0, atol=1e-15)
        J = g.jacobian(p, st)
        n = np.cross(J[..., 0], J[..., 1])
        assert np.all(np.sum(n * x, axis=1) > 0), "outward normal (App. D)"
        hh = 1e-6
        for a in range(2):
            d = np.zeros(2)
            d[a] = hh
            fd = (g.eval(p, st + d) - g.eval(p, st - d)) / (2 * hh)
            np.testing.assert_allclose(J[..., a], fd, atol=1e-8)


def test_sphere6_conforming_mesh():
    """Patches meet at full edges; each element edge is shared by exactly two
    elements and each vertex by 3 (cube corners) or 4 elements (App. D)."""
    sp = S2Space(Sphere6(), 2, 0)
    ids = corner_ids(sp)
    nv = ids.max() + 1
    assert nv == 6 * 16 + 2  # Euler: V - E + F = 2 with F = 96, E = 192
    counts = np.bincount(ids.ravel())
    assert sorted(set(counts.tolist())) == [3, 4]
    assert np.sum(counts == 3) == 8
    edges = {}
    for e in range(sp.nelem):
        for a, b in ((0, 1), (0, 2), (1, 3), (2, 3)):
            key = tuple(sorted((ids[e, a], ids[e, b])))
            edges[key] = edges.get(key, 0) + 1
    assert set(edges.values()) == {2}
    # matching condition: on a shared edge the canonical maps give the same point
    kinds = {"identical": 0, "edge": 0, "vertex": 0, "regular": 0}
    u = np.stack([np.zeros(7), np.linspace(0, 1, 7)], 1)
    for e in range(sp.nelem):
        for f in range(sp.nelem):
            kind, me, mf = canonical_maps(ids[e], ids[f])
            kinds[kind] += 1
            if kind in ("edge", "vertex"):
                from oracle.topology import apply_map

                pe = sp.geom.eval(sp.element(e)[0], sp.to_patch(e, apply_map(me, u if kind == "edge" else u[:1])))
                pf = sp.geom.eval(sp.element(f)[0], sp.to_patch(f, apply_map(mf, u if kind == "edge" else u[:1])))
                np.testing.assert_allclose(pe, pf, atol=1e-14)
    assert kinds["identical"] == 96 and kinds["edge"] == 4 * 96
    assert kinds["vertex"] == 4 * 96 - 8 * 3 * 1  # 8 cube corners: 3 elements, each missing one diagonal neighbour
