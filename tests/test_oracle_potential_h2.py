"""Pins of the compressed potential evaluation (oracle.potential_h2) and the sphere grid.

* With no admissible cluster (eta -> 0) the descent reaches every leaf and the result is
  the plain Gauss potential of oracle.galerkin.potential, to rounding.
* With eta = 1.6 the error against that plain potential falls as the interpolation order q
  grows (Sec. 2: far-field interpolation on the parameter square).
* The sphere grid of Sec. 5 (Util::makeSphereGrid): points at the given radius, n circles
  of latitude with n equally spaced points each.
"""
import numpy as np
import pytest

from inputs import ball_points
from oracle.galerkin import potential
from oracle.geometry import Sphere6
from oracle.potential_h2 import h2_potential, sphere_grid
from oracle.space import S2Space


@pytest.fixture(scope="module")
def setup():
    sp = S2Space(Sphere6(), 3, 1)
    # a smooth density: f(x) = 1 + 0.5 x + 0.3 y z at the degree-1 Greville points (j1, j2) / 2^L
    j = np.arange(sp.ndofs)
    patch, rem = np.divmod(j, sp.n1 * sp.n1)
    j2, j1 = np.divmod(rem, sp.n1)
    x = np.concatenate([sp.geom.eval(p, np.stack([j1[patch == p], j2[patch == p]], 1) * sp.h) for p in range(6)])
    rho = 1.0 + 0.5 * x[:, 0] + 0.3 * x[:, 1] * x[:, 2]
    pts = np.concatenate([sphere_grid(1.6, 5), ball_points(10, 0.5, 2)])
    return sp, rho, pts


def test_no_admissible_cluster_is_plain_potential(setup):
    sp, rho, pts = setup
    ref = potential(sp, rho, pts, "laplace", g=4)
    u = h2_potential(sp, rho, pts, "laplace", q=3, eta=1e-12, leaf_level=2, g=4)
    np.testing.assert_allclose(u, ref, rtol=1e-13, atol=1e-14 * np.abs(ref).max())


def test_interpolation_error_falls_with_q(setup):
    sp, rho, pts = setup
    ref = potential(sp, rho, pts, "laplace", g=4)
    errs = [np.max(np.abs(h2_potential(sp, rho, pts, "laplace", q=q, eta=1.6, leaf_level=2, g=4) - ref))
            / np.max(np.abs(ref)) for q in (2, 3, 4, 5)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[0] > 1e-4 and errs[-1] < 1e-5, errs


def test_helmholtz_no_admissible_cluster(setup):
    sp, rho, pts = setup
    ref = potential(sp, rho.astype(complex), pts[:8], "helmholtz", 2.0, g=4)
    u = h2_potential(sp, rho.astype(complex), pts[:8], "helmholtz", 2.0, q=3, eta=1e-12, leaf_level=2, g=4)
    np.testing.assert_allclose(u, ref, rtol=1e-13, atol=1e-14 * np.abs(ref).max())


def test_sphere_grid():
    p = sphere_grid(6.0, 10)
    assert p.shape == (100, 3)
    np.testing.assert_allclose(np.linalg.norm(p, axis=1), 6.0, rtol=1e-15)
    z = p[:, 2].reshape(10, 10)
    assert np.allclose(z, z[:, :1]) and len(np.unique(np.round(z[:, 0], 12))) == 10  # 10 circles of latitude
    ang = np.arctan2(p[:, 1], p[:, 0]).reshape(10, 10)
    d = np.mod(np.diff(ang, axis=1), 2 * np.pi)
    np.testing.assert_allclose(d, 2 * np.pi / 10, atol=1e-12)  # 10 equally spaced points on each
