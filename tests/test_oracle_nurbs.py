"""Pins of the NURBS patch evaluator (rational tensor B-splines) and of its use in
the oracle's Galerkin assembly."""
import numpy as np

from inputs import nurbs_pillow_box
from oracle.galerkin import Assembler, potential, rhs
from oracle.geometry import NurbsSurface
from oracle.space import S2Space


def quarter_cylinder():
    """Rational quadratic quarter circle in s (weights 1, 1/sqrt2, 1) times a line in t."""
    w = np.sqrt(0.5)
    ctrl = np.zeros((2, 3, 4))
    for i2, z in enumerate((0.0, 1.0)):
        ctrl[i2] = [[1, 0, z, 1], [1, 1, z, w], [0, 1, z, 1]]  # (x, y, z, weight)
    return {"degrees": (2, 1), "knots": (np.array([0, 0, 0, 1, 1, 1.0]), np.array([0, 0, 1, 1.0])), "ctrl": ctrl}


def test_rational_quarter_circle_is_exact():
    g = NurbsSurface([quarter_cylinder()])
    st = np.random.default_rng(0).random((50, 2))
    x = g.eval(0, st)
    assert np.abs(np.hypot(x[:, 0], x[:, 1]) - 1.0).max() < 1e-14
    np.testing.assert_allclose(x[:, 2], st[:, 1], atol=1e-14)


def test_affine_invariance():
    pts = nurbs_pillow_box()
    A = np.array([[0.9, 0.1, 0.0], [-0.2, 1.1, 0.3], [0.0, 0.2, 0.8]])
    b = np.array([0.3, -0.1, 2.0])
    moved = []
    for pt in pts:
        c = pt["ctrl"].copy()
        c[..., :3] = c[..., :3] @ A.T + b
        moved.append({**pt, "ctrl": c})
    g0, g1 = NurbsSurface(pts), NurbsSurface(moved)
    st = np.random.default_rng(1).random((40, 2))
    for P in range(6):
        np.testing.assert_allclose(g1.eval(P, st), g0.eval(P, st) @ A.T + b, atol=1e-13)


def test_pillow_box_edges_match():
    """App. D: every patch edge is shared with exactly one other patch, traversed the same way."""
    g = NurbsSurface(nurbs_pillow_box())
    t = np.linspace(0, 1, 9)
    sides = [np.stack([0 * t, t], 1), np.stack([1 + 0 * t, t], 1), np.stack([t, 0 * t], 1), np.stack([t, 1 + 0 * t], 1)]
    for P in range(6):
        for sp in range(4):
            a = g.eval(P, sides[sp])
            hits = [(Q, sq) for Q in range(6) for sq in range(4) if Q != P and np.abs(g.eval(Q, sides[sq]) - a).max() < 1e-12]
            assert len(hits) == 1


def test_point_charge_reproduced_inside_pillow_box():
    """Single-layer solution for g = 1/|x - x0| (x0 outside) reproduces g inside the box."""
    g = NurbsSurface(nurbs_pillow_box())
    x0 = np.array([0.3, 0.2, 3.0])
    f = lambda x: 1.0 / np.linalg.norm(x - x0, axis=-1)  # noqa: E731
    inside = np.array([[0.0, 0.0, 0.0], [0.3, -0.2, 0.4], [-0.5, 0.1, -0.3]])
    errs = []
    for L in (1, 2):
        sp = S2Space(g, L, 0)
        rho = np.linalg.solve(Assembler(sp, "laplace", 0.0, 4, 5).dense(), rhs(sp, f))
        u = potential(sp, rho, inside, "laplace")
        errs.append(np.abs(u - f(inside)).max() / np.abs(f(inside)).max())
    assert errs[1] < 0.02 and errs[1] < errs[0] / 2
