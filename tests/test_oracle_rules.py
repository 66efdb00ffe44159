"""Pins for the element-pair rules (Duffy-type regularisation, Sec. 2 [SS97]).

On flat unit squares in canonical position the rules must reproduce closed
forms of int int 1/|x-y| (tests/flat_pins.py): the identical-square value
(4/3)(1 - sqrt 2) + 4 ln(1 + sqrt 2), the edge- and vertex-adjacent values from
a fourth antiderivative, and weighted integrals (weights on either element)
from the analytic rectangle potential.  A dropped Jacobian factor, a wrong sign
of z or a mis-mapped variable changes these values at O(1e-2) or more.
"""
import numpy as np
import pytest

from flat_pins import pair_integral, weighted_pair_integral
from oracle import quadrature as Q

U = ((0.0, 1.0), (0.0, 1.0))
EDGE_X = ((-1.0, 0.0), (0.0, 1.0))  # first element mirrored: x = (-s1, s2)
VERT_X = ((-1.0, 0.0), (-1.0, 0.0))  # x = (-s1, -s2)


def test_identical_closed_form():
    exact = 4.0 / 3.0 * (1 - np.sqrt(2)) + 4 * np.log(1 + np.sqrt(2))
    assert abs(pair_integral(U, U) - exact) < 1e-14
    S, T, W = Q.rule_identical(10)
    assert abs(W.sum() - 1.0) < 1e-13
    assert abs(np.sum(W / np.linalg.norm(S - T, axis=1)) - exact) < 1e-12


def _edge_xy(S, T):
    return np.stack([-S[:, 0], S[:, 1]], 1), T


def _vert_xy(S, T):
    return -S, T


W_S = lambda p: p[:, 1] ** 2 * (1 + p[:, 0]) + 0.3 * p[:, 1]  # noqa: E731
W_T = lambda p: (1 + p[:, 0]) ** 3 * (2 - p[:, 1])  # noqa: E731


@pytest.mark.parametrize(
    "rule,xy,X,ends_x,ends_y",
    [
        (Q.rule_edge, _edge_xy, EDGE_X, ([0.0], [0.0, 1.0]), ([0.0], [0.0, 1.0])),
        (Q.rule_vertex, _vert_xy, VERT_X, ([0.0], [0.0]), ([0.0], [0.0])),
    ],
)
def test_adjacent_closed_forms(rule, xy, X, ends_x, ends_y):
    S, T, W = rule(10)
    assert abs(W.sum() - 1.0) < 1e-13
    x, y = xy(S, T)
    r = np.linalg.norm(x - y, axis=1)
    assert abs(np.sum(W / r) - pair_integral(X, U)) < 1e-12
    # weight on the first element: outer integral over X of w * potential of U
    ref_s = weighted_pair_integral(X, U, W_S, *ends_x)
    assert abs(np.sum(W * W_S(x) / r) - ref_s) < 1e-10
    # weight on the second element: outer integral over U of w * potential of X
    ref_t = weighted_pair_integral(U, X, W_T, *ends_y)
    assert abs(np.sum(W * W_T(y) / r) - ref_t) < 1e-10


def test_identical_weighted():
    S, T, W = Q.rule_identical(12)
    r = np.linalg.norm(S - T, axis=1)
    ref = weighted_pair_integral(U, U, W_S, [0.0, 1.0], [0.0, 1.0])
    assert abs(np.sum(W * W_S(S) / r) - ref) < 1e-10


def test_regular_rule_separated():
    X = ((2.0, 3.0), (0.5, 1.5))
    S, T, W = Q.rule_regular(10)
    x = S + np.array([2.0, 0.5])
    r = np.linalg.norm(x - T, axis=1)
    assert abs(np.sum(W / r) - pair_integral(X, U)) < 1e-12


@pytest.mark.parametrize("rule", [Q.rule_identical, Q.rule_edge, Q.rule_vertex])
def test_rules_stay_inside(rule):
    S, T, W = rule(5)
    assert np.all((S > 0) & (S < 1)) and np.all((T > 0) & (T < 1)) and np.all(W > 0)


def test_grid4_per_variable_orders():
    """Variable v of the 4-D grid carries its own Gauss order: monomials of
    degree 2 g_v - 1 in variable v are exact, degree 2 g_v is not (so a
    permuted order assignment fails)."""
    from oracle.quadrature import grid4

    orders = (2, 5, 3, 4)
    P, W = grid4(orders)
    assert len(W) == 2 * 5 * 3 * 4
    for v, g in enumerate(orders):
        for deg, exact in ((2 * g - 1, True), (2 * g, False)):
            val = np.sum(W * P[:, v] ** deg)
            assert (abs(val - 1.0 / (deg + 1)) < 1e-13) == exact, (v, g, deg)


@pytest.mark.parametrize("kind,orders", [("identical", (6, 7, 4, 4)), ("edge", (6, 6, 7, 4)), ("vertex", (7, 7, 7, 7))])
def test_anisotropic_rules_match_closed_forms(kind, orders):
    """Per-variable orders (fewer points along the element) still reproduce the
    closed forms of int int 1/|x-y| over flat unit squares in the canonical
    configurations: identical; sharing the edge x1 = 0; sharing the vertex 0."""
    from oracle.quadrature import rule_edge, rule_identical, rule_vertex

    if kind == "identical":
        S, T, W = rule_identical(orders)
        x, y = S, T
        exact = pair_integral(((0, 1), (0, 1)), ((0, 1), (0, 1)))
    elif kind == "edge":
        S, T, W = rule_edge(orders)
        x, y = S * [-1.0, 1.0], T  # mirror the first square across the shared edge
        exact = pair_integral(((-1, 0), (0, 1)), ((0, 1), (0, 1)))
    else:
        S, T, W = rule_vertex(orders)
        x, y = -S, T  # squares meeting at the origin only
        exact = pair_integral(((-1, 0), (-1, 0)), ((0, 1), (0, 1)))
    val = np.sum(W / np.linalg.norm(x - y, axis=1))
    assert abs(val - exact) < 1e-7 * exact


def test_symmetric_per_variable_orders_do_not_depend_on_pair_order():
    """Exchanging the two elements of a touching pair permutes the eta variables
    of the edge and vertex rules; with equal eta orders the block of (f, e) is the
    transpose of the block of (e, f), with unequal ones it is not."""
    from oracle.galerkin import Assembler
    from oracle.geometry import Sphere6
    from oracle.space import S2Space

    sp = S2Space(Sphere6(), 2, 1)
    sym = Assembler(sp, "laplace", 0.0, 3, ((4, 5, 3, 3), (4, 5, 5, 3), (5, 4, 4, 4)))
    asym = Assembler(sp, "laplace", 0.0, 3, ((4, 5, 3, 3), (4, 4, 5, 3), (5, 4, 4, 3)))
    found = {"edge": False, "vertex": False}
    for e in range(sp.nelem):
        for f in range(sp.nelem):
            kind = sym.classify(e, f)[0]
            if kind not in found or found[kind]:
                continue
            a, b = sym.pair_block(e, f), sym.pair_block(f, e).T
            assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()  # rounding only
            c, d = asym.pair_block(e, f), asym.pair_block(f, e).T
            assert np.abs(c - d).max() > 1e-9 * np.abs(c).max()
            found[kind] = True
        if all(found.values()):
            break
    assert all(found.values())
