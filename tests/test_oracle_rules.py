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
