"""Pins of the converged element-pair reference (oracle.converged) and, through it, of the
oracle's Duffy-type rules on curved elements.

oracle.converged integrates element pairs without any of the regularising transforms of
oracle.quadrature (polar coordinates around the nearest point with sinh substitutions,
tanh-sinh outer rules).  It must

* reproduce the closed forms of int int 1/|x - y| over flat squares (identical, common
  edge, common vertex; tests/flat_pins.py), with polynomial weights on either element;
* agree with the Duffy rules of oracle.quadrature at high order on curved sphere elements
  (inside a patch and across patch edges, Laplace and Helmholtz).

A wrong canonical map, a dropped Jacobian factor or a mis-oriented edge in either code
changes these blocks at 1e-3 or more; the agreement required is 1e-9.
"""
import numpy as np
import pytest

from flat_pins import pair_integral, weighted_pair_integral
from oracle import converged as CV
from oracle.galerkin import Assembler
from oracle.geometry import Sphere6
from oracle.space import S2Space

U = ((0.0, 1.0), (0.0, 1.0))


def _flat(st):
    st = np.atleast_2d(st)
    return np.concatenate([st, np.zeros((len(st), 1))], 1)


def _one(st):
    return np.ones((len(np.atleast_2d(st)), 1))


def _ker(x, y):
    return 1.0 / np.linalg.norm(x - y, axis=-1)


W_S = lambda p: p[:, 1] ** 2 * (1 + p[:, 0]) + 0.3 * p[:, 1]  # noqa: E731
W_T = lambda p: (1 + p[:, 0]) ** 3 * (2 - p[:, 1])  # noqa: E731


def _block(xe, be, xf, bf, kind, shared=()):
    return CV.pair_block(xe, be, xf, bf, _ker, kind, shared, r=1).real[0, 0]


def test_identical_flat_square():
    exact = 4.0 / 3.0 * (1 - np.sqrt(2)) + 4 * np.log(1 + np.sqrt(2))
    assert abs(_block(_flat, _one, _flat, _one, "identical") - exact) < 1e-11


@pytest.mark.parametrize("kind", ["edge", "vertex"])
def test_adjacent_flat_squares(kind):
    # first element mirrored into x1 < 0 (edge) or x1, x2 < 0 (vertex); shared set at its local 0
    if kind == "edge":
        X, sign, shared, ends = ((-1.0, 0.0), (0.0, 1.0)), np.array([-1.0, 1.0]), [(0, 0), (0, 1)], ([0.0], [0.0, 1.0])
    else:
        X, sign, shared, ends = ((-1.0, 0.0), (-1.0, 0.0)), np.array([-1.0, -1.0]), [(0, 0)], ([0.0], [0.0])
    xe = lambda st: _flat(np.atleast_2d(st) * sign)  # noqa: E731
    assert abs(_block(xe, _one, _flat, _one, kind, shared) - pair_integral(X, U)) < 1e-11
    # weights on the first element (functions of the physical point) and on the second
    ws = _block(xe, lambda st: W_S(xe(st))[:, None], _flat, _one, kind, shared)
    assert abs(ws - weighted_pair_integral(X, U, W_S, *ends)) < 1e-10
    wt = _block(xe, _one, _flat, lambda st: W_T(st)[:, None], kind, shared)
    # at refinement 1 the cubic weight on the second element is converged to ~2e-10
    assert abs(wt - weighted_pair_integral(U, X, W_T, *ends)) < 1e-9


def _curved_pairs(sp):
    """(e, f, class) on the level-2 sphere: one pair per touching class inside patch 0, and a
    common edge and a common vertex across patch boundaries."""
    e = sp.element_index(0, 1, 1)
    out = {}
    for f in range(sp.nelem):
        kind, _ = CV.pair_kind(sp, e, f)
        out.setdefault(kind, (e, f))
    e2 = sp.element_index(0, 0, 0)
    for f in range(sp.nelem):
        if sp.element(f)[0] != 0:
            kind, _ = CV.pair_kind(sp, e2, f)
            if kind in ("edge", "vertex"):
                out.setdefault("cross-" + kind, (e2, f))
    return out


@pytest.mark.parametrize("op,k", [("laplace", 0.0), ("helmholtz", 4.0)])
def test_curved_blocks_match_duffy_rules(op, k):
    sp = S2Space(Sphere6(), 2, 1)
    asm = Assembler(sp, op, k, g_reg=14, g_sing=12)
    pairs = _curved_pairs(sp)
    kinds = (["identical", "edge", "vertex", "separated", "cross-edge", "cross-vertex"] if op == "laplace"
             else ["identical", "edge", "cross-vertex"])
    for name in kinds:
        e, f = pairs[name]
        ref = asm.pair_block(e, f)
        blk, _ = CV.space_block(sp, op, k, e, f, r0=1, max_steps=0)
        err = np.max(np.abs(blk - ref)) / np.max(np.abs(ref))
        assert err < 1e-9, (name, err)


def test_bernstein_equals_bspline_basis_at_degree_one():
    """Degree-1 B-splines restricted to an element are the two hat functions, i.e. the
    Bernstein polynomials, so the golden blocks in the Bernstein basis are the oracle's."""
    sp = S2Space(Sphere6(), 3, 1)
    st = np.random.default_rng(0).random((50, 2))
    for e in (0, sp.element_index(3, 7, 0), sp.element_index(5, 4, 7)):
        np.testing.assert_allclose(sp.element_basis(e, st), CV.bernstein(1, st), atol=1e-14)
