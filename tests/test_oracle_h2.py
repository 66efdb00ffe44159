"""Pins for the oracle's H^2 approximant (Sec. 2: kernel interpolation on the
parameter domain per admissible cluster pair).

* The block tree partitions the element-pair set: every (e, f) lies in exactly
  one far or near block, and far blocks satisfy the admissibility reading.
* Interpolation exactness: for a kernel that is a polynomial of degree q-1 in
  each parameter, moments x coupling x moments reproduces the exact Galerkin
  integral (a wrong node, Lagrange factor or moment scaling breaks this).
* Compression error of A~ against the exact-rule matrix A decays with q.
* The sampled-row path (cluster moments of x, no dense matrix) agrees with the
  dense reconstruction.
"""
import numpy as np
import pytest

from inputs import random_vector
from oracle.galerkin import Assembler
from oracle.gauss import tensor2
from oracle.geometry import Sphere6
from oracle.h2 import H2Oracle, block_tree, cluster_elements
from oracle.space import S2Space


def test_block_tree_partition():
    sp = S2Space(Sphere6(), 3, 0)
    far, near, cl = block_tree(sp.geom, 2, 1.6)
    assert len(far) > 0
    cover = np.zeros((sp.nelem, sp.nelem), dtype=int)
    for t, s in far + near:
        E, F = cluster_elements(sp, t), cluster_elements(sp, s)
        cover[np.ix_(E, F)] += 1
    assert np.all(cover == 1)
    for t, s in far:
        (ct, rt), (cs, rs) = cl.ball(t), cl.ball(s)
        assert 2 * max(rt, rs) <= 1.6 * (np.linalg.norm(ct - cs) - rt - rs)
    # touching clusters are never admissible
    for t, s in far:
        assert np.linalg.norm(cl.ball(t)[0] - cl.ball(s)[0]) > cl.ball(t)[1] + cl.ball(s)[1]


@pytest.mark.parametrize("q,d", [(3, 0), (4, 1), (5, 2)])
def test_interpolation_exact_for_polynomial_kernel(q, d):
    sp = S2Space(Sphere6(), 3, d)
    h2 = H2Oracle(sp, "laplace", q=q, eta=1.6, leaf_level=2)
    t, s = h2.far[len(h2.far) // 2]
    rng = np.random.default_rng(5)
    C = rng.standard_normal((q,) * 4)

    def P(a, b):  # polynomial of degree q-1 in each of s1, s2, t1, t2
        out = 0.0
        for i in np.ndindex(*C.shape):
            out = out + C[i] * a[..., 0] ** i[0] * a[..., 1] ** i[1] * b[..., 0] ** i[2] * b[..., 1] ** i[3]
        return out

    xt, xs = h2.cluster_nodes(t), h2.cluster_nodes(s)
    K = P(xt[:, None, :], xs[None, :, :])
    pts, w = tensor2(q + d + 1)
    for e, f in [(cluster_elements(sp, t)[0], cluster_elements(sp, s)[-1]),
                 (cluster_elements(sp, t)[-1], cluster_elements(sp, s)[1])]:
        approx = h2.moment(e, t) @ K @ h2.moment(f, s).T
        se, sf = sp.to_patch(e, pts), sp.to_patch(f, pts)
        Be = sp.element_basis(e, pts) * (w * sp.h**2)[:, None]
        Bf = sp.element_basis(f, pts) * (w * sp.h**2)[:, None]
        exact = Be.T @ P(se[:, None, :], sf[None, :, :]) @ Bf
        np.testing.assert_allclose(approx, exact, rtol=1e-11, atol=1e-13 * np.abs(exact).max())


def test_compression_error_decays_with_q():
    """Relative Frobenius error of the far blocks of A~ against the tensor-rule blocks."""
    sp = S2Space(Sphere6(), 3, 1)
    asm = Assembler(sp, "laplace", 0.0, 6, 5)
    far = block_tree(sp.geom, 2, 1.6)[0]
    exact = {}
    for t, s in far:
        E, F = cluster_elements(sp, t), cluster_elements(sp, s)
        exact[(t, s)] = [[asm.pair_block(e, f, ("regular", None, None)) for f in F] for e in E]
    ref = np.sqrt(sum(np.sum(np.square(b)) for blk in exact.values() for row in blk for b in row))
    errs = []
    for q in (2, 3, 4, 5):
        h2 = H2Oracle(sp, "laplace", q=q, eta=1.6, leaf_level=2)
        assert h2.far == far
        acc = 0.0
        for t, s in far:
            K = h2.coupling(t, s)
            for i, e in enumerate(cluster_elements(sp, t)):
                Me = h2.moment(e, t) @ K
                for j, f in enumerate(cluster_elements(sp, s)):
                    acc += np.sum(np.square(Me @ h2.moment(f, s).T - exact[(t, s)][i][j]))
        errs.append(np.sqrt(acc) / ref)
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[2] < 1e-3, errs


@pytest.mark.parametrize("op,k", [("laplace", 0.0), ("helmholtz", 3.0)])
def test_rows_match_dense(op, k):
    sp = S2Space(Sphere6(), 3, 1)
    h2 = H2Oracle(sp, op, k, q=3, eta=1.6, leaf_level=2, g_reg=3, g_sing=4)
    x = random_vector(sp.ndofs, 11, complex_=(op == "helmholtz"))
    rows = [0, 7, 100, 255, sp.ndofs - 1]
    y_rows = h2.apply_rows(x, rows)
    y = h2.dense() @ x
    np.testing.assert_allclose(y_rows, y[rows], rtol=1e-12, atol=1e-14 * np.abs(y).max())
