"""NURBS geometry (six rational B-spline patches) through the C ABI: assembly
parity with the oracle, the H^2 operator, and the point-charge test on the
pillow box."""
import numpy as np
import pytest
import torch

import paper_1906_00785_gb300 as bem
from inputs import nurbs_pillow_box
from oracle.galerkin import Assembler
from oracle.geometry import NurbsSurface
from oracle.h2 import H2Oracle
from oracle.space import S2Space

pytestmark = pytest.mark.gpu
LAP, HEL = bem.BEMBEL_LAPLACE_SL, bem.BEMBEL_HELMHOLTZ_SL


@pytest.fixture(scope="module")
def box():
    pts = nurbs_pillow_box(degree=2, segments=2)
    return bem.bembel_geom_create(bem.BEMBEL_GEOM_NURBS, patches=pts), NurbsSurface(pts)


def gpu_matrix(op, n, cplx=False):
    eye = torch.eye(n, dtype=torch.complex128 if cplx else torch.float64, device="cuda")
    out = torch.empty_like(eye)
    bem.bembel_matvec(op, eye, out, n)
    torch.cuda.synchronize()
    return out.cpu().numpy().T


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("L,d,op,k", [(2, 1, "laplace", 0.0), (1, 2, "helmholtz", 2.0)])
def test_nurbs_dense_parity(box, L, d, op, k):
    g, geo = box
    gop = bem.bembel_assemble(g, LAP if op == "laplace" else HEL, k, L, d, 0, g_regular=4, g_singular=5)
    sp = S2Space(geo, L, d)
    assert rel(gpu_matrix(gop, sp.ndofs, op == "helmholtz"), Assembler(sp, op, k, 4, 5).dense()) < 1e-12


def test_nurbs_h2_parity(box):
    g, geo = box
    gop = bem.bembel_assemble(g, LAP, 0.0, 3, 0, 3, g_regular=3, g_singular=4, leaf_level=2, eta=1.6)
    sp = S2Space(geo, 3, 0)
    h2 = H2Oracle(sp, "laplace", q=3, eta=1.6, leaf_level=2, g_reg=3, g_sing=4)
    assert bem.bembel_op_info_get(gop)["n_far_blocks"] == len(h2.far) > 0
    assert rel(gpu_matrix(gop, sp.ndofs), h2.dense()) < 1e-12


def test_nurbs_point_charge(box):
    """The single-layer solution for g = 1/|x - x0| reproduces g inside the box (error falling with L)."""
    g, _ = box
    x0 = np.array([[0.3, 0.2, 3.0]])
    pts = np.array([[0.0, 0.0, 0.0], [0.3, -0.2, 0.4], [-0.5, 0.1, -0.3], [0.6, 0.6, 0.6]])
    exact = 1.0 / np.linalg.norm(pts - x0, axis=1)
    errs = []
    for L in (3, 4):
        op = bem.bembel_assemble(g, LAP, 0.0, L, 1, 4)
        n = bem.bembel_ndofs(op)
        b = torch.empty(n, dtype=torch.float64, device="cuda")
        bem.bembel_rhs(op, bem.BEMBEL_RHS_POINT_SOURCE, x0, b)
        x = torch.empty_like(b)
        assert bem.bembel_solve(op, b, x, 1, tol=1e-10, precond=bem.BEMBEL_PRECOND_BLOCK_JACOBI)["converged"]
        u = torch.empty(len(pts), dtype=torch.float64, device="cuda")
        bem.bembel_eval(op, torch.from_numpy(pts).cuda(), x, u, 1, g=6)
        errs.append(np.abs(u.cpu().numpy() - exact).max() / exact.max())
    assert errs[1] < 1e-3 and errs[1] < errs[0] / 2, errs


def test_nurbs_invalid():
    pts = nurbs_pillow_box()
    with pytest.raises(bem.BembelError):
        bem.bembel_geom_create(bem.BEMBEL_GEOM_NURBS, patches=pts[:5])
    bad = [dict(p) for p in pts]
    bad[2] = {**bad[2], "ctrl": bad[2]["ctrl"].copy()}
    bad[2]["ctrl"][0, 0, 3] = 0.0
    with pytest.raises(bem.BembelError):
        bem.bembel_geom_create(bem.BEMBEL_GEOM_NURBS, patches=bad)
    bad = [dict(p) for p in pts]
    kn = bad[0]["knots"][0].copy()
    kn[0] = 0.1  # not open on [0, 1]
    bad[0] = {**bad[0], "knots": (kn, bad[0]["knots"][1])}
    with pytest.raises(bem.BembelError):
        bem.bembel_geom_create(bem.BEMBEL_GEOM_NURBS, patches=bad)
