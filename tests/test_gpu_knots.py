"""S^2 spaces with repeated interior knots (Sec. 4.3 knotRepetition) on the GPU against the
oracle: dense and H^2 matrices (1e-12, rounding only), load vector, solve and potential,
and wide products through the CSR extraction."""
import numpy as np
import pytest
import torch

import paper_1906_00785_gb300 as bem
from inputs import random_vector
from oracle.galerkin import Assembler, potential, rhs
from oracle.geometry import Sphere6
from oracle.h2 import H2Oracle
from oracle.space import S2Space

pytestmark = pytest.mark.gpu
LAP, HEL = bem.BEMBEL_LAPLACE_SL, bem.BEMBEL_HELMHOLTZ_SL


@pytest.fixture(scope="module")
def geom():
    return bem.bembel_geom_create(bem.BEMBEL_GEOM_SPHERE6)


def gpu_matrix(op, n, cplx):
    dt = torch.complex128 if cplx else torch.float64
    eye = torch.eye(n, dtype=dt, device="cuda")
    out = torch.empty_like(eye)
    bem.bembel_matvec(op, eye, out, n)
    torch.cuda.synchronize()
    return out.cpu().numpy().T


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("L,d,r,op,k", [(2, 2, 2, "laplace", 0.0), (2, 2, 3, "helmholtz", 1.5), (2, 1, 2, "laplace", 0.0),
                                        (1, 0, 1, "laplace", 0.0)])
def test_dense_parity(geom, L, d, r, op, k):
    sp = S2Space(Sphere6(), L, d, r)
    gop = bem.bembel_assemble(geom, LAP if op == "laplace" else HEL, k, L, d, 0, g_regular=4, g_singular=5,
                              knot_repetition=r)
    assert bem.bembel_ndofs(gop) == sp.ndofs
    A = gpu_matrix(gop, sp.ndofs, op == "helmholtz")
    assert rel(A, Assembler(sp, op, k, 4, 5).dense()) < 1e-12


def test_h2_parity(geom):
    sp = S2Space(Sphere6(), 3, 2, 2)
    gop = bem.bembel_assemble(geom, LAP, 0.0, 3, 2, 3, g_regular=3, g_singular=4, leaf_level=2, eta=1.6,
                              knot_repetition=2)
    h2 = H2Oracle(sp, "laplace", q=3, eta=1.6, leaf_level=2, g_reg=3, g_sing=4)
    assert rel(gpu_matrix(gop, sp.ndofs, False), h2.dense()) < 1e-12


def test_rhs_solve_eval(geom):
    x0 = np.array([0.0, 0.0, 2.0])
    sp = S2Space(Sphere6(), 2, 2, 3)
    gop = bem.bembel_assemble(geom, LAP, 0.0, 2, 2, 0, g_regular=4, g_singular=5, knot_repetition=3)
    n = bem.bembel_ndofs(gop)
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    bem.bembel_rhs(gop, bem.BEMBEL_RHS_POINT_SOURCE, x0[None, :], b, g=6)
    b_ref = rhs(sp, lambda x: 1.0 / np.linalg.norm(x - x0, axis=1), g=6)
    np.testing.assert_allclose(b.cpu().numpy(), b_ref, rtol=1e-13, atol=1e-16)
    rho = torch.empty_like(b)
    info = bem.bembel_solve(gop, b, rho, 1, tol=1e-13, precond=bem.BEMBEL_PRECOND_BLOCK_JACOBI)
    assert info["converged"]
    rho_ref = np.linalg.solve(Assembler(sp, "laplace", 0.0, 4, 5).dense(), b_ref)
    assert rel(rho.cpu().numpy(), rho_ref) < 1e-9
    pts = np.array([[0.1, 0.2, -0.3], [0.0, 0.4, 0.1]])
    u = torch.empty(2, dtype=torch.float64, device="cuda")
    bem.bembel_eval(gop, torch.from_numpy(pts).cuda(), rho, u, 1, g=6)
    np.testing.assert_allclose(u.cpu().numpy(), potential(sp, rho_ref, pts, "laplace", g=6), rtol=1e-9)


def test_wide_products_equal_columns(geom):
    """40 columns (the width where r = 1 products go through a dof-major copy) equal 40
    single products on the CSR extraction of r = 2."""
    gop = bem.bembel_assemble(geom, LAP, 0.0, 3, 2, 4, leaf_level=2, knot_repetition=2)
    n = bem.bembel_ndofs(gop)
    X = torch.from_numpy(np.ascontiguousarray(random_vector(n, 3, nrhs=40).T)).cuda()
    Y = torch.empty_like(X)
    bem.bembel_matvec(gop, X, Y, 40)
    for c in (0, 17, 39):
        y = torch.empty_like(X[c])
        bem.bembel_matvec(gop, X[c].contiguous(), y, 1)
        assert torch.max(torch.abs(y - Y[c])).item() <= 1e-13 * torch.max(torch.abs(y)).item()


def test_invalid_repetition(geom):
    with pytest.raises(bem.BembelError) as ei:
        bem.bembel_assemble(geom, LAP, 0.0, 2, 1, 0, knot_repetition=3)
    assert ei.value.code == bem.BEMBEL_EINVAL
    with pytest.raises(bem.BembelError) as ei:
        bem.bembel_assemble(geom, bem.BEMBEL_MAXWELL_SL, 2.0, 1, 2, 0, knot_repetition=2)
    assert ei.value.code == bem.BEMBEL_EUNSUPPORTED
