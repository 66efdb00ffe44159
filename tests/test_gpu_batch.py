"""Batched multi-mesh assembly (one persistent launch over all meshes).

Every operator of a batch must be the operator bembel_assemble builds from the
same arguments: the per-pair device code is shared, so products agree to FP64
rounding of the matvec's accumulation order.  One small member is also checked
against the oracle's dense H^2 approximant directly."""
import numpy as np
import pytest
import torch

import paper_1906_00785_gb300 as bem
from inputs import perturbed_sphere_coeffs, random_vector
from oracle.geometry import PerturbedSphere
from oracle.h2 import H2Oracle
from oracle.space import S2Space

pytestmark = pytest.mark.gpu
LAP, HEL = bem.BEMBEL_LAPLACE_SL, bem.BEMBEL_HELMHOLTZ_SL


def matvec(op, x, nrhs=1):
    y = torch.empty_like(x)
    bem.bembel_matvec(op, x, y, nrhs)
    torch.cuda.synchronize()
    return y


@pytest.mark.parametrize("kind,k,p", [(LAP, 0.0, 1), (HEL, 2.0, 2)])
def test_batch_equals_single(kind, k, p):
    sph = bem.bembel_geom_create()
    per = bem.bembel_geom_create(bem.BEMBEL_GEOM_PERTURBED_SPHERE, coeffs=perturbed_sphere_coeffs(2001))
    items = [(sph, k, 2), (per, 1.5 * k, 3), (sph, 0.5 * k + 0.2j * (kind == HEL), 4), (per, k, 2)]
    kw = dict(g_regular=3, g_singular=4, g_edge=5, eta=1.6, precision=bem.BEMBEL_PREC_MIXED,
              g_identical_var=(4, 5, 3, 3) if kind == HEL else (0, 0, 0, 0), g_regular_far=2 if kind == LAP else 0)
    ops = bem.bembel_assemble_batch(items, kind, p, 4, **kw)
    assert len(ops) == len(items)
    for (g, kk, L), op in zip(items, ops):
        ref = bem.bembel_assemble(g, kind, kk, L, p, 4, **kw)
        n = bem.bembel_ndofs(ref)
        assert bem.bembel_ndofs(op) == n
        cplx = kind == HEL
        x = torch.from_numpy(random_vector(n, L, complex_=cplx)).cuda()
        y1, y2 = matvec(op, x), matvec(ref, x)
        rel = (torch.linalg.norm(y1 - y2) / torch.linalg.norm(y2)).item()
        assert rel < 1e-14, (L, kk, rel)
        # the FP32 copies exist and agree too
        x32 = x.to(torch.complex64 if cplx else torch.float32)
        z1, z2 = torch.empty_like(x32), torch.empty_like(x32)
        bem.bembel_matvec(op, x32, z1, 1, fp32=True)
        bem.bembel_matvec(ref, x32, z2, 1, fp32=True)
        torch.cuda.synchronize()
        assert (torch.linalg.norm(z1 - z2) / torch.linalg.norm(z2)).item() < 1e-6
        info = bem.bembel_op_info_get(op)
        assert info["phase_ms"][7] > 0.0 and info["phase_ms"][2] == 0.0


def test_batch_member_matches_oracle():
    a = perturbed_sphere_coeffs(1000)
    per = bem.bembel_geom_create(bem.BEMBEL_GEOM_PERTURBED_SPHERE, coeffs=a, amplitude=0.1)
    sph = bem.bembel_geom_create()
    ops = bem.bembel_assemble_batch([(sph, 0.0, 4), (per, 0.0, 3)], LAP, 0, 3, g_regular=3, g_singular=4,
                                    leaf_level=2, eta=1.6)
    sp = S2Space(PerturbedSphere(a, 0.1), 3, 0)
    h2 = H2Oracle(sp, "laplace", q=3, eta=1.6, leaf_level=2, g_reg=3, g_sing=4)
    n = sp.ndofs
    eye = torch.eye(n, dtype=torch.float64, device="cuda")
    A = matvec(ops[1], eye, n).cpu().numpy().T
    ref = h2.dense()
    assert np.max(np.abs(A - ref)) / np.max(np.abs(ref)) < 1e-12


def test_batch_solves():
    """Batched operators are complete: block-Jacobi mixed solves converge on each."""
    sph = bem.bembel_geom_create()
    ops = bem.bembel_assemble_batch([(sph, 2.0, 3), (sph, 4.0, 3), (sph, 2.0, 4)], HEL, 1, 4,
                                    precision=bem.BEMBEL_PREC_MIXED)
    for op in ops:
        n = bem.bembel_ndofs(op)
        b = torch.empty(n, dtype=torch.complex128, device="cuda")
        bem.bembel_rhs(op, bem.BEMBEL_RHS_PLANE_WAVE, np.array([[0.0, 0.0, 1.0]]), b)
        x = torch.empty_like(b)
        info = bem.bembel_solve(op, b, x, 1, tol=1e-8, precond=bem.BEMBEL_PRECOND_BLOCK_JACOBI)
        assert info["converged"]


def test_batch_invalid():
    sph = bem.bembel_geom_create()
    with pytest.raises(bem.BembelError):
        bem.bembel_assemble_batch([], LAP, 1, 4)
    with pytest.raises(bem.BembelError):
        bem.bembel_assemble_batch([(sph, 0.0, 11)], LAP, 1, 4)
    with pytest.raises(bem.BembelError):
        bem.bembel_assemble_batch([(sph, 0.0, 2)] * 65, LAP, 1, 4)
