"""Two-level preconditioner (block-Jacobi plus the coarse-space correction P A_c^-1 P^T)
on the GPU against the oracle (``oracle.coarse``: Boehm knot insertion, coarse Galerkin
matrix assembled by ``Assembler``, numpy solve).

* The correction alone (two-level minus block-Jacobi applied to the same vectors) equals
  the oracle's P A_c^-1 P^T x: FP64 to 1e-10 relative (rounding of the coarse inverse),
  FP32 to 50 eps_32 cond(A_c).
* Solves with the two-level preconditioner reach the block-Jacobi solution; for Helmholtz
  near an interior resonance (kappa = 8) they take fewer GMRES steps.
* Invalid uses fail with EINVAL / EUNSUPPORTED."""
import numpy as np
import pytest
import torch

import paper_1906_00785_gb300 as bem
from inputs import perturbed_sphere_coeffs, random_vector
from oracle.coarse import coarse_correction, prolongation
from oracle.galerkin import Assembler
from oracle.geometry import Sphere6
from oracle.space import S2Space

pytestmark = pytest.mark.gpu
LAP, HEL = bem.BEMBEL_LAPLACE_SL, bem.BEMBEL_HELMHOLTZ_SL
BJ, TWO = bem.BEMBEL_PRECOND_BLOCK_JACOBI, bem.BEMBEL_PRECOND_TWO_LEVEL


@pytest.fixture(scope="module")
def geom():
    return bem.bembel_geom_create()


@pytest.mark.parametrize("op,k,L,d,Lc,q", [("laplace", 0.0, 3, 1, 1, 0), ("helmholtz", 2.0, 3, 2, 1, 0),
                                           ("laplace", 0.0, 4, 2, 2, 4), ("helmholtz", 3.0, 3, 0, 2, 0)])
def test_coarse_correction_matches_oracle(geom, op, k, L, d, Lc, q):
    kind = LAP if op == "laplace" else HEL
    gop = bem.bembel_assemble(geom, kind, k, L, d, q, g_regular=4, g_singular=5, coarse_level=Lc)
    n = bem.bembel_ndofs(gop)
    cplx = op == "helmholtz"
    nrhs = 3
    X = random_vector(n, 11, nrhs=nrhs, complex_=cplx)  # (n, nrhs)
    Xt = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
    Y_bj, Y_2 = torch.empty_like(Xt), torch.empty_like(Xt)
    bem.bembel_precond_apply(gop, BJ, Xt, Y_bj, nrhs)
    bem.bembel_precond_apply(gop, TWO, Xt, Y_2, nrhs)
    corr = (Y_2 - Y_bj).cpu().numpy().T
    sc, sf = S2Space(Sphere6(), Lc, d), S2Space(Sphere6(), L, d)
    P = prolongation(sc, sf)
    Ac = Assembler(sc, op, k, 4, 5).dense()
    ref = coarse_correction(P, Ac, X)
    rel = np.max(np.abs(corr - ref)) / np.max(np.abs(ref))
    assert rel < 1e-10, rel
    # FP32 application (the inner GMRES of MIXED operators)
    Xf = Xt.to(torch.complex64 if cplx else torch.float32)
    Yf_bj, Yf_2 = torch.empty_like(Xf), torch.empty_like(Xf)
    bem.bembel_precond_apply(gop, BJ, Xf, Yf_bj, nrhs, fp32=True)
    bem.bembel_precond_apply(gop, TWO, Xf, Yf_2, nrhs, fp32=True)
    corr32 = (Yf_2 - Yf_bj).cpu().numpy().T
    # FP32 rounding of the coarse product grows with the conditioning of A_c
    tol32 = 50 * np.finfo(np.float32).eps * np.linalg.cond(Ac)
    err32 = np.max(np.abs(corr32 - ref)) / np.max(np.abs(ref))
    assert err32 < tol32, (err32, tol32)


def test_none_copies(geom):
    gop = bem.bembel_assemble(geom, LAP, 0.0, 2, 1, 0)
    n = bem.bembel_ndofs(gop)
    x = torch.from_numpy(random_vector(n, 2)).cuda()
    y = torch.empty_like(x)
    bem.bembel_precond_apply(gop, bem.BEMBEL_PRECOND_NONE, x, y, 1)
    assert torch.equal(x, y)


@pytest.mark.parametrize("kind,k,L,d,geo", [(LAP, 0.0, 5, 1, "sphere"), (HEL, 8.0, 4, 2, "perturbed")])
def test_two_level_solve_fewer_steps(kind, k, L, d, geo):
    g = (bem.bembel_geom_create() if geo == "sphere" else
         bem.bembel_geom_create(bem.BEMBEL_GEOM_PERTURBED_SPHERE, coeffs=perturbed_sphere_coeffs(2001)))
    gop = bem.bembel_assemble(g, kind, k, L, d, 4)
    n = bem.bembel_ndofs(gop)
    dt = torch.complex128 if kind == HEL else torch.float64
    b = torch.empty(n, dtype=dt, device="cuda")
    if kind == HEL:
        bem.bembel_rhs(gop, bem.BEMBEL_RHS_PLANE_WAVE, [[0.0, 0.0, 1.0]], b)
    else:
        bem.bembel_rhs(gop, bem.BEMBEL_RHS_POINT_SOURCE, [[0.0, 0.0, 2.0]], b)
    x_bj, x_2 = torch.empty_like(b), torch.empty_like(b)
    i_bj = bem.bembel_solve(gop, b, x_bj, 1, tol=1e-10, restart=100, max_iter=5000, precond=BJ)
    i_2 = bem.bembel_solve(gop, b, x_2, 1, tol=1e-10, restart=100, max_iter=5000, precond=TWO)
    print(f"kind {kind} k {k} L {L} d {d}: block-Jacobi {i_bj['iterations']} steps, two-level {i_2['iterations']}")
    assert i_bj["converged"] and i_2["converged"]
    # both at relative residual 1e-10: the solutions agree to about cond(A) 1e-10
    assert (torch.linalg.norm(x_2 - x_bj) / torch.linalg.norm(x_bj)).item() < 1e-6
    if kind == HEL:
        # the coarse space holds the smooth modes near the interior resonances (kappa = 8)
        assert i_2["iterations"] < i_bj["iterations"]
    else:
        # Laplace: the single layer's small eigenvalues belong to oscillating modes, which
        # the coarse space does not hold: no fewer steps (measured 63 vs 64 at level 5)
        assert i_2["iterations"] <= i_bj["iterations"] + 5


def test_invalid_uses(geom):
    with pytest.raises(bem.BembelError) as ei:
        bem.bembel_assemble(geom, LAP, 0.0, 2, 1, 0, coarse_level=3)
    assert ei.value.code == bem.BEMBEL_EINVAL
    rep = bem.bembel_assemble(geom, LAP, 0.0, 2, 2, 0, knot_repetition=2)
    n = bem.bembel_ndofs(rep)
    x = torch.from_numpy(random_vector(n, 3)).cuda()
    y = torch.empty_like(x)
    with pytest.raises(bem.BembelError) as ei:
        bem.bembel_precond_apply(rep, TWO, x, y, 1)
    assert ei.value.code == bem.BEMBEL_EUNSUPPORTED
    with pytest.raises(bem.BembelError) as ei:
        bem.bembel_precond_apply(rep, 7, x, y, 1)
    assert ei.value.code == bem.BEMBEL_EINVAL
    efie = bem.bembel_assemble(geom, bem.BEMBEL_MAXWELL_SL, 2.0, 1, 1, 0)
    ne = bem.bembel_ndofs(efie)
    xe = torch.zeros(ne, dtype=torch.complex128, device="cuda")
    with pytest.raises(bem.BembelError) as ei:
        bem.bembel_precond_apply(efie, BJ, xe, torch.empty_like(xe), 1)
    assert ei.value.code == bem.BEMBEL_EUNSUPPORTED


def test_block_jacobi_leaf_too_large(geom):
    """Leaves of 576 local dofs (level 4, degree 2, leaf level 1): [D | I] of one leaf does not
    fit one CTA's shared memory, and the set-up says so before any device work."""
    gop = bem.bembel_assemble(geom, LAP, 0.0, 4, 2, 4, leaf_level=1)
    n = bem.bembel_ndofs(gop)
    x = torch.from_numpy(random_vector(n, 4)).cuda()
    with pytest.raises(bem.BembelError) as ei:
        bem.bembel_precond_apply(gop, BJ, x, torch.empty_like(x), 1)
    assert ei.value.code == bem.BEMBEL_EUNSUPPORTED
    # the operator stays usable: its product runs
    y = torch.empty_like(x)
    bem.bembel_matvec(gop, x, y, 1)
    assert torch.isfinite(y).all().item()
