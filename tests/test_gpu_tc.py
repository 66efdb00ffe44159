"""Tensor-core (tcgen05) coupling for many right-hand sides.

The single-MMA self-test checks the shared-memory operand layout, the
descriptors and the TMEM read-back on exactly representable data (result must
be exact).  The batched coupling (bf16 operands, FP32 accumulation) is compared
with the FP32 CUDA-core product: the far-field part differs by ~bf16 rounding,
so the whole product agrees to 5e-3 relative; solves with FP64 refinement reach
the FP64 solution."""
import numpy as np
import pytest
import torch

import paper_1906_00785_gb300 as bem
from inputs import random_vector, unit_directions

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [16, 64, 128, 256])
def test_tc_selftest_exact(n):
    assert bem.bembel_tc_selftest(n) == 0.0


def test_bounded_wait_times_out_and_device_stays_usable():
    """The time-out path of the bounded mbarrier waits: a wait on a barrier that nothing
    signals runs out after its short poll limit and is reported as BEMBEL_ETIMEOUT; the
    context stays usable (a self-test MMA right after it is exact)."""
    with pytest.raises(bem.BembelError) as ei:
        bem.bembel_tc_selftest(0)
    assert ei.value.code == bem.BEMBEL_ETIMEOUT
    assert bem.bembel_tc_selftest(64) == 0.0


@pytest.mark.parametrize("op,k,nrhs,tc_used", [("laplace", 0.0, 16, False), ("laplace", 0.0, 32, True),
                                               ("laplace", 0.0, 128, True), ("helmholtz", 3.0, 16, False),
                                               ("helmholtz", 3.0, 32, True), ("helmholtz", 3.0, 64, True)])
def test_tc_coupling_matches_cuda_cores(op, k, nrhs, tc_used):
    g = bem.bembel_geom_create()
    kind = bem.BEMBEL_LAPLACE_SL if op == "laplace" else bem.BEMBEL_HELMHOLTZ_SL
    tc = bem.bembel_assemble(g, kind, k, 4, 1, 4, precision=bem.BEMBEL_PREC_MIXED, tensor_cores=1)
    cc = bem.bembel_assemble(g, kind, k, 4, 1, 4, precision=bem.BEMBEL_PREC_MIXED, tensor_cores=0)
    n = bem.bembel_ndofs(tc)
    cplx = op == "helmholtz"
    X = random_vector(n, 7, nrhs=nrhs, complex_=cplx).T.copy()
    Xt = torch.from_numpy(X).to(torch.complex64 if cplx else torch.float32).cuda()
    Y1, Y2 = torch.empty_like(Xt), torch.empty_like(Xt)
    bem.bembel_matvec(tc, Xt, Y1, nrhs, fp32=True)
    bem.bembel_matvec(cc, Xt, Y2, nrhs, fp32=True)
    torch.cuda.synchronize()
    rel = (torch.linalg.norm(Y1 - Y2) / torch.linalg.norm(Y2)).item()
    # the CUDA-core product accumulates with atomics: two runs differ by FP32
    # rounding order only; bf16 operands differ by ~1e-4..1e-3
    if tc_used:
        assert 1e-5 < rel < 5e-3, rel
    else:
        assert rel < 1e-6, rel  # narrow blocks stay on the CUDA-core product


def test_tc_batched_helmholtz_solve():
    g = bem.bembel_geom_create()
    k = 2.0
    op = bem.bembel_assemble(g, bem.BEMBEL_HELMHOLTZ_SL, k, 4, 2, 4, precision=bem.BEMBEL_PREC_MIXED)
    op64 = bem.bembel_assemble(g, bem.BEMBEL_HELMHOLTZ_SL, k, 4, 2, 4)
    n = bem.bembel_ndofs(op)
    B = torch.empty((64, n), dtype=torch.complex128, device="cuda")
    bem.bembel_rhs(op, bem.BEMBEL_RHS_PLANE_WAVE, unit_directions(64, 3), B)
    X = torch.empty_like(B)
    info = bem.bembel_solve(op, B, X, 64, tol=1e-8, precond=bem.BEMBEL_PRECOND_BLOCK_JACOBI)
    assert info["converged"] and info["rel_residual"] <= 1e-8
    Y = torch.empty_like(B)
    bem.bembel_matvec(op64, X, Y, 64)
    assert (torch.linalg.norm(Y - B) / torch.linalg.norm(B)).item() < 1e-7
