"""bembel_matvec_noalloc: the matrix-vector product for callers that cannot
allocate device memory (their memory belongs to their own pool allocator, or
they cannot afford the synchronisation cudaMalloc/cudaFree may bring).  It runs
the same kernels as bembel_matvec on a fixed scratch array compiled into the
library, so its result must match bembel_matvec's, call after call, while the
array keeps whatever the previous call left in it.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_1906_00785_gb300 as bem
from inputs import random_vector

pytestmark = pytest.mark.gpu


def _noalloc(op, x, y, nrhs, fp32=0):
    """Direct call of the C entry point."""
    return bem.lib().bembel_matvec_noalloc(op.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                           nrhs, fp32)


@pytest.mark.parametrize("op_kind,k,level,p,q,nrhs,prec", [
    (bem.BEMBEL_LAPLACE_SL, 0.0, 5, 1, 4, 1, bem.BEMBEL_PREC_FP64),
    (bem.BEMBEL_HELMHOLTZ_SL, 2.0, 4, 2, 4, 2, bem.BEMBEL_PREC_FP64),
    (bem.BEMBEL_LAPLACE_SL, 0.0, 4, 1, 4, 1, bem.BEMBEL_PREC_MIXED),
])
def test_noalloc_matches_matvec_twice(op_kind, k, level, p, q, nrhs, prec):
    geom = bem.bembel_geom_create(bem.BEMBEL_GEOM_SPHERE6)
    op = bem.bembel_assemble(geom, op_kind, k, level, p, q, precision=prec)
    n = bem.bembel_ndofs(op)
    cplx = op_kind == bem.BEMBEL_HELMHOLTZ_SL
    fp32 = prec == bem.BEMBEL_PREC_MIXED
    dt = (torch.complex64 if fp32 else torch.complex128) if cplx else (torch.float32 if fp32 else torch.float64)
    for seed in (21, 22):  # two calls in a row on different data: nothing may carry over between them
        x = torch.from_numpy(np.ascontiguousarray(random_vector(n, seed, nrhs=nrhs, complex_=cplx).T)).to(dt).cuda()
        y_ref = torch.empty_like(x)
        bem.bembel_matvec(op, x, y_ref, nrhs, fp32=fp32)
        y = torch.full_like(x, float("nan"))
        assert _noalloc(op, x, y, nrhs, int(fp32)) == bem.BEMBEL_OK, bem.lib().bembel_last_error()
        torch.cuda.synchronize()
        tol = 1e-6 if fp32 else 1e-13
        assert torch.max(torch.abs(y - y_ref)).item() <= tol * torch.max(torch.abs(y_ref)).item()


def test_noalloc_first_product_on_fresh_operator():
    """The very first product of a freshly assembled operator is the no-allocation one (no
    bembel_matvec before it), twice; bembel_matvec afterwards must give the same columns."""
    geom = bem.bembel_geom_create(bem.BEMBEL_GEOM_SPHERE6)
    op = bem.bembel_assemble(geom, bem.BEMBEL_LAPLACE_SL, 0.0, 4, 1, 4)
    n = bem.bembel_ndofs(op)
    xs = [torch.from_numpy(random_vector(n, seed)).cuda() for seed in (31, 32)]
    ys = []
    for x in xs:
        y = torch.full_like(x, float("nan"))
        assert _noalloc(op, x, y, 1) == bem.BEMBEL_OK, bem.lib().bembel_last_error()
        ys.append(y)
    torch.cuda.synchronize()
    for x, y in zip(xs, ys):
        y_ref = torch.empty_like(x)
        bem.bembel_matvec(op, x, y_ref, 1)
        torch.cuda.synchronize()
        assert torch.max(torch.abs(y - y_ref)).item() <= 1e-13 * torch.max(torch.abs(y_ref)).item()


def test_noalloc_compressed_efie_twice():
    """Compressed EFIE: three moment channels per cluster in the scratch layout."""
    geom = bem.bembel_geom_create(bem.BEMBEL_GEOM_SPHERE6)
    op = bem.bembel_assemble(geom, bem.BEMBEL_MAXWELL_SL, 2.0, 3, 2, 4, leaf_level=2)
    n = bem.bembel_ndofs(op)
    for seed in (41, 42):
        x = torch.from_numpy(np.ascontiguousarray(random_vector(n, seed, nrhs=2, complex_=True).T)).cuda()
        y = torch.full_like(x, float("nan"))
        assert _noalloc(op, x, y, 2) == bem.BEMBEL_OK, bem.lib().bembel_last_error()
        y_ref = torch.empty_like(x)
        bem.bembel_matvec(op, x, y_ref, 2)
        torch.cuda.synchronize()
        assert torch.max(torch.abs(y - y_ref)).item() <= 1e-13 * torch.max(torch.abs(y_ref)).item()
    # the three channels count in the size check: a request past the fixed array is refused
    info = bem.bembel_op_info_get(op)
    per_rhs = 16 * (2 * info["nlocal"] + 2 * 3 * info["n_clusters"] * 16)
    nbig = (8 << 20) // per_rhs + 1
    xb = torch.zeros((nbig, n), dtype=torch.complex128, device="cuda")
    yb = torch.zeros_like(xb)
    assert _noalloc(op, xb, yb, nbig) == bem.BEMBEL_EINVAL
    assert b"fixed buffer" in bem.lib().bembel_last_error()


def test_noalloc_rejects_oversized_request():
    geom = bem.bembel_geom_create(bem.BEMBEL_GEOM_SPHERE6)
    op = bem.bembel_assemble(geom, bem.BEMBEL_LAPLACE_SL, 0.0, 5, 1, 4)
    n = bem.bembel_ndofs(op)
    nrhs = 16  # 16 columns of the level-5 operator need more than the fixed 8 MiB
    x = torch.zeros((nrhs, n), dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    assert _noalloc(op, x, y, nrhs) == bem.BEMBEL_EINVAL
    assert b"fixed buffer" in bem.lib().bembel_last_error()
