"""Autotuner choices made by timing: leaf level (L-1 or L-2) and, for MIXED operators, the
FP32 far-field coupling evaluated on the fly or streamed from a stored FP32 copy.

* The report's scores are positive for the levels tried and the chosen leaf level is the
  cheapest one; the chosen storage is the faster of the two timed products.
* Both storages give the same FP32 product up to FP32 rounding of the kernel values (5e-6), and
  both stay within FP32 accuracy of the FP64 product."""
import numpy as np
import pytest
import torch

import paper_1906_00785_gb300 as bem
from inputs import random_vector

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,k", [(bem.BEMBEL_LAPLACE_SL, 0.0), (bem.BEMBEL_HELMHOLTZ_SL, 2.0)])
def test_layout_choice(kind, k):
    g = bem.bembel_geom_create()
    L = 5
    opts, rep = bem.bembel_autotune(g, kind, k, L, 1, quad_tol=1e-6, far_tol=1e-4, q_max=4,
                                    precision=bem.BEMBEL_PREC_MIXED, kdiam=4.0 if k else 0.0)
    scores = rep["leaf_score_ms"]
    print("leaf scores (L-1, L-2):", scores, "fp32 products (on the fly, stored):", rep["fp32_product_ms"])
    assert scores[0] > 0 and scores[1] > 0
    assert rep["leaf_level"] == (L - 1 if scores[0] <= scores[1] else L - 2)
    assert opts.leaf_level == rep["leaf_level"]
    onfly, stored = rep["fp32_product_ms"]
    assert onfly > 0 and stored > 0
    assert rep["far_fp32_stored"] == (1 if stored < onfly else 0) == opts.far_fp32_stored

    # both storages: the same product up to FP32 rounding, and close to the FP64 product
    ops = [bem.bembel_assemble(g, kind, k, L, 1, rep["q"], opts=opts, far_fp32_stored=s) for s in (0, 1)]
    n = bem.bembel_ndofs(ops[0])
    cplx = kind == bem.BEMBEL_HELMHOLTZ_SL
    x = torch.from_numpy(random_vector(n, 9, complex_=cplx)).cuda()
    x32 = x.to(torch.complex64 if cplx else torch.float32)
    y = [torch.empty_like(x32) for _ in ops]
    for op, yy in zip(ops, y):
        bem.bembel_matvec(op, x32, yy, 1, fp32=True)
    y64 = torch.empty_like(x)
    bem.bembel_matvec(ops[0], x, y64, 1)
    torch.cuda.synchronize()
    nrm = torch.linalg.norm(y64).item()
    # on the fly: kernel values from absolute FP32 points (distance error up to ~6e-8 |x| / r,
    # about 1e-6 for the closest far blocks); stored: from FP32 offsets to the cluster centres
    assert torch.linalg.norm(y[0] - y[1]).item() / nrm < 5e-6
    for yy in y:
        assert torch.linalg.norm(yy.to(y64.dtype) - y64).item() / nrm < 1e-5


def test_given_leaf_level_is_kept():
    g = bem.bembel_geom_create()
    opts, rep = bem.bembel_autotune(g, bem.BEMBEL_LAPLACE_SL, 0.0, 4, 1, quad_tol=1e-6, far_tol=1e-4, q_max=4,
                                    leaf_level=2)
    assert opts.leaf_level == 2 and rep["leaf_level"] == 2
    assert list(rep["leaf_score_ms"]) == [0.0, 0.0]
    with pytest.raises(bem.BembelError) as ei:
        bem.bembel_assemble(g, bem.BEMBEL_LAPLACE_SL, 0.0, 2, 1, 4, far_fp32_stored=2)
    assert ei.value.code == bem.BEMBEL_EINVAL
