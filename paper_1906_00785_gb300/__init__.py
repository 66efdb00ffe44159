"""GB300 (sm_103a) isogeometric single-layer BEM: H^2 assembly, matvec and GMRES.

The compute path is the CUDA library ``libbembel.so`` behind the C ABI of
``include/bembel.h``; ``capi`` is its ctypes binding with the same names.
Vectors are caller-owned device tensors (``torch`` on ``cuda``), column-major
``n x nrhs``, complex interleaved.  A Laplace solve with an exterior point
charge as data and the potential at interior points::

    import numpy as np, torch
    import paper_1906_00785_gb300 as bem

    geom = bem.bembel_geom_create(bem.BEMBEL_GEOM_SPHERE6)
    op = bem.bembel_assemble(geom, bem.BEMBEL_LAPLACE_SL, 0.0, 6, 1, 4,   # level 6, degree 1, q = 4
                             precision=bem.BEMBEL_PREC_MIXED)
    n = bem.bembel_ndofs(op)
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    bem.bembel_rhs(op, bem.BEMBEL_RHS_POINT_SOURCE, np.array([[0.0, 0.0, 2.0]]), b)
    rho = torch.empty_like(b)
    info = bem.bembel_solve(op, b, rho, 1, tol=1e-8, precond=bem.BEMBEL_PRECOND_BLOCK_JACOBI)
    pts = torch.tensor([[0.0, 0.1, 0.2]], dtype=torch.float64, device="cuda")
    u = torch.empty(1, dtype=torch.float64, device="cuda")
    bem.bembel_eval(op, pts, rho, u, 1)

``bembel_autotune`` picks quadrature orders and q for a target accuracy,
``bembel_assemble_batch`` assembles many meshes in one launch, and
``BEMBEL_HELMHOLTZ_SL`` / ``BEMBEL_MAXWELL_SL`` select the other operators.
"""
from .capi import *  # noqa: F401,F403
from .capi import BembelError, Geometry, Operator, lib  # noqa: F401
