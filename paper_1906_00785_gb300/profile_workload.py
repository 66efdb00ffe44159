"""One assembly plus a few matrix-vector products, for profiling single kernels.

    python -m paper_1906_00785_gb300.profile_workload --level 5 --degree 1 --q 4 --matvecs 3

Unit sphere (6 cube-face patches); prints the operator counters and phase times.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import capi as bem


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", choices=["laplace", "helmholtz"], default="laplace")
    ap.add_argument("--k", type=float, default=2.0)
    ap.add_argument("--level", type=int, default=5)
    ap.add_argument("--degree", type=int, default=1)
    ap.add_argument("--q", type=int, default=4)
    ap.add_argument("--g-regular", type=int, default=4)
    ap.add_argument("--g-singular", type=int, default=5)
    ap.add_argument("--g-regular-far", type=int, default=0, help="separated pairs beyond the ring (0: g-regular)")
    for cls in ("identical", "edge", "vertex"):
        ap.add_argument(f"--g-{cls}-var", type=str, default="", help="four per-variable Duffy orders, e.g. 4,5,3,3")
    ap.add_argument("--matvecs", type=int, default=3)
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--fp32", action="store_true", help="assemble MIXED and time the FP32 matvec")
    ap.add_argument("--solve", action="store_true", help="also solve a point-charge problem to 1e-8")
    ap.add_argument("--precond", action="store_true", help="block-Jacobi preconditioner for --solve")
    a = ap.parse_args()
    torch.cuda.set_device(0)
    geom = bem.bembel_geom_create(bem.BEMBEL_GEOM_SPHERE6)
    op_kind = bem.BEMBEL_LAPLACE_SL if a.op == "laplace" else bem.BEMBEL_HELMHOLTZ_SL
    prec = bem.BEMBEL_PREC_MIXED if a.fp32 else bem.BEMBEL_PREC_FP64
    var = {f"g_{c}_var": [int(v) for v in getattr(a, f"g_{c}_var").split(",")]
           for c in ("identical", "edge", "vertex") if getattr(a, f"g_{c}_var")}
    op = bem.bembel_assemble(geom, op_kind, a.k if a.op == "helmholtz" else 0.0, a.level, a.degree, a.q,
                             g_regular=a.g_regular, g_singular=a.g_singular, g_regular_far=a.g_regular_far,
                             precision=prec, **var)
    n = bem.bembel_ndofs(op)
    cplx = a.op == "helmholtz"
    dt = (torch.complex64 if a.fp32 else torch.complex128) if cplx else (torch.float32 if a.fp32 else torch.float64)
    x = torch.randn((a.nrhs, n), dtype=dt, device="cuda")
    y = torch.empty_like(x)
    for _ in range(a.matvecs):
        bem.bembel_matvec(op, x, y, a.nrhs, fp32=a.fp32)
    torch.cuda.synchronize()
    info = bem.bembel_op_info_get(op)
    if a.solve:
        bdt = torch.complex128 if cplx else torch.float64
        b = torch.empty(n, dtype=bdt, device="cuda")
        bem.bembel_rhs(op, bem.BEMBEL_RHS_POINT_SOURCE, [[0.0, 0.0, 2.0]], b)
        xs = torch.empty_like(b)
        pc = bem.BEMBEL_PRECOND_BLOCK_JACOBI if a.precond else bem.BEMBEL_PRECOND_NONE
        info["solve"] = bem.bembel_solve(op, b, xs, 1, tol=1e-8, precond=pc)
    print(json.dumps({k: v for k, v in info.items()}))


if __name__ == "__main__":
    main()
