"""Timed runs of the batched, multi-mesh and EFIE workloads (one GPU).

    python -m paper_1906_00785_gb300.config_runs helmholtz-batch --level 6 --k 2 --nrhs 64
    python -m paper_1906_00785_gb300.config_runs multimesh
    python -m paper_1906_00785_gb300.config_runs efie --level 4 --degree 2 --k 4 --q 6

Each prints one JSON line.  Inputs are synthetic and seeded: the unit sphere as
six cube-face patches, plane-wave directions uniform on S^2 (seed 3).  Times are
CUDA-event or synchronised wall times on the device; no correctness checks here
(the tests cover them).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import capi as bem


def _directions(n: int, seed: int = 3) -> np.ndarray:
    d = np.random.default_rng(seed).standard_normal((n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def _timed(fn, reps: int = 1):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        out = fn()
    torch.cuda.synchronize()
    return out, (time.perf_counter() - t0) * 1e3 / reps


def _matvec_ms(op, x, nrhs, fp32, reps=10):
    y = torch.empty_like(x)
    for _ in range(2):
        bem.bembel_matvec(op, x, y, nrhs, fp32=fp32)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        bem.bembel_matvec(op, x, y, nrhs, fp32=fp32)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def helmholtz_batch(a):
    g = bem.bembel_geom_create()
    HEL = bem.BEMBEL_HELMHOLTZ_SL
    opts, tune = bem.bembel_autotune(g, HEL, a.k, a.level, a.degree, quad_tol=a.quad_tol, far_tol=1e-4, q_max=4)
    op, t_asm = _timed(lambda: bem.bembel_assemble(g, HEL, a.k, a.level, a.degree, 4, opts=opts,
                                                   precision=bem.BEMBEL_PREC_MIXED))
    n = bem.bembel_ndofs(op)
    dirs = _directions(a.nrhs)
    B = torch.empty((a.nrhs, n), dtype=torch.complex128, device="cuda")
    bem.bembel_rhs(op, bem.BEMBEL_RHS_PLANE_WAVE, dirs, B)
    X = torch.empty_like(B)
    bj = bem.BEMBEL_PRECOND_BLOCK_JACOBI
    info_b, t_b = _timed(lambda: bem.bembel_solve(op, B, X, a.nrhs, tol=1e-8, precond=bj, restart=50,
                                                  max_iter=2000))
    # the same systems one column at a time (mixed, block-Jacobi), on a sample of columns
    ns = min(a.nrhs, a.single_sample)
    t_single = 0.0
    iters_single = []
    for r in range(ns):
        xr = torch.empty_like(B[r])
        info, t = _timed(lambda: bem.bembel_solve(op, B[r].contiguous(), xr, 1, tol=1e-8, precond=bj, restart=50,
                                                  max_iter=2000))
        t_single += t
        iters_single.append(info["iterations"])
    # plain FP64 GPU path (FP64 operator, no preconditioner), one column
    op64 = bem.bembel_assemble(g, HEL, a.k, a.level, a.degree, 4, opts=opts)
    x64 = torch.empty_like(B[0])
    info64, t64 = _timed(lambda: bem.bembel_solve(op64, B[0].contiguous(), x64, 1, tol=1e-8, restart=50,
                                                  max_iter=2000))
    Xr = torch.randn((a.nrhs, n), dtype=torch.complex64, device="cuda")
    mv_tc = _matvec_ms(op, Xr, a.nrhs, True)
    opcc = bem.bembel_assemble(g, HEL, a.k, a.level, a.degree, 4, opts=opts, precision=bem.BEMBEL_PREC_MIXED,
                               tensor_cores=0)
    mv_cc = _matvec_ms(opcc, Xr, a.nrhs, True)
    return {"workload": f"helmholtz_sphere6_L{a.level}_p{a.degree}_k{a.k}_q4_{a.nrhs}rhs", "ndofs": n,
            "assemble_ms": t_asm, "autotune": {k: v for k, v in tune.items() if k.startswith("g_")},
            "batched_solve_ms": t_b, "batched_iters": info_b["iterations"], "batched_relres": info_b["rel_residual"],
            "batched_ms_per_rhs": t_b / a.nrhs, "single_solve_ms_per_rhs": t_single / ns,
            "single_iters": iters_single, "fp64_plain_ms_per_rhs": t64, "fp64_plain_iters": info64["iterations"],
            "speedup_per_rhs_vs_fp64_plain": t64 / (t_b / a.nrhs),
            "fp32_matvec_ms_tensor_cores": mv_tc, "fp32_matvec_ms_cuda_cores": mv_cc,
            "matvec_gdof_rhs_per_s_tensor_cores": n * a.nrhs / mv_tc / 1e6}


def multimesh(a):
    g = bem.bembel_geom_create()
    HEL = bem.BEMBEL_HELMHOLTZ_SL
    levels = [3, 4, 5, 6] * 4
    ks = [2.0, 8.0, 16.0]
    items = [(g, ks[i % 3], L) for i, L in enumerate(levels)]
    kw = dict(precision=bem.BEMBEL_PREC_MIXED, g_identical_var=(4, 5, 3, 3), g_edge_var=(4, 5, 5, 3),
              g_vertex_var=(4, 5, 5, 5), g_regular=5, g_regular_far=4)
    bem.bembel_assemble_batch(items[:2], HEL, a.degree, 4, **kw)  # warm-up
    ops, t_batch = _timed(lambda: bem.bembel_assemble_batch(items, HEL, a.degree, 4, **kw))
    dev_batch = bem.bembel_op_info_get(ops[0])["assemble_ms"]
    del ops

    def sequential():
        out = [bem.bembel_assemble(gg, HEL, k, L, a.degree, 4, **kw) for gg, k, L in items]
        return out

    ops, t_seq = _timed(sequential)
    dev_seq = sum(bem.bembel_op_info_get(o)["assemble_ms"] for o in ops)
    ndofs = sum(bem.bembel_ndofs(o) for o in ops)
    return {"workload": "16 spheres, levels {3,4,5,6} x 4, k cycling {2,8,16}, Helmholtz degree 2, q 4",
            "ndofs_total": ndofs, "batch_wall_ms": t_batch, "batch_device_ms": dev_batch,
            "sequential_wall_ms": t_seq, "sequential_device_ms": dev_seq}


def efie(a):
    g = bem.bembel_geom_create()
    MAX = bem.BEMBEL_MAXWELL_SL
    out = {"workload": f"efie_sphere6_L{a.level}_p{a.degree}_k{a.k}"}
    for q in (0, a.q):
        op, t_asm = _timed(lambda: bem.bembel_assemble(g, MAX, a.k, a.level, a.degree, q))
        info = bem.bembel_op_info_get(op)
        n = bem.bembel_ndofs(op)
        b = torch.empty(n, dtype=torch.complex128, device="cuda")
        bem.bembel_rhs(op, bem.BEMBEL_RHS_EFIE_PLANE_WAVE, np.array([[0, 0, 1.0, 1.0, 0, 0]]), b)
        x = torch.empty_like(b)
        sol, t_sol = _timed(lambda: bem.bembel_solve(op, b, x, 1, tol=a.tol, precond=bem.BEMBEL_PRECOND_BLOCK_JACOBI,
                                                     restart=100, max_iter=4000))
        mv = _matvec_ms(op, torch.randn(n, dtype=torch.complex128, device="cuda"), 1, False)
        out["dense" if q == 0 else f"h2_q{q}"] = {
            "ndofs": n, "assemble_ms": t_asm, "near_bytes": info["near_bytes"],
            "far_blocks": info["n_far_blocks"], "matvec_ms": mv, "solve_ms": t_sol,
            "iterations": sol["iterations"], "rel_residual": sol["rel_residual"]}
        del op
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("run", choices=["helmholtz-batch", "multimesh", "efie"])
    ap.add_argument("--level", type=int, default=6)
    ap.add_argument("--degree", type=int, default=2)
    ap.add_argument("--k", type=float, default=2.0)
    ap.add_argument("--q", type=int, default=6)
    ap.add_argument("--nrhs", type=int, default=64)
    ap.add_argument("--single-sample", type=int, default=4)
    ap.add_argument("--quad-tol", type=float, default=1e-6)
    ap.add_argument("--tol", type=float, default=1e-6)
    a = ap.parse_args()
    torch.cuda.set_device(0)
    fn = {"helmholtz-batch": helmholtz_batch, "multimesh": multimesh, "efie": efie}[a.run]
    print(json.dumps(fn(a)), flush=True)


if __name__ == "__main__":
    main()
