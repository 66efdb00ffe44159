"""Train the learned preconditioner on radially perturbed spheres and compare it
with block-Jacobi on held-out ones (GMRES iterations and time to 1e-8).

    python -m paper_1906_00785_gb300.learned_experiment --train 200 --eval 50 --level 4

Geometry r = 1 + 0.1 sum_{l<=4} a_lm Y_lm, a_lm ~ N(0,1)/l^2 (training seeds
1000.., held-out seeds 2000..), Helmholtz k = 8, degree-2 B-splines, q = 4,
one plane-wave right-hand side per held-out system (incidence +z).  Prints one
JSON line.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from inputs import perturbed_sphere_coeffs

from . import capi as bem


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=200)
    ap.add_argument("--eval", type=int, default=50)
    ap.add_argument("--level", type=int, default=4)
    ap.add_argument("--eval-level", type=int, default=None)
    ap.add_argument("--degree", type=int, default=2)
    ap.add_argument("--k", type=float, default=8.0)
    ap.add_argument("--epochs", type=int, default=150)
    ap.add_argument("--lr", type=float, default=0.02)
    ap.add_argument("--samples", type=int, default=4)
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--fp64", action="store_true", help="solve in FP64 instead of the mixed form")
    a = ap.parse_args()
    torch.cuda.set_device(0)
    el = a.eval_level if a.eval_level is not None else a.level
    t0 = time.perf_counter()
    sets = []
    for i in range(a.train):
        seed = 1000 + i
        g = bem.bembel_geom_create(bem.BEMBEL_GEOM_PERTURBED_SPHERE, coeffs=perturbed_sphere_coeffs(seed))
        op = bem.bembel_assemble(g, bem.BEMBEL_HELMHOLTZ_SL, a.k, a.level, a.degree, 4)
        sets.append(bem.bembel_learned_collect(op, a.samples, seed))
        del op
    t_collect = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    p0 = (rng.standard_normal(bem.BEMBEL_LEARNED_NPARAM) * 0.1).astype(np.float32)
    p0[-17:] = 0.0
    t0 = time.perf_counter()
    params, hist = bem.bembel_learned_train(sets, a.epochs, a.lr, p0)
    t_train = time.perf_counter() - t0
    del sets
    rows, noprec = [], []
    for i in range(a.eval):
        seed = 2000 + i
        g = bem.bembel_geom_create(bem.BEMBEL_GEOM_PERTURBED_SPHERE, coeffs=perturbed_sphere_coeffs(seed))
        op = bem.bembel_assemble(g, bem.BEMBEL_HELMHOLTZ_SL, a.k, el, a.degree, 4,
                                 precision=bem.BEMBEL_PREC_FP64 if a.fp64 else bem.BEMBEL_PREC_MIXED)
        n = bem.bembel_ndofs(op)
        b = torch.empty(n, dtype=torch.complex128, device="cuda")
        bem.bembel_rhs(op, bem.BEMBEL_RHS_PLANE_WAVE, [[0.0, 0.0, 1.0]], b)
        x = torch.empty_like(b)
        bj = bem.bembel_solve(op, b, x, 1, tol=1e-8, restart=a.restart, precond=bem.BEMBEL_PRECOND_BLOCK_JACOBI)
        bem.bembel_learned_attach(op, params)
        ln = bem.bembel_solve(op, b, x, 1, tol=1e-8, restart=a.restart, precond=bem.BEMBEL_PRECOND_LEARNED)
        nop = bem.bembel_solve(op, b, x, 1, tol=1e-8, restart=a.restart) if i < 5 else None
        rows.append((bj["iterations"], ln["iterations"], bj["solve_ms"], ln["solve_ms"], bj["converged"],
                     ln["converged"]))
        if nop is not None:
            noprec.append(nop["iterations"])
        del op
    r = np.array(rows, dtype=float)
    out = {"experiment": "learned_vs_block_jacobi", "k": a.k, "degree": a.degree, "train_level": a.level,
           "eval_level": el, "n_train": a.train, "n_eval": a.eval, "epochs": a.epochs,
           "loss_first": float(hist[0]), "loss_last": float(hist[-1]), "collect_s": t_collect, "train_s": t_train,
           "iters_block_jacobi_mean": float(r[:, 0].mean()), "iters_learned_mean": float(r[:, 1].mean()),
           "ms_block_jacobi_mean": float(r[:, 2].mean()), "ms_learned_mean": float(r[:, 3].mean()),
           "all_converged": bool(r[:, 4:].all()), "params_l2": float(np.linalg.norm(params)),
           "iters_unpreconditioned_first5": noprec, "restart": a.restart, "fp64": a.fp64}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
