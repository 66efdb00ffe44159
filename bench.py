"""Benchmark of the H^2 single-layer hot path on GB300.

Workload (the Laplace H^2 configuration): unit sphere as 6 cube-face patches,
level 6 (24,576 elements), degree-1 B-splines (25,350 dofs), 4 x 4 Chebyshev
interpolation per cluster, eta = 1.6, leaf level 5, quadrature orders chosen by
the autotuner for 1e-6 relative block accuracy (per class and per Duffy
variable; separated pairs next to the touching ones apart from those beyond).
Data: point charge u = 1/|x - x0|, x0 = (0, 0, 2), potential at 100 seeded
points in the ball of radius 0.5.  All inputs are synthetic.

One step = one pass of the whole hot path: assemble the compressed operator
(topology, trees, near-field regular + singular quadrature, coupling), load
vector, GMRES to relative residual 1e-8 (mixed precision: FP32 inner solves,
FP64 refinement) and potential evaluation, then release the operator.
value = dofs solved per second over the timed steps (GDOF/s).  The plain FP64
GPU path (FP64 everywhere, same GMRES) is timed on the same operator size for
the time-to-1e-8 comparison, and the FP64 / FP32 matvec throughputs are timed
separately (median of CUDA-event timings).

Multi-GPU: the path does not shard; N ranks run N independent replicas
(one per GPU), value = total dofs solved / max-over-ranks time.

After the headline numbers the other workloads run at bounded sizes and are
reported under "configs" (batched Helmholtz plane waves at kappa = 2, 8, the
multi-mesh persistent assembly, the EFIE, the learned preconditioner); --no-legs
skips them, --mode <leg> runs one alone, --mode profile runs one assembly and a
few products for ncu.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H² assembly time & matvec GDOF/s; GMRES time-to-1e-8 vs plain FP64 GPU path"
# g_reg / g_sing: the orders the autotuner picks for quad_tol on this workload (separated pairs in
# the ring / beyond it; per-variable Duffy orders identical, edge, vertex): the CPU oracle of the
# reference arm, which cannot run the GPU autotuner, integrates at these
WORKLOAD = dict(level=6, p=1, q=4, eta=1.6, leaf=5, g_reg=(5, 4), g_sing=((4, 5, 3, 3), (4, 5, 5, 3), (4, 5, 5, 5)),
                quad_tol=1e-6, x0=(0.0, 0.0, 2.0), n_eval=100)
# FP64 flops per quadrature point, counted from the formulas:
# regular pair point (x_p, y_q): difference, squared norm, 1/r, 4 (d=1) weighted products
FLOPS_REG_POINT = {0: 12, 1: 18, 2: 28}
# identical-pair Duffy point: rule map + both patch maps + 1/r + (d+1)^4 basis products
FLOPS_SING_POINT = {0: 80, 1: 110, 2: 250}
# one side point of the factorised edge / vertex rules: patch map + weighted Bernstein values
FLOPS_SIDE_POINT = {0: 22, 1: 30, 2: 48}
# DRAM bytes (read + write) per pair of the degree-1 quadrature kernels, from one ncu capture of
# the level-5 launches at the autotuned orders (profiles/quadrature_kernels_laplace_L5_p1.md):
# the traffic is the pair records and geometry read (Duffy kernels; their blocks stay in L2 during
# the launch) and grows with the number of pairs, so it scales to the level-6 launch
DRAM_BYTES_PER_PAIR = {"near_regular": (13671680 + 15446016) / 254412,
                       "singular_identical": (286976 + 2304) / 6144,
                       "singular_edge": (570368 + 256) / 12288,
                       "singular_vertex": (526336 + 1024) / 12276}


def touching_pair_flops(kind, g, p):
    """FP64 flops of one common-edge / common-vertex pair in the factorised rule sums:
    every rule point is one kernel evaluation with its (d+1)^2 row update (the regular-point
    count), every distinct side point one patch map, every outer point one (d+1)^4 outer product."""
    g0, g1, g2, g3 = g
    fk, fp, fo = FLOPS_REG_POINT[p], FLOPS_SIDE_POINT[p], 2 * (p + 1) ** 4
    if kind == "vertex":
        items, staged, moving = 2 * g0 * g2 * g3 + 2 * g0 * g1 * g2, 2 * g0 * g1 + 2 * g0 * g3, 0
    else:
        items = 2 * g0 * g3 * g2 + 4 * g0 * g2 * g3
        staged, moving = 2 * g0 * g3 * g1, 4 * g0 * g2 * g3 * g1
    npts = (4 if kind == "vertex" else 6) * g0 * g1 * g2 * g3
    return npts * fk + items * (fp + fo) + (staged + moving) * fp


def reduce_max(x: float, world: int, device) -> float:
    """Largest value of x over the ranks of the job (x itself on one rank)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gdofs(dofs_per_rank: int, world: int, ms: float) -> float:
    """Dofs solved by all replicas per second (GDOF/s) at the slowest rank's step time ms."""
    return dofs_per_rank * world / (ms / 1e3) / 1e9


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-legs", action="store_true", help="skip the other workloads after the headline step")
    ap.add_argument("--mode", choices=["bench", "profile", "helmholtz-batch", "multimesh", "efie", "learned"],
                    default="bench", help="one workload leg alone (one JSON line), or the profiling workload")
    # legs and the profiling workload
    ap.add_argument("--op", choices=["laplace", "helmholtz"], default=None,
                    help="operator of the profile (default laplace) and learned (default helmholtz) modes")
    ap.add_argument("--k", type=float, default=None)
    ap.add_argument("--level", type=int, default=None)
    ap.add_argument("--degree", type=int, default=None)
    ap.add_argument("--q", type=int, default=4)
    ap.add_argument("--kdiam", type=float, default=0.0)
    ap.add_argument("--nrhs", type=int, default=None)
    ap.add_argument("--g-regular", type=int, default=4)
    ap.add_argument("--g-singular", type=int, default=5)
    ap.add_argument("--g-regular-far", type=int, default=0)
    for cls in ("identical", "edge", "vertex"):
        ap.add_argument(f"--g-{cls}-var", type=str, default="", help="four per-variable Duffy orders, e.g. 4,5,3,3")
    ap.add_argument("--matvecs", type=int, default=3)
    ap.add_argument("--fp32", action="store_true")
    ap.add_argument("--solve", action="store_true", help="profile mode: also a GMRES solve to 1e-8")
    ap.add_argument("--train", type=int, default=40)
    ap.add_argument("--eval", type=int, default=10)
    ap.add_argument("--epochs", type=int, default=150)
    ap.add_argument("--coarse-level", type=int, default=0, help="learned mode: coarse space level (0: level - 3)")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = sorted(float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit())
        mx = max(float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for n, v in zip(names, s[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(self.samples)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def fp64_peak_tflops(sm_mhz: float) -> float:
    # 152 SMs x 2 FP64 FMA lanes per SM per clock x 2 flops (nominal 1.25 TFLOP/s at 2.06 GHz)
    return 152 * 2 * 2 * sm_mhz * 1e6 / 1e12


def oracle_orders(tune=None):
    """Quadrature orders for the oracle: the autotuned ones of the GPU run (separated ring and
    beyond, per-variable Duffy orders), else the workload's defaults."""
    w = WORKLOAD
    if not tune:
        return w["g_reg"], w["g_sing"]
    var = tuple(tuple(tune[f"g_{c}_var"]) if all(tune[f"g_{c}_var"]) else tune[f"g_{c}"]
                for c in ("identical", "edge", "vertex"))
    return (tune["g_regular"], tune["g_regular_far"] or tune["g_regular"]), var


def cpu_baseline_sample(n_rows: int = 1, iters: int = 60, orders=None, seed: int = 5):
    """Time the CPU oracle on a bounded sample of the workload: sampled rows of A~ x.

    First application of a row includes its near-field quadrature and moments
    (assembly work); the second reuses cached element blocks (matvec work).
    Extrapolated time to solve all dofs = ndofs * (t_first + iters * t_again).
    Returns (value GDOF/s, details).
    """
    import numpy as np

    from inputs import random_vector
    from oracle.geometry import Sphere6
    from oracle.h2 import H2Oracle
    from oracle.space import S2Space

    w = WORKLOAD
    g_reg, g_sing = orders if orders else (w["g_reg"], w["g_sing"])
    c_start, w_start = time.process_time(), time.perf_counter()
    sp = S2Space(Sphere6(), w["level"], w["p"])
    t0 = time.perf_counter()
    h2 = H2Oracle(sp, "laplace", q=w["q"], eta=w["eta"], leaf_level=w["leaf"], g_reg=g_reg, g_sing=g_sing)
    t_tree = time.perf_counter() - t0
    rows = np.random.default_rng(seed).choice(sp.ndofs, n_rows, replace=False)
    x = random_vector(sp.ndofs, 2)
    t0 = time.perf_counter()
    h2.apply_rows(x, rows)
    t_first = (time.perf_counter() - t0) / n_rows
    t0 = time.perf_counter()
    h2.apply_rows(x * 0.5, rows)
    t_again = (time.perf_counter() - t0) / n_rows
    total = sp.ndofs * (t_first + iters * t_again) + t_tree
    # cores actually used: process CPU time over wall time of the sample
    cores = max(1, round((time.process_time() - c_start) / (time.perf_counter() - w_start)))
    return sp.ndofs / total / 1e9, dict(t_tree_s=t_tree, t_row_first_s=t_first, t_row_again_s=t_again,
                                        iters=iters, rows=n_rows, extrapolated_s=total, cores=cores)


def _oracle_worker(args):
    """One process of the all-cores CPU baseline (started by spawn, BLAS on one thread)."""
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    os.environ["OMP_NUM_THREADS"] = "1"
    iters, orders, seed = args
    return cpu_baseline_sample(1, iters, orders, seed)[1]


def cpu_baseline_all_cores(iters: int, orders, workers: int):
    """The same sampled-row oracle in `workers` spawned processes, one row each, at once: the
    extrapolated time divides the rows over the processes (tree build once per process)."""
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(workers) as pool:
        dets = pool.map(_oracle_worker, [(iters, orders, 100 + i) for i in range(workers)])
    wall = time.perf_counter() - t0
    t_first = sum(d["t_row_first_s"] for d in dets) / workers
    t_again = sum(d["t_row_again_s"] for d in dets) / workers
    t_tree = max(d["t_tree_s"] for d in dets)
    total = WORKLOAD_NDOFS * (t_first + iters * t_again) / workers + t_tree
    return WORKLOAD_NDOFS / total / 1e9, dict(workers=workers, wall_s=wall, t_row_first_s=t_first,
                                             t_row_again_s=t_again, t_tree_s=t_tree, iters=iters,
                                             extrapolated_s=total)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np  # noqa: F401

    vals = []
    det = None
    for i in range(args.warmup + args.steps):
        v, det = cpu_baseline_sample(1)
        if i >= args.warmup:
            vals.append(v)
    value = float(sorted(vals)[len(vals) // 2]) if vals else 0.0
    ms = 1e3 * WORKLOAD_NDOFS / (value * 1e9) if value else None
    sample = (f"oracle sampled rows at the GPU's autotuned quadrature orders {oracle_orders()}: "
              f"1 row of A~x per step (first application with its near-field quadrature, "
              f"second with cached blocks), extrapolated to all {WORKLOAD_NDOFS} dofs x {det['iters']} GMRES "
              f"applications + tree build; numpy, BLAS limited to 1 thread")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "laplace_h2_sphere6_L6_p1_q4_eta1.6", "ndofs": WORKLOAD_NDOFS, "nrhs": 1},
            "cpu_baseline": {"value": value, "unit": "GDOF/s", "cores": det["cores"], "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "details": det}
    print(json.dumps(line))


WORKLOAD_NDOFS = 6 * (2**6 + 1) ** 2


# ---------------------------------------------------------------------------------------------
# Workload legs beside the headline step: the batched Helmholtz, multi-mesh, EFIE and learned-
# preconditioner configurations at bounded sizes (each a few seconds), and a profiling mode.
# Every leg is one GPU, synthetic seeded inputs, CUDA-event or synchronised device times.
# ---------------------------------------------------------------------------------------------
def _directions(n: int, seed: int = 3):
    import numpy as np

    d = np.random.default_rng(seed).standard_normal((n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def _timed(fn):
    import torch

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, (time.perf_counter() - t0) * 1e3


def _matvec_ms(bem, op, x, nrhs, fp32, reps=10):
    import torch

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


def _sound_soft_series(k, pts, d):
    """Scattered field of the sound-soft unit sphere for u_inc = exp(-i k d.x) (kernel
    exp(-i kappa r)): u_s = -sum_l (2l+1) (-i)^l j_l(k)/h2_l(k) h2_l(k|x|) P_l(cos angle)."""
    import numpy as np
    import scipy.special as ss

    rr = np.linalg.norm(pts, axis=1)
    c = pts @ d / rr
    out = np.zeros(len(pts), dtype=complex)
    for l in range(int(2 * k) + 30):
        h2k = ss.spherical_jn(l, k) - 1j * ss.spherical_yn(l, k)
        h2r = ss.spherical_jn(l, k * rr) - 1j * ss.spherical_yn(l, k * rr)
        out += -(2 * l + 1) * (-1j) ** l * ss.spherical_jn(l, k) / h2k * h2r * ss.eval_legendre(l, c)
    return out


def leg_helmholtz_batch(bem, k: float, level: int, nrhs: int = 64, degree: int = 2, kdiam: float = 0.0,
                        q_max: int = 6, single_sample: int = 2):
    """Sound-soft sphere, nrhs plane waves (seeded directions) solved together (MIXED, block-
    Jacobi, FP64 refinement) vs one column at a time and vs the plain FP64 path; the
    scattered field of the first wave against the partial-wave series."""
    import numpy as np
    import torch

    from inputs import sphere_points

    g = bem.bembel_geom_create()
    HEL = bem.BEMBEL_HELMHOLTZ_SL
    opts, tune = bem.bembel_autotune(g, HEL, k, level, degree, quad_tol=1e-6, far_tol=1e-4, q_max=q_max,
                                     kdiam=kdiam, precision=bem.BEMBEL_PREC_MIXED)
    q = tune["q"]
    op, t_asm = _timed(lambda: bem.bembel_assemble(g, HEL, k, level, degree, q, opts=opts,
                                                   precision=bem.BEMBEL_PREC_MIXED))
    info = bem.bembel_op_info_get(op)
    n = bem.bembel_ndofs(op)
    dirs = _directions(nrhs)
    B = torch.empty((nrhs, n), dtype=torch.complex128, device="cuda")
    bem.bembel_rhs(op, bem.BEMBEL_RHS_PLANE_WAVE, dirs, B)
    B = -B  # Dirichlet data of the scattered field
    X = torch.empty_like(B)
    bj = bem.BEMBEL_PRECOND_BLOCK_JACOBI
    solve = dict(tol=1e-8, restart=50, max_iter=3000)
    info_b, t_b = _timed(lambda: bem.bembel_solve(op, B, X, nrhs, precond=bj, **solve))
    pts = sphere_points(20, 3.0, 11)
    U = torch.empty((1, 20), dtype=torch.complex128, device="cuda")
    bem.bembel_eval(op, torch.from_numpy(pts).cuda(), X[0].contiguous(), U, 1, g=6)
    ref = _sound_soft_series(k, pts, dirs[0])
    err = float(np.max(np.abs(U.cpu().numpy()[0] - ref)) / np.max(np.abs(ref)))
    t_single = []
    for r in range(min(nrhs, single_sample)):
        xr = torch.empty_like(B[r])
        _, t = _timed(lambda: bem.bembel_solve(op, B[r].contiguous(), xr, 1, precond=bj, **solve))
        t_single.append(t)
    op64 = bem.bembel_assemble(g, HEL, k, level, degree, q, opts=opts)
    x64 = torch.empty_like(B[0])
    info64, t64 = _timed(lambda: bem.bembel_solve(op64, B[0].contiguous(), x64, 1, **solve))
    del op64
    # the wide FP32 product: tensor-core coupling on stored bf16 tiles (q = 4 only) against the
    # stored FP32 coupling streamed on the CUDA cores
    Xr = torch.randn((nrhs, n), dtype=torch.complex64, device="cuda")
    mv_default = _matvec_ms(bem, op, Xr, nrhs, True)
    opcc = bem.bembel_assemble(g, HEL, k, level, degree, q, opts=opts, precision=bem.BEMBEL_PREC_MIXED,
                               tensor_cores=0)
    mv_cc = _matvec_ms(bem, opcc, Xr, nrhs, True)
    del opcc
    return {"workload": f"helmholtz_sound_soft_sphere6_L{level}_p{degree}_k{k:g}_{nrhs}rhs", "ndofs": n, "q": q,
            "kdiam": kdiam, "far_blocks": info["n_far_blocks"], "near_gb": info["near_bytes"] / 1e9,
            "far_gb": info["far_bytes"] / 1e9, "autotune_err_far": tune["err_far"],
            "leaf_level": tune["leaf_level"], "leaf_scores_ms": tune["leaf_score_ms"],
            "far_fp32_stored": tune["far_fp32_stored"], "assemble_ms": t_asm,
            "batched_solve_ms": t_b, "batched_iters": info_b["iterations"], "batched_relres": info_b["rel_residual"],
            "batched_ms_per_rhs": t_b / nrhs, "single_ms_per_rhs": float(np.mean(t_single)),
            "fp64_plain_ms_per_rhs": t64, "fp64_plain_iters": info64["iterations"],
            "fp64_plain_converged": info64["converged"],
            "speedup_per_rhs_vs_fp64_plain": t64 / (t_b / nrhs), "field_rel_err_vs_series": err,
            "fp32_matvec_ms_tensor_cores": mv_default if q == 4 else None,
            "fp32_matvec_ms_cuda_cores_stored": mv_cc}


def leg_multimesh(bem, degree: int = 2):
    """16 unit spheres of levels {3, 4, 5, 6} x 4, k cycling {2, 8, 16}: one persistent launch
    for all meshes against 16 separate assemblies."""
    HEL = bem.BEMBEL_HELMHOLTZ_SL
    g = bem.bembel_geom_create()
    levels = [3, 4, 5, 6] * 4
    ks = [2.0, 8.0, 16.0]
    items = [(g, ks[i % 3], L) for i, L in enumerate(levels)]
    kw = dict(precision=bem.BEMBEL_PREC_MIXED, g_identical_var=(4, 5, 3, 3), g_edge_var=(4, 5, 5, 3),
              g_vertex_var=(4, 5, 5, 5), g_regular=5, g_regular_far=4)
    bem.bembel_assemble_batch(items[:2], HEL, degree, 4, **kw)  # warm-up
    ops, t_batch = _timed(lambda: bem.bembel_assemble_batch(items, HEL, degree, 4, **kw))
    dev_batch = bem.bembel_op_info_get(ops[0])["assemble_ms"]
    del ops
    ops, t_seq = _timed(lambda: [bem.bembel_assemble(gg, HEL, k, L, degree, 4, **kw) for gg, k, L in items])
    dev_seq = sum(bem.bembel_op_info_get(o)["assemble_ms"] for o in ops)
    ndofs = sum(bem.bembel_ndofs(o) for o in ops)
    del ops
    return {"workload": "16 spheres, levels {3,4,5,6} x 4, k cycling {2,8,16}, Helmholtz degree 2, q 4",
            "ndofs_total": ndofs, "batch_wall_ms": t_batch, "batch_device_ms": dev_batch,
            "sequential_wall_ms": t_seq, "sequential_device_ms": dev_seq}


def leg_efie(bem, level: int = 4, degree: int = 2, k: float = 4.0, q: int = 6, tol: float = 1e-8,
             restart: int = 200, max_iter: int = 3000):
    """PEC sphere, plane wave along +z polarised in x: dense and H^2 EFIE, assembly, matvec,
    solve, and the scattered field at 40 points of radius 3 against the Mie series."""
    import numpy as np
    import torch

    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from mie import scattered_pec

    g = bem.bembel_geom_create()
    MAX = bem.BEMBEL_MAXWELL_SL
    pts = np.random.default_rng(4).standard_normal((40, 3))
    pts *= (3.0 / np.linalg.norm(pts, axis=1))[:, None]
    ref = scattered_pec(pts, k)
    out = {"workload": f"efie_pec_sphere6_L{level}_p{degree}_k{k:g}"}
    for qq, prec in ((0, bem.BEMBEL_PREC_FP64), (q, bem.BEMBEL_PREC_FP64), (q, bem.BEMBEL_PREC_MIXED)):
        op, t_asm = _timed(lambda: bem.bembel_assemble(g, MAX, k, level, degree, qq, precision=prec))
        info = bem.bembel_op_info_get(op)
        n = bem.bembel_ndofs(op)
        b = torch.empty(n, dtype=torch.complex128, device="cuda")
        bem.bembel_rhs(op, bem.BEMBEL_RHS_EFIE_PLANE_WAVE, np.array([[0, 0, 1.0, 1.0, 0, 0]]), b)
        x = torch.empty_like(b)
        sol, t_sol = _timed(lambda: bem.bembel_solve(op, b, x, 1, tol=tol, precond=bem.BEMBEL_PRECOND_BLOCK_JACOBI,
                                                     restart=restart, max_iter=max_iter))
        E = torch.empty((40, 3), dtype=torch.complex128, device="cuda")
        bem.bembel_eval(op, torch.from_numpy(pts).cuda(), x, E, 1, g=6)
        err = float(np.linalg.norm(E.cpu().numpy() - ref) / np.linalg.norm(ref))
        mv = _matvec_ms(bem, op, torch.randn(n, dtype=torch.complex128, device="cuda"), 1, False)
        mixed = prec == bem.BEMBEL_PREC_MIXED
        out["dense" if qq == 0 else f"h2_q{qq}" + ("_mixed" if mixed else "")] = {
            "ndofs": n, "assemble_ms": t_asm, "near_gb": info["near_bytes"] / 1e9, "far_blocks": info["n_far_blocks"],
            "matvec_ms": mv, "solve_ms": t_sol, "iterations": sol["iterations"], "refinements": sol["refinements"],
            "converged": sol["converged"],
            "rel_residual": sol["rel_residual"], "field_rel_err_vs_mie": err}
        del op
    return out


def leg_learned(bem, n_train: int = 40, n_eval: int = 10, level: int = 6, degree: int = 2, k: float = 8.0,
                epochs: int = 150, samples: int = 4, restart: int = 100, max_iter: int = 4000, coarse_level: int = 0,
                const_weights=(0.25, 0.5, 0.75), pde: str = "helmholtz"):
    """Learned preconditioner on seeded perturbed spheres (training seeds 1000.., held out
    2000..): trained on the GPU, then GMRES iterations and time to 1e-8 on the held-out
    systems (one plane wave each, incidence +z, MIXED) with block-Jacobi, the two-level
    preconditioner (block-Jacobi + coarse correction; the learned form with W = I), the
    learned weights, and, as an ablation, constant weights W = w I (no network).  The
    coarse set-up (coarse assembly + inverse, once per operator) is timed apart and
    added to the two-level and learned times in the *_with_setup ratios."""
    import numpy as np
    import torch

    from inputs import perturbed_sphere_coeffs

    KIND = bem.BEMBEL_HELMHOLTZ_SL if pde == "helmholtz" else bem.BEMBEL_LAPLACE_SL
    if pde != "helmholtz":
        k = 0.0
    t0 = time.perf_counter()
    sets = []
    for i in range(n_train):
        g = bem.bembel_geom_create(bem.BEMBEL_GEOM_PERTURBED_SPHERE, coeffs=perturbed_sphere_coeffs(1000 + i))
        op = bem.bembel_assemble(g, KIND, k, level, degree, 4, coarse_level=coarse_level)
        sets.append(bem.bembel_learned_collect(op, samples, 1000 + i))
        del op
    t_collect = time.perf_counter() - t0
    p0 = (np.random.default_rng(0).standard_normal(bem.BEMBEL_LEARNED_NPARAM) * 0.1).astype(np.float32)
    p0[-17:] = 0.0  # zero output layer: W = I, the two-level preconditioner
    t0 = time.perf_counter()
    params, hist = bem.bembel_learned_train(sets, epochs, 0.02, p0)
    t_train = time.perf_counter() - t0
    del sets

    def const_params(wc):  # w3 = 0, b3 = log(wc): every weight wc
        p = p0.copy()
        p[-1] = np.log(wc)
        return p

    kinds = {"block_jacobi": (bem.BEMBEL_PRECOND_BLOCK_JACOBI, None),
             "two_level": (bem.BEMBEL_PRECOND_TWO_LEVEL, None),
             "learned": (bem.BEMBEL_PRECOND_LEARNED, params)}
    for wc in const_weights:
        kinds[f"const_{wc:g}"] = (bem.BEMBEL_PRECOND_LEARNED, const_params(wc))
    rows = {name: [] for name in kinds}
    setup_ms = []
    for i in range(n_eval):
        g = bem.bembel_geom_create(bem.BEMBEL_GEOM_PERTURBED_SPHERE, coeffs=perturbed_sphere_coeffs(2000 + i))
        op = bem.bembel_assemble(g, KIND, k, level, degree, 4, precision=bem.BEMBEL_PREC_MIXED,
                                 coarse_level=coarse_level)
        n = bem.bembel_ndofs(op)
        b = torch.empty(n, dtype=torch.complex128 if k else torch.float64, device="cuda")
        if k:
            bem.bembel_rhs(op, bem.BEMBEL_RHS_PLANE_WAVE, [[0.0, 0.0, 1.0]], b)
        else:
            bem.bembel_rhs(op, bem.BEMBEL_RHS_POINT_SOURCE, [[0.0, 0.0, 2.0]], b)
        x = torch.empty_like(b)
        # block-Jacobi inverses first, then the coarse set-up alone (wall time)
        bem.bembel_precond_apply(op, bem.BEMBEL_PRECOND_BLOCK_JACOBI, b, x, 1)
        t0 = time.perf_counter()
        bem.bembel_precond_apply(op, bem.BEMBEL_PRECOND_TWO_LEVEL, b, x, 1)
        setup_ms.append(1e3 * (time.perf_counter() - t0))
        for name, (kind, prm) in kinds.items():
            if prm is not None:
                bem.bembel_learned_attach(op, prm)
            inf = bem.bembel_solve(op, b, x, 1, tol=1e-8, restart=restart, max_iter=max_iter, precond=kind)
            rows[name].append((inf["iterations"], inf["solve_ms"], inf["converged"]))
        del op
    r = {name: np.array(v, dtype=float) for name, v in rows.items()}
    su = float(np.mean(setup_ms))
    out = {"workload": f"learned_vs_block_jacobi_perturbed_{pde}_L{level}_p{degree}_k{k:g}", "n_train": n_train,
           "n_eval": n_eval, "epochs": epochs, "coarse_level": coarse_level or max(0, level - 3),
           "loss_first": float(hist[0]), "loss_last": float(hist[-1]), "collect_s": t_collect, "train_s": t_train,
           "coarse_setup_ms_mean": su}
    for name, v in r.items():
        out[f"iters_{name}_mean"] = float(v[:, 0].mean())
        out[f"ms_{name}_mean"] = float(v[:, 1].mean())
        out[f"converged_{name}"] = bool(v[:, 2].all())
    bj = r["block_jacobi"]
    for name in r:
        if name == "block_jacobi":
            continue
        out[f"iteration_ratio_{name}_over_block_jacobi"] = float(r[name][:, 0].mean() / bj[:, 0].mean())
        out[f"time_ratio_{name}_over_block_jacobi_with_setup"] = float(
            (r[name][:, 1].mean() + su) / bj[:, 1].mean())
    out["iteration_ratio_learned_over_two_level"] = float(r["learned"][:, 0].mean() / r["two_level"][:, 0].mean())
    best_const = min((n for n in r if n.startswith("const_")), key=lambda n: r[n][:, 0].mean(), default=None)
    if best_const:
        out["best_constant_weight"] = best_const
        out["iteration_ratio_learned_over_best_constant"] = float(
            r["learned"][:, 0].mean() / r[best_const][:, 0].mean())
    return out


def leg_profile(bem, a):
    """One assembly plus a few products (for capturing single kernels under ncu)."""
    import torch

    geom = bem.bembel_geom_create(bem.BEMBEL_GEOM_SPHERE6)
    a.op = a.op or "laplace"
    kind = bem.BEMBEL_LAPLACE_SL if a.op == "laplace" else bem.BEMBEL_HELMHOLTZ_SL
    prec = bem.BEMBEL_PREC_MIXED if a.fp32 else bem.BEMBEL_PREC_FP64
    var = {f"g_{c}_var": [int(v) for v in getattr(a, f"g_{c}_var").split(",")]
           for c in ("identical", "edge", "vertex") if getattr(a, f"g_{c}_var")}
    op = bem.bembel_assemble(geom, kind, a.k if a.op == "helmholtz" else 0.0, a.level, a.degree, a.q,
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
    if a.solve:  # point charge at (0, 0, 2), GMRES to 1e-8 with block-Jacobi
        b = torch.empty(n, dtype=torch.complex128 if cplx else torch.float64, device="cuda")
        bem.bembel_rhs(op, bem.BEMBEL_RHS_POINT_SOURCE, [[0.0, 0.0, 2.0]], b)
        xs = torch.empty_like(b)
        info["solve"] = bem.bembel_solve(op, b, xs, 1, tol=1e-8, precond=bem.BEMBEL_PRECOND_BLOCK_JACOBI)
    info["phase_ms"] = list(info["phase_ms"])
    return info


def main():
    args = parse()
    if args.impl == "gpu" and args.mode != "bench":
        import torch

        import paper_1906_00785_gb300 as bem

        torch.cuda.set_device(0)
        if args.mode == "profile":
            a = args
            a.k = 2.0 if a.k is None else a.k
            a.level = 5 if a.level is None else a.level
            a.degree = 1 if a.degree is None else a.degree
            a.nrhs = 1 if a.nrhs is None else a.nrhs
            out = leg_profile(bem, a)
        elif args.mode == "helmholtz-batch":
            out = leg_helmholtz_batch(bem, args.k or 2.0, args.level or 5, args.nrhs or 64,
                                      args.degree if args.degree is not None else 2, args.kdiam,
                                      q_max=max(args.q, 2))
        elif args.mode == "multimesh":
            out = leg_multimesh(bem, args.degree if args.degree is not None else 2)
        elif args.mode == "efie":
            out = leg_efie(bem, args.level or 4, args.degree or 2, args.k or 4.0, args.q if args.q != 4 else 6)
        else:
            out = leg_learned(bem, args.train, args.eval, args.level or 6, args.degree or 2, args.k or 8.0,
                              args.epochs, coarse_level=args.coarse_level, pde=args.op or "helmholtz")
        print(json.dumps(out), flush=True)
        return
    if args.impl == "reference":
        os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        run_reference(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1906_00785_gb300 as bem
    from inputs import ball_points

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    w = WORKLOAD

    geom = bem.bembel_geom_create(bem.BEMBEL_GEOM_SPHERE6)
    pts_host = torch.from_numpy(ball_points(w["n_eval"], 0.5, 1)).pin_memory()
    pts = pts_host.to(dev)
    x0 = np.array([w["x0"]])

    # quadrature orders for 1e-6 relative block accuracy, 50x below the q = 4 far-field
    # interpolation error (~5e-5): autotuned once, cached for the run
    # the leaf level and the FP32 coupling storage are chosen by timing (leaf_level -1); the
    # oracle legs use WORKLOAD["leaf"], the tuner's choice on this workload recorded there
    tuned_opts, tune = bem.bembel_autotune(geom, bem.BEMBEL_LAPLACE_SL, 0.0, w["level"], w["p"],
                                           quad_tol=w["quad_tol"], far_tol=1e-4, q_max=w["q"], eta=w["eta"],
                                           leaf_level=-1, precision=bem.BEMBEL_PREC_MIXED,
                                           stream=stream.cuda_stream)
    leaf = tuned_opts.leaf_level

    def assemble(precision):
        o = bem.bembel_opts_default()
        for f in ("g_regular", "g_regular_far", "g_singular", "g_identical", "g_edge", "g_vertex", "bsr_chunk"):
            setattr(o, f, getattr(tuned_opts, f))
        for f in ("g_identical_var", "g_edge_var", "g_vertex_var"):
            for i in range(4):
                getattr(o, f)[i] = getattr(tuned_opts, f)[i]
        return bem.bembel_assemble(geom, bem.BEMBEL_LAPLACE_SL, 0.0, w["level"], w["p"], w["q"], opts=o,
                                   eta=w["eta"], leaf_level=leaf, precision=precision,
                                   far_fp32_stored=tuned_opts.far_fp32_stored, stream=stream.cuda_stream)

    state = {}

    def step(precision=bem.BEMBEL_PREC_MIXED, pts_dev=None, out_host=None):
        op = assemble(precision)
        n = bem.bembel_ndofs(op)
        b = torch.empty(n, dtype=torch.float64, device=dev)
        bem.bembel_rhs(op, bem.BEMBEL_RHS_POINT_SOURCE, x0, b, g=6)
        rho = torch.empty_like(b)
        info = bem.bembel_solve(op, b, rho, 1, tol=1e-8, restart=30, max_iter=1000,
                                precond=bem.BEMBEL_PRECOND_BLOCK_JACOBI if precision == bem.BEMBEL_PREC_MIXED
                                else bem.BEMBEL_PRECOND_NONE)
        u = torch.empty(w["n_eval"], dtype=torch.float64, device=dev)
        bem.bembel_eval(op, pts if pts_dev is None else pts_dev, rho, u, 1, g=6)
        if out_host is not None:
            out_host[0].copy_(rho, non_blocking=True)
            out_host[1].copy_(u, non_blocking=True)
        state["info"] = info
        state["opinfo"] = bem.bembel_op_info_get(op)
        state["u"] = u
        del op
        return n

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # ---- device-resident timed steps ---------------------------------------------------
    for _ in range(args.warmup):
        step()
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    l0 = bem.bembel_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ndofs = 0
    for _ in range(args.steps):
        ndofs += step()
    e1.record(stream)
    barrier()
    sampler.stop()
    launches = bem.bembel_kernel_launches() - l0
    ms = reduce_max(e0.elapsed_time(e1) / args.steps, world, dev)
    n1 = ndofs // args.steps
    value = whole_job_gdofs(n1, world, ms)
    info, opinfo = state["info"], state["opinfo"]
    exact = 1.0 / np.linalg.norm(pts_host.numpy() - np.array(w["x0"]), axis=1)
    pot_err = float(np.max(np.abs(state["u"].cpu().numpy() - exact) / exact))

    # ---- end to end through host buffers -------------------------------------------------
    rho_host = torch.empty(n1, dtype=torch.float64).pin_memory()
    u_host = torch.empty(w["n_eval"], dtype=torch.float64).pin_memory()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        pts_step = pts_host.to(dev, non_blocking=True)
        step(pts_dev=pts_step, out_host=(rho_host, u_host))
        torch.cuda.synchronize(dev)
    barrier()
    ms_e2e = reduce_max((time.perf_counter() - t0) * 1e3 / args.steps, world, dev)
    e2e = {"value": whole_job_gdofs(n1, world, ms_e2e), "unit": "GDOF/s",
           "h2d_bytes_per_step": int(pts_host.numel() * 8 + x0.size * 8),
           "d2h_bytes_per_step": int((n1 + w["n_eval"]) * 8)}

    # ---- plain FP64 path: time to 1e-8, and matvec throughput ---------------------------
    op64 = assemble(bem.BEMBEL_PREC_FP64)
    b = torch.empty(n1, dtype=torch.float64, device=dev)
    bem.bembel_rhs(op64, bem.BEMBEL_RHS_POINT_SOURCE, x0, b, g=6)
    x = torch.empty_like(b)
    bem.bembel_solve(op64, b, x, 1, tol=1e-8)  # warm
    info64 = bem.bembel_solve(op64, b, x, 1, tol=1e-8)
    opmx = assemble(bem.BEMBEL_PREC_MIXED)
    bem.bembel_solve(opmx, b, x, 1, tol=1e-8, precond=bem.BEMBEL_PRECOND_BLOCK_JACOBI)  # warm (builds D^-1)
    infomx = bem.bembel_solve(opmx, b, x, 1, tol=1e-8, precond=bem.BEMBEL_PRECOND_BLOCK_JACOBI)
    infomx_np = bem.bembel_solve(opmx, b, x, 1, tol=1e-8)
    # two-level preconditioner: the first solve includes its set-up (coarse assembly + inverse)
    infomx_2l_first = bem.bembel_solve(opmx, b, x, 1, tol=1e-8, precond=bem.BEMBEL_PRECOND_TWO_LEVEL)
    infomx_2l = bem.bembel_solve(opmx, b, x, 1, tol=1e-8, precond=bem.BEMBEL_PRECOND_TWO_LEVEL)
    bem.bembel_solve(op64, b, x, 1, tol=1e-8, precond=bem.BEMBEL_PRECOND_BLOCK_JACOBI)  # warm (builds D^-1)
    info64_bj = bem.bembel_solve(op64, b, x, 1, tol=1e-8, precond=bem.BEMBEL_PRECOND_BLOCK_JACOBI)

    def time_matvec(op, fp32, reps=20):
        dt = torch.float32 if fp32 else torch.float64
        xx = torch.randn(n1, dtype=dt, device=dev)
        yy = torch.empty_like(xx)
        for _ in range(3):
            bem.bembel_matvec(op, xx, yy, 1, fp32=fp32)
        ts = []
        for _ in range(reps):
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            bem.bembel_matvec(op, xx, yy, 1, fp32=fp32)
            c.record(stream)
            c.synchronize()
            ts.append(a.elapsed_time(c))
        return sorted(ts)[len(ts) // 2]

    mv64_ms = time_matvec(op64, False)
    mv32_ms = time_matvec(opmx, True)

    # ---- roofline of the dominant assembly kernel -----------------------------------------
    peaks, peak_src = measured_peaks()
    clocks = sampler.summary()
    ph = opinfo["phase_ms"]
    names = ["tabulation", "near_regular", "singular_identical", "singular_edge", "singular_vertex", "coupling",
             "fp32_copies"]
    # rule points actually integrated (identical pairs: half of the 8 sub-domains, by symmetry)
    def orders(kind):  # per-variable orders when tuned so
        v = tune[f"g_{kind}_var"]
        return tuple(v) if all(v) else (tune[f"g_{kind}"],) * 4

    def npts4(kind):  # Gauss points of one sub-domain
        return int(np.prod(orders(kind)))

    n_far = opinfo["n_pairs_regular_far"]
    pts_phase = {"near_regular": (opinfo["n_pairs_regular"] - n_far) * tune["g_regular"] ** 4
                 + n_far * tune["g_regular_far"] ** 4,
                 "singular_identical": opinfo["n_pairs_identical"] * 4 * npts4("identical"),
                 "singular_edge": opinfo["n_pairs_edge"] * 6 * npts4("edge"),
                 "singular_vertex": opinfo["n_pairs_vertex"] * 4 * npts4("vertex")}
    flops_phase = {"near_regular": pts_phase["near_regular"] * FLOPS_REG_POINT[w["p"]],
                   "singular_identical": pts_phase["singular_identical"] * FLOPS_SING_POINT[w["p"]],
                   "singular_edge": opinfo["n_pairs_edge"] * touching_pair_flops("edge", orders("edge"), w["p"]),
                   "singular_vertex": opinfo["n_pairs_vertex"] * touching_pair_flops("vertex", orders("vertex"),
                                                                                     w["p"])}
    pairs_key = {"near_regular": "n_pairs_regular", "singular_identical": "n_pairs_identical",
                 "singular_edge": "n_pairs_edge", "singular_vertex": "n_pairs_vertex"}
    dom = max(flops_phase, key=lambda k: ph[names.index(k)])
    dom_ms = ph[names.index(dom)]
    achieved = flops_phase[dom] / (dom_ms / 1e3) / 1e12
    peak = fp64_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
    roofline = {"kernel": f"k_near_singular ({dom})" if dom != "near_regular" else "k_near_regular",
                "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                # ncu DRAM bytes of the level-5 launch scaled by the pairs of this launch; degree 1 only
                "traffic": (DRAM_BYTES_PER_PAIR[dom] * opinfo[pairs_key[dom]] if w["p"] == 1 else None),
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the level-5 launch, "
                                  "scaled by the pair count (level-6 capture not taken: multi-pass metrics); "
                                  "DRAM bytes during the launch: the written blocks stay in L2 and are written "
                                  "back after it (output_bytes)",
                # the blocks a launch writes: every unordered pair writes its block and the mirror
                "output_bytes": opinfo[pairs_key[dom]] * (1 if dom == "singular_identical" else 2)
                * ((w["p"] + 1) ** 2) ** 2 * 8,
                "peak_source": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2 flop x max SM clock (derived; no FP64 peak "
                               "in MEASURED_PEAKS.json)",
                "algorithmic_flops": flops_phase[dom], "launch_ms": dom_ms}
    matvec_bytes = opinfo["near_bytes"] + opinfo["far_bytes"]
    mv = {"fp64_ms": mv64_ms, "fp64_gdofs": n1 / (mv64_ms / 1e3) / 1e9,
          "fp32_ms": mv32_ms, "fp32_gdofs": n1 / (mv32_ms / 1e3) / 1e9,
          "fp64_stream_gbs": matvec_bytes / (mv64_ms / 1e3) / 1e9,
          "fp64_stream_frac_of_measured_hbm": matvec_bytes / (mv64_ms / 1e3) / 1e9 / peaks["hbm_gbs"]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        orders = oracle_orders(tune)
        v1, det1 = cpu_baseline_sample(2, iters=info64["iterations"], orders=orders)
        workers = max(1, min(16, os.cpu_count() or 1))
        vn, detn = cpu_baseline_all_cores(info64["iterations"], orders, workers)
        cpu = {"value": vn, "unit": "GDOF/s", "cores": workers, "kind": "oracle",
               "sample": f"sampled rows of A~x at the GPU's autotuned quadrature orders {orders}: one row per "
                         f"process in {workers} spawned processes (first application with its near-field "
                         f"quadrature, second with cached blocks), extrapolated to {n1} dofs x {det1['iters']} "
                         f"GMRES matvecs + tree build; single-thread figure beside it",
               "single_thread": {"value": v1, "cores": det1["cores"], "details": det1}, "details": detn}

    legs = {}
    if rank == 0 and world == 1 and not args.no_legs:
        for name, fn in (("helmholtz_k2_L5_64rhs", lambda: leg_helmholtz_batch(bem, 2.0, 5, 64, q_max=4)),
                         ("helmholtz_k2_L6_64rhs", lambda: leg_helmholtz_batch(bem, 2.0, 6, 64, q_max=4)),
                         ("helmholtz_k8_L4_64rhs", lambda: leg_helmholtz_batch(bem, 8.0, 4, 64, kdiam=6.0,
                                                                                q_max=8)),
                         ("helmholtz_k16_L5_8rhs", lambda: leg_helmholtz_batch(bem, 16.0, 5, 8, kdiam=6.0,
                                                                                q_max=8, single_sample=1)),
                         ("multimesh_16", lambda: leg_multimesh(bem)),
                         ("efie_L4_p2_k4", lambda: leg_efie(bem)),
                         ("learned_L5_p2_k8", lambda: leg_learned(bem, n_train=20, n_eval=6, level=5))):
            try:
                legs[name] = fn()
            except Exception as exc:  # a leg that fails is reported, the headline line still prints
                legs[name] = {"error": f"{type(exc).__name__}: {exc}"}
            torch.cuda.empty_cache()

    line = {
        "metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": "laplace_h2_sphere6_L6_p1_q4_eta1.6", "ndofs": n1, "nrhs": 1, "level": w["level"],
                   "degree": w["p"], "q": w["q"], "eta": w["eta"], "leaf_level": leaf,
                   "leaf_level_oracle": w["leaf"], "far_fp32_stored": tuned_opts.far_fp32_stored,
                   "quadrature": f"autotuned for {w['quad_tol']:g} relative block accuracy: separated pairs "
                                 f"{tune['g_regular']}^2 per element next to the touching pairs, "
                                 f"{tune['g_regular_far']}^2 beyond, Duffy per-variable orders identical "
                                 f"{tuple(tune['g_identical_var'])}, edge {tuple(tune['g_edge_var'])}, "
                                 f"vertex {tuple(tune['g_vertex_var'])}",
                   "precision": "mixed (FP64 quadrature, "
                   "FP32 inner GMRES with block-Jacobi, FP64 refinement)", "l2": "working set > L2 (near+far FP64 storage "
                   f"{matvec_bytes / 1e9:.2f} GB per step)", "parallelism": f"replicas x{world}"},
        "clocks": clocks, "e2e": e2e, "gpu_launches": int(launches),
        "roofline": roofline, "cpu_baseline": cpu,
        "assembly_ms": opinfo["setup_ms"] + opinfo["assemble_ms"], "assembly_setup_ms": opinfo["setup_ms"],
        "assembly_setup_stage_ms": dict(zip(("corner_ids", "balls_block_tree", "pair_lists",
                                             "extraction_moments_points", "tables_rest"),
                                            opinfo["setup_phase_ms"])),
        "assembly_kernels_ms": opinfo["assemble_ms"], "phase_ms": dict(zip(names, ph)),
        "gmres": {"mixed_bj_ms": infomx["solve_ms"], "mixed_bj_iters": infomx["iterations"],
                  "mixed_noprec_ms": infomx_np["solve_ms"], "mixed_noprec_iters": infomx_np["iterations"],
                  "mixed_two_level_ms": infomx_2l["solve_ms"], "mixed_two_level_iters": infomx_2l["iterations"],
                  "mixed_two_level_with_setup_ms": infomx_2l_first["solve_ms"],
                  "mixed_refinements": infomx["refinements"], "mixed_relres": infomx["rel_residual"],
                  "fp64_ms": info64["solve_ms"], "fp64_iters": info64["iterations"],
                  "fp64_relres": info64["rel_residual"], "speedup_vs_fp64": info64["solve_ms"] / infomx["solve_ms"],
                  "fp64_bj_ms": info64_bj["solve_ms"], "fp64_bj_iters": info64_bj["iterations"],
                  "speedup_mixed_vs_fp64_same_precond": info64_bj["solve_ms"] / infomx["solve_ms"],
                  "speedup_precond_fp64": info64["solve_ms"] / info64_bj["solve_ms"]},
        "matvec": mv, "potential_max_rel_err": pot_err, "peaks_source": peak_src,
        "autotune": {k: v for k, v in tune.items()},
        "configs": legs,
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
