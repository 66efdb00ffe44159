"""Benchmark of the H^2 single-layer hot path on GB300.

Workload (the Laplace H^2 configuration): unit sphere as 6 cube-face patches,
level 6 (24,576 elements), degree-1 B-splines (25,350 dofs), 4 x 4 Chebyshev
interpolation per cluster, eta = 1.6, leaf level 5, Gauss 4 x 4 on separated
near pairs and 5^4 per Duffy sub-domain on touching pairs.  Data: point charge
u = 1/|x - x0|, x0 = (0, 0, 2), potential at 100 seeded points in the ball of
radius 0.5.  All inputs are synthetic.

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
WORKLOAD = dict(level=6, p=1, q=4, eta=1.6, leaf=5, g_reg=4, g_sing=5, quad_tol=1e-6, x0=(0.0, 0.0, 2.0),
                n_eval=100)
# FP64 flops per quadrature point, counted from the formulas:
# regular pair point (x_p, y_q): difference, squared norm, 1/r, 4 (d=1) weighted products
FLOPS_REG_POINT = {0: 12, 1: 18, 2: 28}
# identical-pair Duffy point: rule map + both patch maps + 1/r + (d+1)^4 basis products
FLOPS_SING_POINT = {0: 80, 1: 110, 2: 250}
# one side point of the factorised edge / vertex rules: patch map + weighted Bernstein values
FLOPS_SIDE_POINT = {0: 22, 1: 30, 2: 48}
# DRAM bytes per separated pair of k_near_regular<1, 0> (pair record + written blocks), from an
# ncu capture of the level-5 degree-1 launch: 28.31 MB over 254,412 pairs
REGULAR_DRAM_BYTES_PER_PAIR = 28.31e6 / 254412


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


def cpu_baseline_sample(n_rows: int = 1, iters: int = 60):
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
    c_start, w_start = time.process_time(), time.perf_counter()
    sp = S2Space(Sphere6(), w["level"], w["p"])
    t0 = time.perf_counter()
    h2 = H2Oracle(sp, "laplace", q=w["q"], eta=w["eta"], leaf_level=w["leaf"], g_reg=w["g_reg"],
                  g_sing=w["g_sing"])
    t_tree = time.perf_counter() - t0
    rows = np.random.default_rng(5).choice(sp.ndofs, n_rows, replace=False)
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
    sample = (f"oracle sampled rows: 1 row of A~x per step (first application with its near-field quadrature, "
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


def main():
    args = parse()
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
    tuned_opts, tune = bem.bembel_autotune(geom, bem.BEMBEL_LAPLACE_SL, 0.0, w["level"], w["p"],
                                           quad_tol=w["quad_tol"], far_tol=1e-4, q_max=w["q"], eta=w["eta"],
                                           leaf_level=w["leaf"], stream=stream.cuda_stream)

    def assemble(precision):
        o = bem.bembel_opts_default()
        for f in ("g_regular", "g_regular_far", "g_singular", "g_identical", "g_edge", "g_vertex", "bsr_chunk"):
            setattr(o, f, getattr(tuned_opts, f))
        for f in ("g_identical_var", "g_edge_var", "g_vertex_var"):
            for i in range(4):
                getattr(o, f)[i] = getattr(tuned_opts, f)[i]
        return bem.bembel_assemble(geom, bem.BEMBEL_LAPLACE_SL, 0.0, w["level"], w["p"], w["q"], opts=o,
                                   eta=w["eta"], leaf_level=w["leaf"], precision=precision,
                                   stream=stream.cuda_stream)

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
    dom = max(flops_phase, key=lambda k: ph[names.index(k)])
    dom_ms = ph[names.index(dom)]
    achieved = flops_phase[dom] / (dom_ms / 1e3) / 1e12
    peak = fp64_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
    roofline = {"kernel": f"k_near_singular ({dom})" if dom != "near_regular" else "k_near_regular",
                "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                # ncu DRAM bytes of a level-5 launch scaled by the pairs of this launch (traffic grows
                # with the pair count: records read, blocks written); measured for degree 1 only
                "traffic": (REGULAR_DRAM_BYTES_PER_PAIR * opinfo["n_pairs_regular"]
                            if dom == "near_regular" and w["p"] == 1 else None),
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
        v, det = cpu_baseline_sample(2, iters=info64["iterations"])
        cpu = {"value": v, "unit": "GDOF/s", "cores": det["cores"], "kind": "oracle",
               "sample": f"2 sampled rows of A~x (first: with near-field quadrature, second: cached), "
                         f"extrapolated to {n1} dofs x {det['iters']} GMRES matvecs + tree build", "details": det}

    line = {
        "metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": "laplace_h2_sphere6_L6_p1_q4_eta1.6", "ndofs": n1, "nrhs": 1, "level": w["level"],
                   "degree": w["p"], "q": w["q"], "eta": w["eta"], "leaf_level": w["leaf"],
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
        "assembly_kernels_ms": opinfo["assemble_ms"], "phase_ms": dict(zip(names, ph)),
        "gmres": {"mixed_bj_ms": infomx["solve_ms"], "mixed_bj_iters": infomx["iterations"],
                  "mixed_noprec_ms": infomx_np["solve_ms"], "mixed_noprec_iters": infomx_np["iterations"],
                  "mixed_refinements": infomx["refinements"], "mixed_relres": infomx["rel_residual"],
                  "fp64_ms": info64["solve_ms"], "fp64_iters": info64["iterations"],
                  "fp64_relres": info64["rel_residual"], "speedup_vs_fp64": info64["solve_ms"] / infomx["solve_ms"]},
        "matvec": mv, "potential_max_rel_err": pot_err, "peaks_source": peak_src,
        "autotune": {k: v for k, v in tune.items()},
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
