"""ctypes binding of the C ABI in include/bembel.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  Device
vectors are torch CUDA tensors: a block of nrhs columns of length n is a
contiguous tensor of shape (nrhs, n) (column-major n x nrhs in C terms), dtype
float64 / complex128 (float32 / complex64 for the FP32 matvec).  There is no
fallback: if libbembel.so is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbembel.so")

BEMBEL_OK, BEMBEL_EINVAL, BEMBEL_ENOMEM, BEMBEL_ECUDA, BEMBEL_ENOTCONV, BEMBEL_ETIMEOUT, BEMBEL_EUNSUPPORTED = range(7)
BEMBEL_GEOM_SPHERE6, BEMBEL_GEOM_PERTURBED_SPHERE, BEMBEL_GEOM_NURBS = 0, 1, 2
BEMBEL_LAPLACE_SL, BEMBEL_HELMHOLTZ_SL, BEMBEL_MAXWELL_SL = 0, 1, 2
BEMBEL_PREC_FP64, BEMBEL_PREC_MIXED = 0, 1
BEMBEL_RHS_POINT_SOURCE, BEMBEL_RHS_PLANE_WAVE, BEMBEL_RHS_EFIE_PLANE_WAVE = 0, 1, 2
BEMBEL_PRECOND_NONE, BEMBEL_PRECOND_BLOCK_JACOBI, BEMBEL_PRECOND_LEARNED, BEMBEL_PRECOND_TWO_LEVEL = 0, 1, 2, 3
BEMBEL_LEARNED_NPARAM = 433

EXPORTED = [
    "bembel_opts_default", "bembel_solve_opts_default", "bembel_last_error", "bembel_geom_create",
    "bembel_geom_destroy", "bembel_assemble", "bembel_op_destroy", "bembel_ndofs", "bembel_op_info_get",
    "bembel_matvec", "bembel_rhs", "bembel_solve", "bembel_eval", "bembel_kernel_launches",
    "bembel_matvec_noalloc", "bembel_autotune", "bembel_learned_collect", "bembel_learned_set_destroy",
    "bembel_learned_train", "bembel_learned_attach", "bembel_mlp_eval", "bembel_tc_selftest",
    "bembel_assemble_batch", "bembel_near_block", "bembel_eval_h2", "bembel_sphere_grid",
    "bembel_precond_apply",
]


class BembelError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"bembel error {code}: {msg}")
        self.code = code


class GeomDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_coeffs", C.c_int), ("coeffs", C.POINTER(C.c_double)),
                ("amplitude", C.c_double), ("n_patches", C.c_int), ("degrees", C.POINTER(C.c_int)),
                ("n_ctrl", C.POINTER(C.c_int)), ("knots", C.POINTER(C.c_double)),
                ("ctrl", C.POINTER(C.c_double))]


class Opts(C.Structure):
    _fields_ = [("eta", C.c_double), ("leaf_level", C.c_int), ("g_regular", C.c_int), ("g_singular", C.c_int),
                ("g_identical", C.c_int), ("g_edge", C.c_int), ("g_vertex", C.c_int), ("bsr_chunk", C.c_int),
                ("tensor_cores", C.c_int),
                ("precision", C.c_int), ("stream", C.c_void_p), ("g_identical_var", C.c_int * 4),
                ("g_edge_var", C.c_int * 4), ("g_vertex_var", C.c_int * 4), ("g_regular_far", C.c_int),
                ("knot_repetition", C.c_int), ("kdiam", C.c_double), ("coarse_level", C.c_int),
                ("far_fp32_stored", C.c_int)]


class OpInfo(C.Structure):
    _fields_ = [(n, C.c_int64) for n in (
        "ndofs", "nlocal", "nelements", "n_clusters", "n_far_blocks", "n_near_blocks", "n_pairs_regular",
        "n_pairs_identical", "n_pairs_edge", "n_pairs_vertex", "near_bytes", "far_bytes")] + [
        ("leaf_level", C.c_int), ("q", C.c_int), ("degree", C.c_int), ("level", C.c_int),
        ("assemble_ms", C.c_double), ("setup_ms", C.c_double), ("phase_ms", C.c_double * 8),
        ("n_pairs_regular_far", C.c_int64), ("setup_phase_ms", C.c_double * 5)]


class TuneReport(C.Structure):
    _fields_ = [("g_regular", C.c_int), ("g_identical", C.c_int), ("g_edge", C.c_int), ("g_vertex", C.c_int),
                ("q", C.c_int), ("bsr_chunk", C.c_int), ("err_regular", C.c_double), ("err_identical", C.c_double),
                ("err_edge", C.c_double), ("err_vertex", C.c_double), ("err_far", C.c_double),
                ("chunk_ms", C.c_double * 5), ("tune_ms", C.c_double), ("g_identical_var", C.c_int * 4),
                ("g_edge_var", C.c_int * 4), ("g_vertex_var", C.c_int * 4), ("g_regular_far", C.c_int),
                ("err_regular_far", C.c_double), ("leaf_level", C.c_int), ("leaf_score_ms", C.c_double * 2),
                ("far_fp32_stored", C.c_int), ("fp32_product_ms", C.c_double * 2)]


class BatchItem(C.Structure):
    _fields_ = [("geom", C.c_void_p), ("k_re", C.c_double), ("k_im", C.c_double), ("level", C.c_int)]


class SolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("restart", C.c_int), ("max_iter", C.c_int), ("precond", C.c_int),
                ("refine", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("refinements", C.c_int), ("rel_residual", C.c_double),
                ("solve_ms", C.c_double)]


_lib = None


def lib():
    """Load libbembel.so (raises if it is missing: there is no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing; build it with `python -m paper_1906_00785_gb300.build`")
    L = C.CDLL(LIB_PATH)
    vp, i64, dbl, ci = C.c_void_p, C.c_int64, C.c_double, C.c_int
    L.bembel_opts_default.argtypes = [C.POINTER(Opts)]
    L.bembel_opts_default.restype = None
    L.bembel_solve_opts_default.argtypes = [C.POINTER(SolveOpts)]
    L.bembel_solve_opts_default.restype = None
    L.bembel_last_error.argtypes = []
    L.bembel_last_error.restype = C.c_char_p
    L.bembel_kernel_launches.argtypes = []
    L.bembel_kernel_launches.restype = i64
    L.bembel_geom_create.argtypes = [C.POINTER(GeomDesc), C.POINTER(vp)]
    L.bembel_geom_destroy.argtypes = [vp]
    L.bembel_assemble.argtypes = [vp, ci, dbl, dbl, ci, ci, ci, C.POINTER(Opts), C.POINTER(vp)]
    L.bembel_assemble_batch.argtypes = [ci, ci, ci, C.POINTER(BatchItem), ci, C.POINTER(Opts), C.POINTER(vp)]
    L.bembel_op_destroy.argtypes = [vp]
    L.bembel_ndofs.argtypes = [vp, C.POINTER(i64)]
    L.bembel_op_info_get.argtypes = [vp, C.POINTER(OpInfo)]
    L.bembel_matvec.argtypes = [vp, vp, vp, ci, ci]
    L.bembel_matvec_noalloc.argtypes = [vp, vp, vp, ci, ci]
    fp = C.POINTER(C.c_float)
    L.bembel_learned_collect.argtypes = [vp, ci, C.c_uint64, C.POINTER(vp)]
    L.bembel_learned_set_destroy.argtypes = [vp]
    L.bembel_learned_train.argtypes = [C.POINTER(vp), ci, ci, dbl, fp, C.POINTER(dbl)]
    L.bembel_learned_attach.argtypes = [vp, fp]
    L.bembel_mlp_eval.argtypes = [fp, vp, i64, vp, vp, fp]
    L.bembel_tc_selftest.argtypes = [ci, C.POINTER(dbl)]
    L.bembel_autotune.argtypes = [vp, ci, dbl, dbl, ci, ci, dbl, dbl, ci, C.POINTER(Opts), C.POINTER(TuneReport)]
    L.bembel_rhs.argtypes = [vp, ci, C.POINTER(dbl), ci, ci, vp]
    L.bembel_solve.argtypes = [vp, vp, vp, ci, C.POINTER(SolveOpts), C.POINTER(SolveInfo)]
    L.bembel_eval.argtypes = [vp, vp, i64, vp, ci, ci, vp]
    L.bembel_near_block.argtypes = [vp, ci, ci, ci, ci, ci, ci, C.POINTER(dbl)]
    L.bembel_eval_h2.argtypes = [vp, vp, i64, vp, ci, ci, dbl, vp]
    L.bembel_sphere_grid.argtypes = [dbl, ci, C.POINTER(dbl)]
    L.bembel_precond_apply.argtypes = [vp, ci, vp, vp, ci, ci]
    missing = [n for n in EXPORTED if n not in ("bembel_last_error", "bembel_kernel_launches")
               and getattr(L, n).argtypes is None]
    if missing:  # an undeclared signature would pass 64-bit pointers as C ints
        raise RuntimeError(f"capi: no ctypes signature for {missing}")
    for n in EXPORTED:
        if n not in ("bembel_opts_default", "bembel_solve_opts_default", "bembel_last_error",
                     "bembel_kernel_launches"):
            getattr(L, n).restype = ci
    _lib = L
    return L


def _check(rc: int, allow=()):
    if rc != BEMBEL_OK and rc not in allow:
        raise BembelError(rc, lib().bembel_last_error().decode())
    return rc


def _ptr(t) -> int:
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


class Geometry:
    """Owning wrapper of a bembel_geom handle."""

    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.bembel_geom_destroy(self.handle)
            self.handle = None


class Operator:
    """Owning wrapper of a bembel_op handle (keeps its geometry alive)."""

    def __init__(self, handle, geom: Geometry, op: int):
        self.handle = handle
        self.geom = geom
        self.op = op

    @property
    def complex(self) -> bool:
        return self.op == BEMBEL_HELMHOLTZ_SL

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.bembel_op_destroy(self.handle)
            self.handle = None


def bembel_opts_default() -> Opts:
    o = Opts()
    lib().bembel_opts_default(C.byref(o))
    return o


def bembel_solve_opts_default() -> SolveOpts:
    o = SolveOpts()
    lib().bembel_solve_opts_default(C.byref(o))
    return o


def bembel_geom_create(kind: int = BEMBEL_GEOM_SPHERE6, coeffs=None, amplitude: float = 0.1,
                       patches=None) -> Geometry:
    """patches (NURBS): six dicts with "degrees" (p1, p2), "knots" (s knots, t knots) and
    "ctrl" of shape (k2, k1, 4) = (x, y, z, weight) indexed [i2, i1]."""
    d = GeomDesc()
    d.kind = kind
    keep = None
    if coeffs is not None:
        keep = np.ascontiguousarray(coeffs, dtype=np.float64)
        d.n_coeffs = keep.size
        d.coeffs = keep.ctypes.data_as(C.POINTER(C.c_double))
    d.amplitude = amplitude
    if patches is not None:
        deg = np.ascontiguousarray([v for pt in patches for v in pt["degrees"]], dtype=np.int32)
        nct = np.ascontiguousarray([v for pt in patches for v in (np.shape(pt["ctrl"])[1], np.shape(pt["ctrl"])[0])],
                                   dtype=np.int32)
        kn = np.ascontiguousarray(np.concatenate([np.concatenate(pt["knots"]) for pt in patches]), dtype=np.float64)
        cp = np.ascontiguousarray(np.concatenate([np.asarray(pt["ctrl"], dtype=np.float64).ravel() for pt in patches]))
        keep = (keep, deg, nct, kn, cp)
        d.n_patches = len(patches)
        d.degrees = deg.ctypes.data_as(C.POINTER(C.c_int))
        d.n_ctrl = nct.ctypes.data_as(C.POINTER(C.c_int))
        d.knots = kn.ctypes.data_as(C.POINTER(C.c_double))
        d.ctrl = cp.ctypes.data_as(C.POINTER(C.c_double))
    h = C.c_void_p()
    _check(lib().bembel_geom_create(C.byref(d), C.byref(h)))
    return Geometry(h)


def _apply(o, overrides):
    for key, v in overrides.items():
        if key.endswith("_var"):
            arr = getattr(o, key)
            for i, x in enumerate(v):
                arr[i] = int(x)
        else:
            setattr(o, key, v)
    return o


def bembel_assemble(geom: Geometry, op: int, k: complex, level: int, p: int, q: int, opts: Opts | None = None,
                    **overrides) -> Operator:
    o = _apply(opts if opts is not None else bembel_opts_default(), overrides)
    h = C.c_void_p()
    k = complex(k)
    _check(lib().bembel_assemble(geom.handle, op, k.real, k.imag, level, p, q, C.byref(o), C.byref(h)))
    return Operator(h, geom, op)


def bembel_assemble_batch(items, op: int, p: int, q: int, opts: Opts | None = None, **overrides) -> list:
    """items: sequence of (geometry, k, level).  Returns one Operator per item."""
    o = _apply(opts if opts is not None else bembel_opts_default(), overrides)
    n = len(items)
    arr = (BatchItem * max(1, n))()
    for i, (geom, k, level) in enumerate(items):
        k = complex(k)
        arr[i].geom = geom.handle.value if isinstance(geom.handle, C.c_void_p) else geom.handle
        arr[i].k_re = k.real
        arr[i].k_im = k.imag
        arr[i].level = level
    outs = (C.c_void_p * max(1, n))()
    _check(lib().bembel_assemble_batch(op, p, q, arr, n, C.byref(o), outs))
    return [Operator(C.c_void_p(outs[i]), items[i][0], op) for i in range(n)]


def bembel_autotune(geom: Geometry, op: int, k: complex, level: int, p: int, quad_tol: float = 1e-8,
                    far_tol: float = 1e-5, q_max: int = 8, opts: Opts | None = None, **overrides):
    """Returns (options with the chosen orders, report dict incl. the chosen q)."""
    o = _apply(opts if opts is not None else bembel_opts_default(), overrides)
    rep = TuneReport()
    k = complex(k)
    _check(lib().bembel_autotune(geom.handle, op, k.real, k.imag, level, p, quad_tol, far_tol, q_max, C.byref(o),
                                 C.byref(rep)))
    out = {f: getattr(rep, f) for f, _ in TuneReport._fields_}
    for key in ("chunk_ms", "g_identical_var", "g_edge_var", "g_vertex_var", "leaf_score_ms", "fp32_product_ms"):
        out[key] = list(getattr(rep, key))
    return o, out


class LearnedSet:
    """Owning wrapper of a bembel_learned_set handle."""

    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.bembel_learned_set_destroy(self.handle)
            self.handle = None


def bembel_learned_collect(op: Operator, nsamples: int = 4, seed: int = 0) -> LearnedSet:
    h = C.c_void_p()
    _check(lib().bembel_learned_collect(op.handle, nsamples, seed, C.byref(h)))
    return LearnedSet(h)


def bembel_learned_train(sets, epochs: int, lr: float, params) -> tuple[np.ndarray, np.ndarray]:
    """Returns (trained parameters, loss history)."""
    arr = (C.c_void_p * len(sets))(*[s.handle for s in sets])
    prm = np.ascontiguousarray(params, dtype=np.float32).copy()
    hist = np.zeros(epochs)
    _check(lib().bembel_learned_train(arr, len(sets), epochs, lr, prm.ctypes.data_as(C.POINTER(C.c_float)),
                                      hist.ctypes.data_as(C.POINTER(C.c_double))))
    return prm, hist


def bembel_learned_attach(op: Operator, params) -> None:
    prm = np.ascontiguousarray(params, dtype=np.float32)
    _check(lib().bembel_learned_attach(op.handle, prm.ctypes.data_as(C.POINTER(C.c_float))))


def bembel_mlp_eval(params, feats, gw=None):
    """Weights (device tensor) and, with gw, d/dparams of sum gw * weights (numpy)."""
    import torch

    prm = np.ascontiguousarray(params, dtype=np.float32)
    n = feats.shape[0]
    w = torch.empty(n, dtype=torch.float32, device=feats.device)
    grad = np.zeros(BEMBEL_LEARNED_NPARAM, dtype=np.float32)
    _check(lib().bembel_mlp_eval(prm.ctypes.data_as(C.POINTER(C.c_float)), _ptr(feats), n,
                                 _ptr(gw) if gw is not None else None, _ptr(w),
                                 grad.ctypes.data_as(C.POINTER(C.c_float))))
    return w, grad


def bembel_tc_selftest(n: int) -> float:
    err = C.c_double()
    _check(lib().bembel_tc_selftest(n, C.byref(err)))
    return err.value


def bembel_ndofs(op: Operator) -> int:
    n = C.c_int64()
    _check(lib().bembel_ndofs(op.handle, C.byref(n)))
    return n.value


def bembel_op_info_get(op: Operator) -> dict:
    inf = OpInfo()
    _check(lib().bembel_op_info_get(op.handle, C.byref(inf)))
    out = {f: getattr(inf, f) for f, _ in OpInfo._fields_}
    out["phase_ms"] = list(inf.phase_ms)
    out["setup_phase_ms"] = list(inf.setup_phase_ms)
    return out


def bembel_near_block(op: Operator, e, f) -> np.ndarray:
    """Stored near-field block of elements e = (patch, i1, i2) and f, in the element-local
    Bernstein basis: (nloc, nloc) float64, or complex128 for Helmholtz."""
    info = bembel_op_info_get(op)
    nloc = (info["degree"] + 1) ** 2
    c = 2 if op.complex else 1
    out = np.zeros(nloc * nloc * c)
    _check(lib().bembel_near_block(op.handle, *[int(v) for v in e], *[int(v) for v in f],
                                   out.ctypes.data_as(C.POINTER(C.c_double))))
    return (out.view(np.complex128) if c == 2 else out).reshape(nloc, nloc)


def bembel_kernel_launches() -> int:
    return int(lib().bembel_kernel_launches())


def bembel_matvec(op: Operator, x, y, nrhs: int = 1, fp32: bool = False) -> None:
    _check(lib().bembel_matvec(op.handle, _ptr(x), _ptr(y), nrhs, int(bool(fp32))))


def bembel_matvec_noalloc(op: Operator, x, y, nrhs: int = 1, fp32: bool = False) -> None:
    """y = A x using the library's fixed device scratch (no allocation; see include/bembel.h)."""
    _check(lib().bembel_matvec_noalloc(op.handle, _ptr(x), _ptr(y), nrhs, int(bool(fp32))))


def bembel_rhs(op: Operator, kind: int, params, b, g: int = 6) -> None:
    prm = np.ascontiguousarray(np.atleast_2d(params), dtype=np.float64)
    _check(lib().bembel_rhs(op.handle, kind, prm.ctypes.data_as(C.POINTER(C.c_double)), prm.shape[0], g, _ptr(b)))


def bembel_solve(op: Operator, b, x, nrhs: int = 1, solve_opts: SolveOpts | None = None, **overrides) -> dict:
    so = solve_opts if solve_opts is not None else bembel_solve_opts_default()
    for key, v in overrides.items():
        setattr(so, key, v)
    info = SolveInfo()
    rc = _check(lib().bembel_solve(op.handle, _ptr(b), _ptr(x), nrhs, C.byref(so), C.byref(info)),
                allow=(BEMBEL_ENOTCONV,))
    out = {f: getattr(info, f) for f, _ in SolveInfo._fields_}
    out["converged"] = rc == BEMBEL_OK
    return out


def bembel_precond_apply(op: Operator, precond: int, x, y, nrhs: int = 1, fp32: bool = False) -> None:
    """y = M^-1 x for the preconditioner kind precond (as the solver applies it)."""
    _check(lib().bembel_precond_apply(op.handle, precond, _ptr(x), _ptr(y), nrhs, int(bool(fp32))))


def bembel_eval(op: Operator, pts, rho, out, nrhs: int = 1, g: int = 6) -> None:
    _check(lib().bembel_eval(op.handle, _ptr(pts), pts.shape[0], _ptr(rho), nrhs, g, _ptr(out)))


def bembel_eval_h2(op: Operator, pts, rho, out, nrhs: int = 1, g: int = 6, eta: float = 1.6) -> None:
    _check(lib().bembel_eval_h2(op.handle, _ptr(pts), pts.shape[0], _ptr(rho), nrhs, g, eta, _ptr(out)))


def bembel_sphere_grid(radius: float, n: int) -> np.ndarray:
    """(n * n, 3) host array of points on the sphere of the given radius."""
    out = np.zeros((n * n, 3))
    _check(lib().bembel_sphere_grid(radius, n, out.ctypes.data_as(C.POINTER(C.c_double))))
    return out
