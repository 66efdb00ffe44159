"""CPU checks of the C ABI library: it loads and exports every entry point
include/bembel.h declares (no compute calls without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_1906_00785_gb300", "libbembel.so")


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(bembel_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def built_lib():
    if not os.path.exists(LIB):
        from paper_1906_00785_gb300 import build

        build.build()
    return LIB


def test_library_exports_every_declared_symbol(built_lib):
    out = subprocess.run(["nm", "-D", "--defined-only", built_lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (bembel_\w+)", out))
    declared = declared_functions()
    assert declared, "no declarations found"
    missing = [n for n in declared if n not in exported]
    assert not missing, missing


def test_binding_loads_and_reports_errors(built_lib):
    import ctypes

    import paper_1906_00785_gb300 as bem

    L = bem.lib()
    for n in declared_functions():
        assert hasattr(L, n)
        # every call with arguments has a ctypes signature: an undeclared one would pass
        # 64-bit device pointers as C ints
        if n not in ("bembel_last_error", "bembel_kernel_launches"):
            assert getattr(L, n).argtypes is not None, n
    # NULL operator / vectors and unknown kinds are rejected before any device work
    assert L.bembel_precond_apply(None, 1, None, None, 1, 0) == bem.BEMBEL_EINVAL
    # argument validation happens before any device work
    o = bem.bembel_opts_default()
    assert abs(o.eta - 1.6) < 1e-15 and o.leaf_level == -1
    so = bem.bembel_solve_opts_default()
    assert so.tol == 1e-8 and so.restart == 30
    with pytest.raises(bem.BembelError) as ei:
        bem.bembel_geom_create(kind=7)
    assert ei.value.code == bem.BEMBEL_EINVAL
    with pytest.raises(bem.BembelError):
        bem.bembel_geom_create(bem.BEMBEL_GEOM_PERTURBED_SPHERE, coeffs=[1.0, 2.0])
    g = bem.bembel_geom_create()
    with pytest.raises(bem.BembelError) as ei:
        bem.bembel_assemble(g, bem.BEMBEL_MAXWELL_SL, 4.0, 2, 2, 4, knot_repetition=2)  # S^1: repetition 1
    assert ei.value.code == bem.BEMBEL_EUNSUPPORTED
    with pytest.raises(bem.BembelError) as ei:
        bem.bembel_assemble(g, bem.BEMBEL_MAXWELL_SL, 0.0, 2, 2, 0)  # EFIE needs kappa != 0
    assert ei.value.code == bem.BEMBEL_EINVAL
    with pytest.raises(bem.BembelError) as ei:
        bem.bembel_assemble(g, bem.BEMBEL_LAPLACE_SL, 0.0, 2, 3, 0)
    assert ei.value.code == bem.BEMBEL_EINVAL
    assert L.bembel_ndofs(None, ctypes.byref(ctypes.c_int64())) == bem.BEMBEL_EINVAL


@pytest.mark.parametrize("kw", [dict(g_edge_var=(4, 0, 5, 3)),      # partial
                                dict(g_edge_var=(4, 11, 11, 3)),    # above the largest order
                                dict(g_edge_var=(4, 4, 5, 3)),      # edge rule not symmetric
                                dict(g_vertex_var=(5, 4, 4, 3)),    # vertex rule not symmetric
                                dict(g_regular=11), dict(eta=0.0), dict(leaf_level=7),
                                dict(knot_repetition=3), dict(knot_repetition=-1)])  # degree 1: r <= 2
def test_assemble_rejects_bad_options_before_device_work(built_lib, kw):
    import paper_1906_00785_gb300 as bem

    g = bem.bembel_geom_create()
    with pytest.raises(bem.BembelError) as ei:
        bem.bembel_assemble(g, bem.BEMBEL_LAPLACE_SL, 0.0, 2, 1, 4, **kw)
    assert ei.value.code == bem.BEMBEL_EINVAL


def test_batch_rejects_empty_list(built_lib):
    import paper_1906_00785_gb300 as bem

    with pytest.raises(bem.BembelError) as ei:
        bem.bembel_assemble_batch([], bem.BEMBEL_LAPLACE_SL, 1, 4)
    assert ei.value.code == bem.BEMBEL_EINVAL


def test_sphere_grid_matches_oracle(built_lib):
    """bembel_sphere_grid (host code, no GPU) gives the oracle's sphere grid (Sec. 5)."""
    import numpy as np

    import paper_1906_00785_gb300 as bem
    from oracle.potential_h2 import sphere_grid

    np.testing.assert_allclose(bem.bembel_sphere_grid(6.0, 10), sphere_grid(6.0, 10), rtol=0, atol=1e-14)
    for bad in ((0.0, 10), (1.0, 0)):
        with pytest.raises(bem.BembelError) as ei:
            bem.bembel_sphere_grid(*bad)
        assert ei.value.code == bem.BEMBEL_EINVAL
