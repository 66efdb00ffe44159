"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances (FP64 path, same quadrature rules and H^2 readings on both sides, so
differences are rounding only): matrix entries 1e-12 relative to the largest
entry; H^2 matvec rows 1e-12; solutions 1e-9 (solved to 1e-13 on the GPU,
direct solve in the oracle; the condition numbers here are below 1e3).
"""
import numpy as np
import pytest
import torch

import paper_1906_00785_gb300 as bem
from inputs import ball_points, random_vector
from oracle.galerkin import Assembler, potential, rhs
from oracle.geometry import Sphere6
from oracle.h2 import H2Oracle, block_tree
from oracle.space import S2Space

pytestmark = pytest.mark.gpu
LAP, HEL = bem.BEMBEL_LAPLACE_SL, bem.BEMBEL_HELMHOLTZ_SL


@pytest.fixture(scope="module")
def geom():
    return bem.bembel_geom_create(bem.BEMBEL_GEOM_SPHERE6)


def gpu_matrix(op, n):
    dt = torch.complex128 if op.complex else torch.float64
    eye = torch.eye(n, dtype=dt, device="cuda")
    out = torch.empty_like(eye)
    bem.bembel_matvec(op, eye, out, n)
    torch.cuda.synchronize()
    return out.cpu().numpy().T


def rel_err(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("L,d,op,k", [(2, 0, "laplace", 0.0), (2, 1, "laplace", 0.0), (1, 2, "laplace", 0.0),
                                      (2, 1, "helmholtz", 2.0 + 0.3j), (0, 1, "laplace", 0.0)])
def test_dense_matrix_parity(geom, L, d, op, k):
    gop = bem.bembel_assemble(geom, LAP if op == "laplace" else HEL, k, L, d, 0, g_regular=4, g_singular=5)
    sp = S2Space(Sphere6(), L, d)
    A_ref = Assembler(sp, op, k, 4, 5).dense()
    A = gpu_matrix(gop, sp.ndofs)
    assert rel_err(A, A_ref) < 1e-12


@pytest.mark.parametrize("L,d,q,op,k,leaf", [(3, 1, 4, "laplace", 0.0, 2), (3, 0, 3, "laplace", 0.0, 1),
                                             (3, 2, 4, "helmholtz", 1.5, 2), (4, 0, 2, "laplace", 0.0, 3)])
def test_h2_matrix_parity(geom, L, d, q, op, k, leaf):
    gop = bem.bembel_assemble(geom, LAP if op == "laplace" else HEL, k, L, d, q, g_regular=3, g_singular=4,
                              leaf_level=leaf, eta=1.6)
    sp = S2Space(Sphere6(), L, d)
    h2 = H2Oracle(sp, op, k, q=q, eta=1.6, leaf_level=leaf, g_reg=3, g_sing=4)
    info = bem.bembel_op_info_get(gop)
    assert info["n_far_blocks"] == len(h2.far) and info["n_near_blocks"] == len(h2.near)
    assert info["n_far_blocks"] > 0
    A = gpu_matrix(gop, sp.ndofs)
    assert rel_err(A, h2.dense()) < 1e-12


def test_block_counts_level6(geom):
    """Far/near block counts of the level-6 workload (leaf level 5, eta 1.6)."""
    far, near, _ = block_tree(Sphere6(), 5, 1.6)
    gop = bem.bembel_assemble(geom, LAP, 0.0, 6, 1, 4, leaf_level=5)
    info = bem.bembel_op_info_get(gop)
    assert info["n_far_blocks"] == len(far) and info["n_near_blocks"] == len(near)
    assert info["n_pairs_identical"] == 24576
    assert info["n_pairs_edge"] == 98304 // 2 and info["n_pairs_vertex"] == 98280 // 2


def test_h2_rows_full_size(geom):
    """Sampled rows of A~ x at the full level-6, degree-1, q=4 workload."""
    sp = S2Space(Sphere6(), 6, 1)
    gop = bem.bembel_assemble(geom, LAP, 0.0, 6, 1, 4, leaf_level=5, g_regular=4, g_singular=5)
    n = bem.bembel_ndofs(gop)
    assert n == sp.ndofs == 25350
    x = random_vector(n, 2)
    xt = torch.from_numpy(x).cuda()
    y = torch.empty_like(xt)
    bem.bembel_matvec(gop, xt, y, 1)
    y = y.cpu().numpy()
    rows = np.random.default_rng(9).choice(n, 6, replace=False)
    h2 = H2Oracle(sp, "laplace", q=4, eta=1.6, leaf_level=5, g_reg=4, g_sing=5)
    ref = h2.apply_rows(x, rows)
    np.testing.assert_allclose(y[rows], ref, rtol=1e-11, atol=1e-12 * np.abs(ref).max())


def test_multi_rhs_equals_columns(geom):
    gop = bem.bembel_assemble(geom, HEL, 3.0, 3, 1, 4, leaf_level=2)
    n = bem.bembel_ndofs(gop)
    X = torch.from_numpy(random_vector(n, 4, nrhs=5, complex_=True).T.copy()).cuda()
    Y = torch.empty_like(X)
    bem.bembel_matvec(gop, X, Y, 5)
    for r in range(5):
        y1 = torch.empty_like(X[r])
        bem.bembel_matvec(gop, X[r].contiguous(), y1, 1)
        assert torch.max(torch.abs(y1 - Y[r])) <= 1e-13 * torch.max(torch.abs(Y[r]))


def test_dense_laplace_point_charge_end_to_end(geom):
    """Dense Laplace, level 3, degree 0: load vector, GMRES, potential."""
    x0 = np.array([0.0, 0.0, 2.0])
    sp = S2Space(Sphere6(), 3, 0)
    gop = bem.bembel_assemble(geom, LAP, 0.0, 3, 0, 0, g_regular=4, g_singular=5)
    n = bem.bembel_ndofs(gop)
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    bem.bembel_rhs(gop, bem.BEMBEL_RHS_POINT_SOURCE, x0[None, :], b, g=6)
    b_ref = rhs(sp, lambda x: 1.0 / np.linalg.norm(x - x0, axis=1), g=6)
    np.testing.assert_allclose(b.cpu().numpy(), b_ref, rtol=1e-13, atol=1e-16)
    A_ref = Assembler(sp, "laplace", 0.0, 4, 5).dense()
    rho = torch.empty_like(b)
    info = bem.bembel_solve(gop, b, rho, 1, tol=1e-13)
    assert info["converged"] and info["rel_residual"] <= 1e-13
    rho_ref = np.linalg.solve(A_ref, b_ref)
    assert rel_err(rho.cpu().numpy(), rho_ref) < 1e-9
    pts = ball_points(100, 0.5, 1)
    u = torch.empty(100, dtype=torch.float64, device="cuda")
    bem.bembel_eval(gop, torch.from_numpy(pts).cuda(), rho, u, 1, g=6)
    u_ref = potential(sp, rho_ref, pts, "laplace", g=6)
    np.testing.assert_allclose(u.cpu().numpy(), u_ref, rtol=1e-9)
    exact = 1.0 / np.linalg.norm(pts - x0, axis=1)
    assert np.max(np.abs(u.cpu().numpy() - exact) / exact) < 5e-4


def test_helmholtz_solve_and_eval_parity(geom):
    k = 2.0
    src = np.array([0.1, -0.2, 0.15])
    sp = S2Space(Sphere6(), 2, 1)
    gop = bem.bembel_assemble(geom, HEL, k, 2, 1, 0)
    n = bem.bembel_ndofs(gop)
    b = torch.empty(n, dtype=torch.complex128, device="cuda")
    bem.bembel_rhs(gop, bem.BEMBEL_RHS_POINT_SOURCE, src[None, :], b, g=6)
    r = lambda x: np.linalg.norm(x - src, axis=1)  # noqa: E731
    b_ref = rhs(sp, lambda x: np.exp(-1j * k * r(x)) / r(x), g=6, dtype=complex)
    np.testing.assert_allclose(b.cpu().numpy(), b_ref, rtol=1e-12, atol=1e-15)
    x = torch.empty_like(b)
    info = bem.bembel_solve(gop, b, x, 1, tol=1e-13)
    assert info["converged"]
    A_ref = Assembler(sp, "helmholtz", k, 4, 5).dense()
    x_ref = np.linalg.solve(A_ref, b_ref)
    assert rel_err(x.cpu().numpy(), x_ref) < 1e-9
    pts = np.array([[3.0, 0.0, 0.0], [0.0, -2.5, 1.0]])
    u = torch.empty(2, dtype=torch.complex128, device="cuda")
    bem.bembel_eval(gop, torch.from_numpy(pts).cuda(), x, u, 1, g=6)
    np.testing.assert_allclose(u.cpu().numpy(), potential(sp, x_ref, pts, "helmholtz", k, g=6), rtol=1e-9)


def test_plane_wave_rhs_batch(geom):
    k = 2.0
    sp = S2Space(Sphere6(), 2, 2)
    gop = bem.bembel_assemble(geom, HEL, k, 2, 2, 0)
    dirs = np.array([[0, 0, 1.0], [1.0, 0, 0], [0.6, 0.8, 0]])
    b = torch.empty((3, sp.ndofs), dtype=torch.complex128, device="cuda")
    bem.bembel_rhs(gop, bem.BEMBEL_RHS_PLANE_WAVE, dirs, b, g=5)
    for r in range(3):
        ref = rhs(sp, lambda x: np.exp(-1j * k * (x @ dirs[r])), g=5, dtype=complex)
        np.testing.assert_allclose(b[r].cpu().numpy(), ref, rtol=1e-12, atol=1e-15)


def test_mixed_precision_solution(geom):
    gop64 = bem.bembel_assemble(geom, LAP, 0.0, 4, 1, 4)
    gopmx = bem.bembel_assemble(geom, LAP, 0.0, 4, 1, 4, precision=bem.BEMBEL_PREC_MIXED)
    n = bem.bembel_ndofs(gop64)
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    bem.bembel_rhs(gop64, bem.BEMBEL_RHS_POINT_SOURCE, np.array([[0.0, 0.0, 2.0]]), b)
    x64, xmx = torch.empty_like(b), torch.empty_like(b)
    i64 = bem.bembel_solve(gop64, b, x64, 1, tol=1e-10)
    imx = bem.bembel_solve(gopmx, b, xmx, 1, tol=1e-10)
    assert i64["converged"] and imx["converged"] and imx["refinements"] >= 1
    assert (torch.linalg.norm(xmx - x64) / torch.linalg.norm(x64)).item() < 1e-6


def test_mixed_precision_restarts(geom):
    """Short restart cycles with FP64 residuals between graph-replayed FP32
    Arnoldi steps, on device memory that held NaN before."""
    gop64 = bem.bembel_assemble(geom, LAP, 0.0, 4, 1, 4)
    gopmx = bem.bembel_assemble(geom, LAP, 0.0, 4, 1, 4, precision=bem.BEMBEL_PREC_MIXED)
    n = bem.bembel_ndofs(gop64)
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    bem.bembel_rhs(gop64, bem.BEMBEL_RHS_POINT_SOURCE, np.array([[0.0, 0.0, 2.0]]), b)
    x64, xmx = torch.empty_like(b), torch.empty_like(b)
    bem.bembel_solve(gop64, b, x64, 1, tol=1e-10)
    # leave NaN in freed device memory: the solver's fresh buffers may reuse it,
    # and Krylov columns a cycle did not build must never be read
    poison = torch.full((64 << 20,), float("nan"), dtype=torch.float32, device="cuda")
    del poison
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    imx = bem.bembel_solve(gopmx, b, xmx, 1, tol=1e-10, restart=4)
    assert imx["converged"] and torch.isfinite(xmx).all().item()
    assert (torch.linalg.norm(xmx - x64) / torch.linalg.norm(x64)).item() < 1e-6


def test_invalid_arguments(geom):
    gop = bem.bembel_assemble(geom, LAP, 0.0, 1, 0, 0)
    x = torch.zeros(24, dtype=torch.float64, device="cuda")
    with pytest.raises(bem.BembelError):
        bem.bembel_matvec(gop, x, x, 1)  # aliasing
    with pytest.raises(bem.BembelError):
        bem.bembel_matvec(gop, x, torch.empty_like(x), 0)
    with pytest.raises(bem.BembelError):
        bem.bembel_matvec(gop, x, torch.empty_like(x), 1, fp32=True)  # FP64 operator has no FP32 copy
    out = bem.bembel_solve(gop, x, torch.empty_like(x), 1)  # zero right-hand side
    assert out["converged"] and out["iterations"] == 0


@pytest.mark.parametrize("op,k,d", [("laplace", 0.0, 1), ("helmholtz", 2.5, 2), ("laplace", 0.0, 0)])
def test_block_jacobi_solve_parity(geom, op, k, d):
    """Right block-Jacobi preconditioning changes iterations, not the solution.

    Both solves run to relative residual 1e-13; the solution error is bounded by
    cond(A) x residual (cond(A) < 1e4 for these operators), so 1e-8.
    """
    L = 3
    sp = S2Space(Sphere6(), L, d)
    gop = bem.bembel_assemble(geom, LAP if op == "laplace" else HEL, k, L, d, 0)
    n = bem.bembel_ndofs(gop)
    dt = torch.complex128 if op == "helmholtz" else torch.float64
    b = torch.empty(n, dtype=dt, device="cuda")
    bem.bembel_rhs(gop, bem.BEMBEL_RHS_POINT_SOURCE, np.array([[0.1, 0.2, -0.3]]), b)
    x0, x1 = torch.empty_like(b), torch.empty_like(b)
    i0 = bem.bembel_solve(gop, b, x0, 1, tol=1e-13, precond=bem.BEMBEL_PRECOND_NONE)
    i1 = bem.bembel_solve(gop, b, x1, 1, tol=1e-13, precond=bem.BEMBEL_PRECOND_BLOCK_JACOBI)
    assert i0["converged"] and i1["converged"]
    assert i1["iterations"] < i0["iterations"]
    A_ref = Assembler(sp, op, k, 4, 5).dense()
    x_ref = np.linalg.solve(A_ref, b.cpu().numpy())
    assert rel_err(x1.cpu().numpy(), x_ref) < 1e-8
    assert rel_err(x0.cpu().numpy(), x_ref) < 1e-8


def test_batched_solve_matches_single(geom):
    gop = bem.bembel_assemble(geom, HEL, 2.0, 3, 1, 4, precision=bem.BEMBEL_PREC_MIXED)
    n = bem.bembel_ndofs(gop)
    dirs = np.array([[0, 0, 1.0], [1.0, 0, 0], [0.6, 0.8, 0], [0, -0.6, 0.8]])
    B = torch.empty((4, n), dtype=torch.complex128, device="cuda")
    bem.bembel_rhs(gop, bem.BEMBEL_RHS_PLANE_WAVE, dirs, B)
    X = torch.empty_like(B)
    info = bem.bembel_solve(gop, B, X, 4, tol=1e-10, precond=bem.BEMBEL_PRECOND_BLOCK_JACOBI)
    assert info["converged"] and info["rel_residual"] <= 1e-10
    for r in range(4):
        x1 = torch.empty_like(B[r])
        bem.bembel_solve(gop, B[r].contiguous(), x1, 1, tol=1e-10, precond=bem.BEMBEL_PRECOND_BLOCK_JACOBI)
        assert (torch.linalg.norm(x1 - X[r]) / torch.linalg.norm(x1)).item() < 1e-8
    # residual of the batch checked with the FP64 operator product
    Y = torch.empty_like(B)
    bem.bembel_matvec(gop, X, Y, 4)
    assert (torch.linalg.norm(Y - B) / torch.linalg.norm(B)).item() < 1e-9


def test_perturbed_sphere_parity():
    """Perturbed sphere (dense Helmholtz, and H^2 Laplace): the device harmonics vs the oracle's."""
    from inputs import perturbed_sphere_coeffs
    from oracle.geometry import PerturbedSphere

    a = perturbed_sphere_coeffs(1000)
    g = bem.bembel_geom_create(bem.BEMBEL_GEOM_PERTURBED_SPHERE, coeffs=a, amplitude=0.1)
    geo = PerturbedSphere(a, 0.1)
    gop = bem.bembel_assemble(g, HEL, 3.0, 2, 1, 0, g_regular=4, g_singular=5)
    sp = S2Space(geo, 2, 1)
    A_ref = Assembler(sp, "helmholtz", 3.0, 4, 5).dense()
    assert rel_err(gpu_matrix(gop, sp.ndofs), A_ref) < 1e-12
    gop2 = bem.bembel_assemble(g, LAP, 0.0, 3, 0, 3, g_regular=3, g_singular=4, leaf_level=2)
    sp2 = S2Space(geo, 3, 0)
    h2 = H2Oracle(sp2, "laplace", q=3, eta=1.6, leaf_level=2, g_reg=3, g_sing=4)
    info = bem.bembel_op_info_get(gop2)
    assert info["n_far_blocks"] == len(h2.far) > 0
    assert rel_err(gpu_matrix(gop2, sp2.ndofs), h2.dense()) < 1e-12


def test_per_class_orders_parity(geom):
    gop = bem.bembel_assemble(geom, LAP, 0.0, 2, 1, 0, g_regular=3, g_singular=4, g_identical=6, g_edge=5,
                              g_vertex=3)
    sp = S2Space(Sphere6(), 2, 1)
    A_ref = Assembler(sp, "laplace", 0.0, 3, (6, 5, 3)).dense()
    assert rel_err(gpu_matrix(gop, sp.ndofs), A_ref) < 1e-12


@pytest.mark.parametrize("op,k,d", [("laplace", 0.0, 1), ("helmholtz", 2.5 + 0.3j, 2)])
def test_per_variable_orders_parity(geom, op, k, d):
    """Duffy rules with a Gauss order per variable (xi, eta.., u..) against the oracle's."""
    var = ((4, 5, 3, 3), (4, 5, 5, 3), (5, 4, 4, 4))
    gop = bem.bembel_assemble(geom, LAP if op == "laplace" else HEL, k, 2, d, 0, g_regular=3, g_singular=4,
                              g_identical_var=var[0], g_edge_var=var[1], g_vertex_var=var[2])
    sp = S2Space(Sphere6(), 2, d)
    A_ref = Assembler(sp, op, k, 3, var).dense()
    assert rel_err(gpu_matrix(gop, sp.ndofs), A_ref) < 1e-12


@pytest.mark.parametrize("op,k,d", [("laplace", 0.0, 1), ("helmholtz", 1.5, 0)])
def test_graded_separated_orders_parity(geom, op, k, d):
    """Separated pairs beyond the ring next to the touching pairs at their own order."""
    gop = bem.bembel_assemble(geom, LAP if op == "laplace" else HEL, k, 3, d, 0, g_regular=4, g_regular_far=2,
                              g_singular=4)
    sp = S2Space(Sphere6(), 3, d)
    asm = Assembler(sp, op, k, (4, 2), 4)
    info = bem.bembel_op_info_get(gop)
    far = sum(1 for e in range(sp.nelem) for f in range(e + 1, sp.nelem)
              if asm.classify(e, f)[0] == "regular" and not asm.ring(e, f))
    assert info["n_pairs_regular_far"] == far > 0
    assert rel_err(gpu_matrix(gop, sp.ndofs), asm.dense()) < 1e-12


def test_per_variable_orders_invalid(geom):
    for kw in (dict(g_edge_var=(4, 0, 5, 3)), dict(g_edge_var=(4, 11, 11, 3)),
               dict(g_edge_var=(4, 4, 5, 3)), dict(g_vertex_var=(5, 4, 4, 3))):  # partial, too large, asymmetric
        with pytest.raises(bem.BembelError):
            bem.bembel_assemble(geom, LAP, 0.0, 2, 1, 0, **kw)


@pytest.mark.parametrize("op,k,d", [("laplace", 0.0, 1), ("helmholtz", 4.0, 2)])
def test_autotune_meets_target(geom, op, k, d):
    """Tuned orders meet the accuracy target: the operator assembled with them
    differs from a high-order assembly by about the target, and q meets far_tol on far
    blocks of every level (Helmholtz: with the block tree's |kappa| diam <= 2 limit, without
    which the top-level clusters of kappa = 4 cannot be interpolated to 1e-4 by q <= 6)."""
    kind = LAP if op == "laplace" else HEL
    quad_tol, far_tol = 1e-6, 1e-4
    kw = dict(kdiam=2.0) if op == "helmholtz" else {}
    opts, rep = bem.bembel_autotune(geom, kind, k, 4, d, quad_tol=quad_tol, far_tol=far_tol, q_max=6, **kw)
    for key in ("err_regular", "err_identical", "err_edge", "err_vertex"):
        assert rep[key] <= quad_tol, rep
    assert rep["err_far"] <= far_tol and 2 <= rep["q"] <= 6, rep
    assert all(2 <= opts.__getattribute__(f) <= 9 for f in ("g_regular", "g_identical", "g_edge", "g_vertex"))
    tuned = bem.bembel_assemble(geom, kind, k, 4, d, 0, opts=opts)
    ref = bem.bembel_assemble(geom, kind, k, 4, d, 0, g_regular=8, g_singular=8)
    n = bem.bembel_ndofs(tuned)
    dt = torch.complex128 if op == "helmholtz" else torch.float64
    x = torch.from_numpy(random_vector(n, 5, complex_=(op == "helmholtz"))).to(dt).cuda()
    y1, y2 = torch.empty_like(x), torch.empty_like(x)
    bem.bembel_matvec(tuned, x, y1, 1)
    bem.bembel_matvec(ref, x, y2, 1)
    assert (torch.linalg.norm(y1 - y2) / torch.linalg.norm(y2)).item() < 10 * quad_tol


def test_sound_soft_scattering_batch(geom):
    """Sound-soft unit sphere, 6 plane waves solved as one batch (degree 2, q = 4,
    mixed precision): the scattered field at |x| = 3 against the partial-wave
    series for the exp(-i k r) convention,
    u_s = -sum_l (2l+1) (-i)^l j_l(k)/h2_l(k) h2_l(k|x|) P_l(cos angle(x, d))."""
    import scipy.special as ss

    from inputs import sphere_points, unit_directions

    k = 2.0
    gop = bem.bembel_assemble(geom, HEL, k, 4, 2, 4, precision=bem.BEMBEL_PREC_MIXED)
    n = bem.bembel_ndofs(gop)
    dirs = unit_directions(6, 3)
    B = torch.empty((6, n), dtype=torch.complex128, device="cuda")
    bem.bembel_rhs(gop, bem.BEMBEL_RHS_PLANE_WAVE, dirs, B, g=6)
    B = -B  # Dirichlet data of the scattered field: u_s = -u_inc on the sphere
    X = torch.empty_like(B)
    info = bem.bembel_solve(gop, B, X, 6, tol=1e-10, precond=bem.BEMBEL_PRECOND_BLOCK_JACOBI)
    assert info["converged"]
    pts = sphere_points(10, 3.0, 11)
    U = torch.empty((6, 10), dtype=torch.complex128, device="cuda")
    bem.bembel_eval(gop, torch.from_numpy(pts).cuda(), X, U, 6, g=6)
    U = U.cpu().numpy()
    rr = np.linalg.norm(pts, axis=1)
    h2 = lambda l, z: ss.spherical_jn(l, z) - 1j * ss.spherical_yn(l, z)  # noqa: E731
    for r in range(6):
        c = pts @ dirs[r] / rr
        ref = np.zeros(10, dtype=complex)
        for l in range(25):
            ref += -(2 * l + 1) * (-1j) ** l * ss.spherical_jn(l, k) / h2(l, k) * h2(l, k * rr) * ss.eval_legendre(l, c)
        assert np.max(np.abs(U[r] - ref)) / np.max(np.abs(ref)) < 1e-4, r
