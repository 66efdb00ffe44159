"""Helmholtz at kappa = 8 and 16 (the batched Helmholtz configuration's wavenumbers).

The far field uses the block tree's |kappa| max(diam) <= kdiam limit (App. B eq. (HS):
exp(-i kappa r) must be resolvable by q Chebyshev points over a far block) with q chosen by
the autotuner from far blocks of every level.  Checks: block counts and the H^2 matrix
against the oracle with the same limit (rounding only), and the sound-soft sphere's
scattered field at |x| = 3 against the partial-wave series
u_s = -sum_l (2l+1) (-i)^l j_l(k)/h2_l(k) h2_l(k|x|) P_l(cos angle)
(discretisation + compression error; measured ~1e-6 at kappa = 8, level 4 and kappa = 16,
level 5, degree 2)."""
import numpy as np
import pytest
import scipy.special as ss
import torch

import paper_1906_00785_gb300 as bem
from inputs import sphere_points, unit_directions
from oracle.geometry import Sphere6
from oracle.h2 import H2Oracle
from oracle.space import S2Space

pytestmark = pytest.mark.gpu
HEL = bem.BEMBEL_HELMHOLTZ_SL


@pytest.fixture(scope="module")
def geom():
    return bem.bembel_geom_create()


def series(k, pts, d):
    rr = np.linalg.norm(pts, axis=1)
    c = pts @ d / rr
    h2 = lambda l, z: ss.spherical_jn(l, z) - 1j * ss.spherical_yn(l, z)  # noqa: E731
    out = np.zeros(len(pts), dtype=complex)
    for l in range(int(2 * k) + 30):
        out += -(2 * l + 1) * (-1j) ** l * ss.spherical_jn(l, k) / h2(l, k) * h2(l, k * rr) * ss.eval_legendre(l, c)
    return out


def test_kdiam_block_tree_and_matrix_parity(geom):
    k, kd = 8.0, 4.0
    gop = bem.bembel_assemble(geom, HEL, k, 3, 1, 4, g_regular=3, g_singular=4, leaf_level=2, eta=1.6, kdiam=kd)
    sp = S2Space(Sphere6(), 3, 1)
    h2 = H2Oracle(sp, "helmholtz", k, q=4, eta=1.6, leaf_level=2, g_reg=3, g_sing=4, kdiam=kd)
    info = bem.bembel_op_info_get(gop)
    assert info["n_far_blocks"] == len(h2.far) and info["n_near_blocks"] == len(h2.near)
    plain = bem.bembel_op_info_get(bem.bembel_assemble(geom, HEL, k, 3, 1, 4, leaf_level=2, eta=1.6))
    assert info["n_far_blocks"] != plain["n_far_blocks"]  # the limit changes the tree
    n = sp.ndofs
    eye = torch.eye(n, dtype=torch.complex128, device="cuda")
    out = torch.empty_like(eye)
    bem.bembel_matvec(gop, eye, out, n)
    A = out.cpu().numpy().T
    ref = h2.dense()
    assert np.max(np.abs(A - ref)) / np.max(np.abs(ref)) < 1e-12


@pytest.mark.parametrize("k,L", [(8.0, 4), (16.0, 5)])
def test_sound_soft_high_wavenumber(geom, k, L):
    opts, rep = bem.bembel_autotune(geom, HEL, k, L, 2, quad_tol=1e-6, far_tol=1e-4, q_max=8, kdiam=6.0)
    assert rep["err_far"] <= 1e-4, rep
    op = bem.bembel_assemble(geom, HEL, k, L, 2, rep["q"], opts=opts, precision=bem.BEMBEL_PREC_MIXED)
    n = bem.bembel_ndofs(op)
    d = unit_directions(2, 3)
    B = torch.empty((2, n), dtype=torch.complex128, device="cuda")
    bem.bembel_rhs(op, bem.BEMBEL_RHS_PLANE_WAVE, d, B, g=6)
    B = -B
    X = torch.empty_like(B)
    info = bem.bembel_solve(op, B, X, 2, tol=1e-8, restart=50, max_iter=5000, precond=bem.BEMBEL_PRECOND_BLOCK_JACOBI)
    assert info["converged"], info
    pts = sphere_points(20, 3.0, 11)
    U = torch.empty((2, 20), dtype=torch.complex128, device="cuda")
    bem.bembel_eval(op, torch.from_numpy(pts).cuda(), X, U, 2, g=6)
    for r in range(2):
        ref = series(k, pts, d[r])
        err = np.max(np.abs(U[r].cpu().numpy() - ref)) / np.max(np.abs(ref))
        print(f"kappa {k} level {L} q {rep['q']}: field error {err:.2e}, {info['iterations']} iterations")
        assert err < 1e-4, (r, err)
