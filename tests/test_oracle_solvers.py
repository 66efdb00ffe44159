"""Pins for the oracle's solvers: restarted GMRES against LAPACK's direct solve."""
import numpy as np
import pytest

from oracle.solvers import direct_solve, gmres


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("restart", [5, 30])
def test_gmres_matches_direct(cplx, restart):
    rng = np.random.default_rng(3)
    n = 60
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    if cplx:
        A = A + 1j * rng.standard_normal((n, n)) / np.sqrt(n)
        b = b + 1j * rng.standard_normal(n)
    x, it, hist = gmres(lambda v: A @ v, b, tol=1e-12, restart=restart, maxit=500)
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) <= 1e-12
    np.testing.assert_allclose(x, direct_solve(A, b), rtol=1e-10, atol=1e-12)
    # Arnoldi residual estimates never increase within a cycle
    est = hist[: min(restart, it) + 1]  # initial residual + estimates of the first cycle
    assert all(b_ <= a_ * (1 + 1e-12) for a_, b_ in zip(est, est[1:]))


def test_gmres_zero_rhs():
    x, it, hist = gmres(lambda v: v, np.zeros(5))
    assert it == 0 and not np.any(x)
