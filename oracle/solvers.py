"""Linear solvers for the Galerkin systems (test infrastructure).

Sec. 4.6: the reference solves with Eigen's matrix-free GMRES and no
preconditioner.  Here: a dense direct solve (LAPACK through numpy) and a
textbook restarted GMRES(m) (Saad & Schultz 1986) with modified Gram-Schmidt
Arnoldi and Givens rotations, x0 = 0, stopping on the relative residual
||b - A x|| / ||b||.
"""
from __future__ import annotations

import numpy as np


def direct_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    return np.linalg.solve(A, b)


def gmres(matvec, b: np.ndarray, tol: float = 1e-8, restart: int = 30, maxit: int = 1000):
    """Restarted GMRES.  Returns (x, iterations, relative residual history)."""
    b = np.asarray(b)
    dtype = np.result_type(b.dtype, float)
    n = b.size
    x = np.zeros(n, dtype=dtype)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, [0.0]
    hist = []
    it = 0
    while it < maxit:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta / bnorm <= tol:
            break
        V = np.zeros((restart + 1, n), dtype=dtype)
        H = np.zeros((restart + 1, restart), dtype=dtype)
        cs = np.zeros(restart, dtype=dtype)
        sn = np.zeros(restart, dtype=dtype)
        g = np.zeros(restart + 1, dtype=dtype)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(restart):
            w = matvec(V[j])
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[j + 1] = w / H[j + 1, j]
            # apply previous rotations to the new column
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            # new rotation zeroing H[j+1, j]
            a, bb = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            cs[j] = abs(a) / den if den else 1.0
            sn[j] = (a / abs(a)) * np.conj(bb) / den if abs(a) > 0 else 1.0
            H[j, j] = cs[j] * a + sn[j] * bb
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) / bnorm <= tol or it >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + V[:j_done].T @ y
        if hist[-1] <= tol:
            r = b - matvec(x)
            hist.append(np.linalg.norm(r) / bnorm)
            if hist[-1] <= tol:
                break
    return x, it, hist
