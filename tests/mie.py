"""Mie series for a perfectly conducting unit sphere (test helper).

Textbook vector spherical wave functions (Bohren & Huffman, ch. 4) for
x-polarised plane-wave incidence in the exp(-i omega t) convention:
    E_inc = x_hat exp(i k z) = sum_n E_n (M_o1n^(1) - i N_e1n^(1)),
    E_sca = sum_n E_n (i a_n N_e1n^(3) - b_n M_o1n^(3)),   E_n = i^n (2n+1)/(n(n+1)),
with, for a perfect conductor, a_n = [x j_n(x)]' / [x h_n(x)]', b_n = j_n(x) / h_n(x), x = k.
The library's kernel exp(-i kappa r) is the exp(+i omega t) convention: for real
k its fields are the complex conjugates, E_inc = x_hat exp(-i k z).
"""
from __future__ import annotations

import numpy as np
from scipy.special import spherical_jn, spherical_yn


def _pi_tau(mu: np.ndarray, nmax: int):
    pi = np.zeros((nmax + 1,) + mu.shape)
    tau = np.zeros_like(pi)
    pi[1] = 1.0
    for n in range(2, nmax + 1):
        pi[n] = (2 * n - 1) / (n - 1) * mu * pi[n - 1] - n / (n - 1) * pi[n - 2]
    for n in range(1, nmax + 1):
        tau[n] = n * mu * pi[n] - (n + 1) * pi[n - 1]
    return pi, tau


def _fields(pts: np.ndarray, k: float, kind: str, nmax: int, coef_M, coef_N):
    """sum_n coef_M[n] M_o1n + coef_N[n] N_e1n at Cartesian points, with radial
    functions j_n (kind 'j') or h_n^(1) (kind 'h')."""
    x, y, z = pts.T
    r = np.linalg.norm(pts, axis=1)
    th = np.arccos(np.clip(z / r, -1, 1))
    ph = np.arctan2(y, x)
    mu = np.cos(th)
    pi, tau = _pi_tau(mu, nmax)
    rho = k * r
    Er = np.zeros(len(r), dtype=complex)
    Et = np.zeros_like(Er)
    Ep = np.zeros_like(Er)
    for n in range(1, nmax + 1):
        jn = spherical_jn(n, rho)
        djn = spherical_jn(n, rho, derivative=True)
        if kind == "j":
            zn, dzn = jn, djn
        else:
            zn = jn + 1j * spherical_yn(n, rho)
            dzn = djn + 1j * spherical_yn(n, rho, derivative=True)
        drz = (zn + rho * dzn) / rho  # [rho z_n]' / rho
        # M_o1n = cos(ph) pi_n z_n e_th - sin(ph) tau_n z_n e_ph
        Mt = np.cos(ph) * pi[n] * zn
        Mp = -np.sin(ph) * tau[n] * zn
        # N_e1n = cos(ph) n(n+1) sin(th) pi_n z_n/rho e_r + cos(ph) tau_n drz e_th - sin(ph) pi_n drz e_ph
        Nr = np.cos(ph) * n * (n + 1) * np.sin(th) * pi[n] * zn / rho
        Nt = np.cos(ph) * tau[n] * drz
        Np = -np.sin(ph) * pi[n] * drz
        Er += coef_N[n] * Nr
        Et += coef_M[n] * Mt + coef_N[n] * Nt
        Ep += coef_M[n] * Mp + coef_N[n] * Np
    st, ct, sp, cp = np.sin(th), np.cos(th), np.sin(ph), np.cos(ph)
    ex = Er * st * cp + Et * ct * cp - Ep * sp
    ey = Er * st * sp + Et * ct * sp + Ep * cp
    ez = Er * ct - Et * st
    return np.stack([ex, ey, ez], axis=1)


def nmax_for(k: float) -> int:
    return int(k + 4 * k ** (1 / 3) + 8)


def incident_series_bh(pts, k: float, nmax: int | None = None):
    """The BH expansion of x_hat exp(i k z) (exp(-i omega t) convention)."""
    nmax = nmax or nmax_for(k)
    En = np.array([0] + [1j**n * (2 * n + 1) / (n * (n + 1)) for n in range(1, nmax + 1)])
    return _fields(np.asarray(pts, float), k, "j", nmax, En, -1j * En)


def scattered_pec(pts, k: float, nmax: int | None = None):
    """Scattered field of a PEC unit sphere for E_inc = x_hat exp(-i k z) in the
    exp(+i omega t) convention of the kernel exp(-i kappa r) (conjugate of BH)."""
    nmax = nmax or nmax_for(k)
    a = np.zeros(nmax + 1, dtype=complex)
    b = np.zeros(nmax + 1, dtype=complex)
    En = np.zeros(nmax + 1, dtype=complex)
    for n in range(1, nmax + 1):
        jn, djn = spherical_jn(n, k), spherical_jn(n, k, derivative=True)
        hn = jn + 1j * spherical_yn(n, k)
        dhn = djn + 1j * spherical_yn(n, k, derivative=True)
        a[n] = (jn + k * djn) / (hn + k * dhn)
        b[n] = jn / hn
        En[n] = 1j**n * (2 * n + 1) / (n * (n + 1))
    E_bh = _fields(np.asarray(pts, float), k, "h", nmax, -b * En, 1j * a * En)
    return np.conj(E_bh)
