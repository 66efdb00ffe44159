"""Real orthonormal spherical harmonics from scipy (test helper)."""
import numpy as np
import scipy.special as ss


def real_ylm(l, m, x):
    th = np.arccos(np.clip(x[:, 2], -1, 1))
    ph = np.arctan2(x[:, 1], x[:, 0])
    y = ss.sph_harm_y(l, abs(m), th, ph)
    if m == 0:
        return y.real
    return np.sqrt(2) * (-1) ** m * (y.real if m > 0 else y.imag)


def helmholtz_sl_eig(l, k):
    """Single-layer eigenvalue on the unit sphere for exp(-ikr)/(4 pi r): -i k j_l(k) h_l^(2)(k)."""
    j = ss.spherical_jn(l, k)
    return -1j * k * j * (j - 1j * ss.spherical_yn(l, k))
