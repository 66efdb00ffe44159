"""Pins for the perturbed sphere geometry: the real harmonics are orthonormal on
the sphere (quadrature on the cube-face patches), agree with scipy's complex
harmonics up to the documented phase, and the coefficient draw keeps r > 0.5."""
import numpy as np
import scipy.special as ss

from inputs import perturbed_sphere_coeffs
from oracle.gauss import tensor2
from oracle.geometry import PerturbedSphere, Sphere6, real_harmonic


def test_real_harmonics_orthonormal():
    g = Sphere6()
    pts, w = tensor2(16)
    X, W = [], []
    for p in range(6):
        st = pts
        x = g.eval(p, st)
        J = g.jacobian(p, st)
        area = np.linalg.norm(np.cross(J[..., 0], J[..., 1]), axis=-1)
        X.append(x)
        W.append(w * area)
    X, W = np.concatenate(X), np.concatenate(W)
    lm = [(l, m) for l in range(1, 5) for m in range(-l, l + 1)]
    Y = np.stack([real_harmonic(l, m, X) for l, m in lm])
    G = (Y * W) @ Y.T
    np.testing.assert_allclose(G, np.eye(len(lm)), atol=1e-6)


def test_real_harmonics_vs_scipy():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((20, 3))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    th, ph = np.arccos(x[:, 2]), np.arctan2(x[:, 1], x[:, 0])
    for l in range(1, 5):
        for m in range(1, l + 1):
            y = ss.sph_harm_y(l, m, th, ph)  # includes (-1)^m
            np.testing.assert_allclose(real_harmonic(l, m, x), (-1) ** m * np.sqrt(2) * y.real, atol=1e-12)
            np.testing.assert_allclose(real_harmonic(l, -m, x), (-1) ** m * np.sqrt(2) * y.imag, atol=1e-12)
        np.testing.assert_allclose(real_harmonic(l, 0, x), ss.sph_harm_y(l, 0, th, ph).real, atol=1e-12)


def test_perturbed_radius_bounds():
    for seed in (1000, 1001, 2000):
        a = perturbed_sphere_coeffs(seed)
        geo = PerturbedSphere(a, 0.1)
        st = np.stack(np.meshgrid(np.linspace(0, 1, 21), np.linspace(0, 1, 21)), -1).reshape(-1, 2)
        for p in range(6):
            r = np.linalg.norm(geo.eval(p, st), axis=1)
            assert r.min() > 0.5
