"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws random numbers and fixes workload sizes; it holds none
of the boundary element method's arithmetic (no geometry, quadrature, kernel or
basis evaluation).  Both the CUDA path and the CPU oracle take their inputs from
here so that a parity test compares the two on identical data.

Workloads (the paper publishes no data sets; these stand in for its examples):

* ``ball_points``: evaluation points uniform in a ball (interior Laplace check,
  Remark in App. B: the single-layer potential also solves the interior problem).
* ``sphere_points``: evaluation points on a sphere of given radius (exterior
  scattered-field checks, in the spirit of the example's ``makeSphereGrid``).
* ``unit_directions``: plane-wave incidence directions uniform on S^2.
* ``perturbed_sphere_coeffs``: real spherical-harmonic coefficients a_lm for a
  radially perturbed sphere r = 1 + 0.1 * sum_{1<=l<=4} a_lm Y_lm.
* ``random_vector``: N(0,1) coefficient vectors for matvec parity.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(int(seed))


def ball_points(n: int, radius: float, seed: int) -> np.ndarray:
    """n points uniform in the ball of given radius: r = R*U^(1/3), direction = N(0,I)/|.|."""
    g = _rng(seed)
    d = g.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = radius * g.random(n) ** (1.0 / 3.0)
    return np.ascontiguousarray(d * r[:, None])


def sphere_points(n: int, radius: float, seed: int) -> np.ndarray:
    """n points uniform on the sphere of given radius."""
    g = _rng(seed)
    d = g.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return np.ascontiguousarray(d * radius)


def unit_directions(n: int, seed: int) -> np.ndarray:
    """n unit vectors uniform on S^2 (plane-wave incidence directions)."""
    return sphere_points(n, 1.0, seed)


def random_vector(n: int, seed: int, nrhs: int = 1, complex_: bool = False) -> np.ndarray:
    """Column-major (n, nrhs) N(0,1) data; complex draws real and imaginary parts independently."""
    g = _rng(seed)
    if complex_:
        v = g.standard_normal((nrhs, n)) + 1j * g.standard_normal((nrhs, n))
    else:
        v = g.standard_normal((nrhs, n))
    v = v.T
    return np.asfortranarray(v[:, 0] if nrhs == 1 else v)


def perturbed_sphere_coeffs(seed: int, lmax: int = 4, amp: float = 0.1) -> np.ndarray:
    """Coefficients a_lm ~ N(0,1)/l^2 for 1 <= l <= lmax, ordered (l, m = -l..l).

    Returned array has length (lmax+1)^2 - 1.  The draw is repeated (same
    generator, next numbers) while the coefficient-only bound
    amp * sum |a_lm| * sqrt(2) * sqrt((2l+1)/(4 pi)) reaches 0.5; real orthonormal
    harmonics satisfy |Y_lm| <= sqrt(2) sqrt((2l+1)/(4 pi)), so every accepted
    draw keeps the radius above 0.5.
    """
    g = _rng(seed)
    ls = np.concatenate([[l] * (2 * l + 1) for l in range(1, lmax + 1)]).astype(float)
    bound_w = np.sqrt(2.0) * np.sqrt((2 * ls + 1) / (4 * np.pi))
    for _ in range(1000):
        a = g.standard_normal(ls.size) / ls**2
        if amp * np.sum(np.abs(a) * bound_w) < 0.5:
            return a
    raise RuntimeError("perturbed_sphere_coeffs: no admissible draw")


# Workload definitions (sizes only).  Level L gives 2^L x 2^L elements per patch
# on the 6-patch sphere (App. E: equidistant knots with 2^L elements).
WORKLOADS = {
    "laplace_dense_L3_p0": dict(op="laplace", level=3, p=0, q=0, eta=1.6, x0=(0.0, 0.0, 2.0),
                                 n_eval=100, eval_radius=0.5, eval_seed=1),
    "laplace_h2_L6_p1_q4": dict(op="laplace", level=6, p=1, q=4, eta=1.6, x_seed=2),
    "helmholtz_h2_p2": dict(op="helmholtz", ks=(2.0, 8.0, 16.0), levels=(4, 5, 6), p=2,
                            nrhs=64, dir_seed=3),
    "efie_L4_p2_q6": dict(op="maxwell", k=4.0, level=4, p=2, q=6, n_eval=100, eval_radius=3.0,
                          eval_seed=4),
}


# (o, e1, e2) per cube face, e1 x e2 = o, in the patch order of the cube-face
# sphere: +x, -x, +y, -y, +z, -z (neighbouring faces then run the same way
# along every shared edge).
CUBE_FACES = (
    ((1, 0, 0), (0, 1, 0), (0, 0, 1)),
    ((-1, 0, 0), (0, 0, 1), (0, 1, 0)),
    ((0, 1, 0), (0, 0, 1), (1, 0, 0)),
    ((0, -1, 0), (1, 0, 0), (0, 0, 1)),
    ((0, 0, 1), (1, 0, 0), (0, 1, 0)),
    ((0, 0, -1), (0, 1, 0), (1, 0, 0)),
)


def nurbs_pillow_box(degree: int = 2, segments: int = 2, bulge: float = 0.3, weight: float = 1.6):
    """Six NURBS patches forming a closed 'pillow box' around the cube [-1, 1]^3.

    Each face is a degree-``degree`` B-spline patch with ``segments`` uniform knot
    spans per direction; control points sit at the Greville abscissae g of the
    face, pushed outward by bulge * b(g1) b(g2) (b(g) = 4 g (1 - g)) with weights
    1 + (weight - 1) b(g1) b(g2).  Boundary control points lie on the cube edges
    with weight 1, so neighbouring faces share their edge curves exactly.
    Returns six dicts: degrees, knots (s, t) and ctrl[i2, i1] = (x, y, z, w)."""
    p = degree
    kn = np.concatenate([np.zeros(p + 1), np.arange(1, segments) / segments, np.ones(p + 1)])
    k = segments + p
    grev = np.array([kn[i + 1 : i + p + 1].mean() for i in range(k)])
    bump = 4.0 * grev * (1.0 - grev)
    patches = []
    for o, e1, e2 in CUBE_FACES:
        o, e1, e2 = (np.array(v, dtype=float) for v in (o, e1, e2))
        ctrl = np.zeros((k, k, 4))
        for i2 in range(k):
            for i1 in range(k):
                b = bump[i1] * bump[i2]
                ctrl[i2, i1, :3] = o * (1.0 + bulge * b) + (2 * grev[i1] - 1) * e1 + (2 * grev[i2] - 1) * e2
                ctrl[i2, i1, 3] = 1.0 + (weight - 1.0) * b
        patches.append({"degrees": (p, p), "knots": (kn.copy(), kn.copy()), "ctrl": ctrl})
    return patches
