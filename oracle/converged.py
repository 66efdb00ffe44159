"""Converged element-pair integrals without the Duffy rule set (test infrastructure).

An independent reference for the Galerkin entries of Sec. 2 and App. B, eq. (LS)/(HS):

    B_ij = int_e int_f G(gamma(s), gamma(t)) phi_i(s) phi_j(t) dt ds

for curved elements e, f, by a technique that shares nothing with the
regularising (Duffy-type) transforms of ``oracle.quadrature``:

* Inner integral, for one outer point x = gamma_e(s): f's local square is cut
  into four triangles with a common apex p, the point of f's square whose image
  is nearest x (p = s when f = e).  Triangle (p, a, b) is integrated in the
  coordinates (rho, theta) -> t = p + rho (a + theta (b - a) - p), whose
  Jacobian rho |(a - p) x (b - a)| cancels the 1/|x - y| growth at the apex.
  theta is integrated after the substitution theta = theta0 + delta sinh(u)
  (theta0 the foot of p on the side, delta its height), which removes the
  near-singularity of thin triangles; rho by Gauss-Legendre when x = gamma(p),
  else after rho = (d / |D gamma v|) sinh(u) with d = |x - gamma_f(p)|, which
  removes the near-singularity of outer points close to f.  Outer points
  farther from f than its diameter take a plain tensor Gauss rule.
* Outer integral: the inner integral, as a function of s, is smooth inside e but
  not at the set where e meets f (its derivatives grow like log distance): the
  whole boundary of e when f = e, the shared edge or the shared vertex for
  touching pairs.  The outer rule is the tanh-sinh rule in both directions for
  touching pairs (exponentially convergent for such end-point singularities)
  and Gauss-Legendre for separated ones.

Both parts are refined together (more panels, more points per panel) until the
block stops changing; ``converged_block`` returns the finest block and the
largest change of its last refinement as an error estimate.

The elements are given as callables, so the same code integrates flat squares
in closed-form position (the pins) and elements of any patch geometry.
"""
from __future__ import annotations

import numpy as np

from .gauss import gauss_legendre01

CORNERS = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])  # counter-clockwise
T_MAX = 3.0  # tanh-sinh cut-off: 1 - x >= 1/(1 + e^(pi sinh 3)) ~ 1e-14


# --------------------------------------------------------------------------- 1-D rules
def _panels_rule(bp, n):
    """Composite n-point Gauss on the panels between consecutive breakpoints (any shape
    (..., k+1)); returns nodes and weights of shape (..., k * n)."""
    x, w = gauss_legendre01(n)
    lo, hi = bp[..., :-1, None], bp[..., 1:, None]
    nodes = lo + (hi - lo) * x
    wts = (hi - lo) * w
    shp = bp.shape[:-1] + ((bp.shape[-1] - 1) * n,)
    return nodes.reshape(shp), wts.reshape(shp)


def tanh_sinh(level: int) -> tuple[np.ndarray, np.ndarray]:
    """Tanh-sinh rule on [0, 1] with step 2^-level: x = 1 / (1 + exp(-pi sinh t)),
    w = h pi cosh t x (1 - x), t = -T_MAX .. T_MAX.  It converges exponentially for
    integrands analytic inside (0, 1) whatever their (integrable) singularities at the ends."""
    h = 2.0 ** -level
    t = np.arange(-T_MAX, T_MAX + 0.5 * h, h)
    x = 1.0 / (1.0 + np.exp(-np.pi * np.sinh(t)))
    xc = 1.0 / (1.0 + np.exp(np.pi * np.sinh(t)))  # 1 - x without cancellation
    return x, h * np.pi * np.cosh(t) * x * xc


def outer_rule_1d(r: int, singular: bool):
    """Outer rule in one direction: tanh-sinh of level 2 + r where the inner integral may be
    singular at an end of [0, 1], else Gauss-Legendre with 2 panels of 8 + 2r points."""
    if singular:
        return tanh_sinh(2 + r)
    return _panels_rule(np.array([0.0, 0.5, 1.0]), 8 + 2 * r)


def _sinh_nodes(c, scale, lo, hi, panels: int, n: int):
    """Nodes and weights in y on [lo, hi] (arrays of any common shape S) for an integrand
    near-singular at y = c with width scale: y = c + scale sinh(u), u on equal panels.
    Returns arrays of shape S + (panels * n,)."""
    ua = np.arcsinh((lo - c) / scale)
    ub = np.arcsinh((hi - c) / scale)
    bp = ua[..., None] + (ub - ua)[..., None] * np.linspace(0.0, 1.0, panels + 1)
    u, wu = _panels_rule(bp, n)
    y = c[..., None] + scale[..., None] * np.sinh(u)
    return y, wu * scale[..., None] * np.cosh(u)


# --------------------------------------------------------------------------- inner rules
def polar_rule(p, d, jac, r: int):
    """Rule on the unit square for apexes p (B, 2) at physical distance d (B,) from the outer
    point (d = 0: the apex is the outer point's own parameter), jac (B, 3, 2) the patch
    Jacobian of the element map at p.  Four triangles (p, c_k, c_k+1) in (rho, theta):
    theta by a sinh substitution around the foot of p on the side (width: the height of p),
    rho by Gauss-Legendre (d = 0) or a sinh substitution around rho = 0 of width
    d / |jac v(theta)|.  Returns points (B, N, 2) and weights (B, N)."""
    n = 6 + 2 * r
    panels = 2 + r
    B = p.shape[0]
    pts, wts = [], []
    for k in range(4):
        a, b = CORNERS[k], CORNERS[(k + 1) % 4]
        ab = b - a  # unit length side
        ap = a[None, :] - p  # (B, 2)
        det = np.abs(ap[:, 0] * ab[1] - ap[:, 1] * ab[0])  # height of p over the side
        th0 = np.clip(-(ap @ ab), 0.0, 1.0)  # foot of p on the side, in theta
        zero, one = np.zeros(B), np.ones(B)
        th, wth = _sinh_nodes(th0, np.maximum(det, 1e-15), zero, one, panels, n)  # (B, T)
        v = ap[:, None, :] + th[:, :, None] * ab[None, None, :]  # (B, T, 2)
        T = th.shape[1]
        if d is None:
            rho, wr = _panels_rule(np.linspace(0.0, 1.0, panels + 1), n)
            rho = np.broadcast_to(rho, (B, T, len(rho)))
            wr = np.broadcast_to(wr, (B, T, len(wr)))
        else:
            vlen = np.linalg.norm(np.einsum("bkj,btj->btk", jac, v), axis=-1)  # physical |dgamma v|
            scale = np.maximum(d[:, None] / np.maximum(vlen, 1e-300), 1e-15)
            rho, wr = _sinh_nodes(np.zeros((B, T)), scale, np.zeros((B, T)), np.ones((B, T)), panels, n)
        # t = p + rho v(theta); Jacobian rho * det
        t = p[:, None, None, :] + rho[..., None] * v[:, :, None, :]  # (B, T, R, 2)
        w = wth[:, :, None] * wr * rho * det[:, None, None]
        pts.append(t.reshape(B, -1, 2))
        wts.append(w.reshape(B, -1))
    return np.concatenate(pts, axis=1), np.concatenate(wts, axis=1)


def _jacobian(xf, p, h: float = 1e-6):
    """Central-difference Jacobian (B, 3, 2) of the element map at local points p (B, 2)
    (one-sided at the square's boundary)."""
    cols = []
    for i, e in enumerate(np.eye(2)):
        hi, lo = np.clip(p + h * e, 0, 1), np.clip(p - h * e, 0, 1)
        cols.append((xf(hi) - xf(lo)) / (hi - lo)[:, [i]])
    return np.stack(cols, axis=-1)


def nearest_point(xf, x, grid: int = 17, iters: int = 25):
    """Point of the unit square whose image under xf is nearest each x (B, 3): a grid search
    then projected Gauss-Newton steps.  Any point of the square is a valid apex; nearness
    only speeds up convergence."""
    g = (np.arange(grid) + 0.5) / grid
    G = np.stack(np.meshgrid(g, g, indexing="xy"), -1).reshape(-1, 2)
    XG = xf(G)  # (grid^2, 3)
    d2 = np.sum((x[:, None, :] - XG[None, :, :]) ** 2, axis=-1)
    p = G[np.argmin(d2, axis=1)].copy()
    for _ in range(iters):
        J = _jacobian(xf, p)
        r = xf(p) - x
        JtJ = np.einsum("bki,bkj->bij", J, J)
        Jtr = np.einsum("bki,bk->bi", J, r)
        step = np.linalg.solve(JtJ + 1e-30 * np.eye(2), Jtr[..., None])[..., 0]
        p = np.clip(p - step, 0.0, 1.0)
    return p


# --------------------------------------------------------------------------- the block
def _outer_singular(kind: str):
    """Per direction of e's local square: may the inner integral be singular at an end of it?
    For touching pairs yes in both directions (across a shared edge, and at its end points
    along it); tanh-sinh costs little where an end is smooth after all."""
    return (kind != "separated",) * 2


def pair_block(xe, be, xf, bf, kernel, kind: str, shared=(), r: int = 2, chunk: int = 32, diam_f=None):
    """int_[0,1]^2 int_[0,1]^2 kernel(xe(s), xf(t)) be(s)_i bf(t)_j dt ds at refinement r.

    xe, xf: local points (N, 2) -> physical points (N, 3); be, bf: local points -> basis
    values (N, ni) / (N, nj).  kind: 'identical' (xf = xe), 'edge', 'vertex' or 'separated';
    shared: e's local corners that are corners of f (informative; the rules depend on kind)."""
    sg1, sg2 = _outer_singular(kind)
    s1, w1 = outer_rule_1d(r, sg1)
    s2, w2 = outer_rule_1d(r, sg2)
    S = np.stack(np.meshgrid(s1, s2, indexing="ij"), -1).reshape(-1, 2)
    WS = np.outer(w1, w2).ravel()
    X = xe(S)
    BE = be(S)
    if diam_f is None:
        C = xf(CORNERS)
        diam_f = max(np.linalg.norm(C[i] - C[j]) for i in range(4) for j in range(i))
    # plain tensor Gauss for outer points far from f
    tg, tw = _panels_rule(np.array([0.0, 0.5, 1.0]), 8 + 2 * r)
    TP = np.stack(np.meshgrid(tg, tg, indexing="ij"), -1).reshape(-1, 2)
    TW = np.outer(tw, tw).ravel()
    YP, BP = xf(TP), bf(TP)
    out = None
    for lo in range(0, len(S), chunk):
        sl = slice(lo, lo + chunk)
        x = X[sl]
        if kind == "identical":
            p = S[sl].copy()
            d = np.zeros(len(p))
        else:
            p = nearest_point(xf, x)
            d = np.linalg.norm(xf(p) - x, axis=1)
        far = d > diam_f
        inner = np.zeros((len(x), BP.shape[1]), dtype=complex)
        if far.any():
            Kf = kernel(x[far][:, None, :], YP[None, :, :])
            inner[far] = (Kf * TW) @ BP
        near = ~far
        if near.any():
            pn = p[near]
            T, WT = polar_rule(pn, None if kind == "identical" else d[near], _jacobian(xf, pn), r)
            B, N = T.shape[:2]
            Y = xf(T.reshape(-1, 2)).reshape(B, N, 3)
            BF = bf(T.reshape(-1, 2)).reshape(B, N, -1)
            with np.errstate(divide="ignore", invalid="ignore"):
                Kn = kernel(x[near][:, None, :], Y)
            # an inner point can round onto the outer point only where rho * height is below
            # 1e-16 (apex within rounding of a side), i.e. at a weight far below any digit kept
            Kn = np.where(np.isfinite(Kn), Kn, 0.0)
            inner[near] = np.einsum("bn,bnj->bj", Kn * WT, BF)
        blk = (BE[sl] * WS[sl, None]).T @ inner
        out = blk if out is None else out + blk
    return out


def converged_block(xe, be, xf, bf, kernel, kind: str, shared=(), tol: float = 1e-12, r0: int = 1,
                    max_steps: int = 4, **kw):
    """Refine r -> r + 1 until two successive blocks differ by at most tol relative to the
    block's largest entry.  Returns (block, estimated relative error)."""
    r = r0
    prev = pair_block(xe, be, xf, bf, kernel, kind, shared, r=r, **kw)
    err = np.inf
    for _ in range(max_steps):
        r += 1
        cur = pair_block(xe, be, xf, bf, kernel, kind, shared, r=r, **kw)
        err = np.max(np.abs(cur - prev)) / np.max(np.abs(cur))
        prev = cur
        if err <= tol:
            break
    return prev, err


# --------------------------------------------------------------------------- S2 spaces
def _shared_corners(space, e: int, f: int, tol: float = 1e-9):
    """Local corners of e that are also corners of f (physical positions compared)."""
    ce, cf = space.corners(e), space.corners(f)
    loc = [(0.0, 0.0), (1.0, 0.0), (0.0, 1.0), (1.0, 1.0)]
    return [loc[i] for i in range(4) if np.min(np.linalg.norm(cf - ce[i], axis=1)) < tol]


def pair_kind(space, e: int, f: int):
    """('identical' | 'edge' | 'vertex' | 'separated', shared local corners of e)."""
    if e == f:
        return "identical", []
    sh = _shared_corners(space, e, f)
    return {0: "separated", 1: "vertex", 2: "edge"}[len(sh)], sh


def bernstein(d: int, st):
    """Tensor Bernstein polynomials of degree d on the unit square, index k1 + (d+1) k2."""
    from math import comb

    st = np.atleast_2d(st)
    k = np.arange(d + 1)
    c = np.array([comb(d, i) for i in k], dtype=float)
    b1 = c * st[:, 0:1] ** k * (1 - st[:, 0:1]) ** (d - k)
    b2 = c * st[:, 1:2] ** k * (1 - st[:, 1:2]) ** (d - k)
    return np.einsum("na,nb->nba", b1, b2).reshape(len(st), -1)


def space_block(space, op: str, kappa: complex, e: int, f: int, basis: str = "bspline", tol: float = 1e-12,
                **kw):
    """Converged (nloc x nloc) block of elements e, f of an S2Space for the kernel of (LS)/(HS),
    in the parameter measure (Piola 2-form lift: measures cancel), i.e. h^4 times the local
    integral.  basis 'bspline' (the space's element-restricted B-splines, the oracle's basis) or
    'bernstein' (tensor Bernstein polynomials of the space's degree on the element)."""
    from .galerkin import green

    kind, shared = pair_kind(space, e, f)
    pe, pf = space.element(e)[0], space.element(f)[0]

    def xe(st):
        return space.geom.eval(pe, space.to_patch(e, st))

    def xf(st):
        return space.geom.eval(pf, space.to_patch(f, st))

    if basis == "bspline":
        def be(st):
            return space.element_basis(e, st)

        def bf(st):
            return space.element_basis(f, st)
    else:
        def be(st):
            return bernstein(space.d, st)

        bf = be

    def kernel(x, y):
        return green(op, kappa, x, y)

    blk, err = converged_block(xe, be, xf, bf, kernel, kind, shared, tol=tol, **kw)
    blk = blk * space.h**4
    return (blk.real if op == "laplace" else blk), err
