"""Element adjacency and canonical orientation for singular pairs (test infrastructure).

App. D: patches meet at full edges or vertices and neighbouring parametrisations
agree on a shared edge up to an affine map.  Two elements therefore touch iff
they share physical corner points; the shared corners tell which Duffy rule
applies (4 shared: identical, 2: common edge, 1: common vertex) and how to map
the canonical square of the rule onto each element.

A canonical map is T(u) = A + u1 D1 + u2 D2 from the rule's square to the
element's local square, with A a corner and D1, D2 the two unit directions
pointing into the square from A.
* common edge: A, B are the two shared corners, A the one listed first in the
  first element's corner order (0,0),(1,0),(0,1),(1,1); on both elements
  D2 = B - A runs along the edge and D1 points into the element, so u1 = 0 is
  the shared edge and u2 is the same physical point on both sides (matching
  condition of App. D).
* common vertex: A is the shared corner, D1 along the first local axis, D2 along
  the second.
"""
from __future__ import annotations

import numpy as np

LOCAL_CORNERS = np.array([[0, 0], [1, 0], [0, 1], [1, 1]], dtype=float)


def corner_ids(space, tol: float = 1e-9) -> np.ndarray:
    """Global vertex id of each element corner, (nelem, 4), by matching physical positions."""
    ids = np.empty((space.nelem, 4), dtype=np.int64)
    table: dict[tuple, int] = {}
    for e in range(space.nelem):
        for c, x in enumerate(space.corners(e)):
            key = tuple(np.round(x / tol).astype(np.int64))
            if key not in table:
                table[key] = len(table)
            ids[e, c] = table[key]
    return ids


def _inward(corner: np.ndarray, axis: int) -> np.ndarray:
    d = np.zeros(2)
    d[axis] = 1.0 if corner[axis] == 0.0 else -1.0
    return d


def canonical_maps(ids_e: np.ndarray, ids_f: np.ndarray):
    """Classify the pair (e, f) and return (kind, map_e, map_f).

    kind is 'identical', 'edge', 'vertex' or 'regular'; each map is (A, D1, D2)
    with T(u) = A + u1 D1 + u2 D2 (identity maps for 'identical' and 'regular').
    """
    ident = (np.zeros(2), np.array([1.0, 0.0]), np.array([0.0, 1.0]))
    shared = [c for c in range(4) if ids_e[c] in set(ids_f.tolist())]
    if len(shared) == 4:
        return "identical", ident, ident
    if len(shared) == 0:
        return "regular", ident, ident
    if len(shared) == 2:
        ca, cb = shared  # ascending corner order in e
        fa = int(np.nonzero(ids_f == ids_e[ca])[0][0])
        fb = int(np.nonzero(ids_f == ids_e[cb])[0][0])
        maps = []
        for a, b in ((ca, cb), (fa, fb)):
            A, B = LOCAL_CORNERS[a], LOCAL_CORNERS[b]
            D2 = B - A
            axis_along = 0 if D2[0] != 0 else 1
            D1 = _inward(A, 1 - axis_along)
            maps.append((A, D1, D2))
        return "edge", maps[0], maps[1]
    if len(shared) == 1:
        ca = shared[0]
        fa = int(np.nonzero(ids_f == ids_e[ca])[0][0])
        maps = []
        for a in (ca, fa):
            A = LOCAL_CORNERS[a]
            maps.append((A, _inward(A, 0), _inward(A, 1)))
        return "vertex", maps[0], maps[1]
    raise ValueError(f"elements share {len(shared)} corners: not a conforming mesh (App. D)")


def apply_map(m, u: np.ndarray) -> np.ndarray:
    A, D1, D2 = m
    u = np.asarray(u, dtype=float)
    return A + u[:, 0:1] * D1 + u[:, 1:2] * D2
