"""Write tests/golden/converged_blocks_L6_p1.txt: converged near-field element-pair blocks
of the level-6, degree-1 cube-face sphere (Laplace single layer, App. B eq. (LS)).

Every value comes from ``oracle.converged`` (graded polar/tanh-sinh integration, no Duffy
rules), in the element-local tensor Bernstein basis of degree 1, parameter measure (Piola
2-form lift of App. E).  Pairs are chosen from the near field of the block tree at leaf
level 5, eta = 1.6 (``oracle.h2.block_tree``), one of each class (identical, common edge,
common vertex, separated in the ring next to the touching pairs, separated beyond it) for
each of three elements: inside a patch, on a patch edge and at a cube corner.

Usage: python tests/golden/make_converged_blocks.py   (about ten minutes on one core)
"""
from __future__ import annotations

import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import converged as CV  # noqa: E402
from oracle.galerkin import Assembler  # noqa: E402
from oracle.geometry import Sphere6  # noqa: E402
from oracle.h2 import block_tree, cluster_elements, cluster_of  # noqa: E402
from oracle.space import S2Space  # noqa: E402

LEVEL, DEGREE, LEAF, ETA = 6, 1, 5, 1.6
ELEMENTS = [(2, 20, 37), (0, 0, 30), (4, 63, 63)]
OUT = os.path.join(HERE, "converged_blocks_L6_p1.txt")


def main():
    sp = S2Space(Sphere6(), LEVEL, DEGREE)
    asm = Assembler(sp, "laplace")
    _, near, _ = block_tree(sp.geom, LEAF, ETA)
    near_of = {}
    for t, s in near:
        near_of.setdefault(t, []).append(s)
    lines = [f"# converged Laplace single-layer blocks, sphere6 level {LEVEL}, degree {DEGREE} (Bernstein), "
             f"parameter measure; written by tests/golden/make_converged_blocks.py from oracle.converged",
             "# kind  e_patch e_i1 e_i2  f_patch f_i1 f_i2  est_rel_err  block row-major"]
    t0 = time.time()
    for ep in ELEMENTS:
        e = sp.element_index(*ep)
        cands = [f for s in near_of[cluster_of(sp, e, LEAF)] for f in cluster_elements(sp, s)]
        picked = {}
        for f in sorted(cands, key=lambda f: (sp.element(f)[0] == ep[0], f)):  # cross-patch first
            kind, _ = CV.pair_kind(sp, e, f)
            if kind == "separated":
                kind = "ring" if asm.ring(e, f) else "beyond"
            picked.setdefault(kind, f)
        for kind in ("identical", "edge", "vertex", "ring", "beyond"):
            f = picked[kind]
            blk, err = CV.space_block(sp, "laplace", 0.0, e, f, basis="bernstein", r0=1, max_steps=1)
            fp = sp.element(f)
            lines.append(" ".join([kind, *map(str, ep), *map(str, fp), f"{err:.3e}", *(repr(float(v)) for v in
                                                                                     blk.ravel())]))
            print(f"{kind:9s} e={ep} f={fp} est {err:.1e} ({time.time() - t0:.0f} s)", flush=True)
    with open(OUT, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
