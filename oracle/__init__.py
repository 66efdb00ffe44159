"""Plain FP64 CPU oracle for the isogeometric single-layer boundary element method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path (the
CUDA library and its Python binding) never imports, links or executes it, and
this package imports nothing from the product package.

What it computes, written from the paper (Doelz et al., "Bembel", App. A-E):

* Geometry: the 6-patch cube-face sphere (arbitrary smooth parametric mappings,
  Sec. 4.1) and the radially perturbed sphere; patches satisfy the matching
  condition of App. D.
* Spaces: the S^2 space of App. E (tensor B-splines of degree p-1 on the
  truncated open knot vector, lifted by the 2-form Piola transform) evaluated
  with the B-spline recursion of App. C.
* The Galerkin matrix A_ij = <S phi_j, phi_i> of the single-layer operators (LS)
  and (HS) of App. B, with tensor Gauss quadrature on separated element pairs
  and Duffy-type regularising transforms (the "regularization techniques" cited
  in Sec. 2) on identical, edge- and vertex-adjacent element pairs.
* Load vectors (Sec. 4.4) and potential evaluation (Sec. 4.7).
* The H^2 approximant of Sec. 2 (kernel interpolated on the parameter domain per
  cluster pair), written as a dense block-wise reconstruction without nested
  bases.
* Dense LU and textbook restarted GMRES (Sec. 4.6).

Every function states the passage it follows.  Pins against closed forms,
library routines and brute force live in ``tests/test_oracle_*.py``.
"""
