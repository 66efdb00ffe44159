/*
 * bembel.h - C ABI of the GB300 (sm_103a) isogeometric single-layer BEM library.
 *
 * The library assembles and applies the Galerkin matrix of the single-layer
 * boundary integral operators of the Bembel paper (Doelz, Harbrecht, Kurz,
 * Multerer, Schoeps, Wolf), App. B eq. (LS) Laplace and eq. (HS) Helmholtz,
 *   <S phi_j, phi_i> = int_Gamma int_Gamma G(x, y) phi_j(y) phi_i(x),
 * on the B-spline space S^2 of App. E lifted to the patches of App. D by the
 * 2-form Piola transform, with the far field compressed by interpolating the
 * kernel on the parameter domain (Sec. 2, embedded fast multipole / H^2) and
 * the near field integrated by Gauss rules and Duffy-type regularisation
 * (Sec. 2).  All compute runs in CUDA kernels on the current device; there is
 * no CPU fallback.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Return value: BEMBEL_OK (0) or one of the BEMBEL_E* codes below; on error
 *   bembel_last_error() returns a message (thread-local, valid until the next
 *   call on the same thread).  No C++ exception crosses this boundary.
 * - Handles (bembel_geom*, bembel_op*) are created and owned by the library;
 *   release them with the matching *_destroy call.  A handle may be used by one
 *   host thread at a time.
 * - Vector arguments named *_dev are caller-owned DEVICE pointers.  Block
 *   vectors are column-major n x nrhs (column r starts at r*n elements).
 *   Real operators (Laplace) use double; complex operators (Helmholtz) use
 *   interleaved complex double {re, im}, i.e. 2*n*nrhs doubles.
 * - Work is ordered on the stream given in bembel_opts.stream at assembly
 *   (NULL = legacy default stream).  bembel_matvec and bembel_eval return
 *   without synchronising; bembel_assemble, bembel_rhs and bembel_solve
 *   return after the stream has drained.
 * - Global dof numbering of S^2 on level L and degree d (n1 = 2^L + d):
 *   dof = patch * n1^2 + j2 * n1 + j1, with (j1, j2) the B-spline indices along
 *   the first and second patch parameter.
 */
#ifndef BEMBEL_H
#define BEMBEL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define BEMBEL_OK 0
#define BEMBEL_EINVAL 1        /* invalid argument or handle                   */
#define BEMBEL_ENOMEM 2        /* device or host allocation failed             */
#define BEMBEL_ECUDA 3         /* a CUDA call failed (message has the reason)  */
#define BEMBEL_ENOTCONV 4      /* GMRES reached max_iter; x holds its iterate  */
#define BEMBEL_ETIMEOUT 5      /* a bounded device wait (tensor-core MMA completion) expired;
                                  reported after a solve or by the next call on the operator */
#define BEMBEL_EUNSUPPORTED 6  /* valid request the library does not implement */

/* ---- enumerations ---------------------------------------------------------- */
enum bembel_geom_kind {
  BEMBEL_GEOM_SPHERE6 = 0,          /* unit sphere, 6 cube-face patches gamma = c/|c| */
  BEMBEL_GEOM_PERTURBED_SPHERE = 1, /* r(x) = 1 + amp * sum a_lm Y_lm(x), 1 <= l <= 4   */
  BEMBEL_GEOM_NURBS = 2             /* six rational B-spline patches (Sec. 4.1, App. C) */
};
enum bembel_op_kind {
  BEMBEL_LAPLACE_SL = 0,   /* App. B (LS): G = 1/(4 pi r)                 */
  BEMBEL_HELMHOLTZ_SL = 1, /* App. B (HS): G = exp(-i kappa r)/(4 pi r)    */
  BEMBEL_MAXWELL_SL = 2    /* App. B (MS): electric field integral equation on the S^1
                              space of App. E (see "EFIE" below)                 */
};
enum bembel_precision {
  BEMBEL_PREC_FP64 = 0,  /* everything in FP64                                       */
  BEMBEL_PREC_MIXED = 1  /* FP64 assembly and residuals; FP32 inner solves/matvecs    */
};
enum bembel_rhs_kind {
  BEMBEL_RHS_POINT_SOURCE = 0, /* g(x) = exp(-i kappa |x-x0|)/|x-x0| (kappa = 0: 1/|x-x0|); params: 3 per rhs */
  BEMBEL_RHS_PLANE_WAVE = 1,   /* g(x) = exp(-i kappa d.x); params: direction d, 3 per rhs */
  BEMBEL_RHS_EFIE_PLANE_WAVE = 2 /* EFIE only: E_inc(x) = pol exp(-i kappa d.x); params:
                                    direction d then polarisation pol, 6 per rhs;
                                    b_i = -int_Gamma E_inc . mu_i */
};
enum bembel_precond_kind {
  BEMBEL_PRECOND_NONE = 0,
  BEMBEL_PRECOND_BLOCK_JACOBI = 1, /* M^-1 = E^T D^-1 E, D = near-field diagonal leaf blocks */
  BEMBEL_PRECOND_LEARNED = 2,      /* M^-1 = E^T W D^-1 W E + P A_c^-1 P^T, W from
                                      bembel_learned_attach (W = I: TWO_LEVEL)              */
  BEMBEL_PRECOND_TWO_LEVEL = 3     /* M^-1 = E^T D^-1 E + P A_c^-1 P^T: block-Jacobi plus the
                                      coarse-space correction (opts.coarse_level)           */
};
#define BEMBEL_LEARNED_NPARAM 433  /* parameters of the learned preconditioner's network */

typedef struct bembel_geom bembel_geom;
typedef struct bembel_op bembel_op;
typedef struct bembel_learned_set bembel_learned_set;

/* Geometry description (App. D boundary representation; Sec. 4.1 allows
 * arbitrary smooth parametric patch maps).  Host memory; copied by
 * bembel_geom_create. */
typedef struct {
  int kind;              /* enum bembel_geom_kind                                    */
  int n_coeffs;          /* PERTURBED_SPHERE: number of a_lm, must be 24 (l = 1..4)  */
  const double* coeffs;  /* PERTURBED_SPHERE: a_lm ordered (l, m = -l..l), host ptr   */
  double amplitude;      /* PERTURBED_SPHERE: amp (0.1 in the perturbed workload)     */
  /* NURBS: gamma_P(s,t) = sum N_a(s) N_b(t) w_ab P_ab / sum N_a(s) N_b(t) w_ab with
   * B-splines N on open knot vectors over [0,1] (App. C).  Six patches in the
   * order and orientation of the cube-face sphere (patch 0 faces +x, 1 -x, 2 +y,
   * 3 -y, 4 +z, 5 -z; d_s gamma x d_t gamma outward), meeting at full edges with
   * matching parametrisations (App. D).  Host arrays, read during the call:    */
  int n_patches;          /* must be 6                                              */
  const int* degrees;     /* (p1, p2) per patch, 1 <= p <= 4                        */
  const int* n_ctrl;      /* (k1, k2) control points per direction per patch       */
  const double* knots;    /* per patch: k1 + p1 + 1 knots in s, then k2 + p2 + 1 in t */
  const double* ctrl;     /* per patch: k1 k2 points (x, y, z, w > 0), index i1 + k1 i2 */
} bembel_geom_desc;

/* Assembly options.  Fill with bembel_opts_default, then override. */
typedef struct {
  double eta;        /* admissibility max(diam) <= eta * dist of the cluster balls (1.6)   */
  int leaf_level;    /* quadtree leaf level; -1: max(0, level - 1)                           */
  int g_regular;     /* Gauss points per direction on separated near-field pairs (4)         */
  int g_singular;    /* Gauss points per variable of the Duffy rules (5)                     */
  int g_identical;   /* per-class overrides of g_singular for identical, common-edge and     */
  int g_edge;        /* common-vertex pairs; 0 = use g_singular (0)                          */
  int g_vertex;
  int bsr_chunk;     /* blocks per warp in the block-sparse products; 0 = 32                 */
  int tensor_cores;  /* MIXED, q = 4: coupling for 8..128 right-hand sides on tcgen05 (1)    */
  int precision;     /* enum bembel_precision (FP64)                                         */
  void* stream;      /* cudaStream_t used by every call on the operator (NULL: default)      */
  /* Per-variable Gauss orders of the Duffy rules, in the order of each rule's
   * variables: identical (xi, eta, u1, u2), common edge (xi, eta1, eta2, u),
   * common vertex (xi, eta1, eta2, eta3).  All four > 0 override the class's
   * single order; zeros keep it (default: zeros).  The rules must not depend on
   * which element of a pair comes first, which needs edge eta1 = eta2 and vertex
   * eta1 = eta2 = eta3 (EINVAL otherwise). */
  int g_identical_var[4];
  int g_edge_var[4];
  int g_vertex_var[4];
  /* Gauss points per direction on separated pairs beyond the ring next to the
   * touching pairs (no element holds a corner of both); g_regular then applies
   * to the ring only.  0 = g_regular (default 0). */
  int g_regular_far;
  /* Repetition r of every interior knot of the S^2 spline space (Sec. 4.3,
   * Discretization(geom, pde, P, knotRepetition, L)): smoothness C^(d-r) inside a
   * patch, d + 1 + (2^level - 1) r functions per direction, r = d + 1 gives
   * discontinuous piecewise polynomials.  1 <= r <= p + 1; 0 = 1 (default 1).
   * The EFIE, the learned preconditioner and bembel_assemble_batch take r = 1 only. */
  int knot_repetition;
  /* Helmholtz: a cluster pair is admissible only if also |kappa| max(diam) <= kdiam,
   * so that the oscillation of exp(-i kappa r) over a far block stays within what
   * q Chebyshev points resolve (diameters of the bounding balls; App. B eq. (HS)).
   * 0 = no such limit (default 0). */
  double kdiam;
  /* Coarse space of the two-level and learned preconditioners (not in the paper): the
   * S^2 space of the same degree on level coarse_level, nested in the operator's space
   * (App. E), with P its refinement (knot insertion) into the fine space and A_c its
   * Galerkin matrix, assembled densely on that level with the operator's quadrature
   * orders and inverted once on the device (6 (p + 2^coarse_level)^2 <= 8192 dofs,
   * EINVAL above).  1 <= coarse_level <= level; 0 = max(0, level - 3) (default 0).
   * S^2 operators with knot_repetition 1 only (EUNSUPPORTED otherwise). */
  int coarse_level;
  /* FP32 products with fewer than 8 real columns (MIXED operators): 0 evaluates the
   * far-field coupling on the fly from the FP32 cluster points (default), 1 streams
   * an FP32 copy of the stored coupling (made at the first FP32 product, outside graph
   * capture).  Wider products always use the stored copy or the tensor cores. */
  int far_fp32_stored;
} bembel_opts;

/* Counters describing an assembled operator (host struct). */
typedef struct {
  int64_t ndofs;            /* global S^2 dofs                                  */
  int64_t nlocal;           /* element-local dofs (elements * (d+1)^2)          */
  int64_t nelements;
  int64_t n_clusters;       /* clusters over all levels                         */
  int64_t n_far_blocks;     /* ordered admissible cluster pairs                 */
  int64_t n_near_blocks;    /* ordered non-admissible leaf cluster pairs        */
  int64_t n_pairs_regular;  /* unordered separated near element pairs           */
  int64_t n_pairs_identical;
  int64_t n_pairs_edge;
  int64_t n_pairs_vertex;
  int64_t near_bytes;       /* FP64 near-field storage                          */
  int64_t far_bytes;        /* FP64 coupling storage                            */
  int leaf_level;
  int q;
  int degree;
  int level;
  double assemble_ms;       /* device time of the assembly kernels               */
  double setup_ms;          /* host time of topology, trees and pair lists      */
  /* device time per assembly phase (CUDA events on the operator's stream):
   * 0 tabulation, 1 regular near field, 2 identical, 3 common edge,
   * 4 common vertex, 5 coupling, 6 FP32 copies, 7 the persistent multi-mesh
   * kernel (operators from bembel_assemble_batch: phases 0, 6 and 7 are the
   * whole batch's, 1-5 are zero) */
  double phase_ms[8];
  int64_t n_pairs_regular_far; /* separated pairs integrated at g_regular_far      */
  /* host wall time per set-up stage (part of setup_ms): 0 element corner ids, 1 cluster
   * balls + block tree, 2 near-field pair lists, 3 extraction, moments, transfers and
   * cluster points, 4 quadrature tables and the rest */
  double setup_phase_ms[5];
} bembel_op_info;

/* Solver options and report (Sec. 4.6: GMRES, restarted). */
typedef struct {
  double tol;         /* relative residual ||b - A x|| / ||b|| per column (1e-8) */
  int restart;        /* Krylov dimension m (30)                                  */
  int max_iter;       /* total Arnoldi steps per column (1000)                    */
  int precond;        /* enum bembel_precond_kind (NONE)                          */
  int refine;         /* MIXED operators: FP64 iterative refinement on/off (1)    */
} bembel_solve_opts;

typedef struct {
  int iterations;        /* Arnoldi steps of the slowest column (inner steps summed over refinement) */
  int refinements;       /* outer FP64 refinement steps (0 for FP64 solves)       */
  double rel_residual;   /* largest final relative residual over columns (FP64)   */
  double solve_ms;       /* host wall time of the call                            */
} bembel_solve_info;

/* Defaults: eta 1.6, leaf_level -1, g_regular 4, g_singular 5 (no per-class overrides),
 * bsr_chunk 32, tensor_cores 1, FP64, stream NULL. */
void bembel_opts_default(bembel_opts* o);
/* Result of bembel_autotune: chosen orders and the estimated errors at them. */
typedef struct {
  int g_regular, g_identical, g_edge, g_vertex;  /* Gauss points per variable               */
  int q;                                          /* interpolation points per direction      */
  int bsr_chunk;                                  /* fastest chunk of the block products     */
  double err_regular, err_identical, err_edge, err_vertex; /* max relative block error, sample */
  double err_far;                                 /* relative error of sampled far blocks    */
  double chunk_ms[5];                             /* FP64 matvec ms for chunks 8..128         */
  double tune_ms;                                 /* host wall time of the call              */
  int g_identical_var[4], g_edge_var[4], g_vertex_var[4]; /* chosen per-variable Duffy orders  */
  int g_regular_far;                              /* separated pairs beyond the ring          */
  double err_regular_far;
  int leaf_level;                                 /* chosen (or given) leaf level              */
  double leaf_score_ms[2];                        /* set-up + assembly + 100 products at leaf
                                                     L-1, L-2 (0: not tried, -1: did not fit) */
  int far_fp32_stored;                            /* chosen FP32 coupling storage (MIXED)      */
  double fp32_product_ms[2];                      /* FP32 product: on the fly, stored copy     */
} bembel_tune_report;

/* Defaults: tol 1e-8, restart 30, max_iter 1000, NONE, refine 1. */
void bembel_solve_opts_default(bembel_solve_opts* o);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* bembel_last_error(void);

/* Number of CUDA kernel launches issued by this library since it was loaded
 * (all threads).  Diagnostic counter for launch accounting; never fails. */
int64_t bembel_kernel_launches(void);

/* Create a geometry (App. D: patches with outward normals meeting at full
 * edges or vertices; the matching condition holds for both kinds by
 * construction).  desc and desc->coeffs are read during the call only.
 * Errors: EINVAL (NULL pointers, unknown kind, wrong n_coeffs, NURBS data that is
 * not 6 patches of degree 1..4 on open knot vectors with positive weights),
 * ENOMEM, ECUDA.  The geometry must outlive every operator assembled on it. */
int bembel_geom_create(const bembel_geom_desc* desc, bembel_geom** out);
int bembel_geom_destroy(bembel_geom* g);

/* EFIE (op = BEMBEL_MAXWELL_SL).  App. B (MS) with the kernel of (HS); the
 * Galerkin form moves the kappa^-2 gradient onto the test function:
 *   a(j, mu) = int int G(x,y) [ j(y) . mu(x) - kappa^-2 div j(y) div mu(x) ],
 * and the perfect-conductor condition n x (E_inc + E) = 0 of (MP) reads
 * a(j, mu) = -int E_inc . mu (BEMBEL_RHS_EFIE_PLANE_WAVE builds that right-hand
 * side).  Space: S^1 of App. E, p in [1, 3] (degree p across, p-1 along each
 * component), lifted by the div-conforming Piola transform, with the normal
 * component glued across patch edges.  Dofs per patch 2 (2^L+p)(2^L+p-1), minus
 * one per glued edge function: ndofs = 12 (2^L+p)(2^L+p-1) - 12 (2^L+p-1).
 * Global numbering: patches in order; inside a patch the first component
 * i1 + np j2 (i1 < np = 2^L+p, j2 < np-1), then the second component
 * np (np-1) + j1 + (np-1) i2; a function glued to one numbered earlier shares
 * its number, with sign -s_own s_partner (s = +1 on the sides s = 1, t = 1,
 * -1 on s = 0, t = 0).  The EFIE is available on the cube-face sphere, dense
 * (q = 0) or H^2-compressed (q > 0: the kernel times the Jacobian dot
 * products and G itself are interpolated per far block, the three moment
 * channels int phi^1 L_a, int phi^2 L_a, int div phi L_a run through the same
 * nested transfers; MIXED operators keep FP32 copies of the near field and of
 * the five coupling matrices for the inner solves, FP64 for the refinement);
 * bembel_eval returns the scattered field (MS) at the points,
 * 3 complex values per point (out: [rhs][point][3] interleaved complex).
 * bembel_autotune, bembel_assemble_batch and the learned preconditioner are
 * for the scalar operators only (EUNSUPPORTED). */

/* Assemble the compressed single-layer Galerkin matrix (Sec. 2, Sec. 4.5).
 *   op     enum bembel_op_kind; Laplace (LS) or Helmholtz (HS)
 *   k_re, k_im  complex wavenumber kappa (Sec. 4.2); ignored for Laplace
 *   level  refinement level L: 2^L x 2^L elements per patch (App. E)
 *   p      ansatz degree d of S^2 (d = 0: piecewise constants), 0 <= d <= 2
 *   q      interpolation points per direction per cluster; q = 0 assembles
 *          the matrix densely (no admissible blocks); 1 <= q <= 8 otherwise
 *   o      options (NULL: defaults); copied
 * Builds the element topology, cluster tree and block tree on the host, then
 * runs the tabulation, near-field (regular + singular) quadrature and
 * coupling kernels.  The geometry must outlive the operator.
 * Errors: EINVAL (bad sizes, 0 <= level <= 10 required, EFIE with k = 0 or
 * p = 0, leaf clusters whose moment matrix (nld x q^2 FP64, nld = 4^(level - leaf)
 * times the functions per element) exceeds 227 KiB), EUNSUPPORTED (the EFIE on
 * another geometry or with knot_repetition > 1), ENOMEM, ECUDA. */
int bembel_assemble(bembel_geom* g, int op, double k_re, double k_im, int level, int p, int q,
                    const bembel_opts* o, bembel_op** out);

/* One mesh of a batched assembly. */
typedef struct {
  bembel_geom* geom;  /* geometry of this mesh (must outlive the operator)   */
  double k_re, k_im;  /* wavenumber (Helmholtz; ignored for Laplace)          */
  int level;          /* refinement level L of this mesh                      */
} bembel_batch_item;

/* Assemble n operators that share op, p, q and the options (same quadrature
 * orders, eta, leaf rule, precision) but may differ in geometry, level and
 * wavenumber -- e.g. a family of meshes or a frequency sweep.  No counterpart
 * in the paper, which assembles one operator at a time: every operator is the
 * one bembel_assemble builds from the same arguments (bit-identical blocks).
 * The host set-up runs per mesh; then one tabulation launch, ONE persistent
 * launch that walks a global work list of (mesh, phase, pair or block range)
 * items over the near field and coupling of all meshes, and one FP32-copy
 * launch (MIXED).  out[0..n-1] receive independent handles (destroy each);
 * info.assemble_ms is the batch's device time and phase_ms 0 / 7 / 6 the
 * tabulation, persistent and copy launches.  items and out: host arrays of n.
 * On failure every out[i] is NULL and nothing is left allocated.
 * Errors: EINVAL (NULL, n outside [1, 64], bad item), EUNSUPPORTED (Maxwell),
 * ENOMEM, ECUDA. */
int bembel_assemble_batch(int op, int p, int q, const bembel_batch_item* items, int n, const bembel_opts* o,
                          bembel_op** out);
int bembel_op_destroy(bembel_op* op);

/* Choose quadrature orders, the interpolation order q and the block-product
 * chunk for an operator (the paper fixes none of them).  For each pair kind
 * (separated near pairs, identical, common edge, common vertex) a sample of the
 * kind's element pairs is integrated on the device at Gauss orders 2, 3, ...
 * against order 10; the first order with worst relative block difference
 * <= quad_tol is chosen.  q is the smallest in [2, q_max] for which sampled
 * leaf-level far blocks V K V^T (Sec. 2 interpolation) differ from a converged
 * Gauss integration by <= far_tol (relative Frobenius norm).  The chunk is the
 * fastest of 8..128 for the FP64 matvec.  inout (options used for the sampling
 * assembly: eta, leaf level, stream) receives g_regular, g_identical, g_edge,
 * g_vertex, g_singular and bsr_chunk; rep (may be NULL) receives the choices,
 * q and the error estimates.  When inout->leaf_level < 0 the leaf level is chosen
 * too: operators at the chosen orders and q with leaves on levels L-1 and L-2 are
 * assembled and scored by host set-up + assembly + 100 products (FP32 for MIXED
 * options, else FP64), and for MIXED options the FP32 product of the chosen layout is
 * timed with on-the-fly and stored FP32 coupling (inout->leaf_level and
 * inout->far_fp32_stored receive the choices).  Assembles and releases these
 * operators internally.
 * Errors: EINVAL, ENOMEM, ECUDA, EUNSUPPORTED. */
int bembel_autotune(bembel_geom* g, int op, double k_re, double k_im, int level, int p, double quad_tol,
                    double far_tol, int q_max, bembel_opts* inout, bembel_tune_report* rep);

/* Number of global dofs (rows = cols of the Galerkin matrix, Sec. 4.5 rows()/cols()). */
int bembel_ndofs(const bembel_op* op, int64_t* n);
/* Fill *info with the operator's counters. */
int bembel_op_info_get(const bembel_op* op, bembel_op_info* info);
/* Diagnostic read of one element-pair block of the near field as assembled:
 * int_e int_f G(gamma(s), gamma(t)) phi_k(s) phi_l(t) dt ds in the parameter
 * measure (App. B eq. (LS)/(HS) with the Piola lift of App. E), for the
 * element-local tensor Bernstein polynomials of degree p on e and f, index
 * k = k1 + (p+1) k2 with k1 along the patch's first parameter.  Elements are
 * named by (patch, i1, i2), 0 <= i1, i2 < 2^level.  out (host) receives the
 * (p+1)^2 x (p+1)^2 block row-major (k row, l column), interleaved complex for
 * Helmholtz.  Synchronises the operator's stream.  S^2 operators only.
 * Errors: EINVAL (NULL, element out of range, pair not in the near field),
 * EUNSUPPORTED (EFIE operator), ECUDA. */
int bembel_near_block(const bembel_op* op, int e_patch, int e_i1, int e_i2, int f_patch, int f_i1, int f_i2,
                      double* out);

/* y = A x for nrhs columns (Sec. 4.5 "H * x"): gather to element-local
 * coefficients, leaf moments, upward transfer, coupling, downward transfer,
 * near field, scatter.  x_dev, y_dev: device, column-major ndofs x nrhs, real
 * or interleaved complex per the operator; must not overlap.  Uses library
 * scratch owned by the operator (grown on demand, so the first call with a
 * larger nrhs allocates).  Precision: FP64 unless the operator is MIXED and
 * fp32 != 0, in which case x and y are FP32 (float / interleaved complex
 * float) and the FP32 copies of the near and coupling matrices are used.
 * Errors: EINVAL (NULL, nrhs < 1), ENOMEM, ECUDA. */
int bembel_matvec(const bembel_op* op, const void* x_dev, void* y_dev, int nrhs, int fp32);
/* Note: for MIXED operators with q = 4 and tensor_cores = 1, the FP32 product
 * with nrhs (x2 complex) real columns a multiple of 16 in [32, 256] (Laplace)
 * or [64, 256] (Helmholtz) evaluates the far-field coupling on the tensor cores
 * in bf16 with FP32 accumulation (relative error ~1e-3 of the far-field part);
 * other FP32 products use FP32 CUDA-core arithmetic. */

/* y = A x like bembel_matvec, but without allocating anything.  The paper has
 * no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc themselves or through us -- for example code whose device memory
 * is owned by its own pool allocator (a framework's caching allocator that has
 * reserved the free memory, so an outside cudaMalloc fails or fragments it),
 * code on a latency-critical path that cannot afford the device-wide
 * synchronisation cudaMalloc and cudaFree may imply, or code that must keep
 * this library to a fixed, known memory footprint.  The operator (made by
 * bembel_assemble) and the x and y buffers are still the caller's inputs and
 * outputs, exactly as for bembel_matvec.
 * Scratch: a fixed array of 8 MiB compiled into the library as device memory.
 * It is part of the library's matvec module, which the CUDA runtime may load
 * lazily; bembel_assemble and bembel_assemble_batch look the array's address up
 * on the current device, which loads the module there, so the memory is taken
 * at assembly and a later bembel_matvec_noalloc on that device loads and
 * allocates nothing.  A device keeps the array until the process exits.  A
 * product needs (2 * nlocal + 2 * n_clusters * q^2) * nrhs values (x2 for
 * complex operators, 8 bytes each in FP64, 4 in FP32; counts from
 * bembel_op_info_get); larger requests are rejected with BEMBEL_EINVAL and a
 * message giving the size needed -- use bembel_matvec for them.  The level-6,
 * degree-1, q = 4 Laplace operator needs 3.7 MB per right-hand side.
 * The address lookup (one cudaGetSymbolAddress per device, with that device
 * current) happens at the first assembly on the device and is cached; call
 * bembel_assemble before any stream capture.  Every call uses the same array and
 * leaves its contents behind; each call writes every scratch value before
 * reading it, so nothing carries over.  Calls that overlap on the GPU (on
 * different streams, from different threads, or from different operators)
 * race on the array and give wrong results: order them on one stream or
 * synchronise between them.
 * Arguments, layouts and the fp32 flag are those of bembel_matvec.  The
 * kernels are those of bembel_matvec with one exception: this call never
 * builds what wide FP32 products allocate on first use (the tensor-core
 * groups and tiles, the FP32 copy of the stored coupling), so a wide FP32
 * product on a MIXED operator uses them only after a bembel_matvec or
 * bembel_solve with as many columns has made them; before that it evaluates
 * the FP32 coupling on the fly on the CUDA cores (results then differ from
 * bembel_matvec's tensor-core product by the bf16 rounding, ~1e-3 of the far
 * field).
 * Errors: EINVAL (NULL, nrhs < 1, aliasing, scratch too small, fp32 on an FP64
 * operator), ECUDA. */
int bembel_matvec_noalloc(const bembel_op* op, const void* x_dev, void* y_dev, int nrhs, int fp32);

/* Diagnostic: one tcgen05.mma (M = 128, N = n, K = 16, bf16 operands in the
 * canonical K-major shared-memory layout used by the tensor-core coupling, FP32
 * accumulation in TMEM) on exactly representable data, compared with a host
 * product; *max_abs_err receives the largest difference (0 when the layout and
 * descriptors are right).  n: multiple of 16 in [16, 256].  n = 0 exercises the
 * time-out path of the bounded waits instead: one thread waits, with a short
 * poll limit, on an mbarrier that nothing signals; the call then returns
 * BEMBEL_ETIMEOUT (the expected outcome) with the device still usable.  The
 * paper has no counterpart.  Errors: EINVAL, ETIMEOUT (bounded wait expired),
 * ECUDA. */
int bembel_tc_selftest(int n, double* max_abs_err);

/* ---- learned preconditioner (not in the paper: the solver's own extension) ----
 * M_W^-1 = E^T W D^-1 W E with W = diag(exp(MLP(f_i))) over element-local dofs,
 * f_i 8 local features (basis position in the element, element position in its
 * leaf, patch/leaf boundary flags, log element distortion, |kappa| * element
 * size); MLP 8 -> 16 -> 16 -> 1 with tanh, parameters packed [W1 (16x8, row-
 * major), b1, W2 (16x16), b2, w3 (16), b3] (BEMBEL_LEARNED_NPARAM floats).
 * The coarse-space correction P A_c^-1 P^T of the two-level preconditioner is added
 * to it: M_W^-1 = E^T W D^-1 W E + P A_c^-1 P^T (opts.coarse_level).  Zero w3, b3
 * gives W = I, i.e. the two-level preconditioner.  Trained with the unsupervised
 * loss sum_s |M_W^-1 A z_s - z_s|^2 / |z_s|^2 on systems the solver generates. */

/* Training data of one operator: builds the block-Jacobi inverses and the coarse
 * correction, the dof features and nsamples pairs (z ~ N(0,1) seeded, y = A z by the
 * FP64 product, and the part z - P A_c^-1 P^T y that the weighted block-Jacobi term
 * is trained to reproduce), and keeps only those (the operator may be destroyed
 * afterwards).  1 <= nsamples <= 64. */
int bembel_learned_collect(bembel_op* op, int nsamples, uint64_t seed, bembel_learned_set** out);
int bembel_learned_set_destroy(bembel_learned_set* s);
/* Adam on the loss over all sets, one step per epoch (full batch); params (host,
 * BEMBEL_LEARNED_NPARAM floats) in/out; loss_history (host, epochs doubles, may
 * be NULL) receives the mean loss before each step.  Forward and backward run
 * in this library's kernels. */
int bembel_learned_train(bembel_learned_set* const* sets, int nsets, int epochs, double lr, float* params,
                         double* loss_history);
/* Evaluate the network on the operator's dofs and keep the weights for
 * bembel_solve with precond = BEMBEL_PRECOND_LEARNED. */
int bembel_learned_attach(bembel_op* op, const float* params);
/* Network evaluation on n feature rows (device, n x 8 FP32): weights to w_dev
 * (device, n); when gw_dev (device, n) is given, grad_host (host, NPARAM) gets
 * d/dparams of sum_i gw_i w_i.  For checking the kernels. */
int bembel_mlp_eval(const float* params, const float* feat_dev, int64_t n, const float* gw_dev, float* w_dev,
                    float* grad_host);

/* Load vectors b_i = int_Gamma g phi_i (Sec. 4.4) for nrhs data functions of
 * the given kind (enum bembel_rhs_kind), with params (host, 3 doubles per rhs).
 * b_dev: device, column-major ndofs x nrhs, FP64 (complex for Helmholtz).
 * Tensor Gauss with g points per direction on every element (g <= 10).
 * Errors: EINVAL, ECUDA. */
int bembel_rhs(const bembel_op* op, int kind, const double* params, int nrhs, int g, void* b_dev);

/* Solve A x = b for nrhs columns with restarted GMRES (Sec. 4.6), x0 = 0.
 * b_dev, x_dev: device FP64 (complex for Helmholtz), column-major.  MIXED
 * operators with refine = 1 run FP32 inner GMRES inside FP64 iterative
 * refinement (residual r = b - A x in FP64 each outer step).  info may be NULL.
 * Errors: EINVAL, ENOMEM, ECUDA, ENOTCONV (x holds the last iterate), EUNSUPPORTED
 * (a preconditioner the operator cannot take: block-Jacobi leaves whose [D | I] exceeds
 * 227 KiB, a coarse space with knot_repetition > 1). */
int bembel_solve(const bembel_op* op, const void* b_dev, void* x_dev, int nrhs, const bembel_solve_opts* so,
                 bembel_solve_info* info);

/* Apply the preconditioner M^-1 of kind precond (enum bembel_precond_kind; NONE
 * copies) to nrhs columns: y = M^-1 x, as the solver applies it.  x_dev, y_dev:
 * device, column-major ndofs x nrhs, FP64 (fp32 = 0) or FP32 (complex for
 * Helmholtz), not overlapping.  Builds the block-Jacobi inverses and the coarse
 * correction on first use (allocates); LEARNED needs bembel_learned_attach first.
 * Not in the paper (which solves without a preconditioner).  Synchronous on the
 * operator's stream.  Errors: EINVAL, EUNSUPPORTED (EFIE; coarse space with
 * knot_repetition > 1), ENOMEM, ECUDA. */
int bembel_precond_apply(const bembel_op* op, int precond, const void* x_dev, void* y_dev, int nrhs, int fp32);

/* Potential u(x) = sum_j rho_j int G(x, gamma(t)) phi_hat_j(t) dt (Sec. 4.7;
 * (LS)/(HS)) at npts points.  pts_dev: device, npts x 3 row-major FP64;
 * rho_dev: device ndofs x nrhs; out_dev: device npts x nrhs column-major
 * (complex for Helmholtz).  Tensor Gauss with g points per direction per
 * element (g <= 10); points should keep a distance of a few elements from Gamma.
 * EFIE operators: the scattered field E(x) of (MS) instead, out_dev holding
 * 3 complex values per point and column ([rhs][point][x, y, z] interleaved).
 * Errors: EINVAL, ECUDA. */
int bembel_eval(const bembel_op* op, const double* pts_dev, int64_t npts, const void* rho_dev, int nrhs, int g,
                void* out_dev);

/* The same potential through the cluster tree (Sec. 4.7 evaluated with the far-field
 * machinery of Sec. 2) for many points: a source cluster sigma that is admissible
 * for the point x, 2 r_sigma <= eta max(0, |x - c_sigma| - r_sigma) with the block
 * tree's bounding balls, contributes sum_b G(x, gamma(x_b)) rhohat_sigma[b] over
 * its q x q Chebyshev points x_b, rhohat_sigma[b] = sum_j rho_j int phi_hat_j L_b
 * (the operator's leaf moments and upward transfers); elements of non-admissible
 * leaf clusters take the g x g Gauss rule of bembel_eval; every other cluster is
 * split into its children, starting from the six patches.  Work per point grows
 * like the logarithm of the number of elements instead of linearly.  Arguments and
 * layouts as bembel_eval; eta > 0 (the operator's eta is a good choice).  Compressed
 * S^2 operators (q > 0) only.
 * Errors: EINVAL (NULL, sizes, eta <= 0, a point whose cluster frontier exceeds
 * 1024 clusters), EUNSUPPORTED (q = 0 or EFIE), ENOMEM, ECUDA. */
int bembel_eval_h2(const bembel_op* op, const double* pts_dev, int64_t npts, const void* rho_dev, int nrhs, int g,
                   double eta, void* out_dev);

/* Evaluation points on a sphere about the origin (Sec. 5, Util::makeSphereGrid):
 * n points on each of n circles of latitude, polar angles pi (i + 1/2) / n and
 * azimuths 2 pi j / n; point i n + j at out_host[3 (i n + j)].  out_host: host,
 * 3 n^2 doubles.  Errors: EINVAL (NULL, radius <= 0, n < 1 or n > 46340). */
int bembel_sphere_grid(double radius, int n, double* out_host);

#ifdef __cplusplus
}
#endif
#endif /* BEMBEL_H */
