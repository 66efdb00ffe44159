// op.h - internal operator state of the single-layer BEM library (host side).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/bembel.h"
#include "common.cuh"

namespace bembel {

// One element pair of the near field.  e < f, or e == f for identical pairs.
// code: bits 0-1 kind (0 regular, 1 identical, 2 edge, 3 vertex), bits 2-4
// canonical map of e, bits 5-7 canonical map of f (see apply_cmap).
// off1: offset of entry (row i of e, col j of f) = off1 + i * nld + j in the
// near-field storage (row-major blocks); off2 likewise for the mirrored block
// (row j of f, col i of e) = off2 + j * nld + i, or -1 when the pair is its own
// mirror.
struct PairRec {
  int e, f;
  int code, pad;
  long long off1, off2;
};

enum PairKind { kRegular = 0, kIdentical = 1, kEdge = 2, kVertex = 3 };

struct Op {
  Geom geom{};
  int op = 0;          // bembel_op_kind
  bool cplx = false;   // Helmholtz
  double kre = 0, kim = 0;
  int L = 0, d = 0, q = 0, leaf = 0;
  int rep = 1;         // knot repetition of the S^2 space; > 1: CSR extraction (d_e_*)
  int nloc = 1, n1 = 1, nel1 = 1, q2 = 0;
  int m = 1;           // elements per leaf side
  int nld = 1;         // local dofs per leaf cluster (m*m*nloc)
  int64_t nelem = 0, ndofs = 0, nlocal = 0, nleaf = 0;
  double h = 1.0;      // element side in the parameter square
  bembel_opts opts{};
  cudaStream_t stream = nullptr;

  // cluster tree (levels 0..leaf), global cluster id = lvl_off[l] + patch*4^l + morton
  std::vector<int64_t> lvl_off;
  int64_t nclusters = 0;
  double* d_balls = nullptr;  // compressed operators: (centre, radius) per cluster, 4 doubles

  // far field: CSR over target cluster ids
  int64_t nfar = 0;
  long long* d_far_ptr = nullptr;  // nclusters + 1
  int* d_far_src = nullptr;        // source cluster id per block
  int* d_far_tgt = nullptr;        // target cluster id per block
  double* d_K = nullptr;           // nfar * q2 * q2 (x2 complex), row-major: entry (a, b) at a*q2 + b
  float* d_K32 = nullptr;

  // near field: CSR over leaf clusters, blocks nld x nld, row-major: entry (i, j) at i*nld + j
  int64_t nnear = 0;
  long long* d_near_ptr = nullptr;  // nleaf + 1
  int* d_near_col = nullptr;
  int* d_near_tgt = nullptr;       // target leaf per block
  double* d_N = nullptr;
  float* d_N32 = nullptr;

  // element-pair lists by kind
  PairRec* d_pairs[4] = {nullptr, nullptr, nullptr, nullptr};
  int64_t npairs[4] = {0, 0, 0, 0};

  // geometry-independent matrices
  double* d_V = nullptr;   // nld x q2, entry (i, a) at i*q2 + a
  double* d_T = nullptr;   // 4 x q2 x q2, child c entry (a', a) at c*q2*q2 + a'*q2 + a
  float* d_V32 = nullptr;
  float* d_T32 = nullptr;
  double* d_ex = nullptr;  // 1-D Bezier extraction: (i*(d+1) + j)*(d+1) + k

  // quadrature tabulation (A1)
  int g_reg = 4, g_sing = 5;
  int g_kind[4] = {4, 5, 5, 5};  // Gauss points per variable per pair kind (largest of g_var)
  int g_var[4][4] = {};          // per-variable orders per pair kind (regular: g_reg x 4)
  int g_reg_far = 4;             // separated pairs beyond the ring next to the touching ones
  int gauss_off_far = 0;         // its [nodes][weights] in d_gauss
  int64_t npairs_regular_far = 0;
  double* d_Xq_far = nullptr;    // gamma at the far order's points
  float* d_Xq_far32 = nullptr;   // MIXED: the same as FP32 offsets (x, y, z, 0) from the element centre
  double* d_cen = nullptr;       // MIXED: element centres (x, y, z, 0) of those points
  float* d_BW_far32 = nullptr;   // MIXED: FP32 copy of d_BW_far
  double* d_nodes_jac = nullptr; // EFIE: d_s gamma, d_t gamma at the cluster points
  double* d_BW_far = nullptr;
  double* d_Xq = nullptr;  // nelem * g_reg^2 * 3
  double* d_BW = nullptr;  // g_reg^2 * nloc: w_p h^2 B_k(u_p)
  double* d_gauss = nullptr;  // [g_reg nodes] then per singular kind [nodes, weights]
  int gauss_off[4] = {0, 0, 0, 0};  // offset of each pair kind's [nodes][weights] table in d_gauss
  double* d_nodes = nullptr;  // nclusters * q2 * 3 cluster interpolation points
  float* d_nodes32 = nullptr; // FP32 copy (x, y, z, 0) per point for the on-the-fly FP32 coupling
  double* d_ccen = nullptr;     // MIXED: cluster centres (x, y, z), mean of the cluster's points
  float* d_nodes_rel32 = nullptr;  // MIXED: points as FP32 offsets (x, y, z, 0) from their centre

  // EFIE on the S^1 space, or S^2 with knot repetition > 1: extraction E (element-local
  // <- global, signed for S^1) as CSR and its transpose; set means "CSR mode"
  bool efie = false;
  int* d_e_ptr = nullptr;
  int* d_e_col = nullptr;
  double* d_e_val = nullptr;
  int* d_et_ptr = nullptr;
  int* d_et_col = nullptr;
  double* d_et_val = nullptr;

  // matvec scratch (grown on demand), FP64 and FP32 views share the bytes
  int bsr_chunk = 32;        // blocks per warp in the block-sparse products
  // tensor-core coupling for many right-hand sides (tc_coupling.cu)
  int* d_tc_gptr = nullptr;        // CSR over sibling-target groups
  int* d_tc_gsrc = nullptr;        // union of far sources per group
  unsigned* d_tc_gmask = nullptr;  // which group targets interact with the source
  int* d_tc_gfirst = nullptr;      // first target of the group
  int* d_tc_gcnt = nullptr;        // targets in the group
  int* d_tc_err = nullptr;         // device alias of h_tc_err
  int* h_tc_err = nullptr;         // host-mapped flag: set when a bounded MMA wait timed out
  int64_t tc_ngroups = 0, tc_nentries = 0;
  unsigned char* d_tc_A = nullptr;  // stored A tiles, 4 KB per group entry (bf16, canonical layout)
  unsigned char* d_tc_B = nullptr;  // packed source moments, nclusters x 256 columns x 32 B
  int* d_tc_items = nullptr;        // (group, first entry, end) runs of at most 128 entries
  int64_t tc_nitems = 0;
  void* d_scratch = nullptr;
  void* d_dofmajor = nullptr;  // dof-major staging of wide S^2 products (ndofs x ncol)
  size_t dofmajor_bytes = 0;
  size_t scratch_bytes = 0;

  // block-Jacobi preconditioner: inverses of the near-field diagonal blocks
  double* d_bj = nullptr;         // nleaf * nld * nld (x2 complex), leaf order, column-major blocks
  float* d_bj32 = nullptr;
  int* d_diag_blk = nullptr;      // near-field block index of the diagonal block of each leaf
  int* d_leaf_ids = nullptr;      // 0 .. nleaf-1 (target = source list of the block diagonal)
  float* d_lw = nullptr;          // learned weights per element-local dof (learned.cu)
  int active_precond = 0;         // preconditioner of the running solve (enum bembel_precond_kind)
  // two-level preconditioner: coarse S^2 space of level coarse_level (coarse.cu)
  int coarse_level = -1;          // level of the built coarse space (-1: not built)
  int n1c = 0;                    // coarse functions per direction
  int64_t ncoarse = 0;            // coarse dofs (6 n1c^2)
  double* d_R = nullptr;          // 1-D refinement matrix, n1 x n1c row-major
  int* d_rcol = nullptr;          // per fine row i: first and end nonzero column (2 n1)
  int* d_rrow = nullptr;          // per coarse column a: first and end nonzero row (2 n1c)
  double* d_cinv = nullptr;       // A_c^-1, ncoarse x ncoarse row-major (x2 complex)
  float* d_cinv32 = nullptr;
  void* d_cbuf = nullptr;         // coarse vectors: restriction and correction (2 x ncoarse x ncol)
  double* d_evalY = nullptr;      // potential evaluation: quadrature points of every element (rhs_eval.cu)
  int evalG = 0;                  // their Gauss order
  double* d_evalC = nullptr;      // MIXED: element centres of those points
  float* d_evalRel = nullptr;     // MIXED: the points as FP32 offsets (x, y, z, 0) from the centres
  size_t cbuf_bytes = 0;

  bembel_op_info info{};
};

struct GeomHandle {
  Geom g;
  std::vector<double> nurbs;  // host copy of the NURBS buffer (g.nurbs_host points here)
  double* nurbs_dev = nullptr;
  ~GeomHandle() {
    if (nurbs_dev) cudaFree(nurbs_dev);
  }
};

// setup.cu
void build_structure(Op& o);            // topology, trees, pairs, moments (host) + uploads
void gauss01(int n, std::vector<double>& x, std::vector<double>& w);  // Gauss-Legendre on [0,1]
double chebyshev01(int q, int a);
double lagrange01(int q, int a, double x);
double bernstein_h(int d, int k, double u);
// quad.cu: max over a sample of pairs of |B_g - B_ref|_F / |B_ref|_F for one pair kind
double sample_pair_error(Op& o, int kind, const int g[4], int g_ref, int max_pairs, std::vector<double>* ref_cache,
                         int cls = -1);
// autotune.cu
int autotune_impl(bembel_geom* g, int op, double k_re, double k_im, int level, int p, double quad_tol,
                  double far_tol, int q_max, bembel_opts* inout, bembel_tune_report* rep);
// quad.cu
void run_assembly_kernels(Op& o);       // tabulation, near field, coupling
void alloc_assembly_outputs(Op& o);     // Xq, near field, coupling, FP32 near copy
// MIXED: FP32 points (offsets from element centres) and weights of the far separated order
void points_f32(Op& o, cudaStream_t s);
void coupling_f32(Op& o, cudaStream_t s);  // MIXED: d_K32 = float(d_K)
// MIXED S^2: the FP32 coupling copy that wide FP32 products stream, made on first use
// (never under graph capture)
void coupling_f32_prepare(Op& o, int nrhs);
// several operators sharing (op, degree, q, options): tabulation, one
// persistent launch for all near-field pairs and coupling blocks, FP32 copies
void run_assembly_batch(const std::vector<Op*>& ops);
// efie.cu: S^1 element-pair quadrature (phases 1-4 with events ev[2..5]),
// local load vectors of plane waves, and the scattered field at points
void efie_pair_kernels(Op& o, cudaEvent_t* ev);
void efie_coupling_assemble(Op& o);  // compressed EFIE: 5 coupling matrices per far block
void efie_coupling_apply(const Op& o, const double* xh, double* yh, int nrhs, cudaStream_t s);
void efie_coupling_apply(const Op& o, const float* xh, float* yh, int nrhs, cudaStream_t s);  // MIXED
void efie_rhs_local(const Op& o, const double* gx, const double* gw, int G, const double* prm_dev, int nrhs,
                    double* bl, cudaStream_t s);
void efie_field(const Op& o, const double* rl, const double* gx, const double* gw, int G, const double* pts,
                int64_t npts, int nrhs, double* out, cudaStream_t s);
// h2mv.cu
void matvec_device(const Op& o, const void* x, void* y, int nrhs, bool fp32, cudaStream_t s);
void ensure_scratch(Op& o, size_t bytes);
void ensure_dofmajor(Op& o, size_t bytes);
size_t matvec_scratch_bytes(const Op& o, int nrhs, bool fp32);
// same product with the fixed file-scope scratch of h2mv.cu; allocates nothing
void matvec_noalloc(const Op& o, const void* x, void* y, int nrhs, bool fp32, cudaStream_t s);
size_t matvec_noalloc_limit();
void noalloc_prepare();
// y = E^T D^-1 E x (block-Jacobi), uses the matvec scratch
void precond_apply(const Op& o, const void* x, void* y, int nrhs, bool fp32, cudaStream_t s);
// element-local helpers (h2mv.cu): gather E x, scatter E^T y, block-diagonal D^-1 x_loc
void local_gather(const Op& o, const void* x, void* xl, int nrhs, bool fp32, cudaStream_t s);
void local_scatter(const Op& o, const void* yl, void* y, int nrhs, bool fp32, cudaStream_t s);
void blockdiag_apply(const Op& o, const void* Dinv, const void* xl, void* yl, int nrhs, bool fp32, cudaStream_t s);
// tc_coupling.cu
bool tc_coupling_usable(const Op& o, int nrhs);  // groups built and the product wide enough
bool tc_coupling_wanted(const Op& o, int nrhs);  // operator and width qualify
void tc_prepare(Op& o, int nrhs);                // build the groups if wanted (never under capture)
void tc_coupling(const Op& o, const float* xh, float* yh, int nrhs, cudaStream_t s);
void tc_build_groups(Op& o, const std::vector<long long>& fptr, const std::vector<int>& fsrc);
double tc_selftest(int N);
bool tc_timeout_probe();  // true when the bounded wait on an unsignalled mbarrier ran out
// fails with BEMBEL_ETIMEOUT if an earlier tensor-core product on o timed out
void tc_check(const Op& o);
// precond.cu
void precond_setup(Op& o);
// coarse.cu: coarse correction P A_c^-1 P^T of the two-level and learned preconditioners
void coarse_setup(Op& o, int nrhs);
void coarse_apply_add(const Op& o, const void* x, void* y, int nrhs, bool fp32, cudaStream_t s);
// capi.cu: the dense operator of the same kernel, degree and quadrature on another level
Op* assemble_level(const Op& o, int level);
void destroy_op(Op* o);
// learned.cu
struct LearnedSet;
LearnedSet* learned_collect(Op& src, int ns, unsigned long long seed);
void learned_train(LearnedSet* const* sets, int nsets, int epochs, double lr, float* params, double* hist);
void learned_attach(Op& o, const float* params);
void learned_scale_local(const Op& o, void* yl, int nrhs, bool fp32, cudaStream_t s);
void mlp_eval_dev(const float* params_host, const float* F, int64_t n, const float* gw, float* W, float* grad_host);
void learned_set_free(LearnedSet* s);
// element-local layout: dof-major, nrhs (x2 complex) real columns contiguous
void gather_to_local(const Op& o, const double* x, double* xl, int nrhs, cudaStream_t s);
void scatter_to_global(const Op& o, const double* yl, double* y, int nrhs, cudaStream_t s);
// solve.cu
int solve_gmres(const Op& o, const void* b, void* x, int nrhs, const bembel_solve_opts& so, bembel_solve_info* info);
void rhs_device(const Op& o, int kind, const double* params, int nrhs, int g, void* b);
void eval_device(const Op& o, const double* pts, int64_t npts, const void* rho, int nrhs, int g, void* out);
// compressed evaluation (S^2 operators with q > 0): far clusters by their interpolated moments
void eval_h2_device(const Op& o, const double* pts, int64_t npts, const void* rho, int nrhs, int g, double eta,
                    void* out);
// h2mv.cu: cluster moments of a global vector x (FP64): gather + leaf moments + upward
// transfers; xl (nlocal x ncol) and xh (nclusters x q2 x ncol) are caller-provided
void cluster_moments(const Op& o, const double* x, double* xl, double* xh, int nrhs, cudaStream_t s);

// error plumbing (capi.cu)
struct Error {
  int code;
  std::string msg;
};
[[noreturn]] void fail(int code, const std::string& msg);
void cuda_check(cudaError_t e, const char* what);
// check the launch that was just issued and count it
void launched(const char* what);
// stream capture of a CUDA graph on this thread; capture_end returns the
// number of kernels captured (launch accounting adds them per replay)
void capture_begin(cudaStream_t s);
long long capture_end(cudaStream_t s, cudaGraph_t* g);
void note_graph_kernels(long long n);
// true between capture_begin and capture_end on this thread
bool capturing();
void* dev_alloc(size_t bytes);
void dev_free(void* p);
// scoped device allocation
struct DevBuf {
  void* p = nullptr;
  explicit DevBuf(size_t bytes) { p = dev_alloc(bytes); }
  ~DevBuf() { dev_free(p); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
};

}  // namespace bembel
