// capi.cu - extern "C" entry points declared in include/bembel.h.
//
// Every entry point catches the library's internal errors and turns them into
// status codes plus a thread-local message; no exception crosses the ABI.
#include <algorithm>
#include <cmath>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <unordered_map>
#include <new>
#include <stdexcept>

#include "op.h"

namespace bembel {

namespace {
thread_local std::string g_last_error;

struct LibError : std::exception {
  int code;
  std::string msg;
  LibError(int c, std::string m) : code(c), msg(std::move(m)) {}
  const char* what() const noexcept override { return msg.c_str(); }
};

template <typename F>
int guarded(F&& f) {
  try {
    g_last_error.clear();
    return f();
  } catch (const LibError& e) {
    g_last_error = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return BEMBEL_ENOMEM;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return BEMBEL_EINVAL;
  }
}

void free_op(Op* o) {
  if (!o) return;
  void* ptrs[] = {o->d_far_ptr, o->d_balls, o->d_far_src, o->d_far_tgt, o->d_K,     o->d_K32,   o->d_near_ptr, o->d_near_col,
                  o->d_N,       o->d_N32,     o->d_V,       o->d_T,     o->d_V32,   o->d_T32,      o->d_ex,
                  o->d_Xq,      o->d_BW,      o->d_gauss,   o->d_Xq_far, o->d_Xq_far32, o->d_cen, o->d_BW_far32, o->d_BW_far, o->d_nodes_jac, o->d_dofmajor,   o->d_nodes, o->d_scratch, o->d_bj,
                  o->d_near_tgt, o->d_nodes32, o->d_bj32, o->d_diag_blk, o->d_leaf_ids, o->d_lw,
                  o->d_tc_gptr, o->d_tc_A, o->d_tc_B, o->d_tc_items, o->d_tc_gsrc, o->d_tc_gmask, o->d_tc_gfirst, o->d_tc_gcnt,
                  o->d_e_ptr, o->d_e_col, o->d_e_val, o->d_et_ptr, o->d_et_col, o->d_et_val,
                  o->d_R, o->d_rcol, o->d_rrow, o->d_cinv, o->d_cinv32, o->d_cbuf, o->d_evalY,
                  o->d_ccen, o->d_nodes_rel32, o->d_evalC, o->d_evalRel};
  for (void* p : ptrs) dev_free(p);
  for (auto* p : o->d_pairs) dev_free(p);
  if (o->h_tc_err) cudaFreeHost(o->h_tc_err);
  delete o;
}

double factorial(int n) {
  double r = 1.0;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}
}  // namespace

void fail(int code, const std::string& msg) { throw LibError(code, msg); }

void cuda_check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    const int code = (e == cudaErrorMemoryAllocation) ? BEMBEL_ENOMEM : BEMBEL_ECUDA;
    throw LibError(code, std::string(what) + ": " + cudaGetErrorString(e));
  }
}

static std::atomic<long long> g_launches{0};
static thread_local bool t_capturing = false;
static thread_local long long t_captured = 0;

void capture_begin(cudaStream_t s) {
  cuda_check(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
  t_capturing = true;
  t_captured = 0;
}

long long capture_end(cudaStream_t s, cudaGraph_t* g) {
  t_capturing = false;
  cuda_check(cudaStreamEndCapture(s, g), "cudaStreamEndCapture");
  return t_captured;
}

bool capturing() { return t_capturing; }

void note_graph_kernels(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void launched(const char* what) {
  if (t_capturing) {  // counted when the graph is replayed
    ++t_captured;
    cuda_check(cudaGetLastError(), what);
    return;
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cuda_check(cudaGetLastError(), what);
}

long long launches_total() { return g_launches.load(); }

// Device memory through a small caching allocator.  Operators allocate and release the same
// sizes every time one is assembled and destroyed, and cudaMalloc / cudaFree (which
// synchronises the device) cost milliseconds per operator.  Released blocks first wait in a
// per-device pending list (work in flight may still read them); when an allocation finds no
// idle block of its size class, one cudaDeviceSynchronize moves the pending blocks to the
// idle lists.  The cache holds at most kCacheCap bytes per device (beyond that, blocks are
// returned with cudaFree), and an allocation that fails releases every idle block and
// retries once.  Not used under graph capture (no synchronisation is allowed there).
namespace {
constexpr int kMaxDevices = 64;
constexpr size_t kCacheCap = size_t(32) << 30;

struct AllocCache {
  std::mutex mu;
  std::multimap<size_t, void*> idle[kMaxDevices];
  std::vector<void*> pending[kMaxDevices];
  std::unordered_map<void*, std::pair<size_t, int>> blocks;  // live or cached: size class, device
  size_t cached[kMaxDevices] = {};
};

AllocCache& alloc_cache() {
  static AllocCache* c = new AllocCache();  // never destroyed: usable until the process ends
  return *c;
}

size_t size_class(size_t b) {
  if (b <= (size_t(1) << 20)) return (b + 511) & ~size_t(511);
  const size_t g = size_t(2) << 20;
  return (b + g - 1) / g * g;
}

// idle and pending blocks of the device back to the driver (caller holds the lock)
void release_cached(AllocCache& c, int dev) {
  if (!c.pending[dev].empty()) cudaDeviceSynchronize();
  for (void* p : c.pending[dev]) {
    c.blocks.erase(p);
    cudaFree(p);
  }
  c.pending[dev].clear();
  for (auto& kv : c.idle[dev]) {
    c.blocks.erase(kv.second);
    cudaFree(kv.second);
  }
  c.idle[dev].clear();
  c.cached[dev] = 0;
}
}  // namespace

void* dev_alloc(size_t bytes) {
  if (bytes == 0) bytes = 16;
  const size_t rb = size_class(bytes);
  int dev = 0;
  cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) fail(BEMBEL_EINVAL, "device index outside the allocator's range");
  AllocCache& c = alloc_cache();
  std::lock_guard<std::mutex> lock(c.mu);
  auto it = c.idle[dev].find(rb);
  if (it == c.idle[dev].end() && !c.pending[dev].empty() && !capturing()) {
    cuda_check(cudaDeviceSynchronize(), "allocator synchronisation");
    for (void* p : c.pending[dev]) c.idle[dev].emplace(c.blocks[p].first, p);
    c.pending[dev].clear();
    it = c.idle[dev].find(rb);
  }
  if (it != c.idle[dev].end()) {
    void* p = it->second;
    c.idle[dev].erase(it);
    c.cached[dev] -= rb;
    return p;
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, rb);
  if (e != cudaSuccess && !capturing()) {
    cudaGetLastError();
    release_cached(c, dev);
    e = cudaMalloc(&p, rb);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw LibError(BEMBEL_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
  }
  c.blocks[p] = {rb, dev};
  return p;
}

void dev_free(void* p) {
  if (!p) return;
  AllocCache& c = alloc_cache();
  std::lock_guard<std::mutex> lock(c.mu);
  const auto it = c.blocks.find(p);
  if (it == c.blocks.end()) {  // not from dev_alloc
    cudaFree(p);
    return;
  }
  const size_t rb = it->second.first;
  const int dev = it->second.second;
  if (c.cached[dev] + rb > kCacheCap) {
    c.blocks.erase(it);
    cudaFree(p);
    return;
  }
  c.pending[dev].push_back(p);
  c.cached[dev] += rb;
}

}  // namespace bembel

using namespace bembel;

extern "C" {

void bembel_opts_default(bembel_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));  // every field not named below defaults to 0
  o->eta = 1.6;
  o->leaf_level = -1;
  o->g_regular = 4;
  o->g_singular = 5;
  o->g_identical = 0;
  o->g_edge = 0;
  o->g_vertex = 0;
  o->bsr_chunk = 0;
  o->tensor_cores = 1;
  o->precision = BEMBEL_PREC_FP64;
  o->stream = nullptr;
  o->knot_repetition = 1;
}

void bembel_solve_opts_default(bembel_solve_opts* o) {
  if (!o) return;
  o->tol = 1e-8;
  o->restart = 30;
  o->max_iter = 1000;
  o->precond = BEMBEL_PRECOND_NONE;
  o->refine = 1;
}

const char* bembel_last_error(void) { return g_last_error.c_str(); }

int64_t bembel_kernel_launches(void) { return launches_total(); }

int bembel_geom_create(const bembel_geom_desc* desc, bembel_geom** out) {
  return guarded([&] {
    if (!desc || !out) fail(BEMBEL_EINVAL, "geom_create: NULL argument");
    auto* g = new GeomHandle();
    std::memset(&g->g, 0, sizeof(Geom));
    if (desc->kind == BEMBEL_GEOM_SPHERE6) {
      g->g.kind = kSphere6;
    } else if (desc->kind == BEMBEL_GEOM_PERTURBED_SPHERE) {
      if (desc->n_coeffs != 24 || !desc->coeffs) {
        delete g;
        fail(BEMBEL_EINVAL, "geom_create: perturbed sphere needs 24 coefficients (l = 1..4)");
      }
      g->g.kind = kPerturbedSphere;
      for (int l = 1; l <= 4; ++l)
        for (int m = -l; m <= l; ++m) {
          const int idx = l * l - 1 + l + m;
          const int am = m < 0 ? -m : m;
          double nlm = std::sqrt((2 * l + 1) / (4 * M_PI) * factorial(l - am) / factorial(l + am));
          if (m != 0) nlm *= std::sqrt(2.0);
          g->g.w[idx] = desc->amplitude * desc->coeffs[idx] * nlm;
        }
    } else if (desc->kind == BEMBEL_GEOM_NURBS) {
      std::unique_ptr<GeomHandle> own(g);
      if (desc->n_patches != 6 || !desc->degrees || !desc->n_ctrl || !desc->knots || !desc->ctrl)
        fail(BEMBEL_EINVAL, "geom_create: NURBS needs 6 patches with degrees, control-net sizes, knots and points");
      std::vector<double>& buf = g->nurbs;
      buf.assign(6, 0.0);
      const double* kn = desc->knots;
      const double* cp = desc->ctrl;
      for (int P = 0; P < 6; ++P) {
        const int p1 = desc->degrees[2 * P], p2 = desc->degrees[2 * P + 1];
        const int k1 = desc->n_ctrl[2 * P], k2 = desc->n_ctrl[2 * P + 1];
        if (p1 < 1 || p2 < 1 || p1 > kMaxNurbsDeg || p2 > kMaxNurbsDeg || k1 < p1 + 1 || k2 < p2 + 1 || k1 > 4096 ||
            k2 > 4096)
          fail(BEMBEL_EINVAL, "geom_create: NURBS degrees must be in [1, 4] with at least degree + 1 points");
        buf[P] = double(buf.size());
        buf.insert(buf.end(), {double(p1), double(p2), double(k1), double(k2)});
        for (int dir = 0; dir < 2; ++dir) {
          const int p = dir ? p2 : p1, k = dir ? k2 : k1, n = k + p + 1;
          for (int i = 0; i < n; ++i) {
            if (i > 0 && kn[i] < kn[i - 1]) fail(BEMBEL_EINVAL, "geom_create: NURBS knots must not decrease");
            if ((i <= p && kn[i] != 0.0) || (i >= k && kn[i] != 1.0))
              fail(BEMBEL_EINVAL, "geom_create: NURBS knot vectors must be open on [0, 1]");
          }
          buf.insert(buf.end(), kn, kn + n);
          kn += n;
        }
        for (int i = 0; i < k1 * k2; ++i)
          if (!(cp[4 * i + 3] > 0.0)) fail(BEMBEL_EINVAL, "geom_create: NURBS weights must be positive");
        buf.insert(buf.end(), cp, cp + 4 * k1 * k2);
        cp += 4 * k1 * k2;
      }
      cuda_check(cudaMalloc(&g->nurbs_dev, sizeof(double) * buf.size()), "nurbs alloc");
      cuda_check(cudaMemcpy(g->nurbs_dev, buf.data(), sizeof(double) * buf.size(), cudaMemcpyHostToDevice),
                 "nurbs upload");
      g->g.kind = kNurbs;
      g->g.nurbs_host = buf.data();
      g->g.nurbs_dev = g->nurbs_dev;
      own.release();
    } else {
      delete g;
      fail(BEMBEL_EINVAL, "geom_create: unknown geometry kind");
    }
    *out = reinterpret_cast<bembel_geom*>(g);
    return BEMBEL_OK;
  });
}

int bembel_geom_destroy(bembel_geom* g) {
  delete reinterpret_cast<GeomHandle*>(g);
  return BEMBEL_OK;
}

namespace {
// Validated operator description (no device work yet).
Op* make_op(bembel_geom* g, int op, double k_re, double k_im, int level, int p, int q, const bembel_opts* o) {
  if (!g) fail(BEMBEL_EINVAL, "assemble: NULL geometry");
  if (op != BEMBEL_LAPLACE_SL && op != BEMBEL_HELMHOLTZ_SL && op != BEMBEL_MAXWELL_SL)
    fail(BEMBEL_EINVAL, "assemble: unknown operator");
  if (op == BEMBEL_MAXWELL_SL) {
    if (p < 1 || p > kMaxEfieDeg) fail(BEMBEL_EINVAL, "assemble: the EFIE needs the S^1 degree p in [1, 3]");
    if (reinterpret_cast<GeomHandle*>(g)->g.kind != BEMBEL_GEOM_SPHERE6)
      fail(BEMBEL_EUNSUPPORTED, "assemble: the EFIE is available on the cube-face sphere");
    if (k_re == 0.0 && k_im == 0.0) fail(BEMBEL_EINVAL, "assemble: the EFIE needs a nonzero wavenumber");
  }
  if (level < 0 || level > 10) fail(BEMBEL_EINVAL, "assemble: level must be in [0, 10]");
  if (op != BEMBEL_MAXWELL_SL && (p < 0 || p > kMaxDeg)) fail(BEMBEL_EINVAL, "assemble: degree p must be in [0, 2]");
  if (q < 0 || q > kMaxQ) fail(BEMBEL_EINVAL, "assemble: q must be in [0, 8]");
  bembel_opts opts;
  bembel_opts_default(&opts);
  if (o) opts = *o;
  if (opts.g_regular < 1 || opts.g_regular > kMaxG || opts.g_singular < 1 || opts.g_singular > kMaxG)
    fail(BEMBEL_EINVAL, "assemble: Gauss orders must be in [1, 10]");
  for (int gk : {opts.g_identical, opts.g_edge, opts.g_vertex})
    if (gk < 0 || gk > kMaxG) fail(BEMBEL_EINVAL, "assemble: per-class Gauss orders must be in [0, 10]");
  if (opts.precision != BEMBEL_PREC_FP64 && opts.precision != BEMBEL_PREC_MIXED)
    fail(BEMBEL_EINVAL, "assemble: unknown precision");
  if (q > 0 && !(opts.eta > 0)) fail(BEMBEL_EINVAL, "assemble: eta must be positive");
  if (!(opts.kdiam >= 0.0)) fail(BEMBEL_EINVAL, "assemble: kdiam must be >= 0");
  if (opts.bsr_chunk < 0 || opts.bsr_chunk > 4096) fail(BEMBEL_EINVAL, "assemble: bsr_chunk must be in [0, 4096]");
  const int leaf = opts.leaf_level < 0 ? (level > 0 ? level - 1 : 0) : opts.leaf_level;
  if (leaf > level) fail(BEMBEL_EINVAL, "assemble: leaf_level above level");
  const int rep = opts.knot_repetition == 0 ? 1 : opts.knot_repetition;
  if (rep < 1 || rep > p + 1) fail(BEMBEL_EINVAL, "assemble: knot_repetition must be in [1, p + 1]");
  if (rep > 1 && op == BEMBEL_MAXWELL_SL) fail(BEMBEL_EUNSUPPORTED, "assemble: the EFIE takes knot_repetition 1");
  {
    // the leaf transfer kernels hold a leaf's moment matrix (nld x q^2 FP64) in shared memory
    const int nloc = op == BEMBEL_MAXWELL_SL ? 2 * p * (p + 1) : (p + 1) * (p + 1);
    const int64_t side = int64_t(1) << (level - leaf);
    if (q > 0 && 8 * side * side * nloc * q * q > 227 * 1024)
      fail(BEMBEL_EINVAL, "assemble: leaf clusters too large for q (leaf moment matrix above 227 KiB)");
  }
  if (opts.coarse_level < 0 || opts.coarse_level > level)
    fail(BEMBEL_EINVAL, "assemble: coarse_level must be in [0, level]");
  if (opts.far_fp32_stored != 0 && opts.far_fp32_stored != 1)
    fail(BEMBEL_EINVAL, "assemble: far_fp32_stored must be 0 or 1");
  Op* res = new Op();
  res->rep = rep;
  res->geom = reinterpret_cast<GeomHandle*>(g)->g;
  res->op = op;
  res->efie = op == BEMBEL_MAXWELL_SL;
  res->cplx = op == BEMBEL_HELMHOLTZ_SL || res->efie;
  res->kre = res->cplx ? k_re : 0.0;
  res->kim = res->cplx ? k_im : 0.0;
  res->L = level;
  res->d = p;
  res->q = q;
  res->leaf = leaf;
  res->opts = opts;
  res->g_reg = opts.g_regular;
  if (opts.g_regular_far < 0 || opts.g_regular_far > kMaxG) fail(BEMBEL_EINVAL, "assemble: g_regular_far in [0, 10]");
  res->g_reg_far = opts.g_regular_far > 0 ? opts.g_regular_far : opts.g_regular;
  res->g_sing = opts.g_singular;
  res->g_kind[kIdentical] = opts.g_identical > 0 ? opts.g_identical : opts.g_singular;
  res->g_kind[kEdge] = opts.g_edge > 0 ? opts.g_edge : opts.g_singular;
  res->g_kind[kVertex] = opts.g_vertex > 0 ? opts.g_vertex : opts.g_singular;
  const int* var[4] = {nullptr, opts.g_identical_var, opts.g_edge_var, opts.g_vertex_var};
  for (int k = kRegular; k <= kVertex; ++k) {
    for (int v = 0; v < 4; ++v) res->g_var[k][v] = k == kRegular ? res->g_reg : res->g_kind[k];
    if (!var[k]) continue;
    int set = 0;
    for (int v = 0; v < 4; ++v) {
      if (var[k][v] < 0 || var[k][v] > kMaxG) fail(BEMBEL_EINVAL, "assemble: per-variable orders must be in [0, 10]");
      set += var[k][v] > 0;
    }
    if (set != 0 && set != 4) fail(BEMBEL_EINVAL, "assemble: give all four per-variable orders of a class or none");
    // the rule must not depend on which element of the pair comes first: exchanging
    // the elements swaps eta1 and eta2 of the edge rule and permutes all three eta
    // of the vertex rule, so those orders must be equal
    if (set == 4 && ((k == kEdge && var[k][1] != var[k][2]) ||
                     (k == kVertex && (var[k][1] != var[k][2] || var[k][2] != var[k][3]))))
      fail(BEMBEL_EINVAL, "assemble: per-variable Duffy orders must keep the rule symmetric (edge eta1 = eta2, "
                          "vertex eta1 = eta2 = eta3)");
    if (set == 4) {
      int mx = 0;
      for (int v = 0; v < 4; ++v) {
        res->g_var[k][v] = var[k][v];
        mx = std::max(mx, var[k][v]);
      }
      res->g_kind[k] = mx;
    }
  }
  res->stream = static_cast<cudaStream_t>(opts.stream);
  res->bsr_chunk = opts.bsr_chunk > 0 ? opts.bsr_chunk : 32;
  return res;
}

// host set-up of one operator, timed into info.setup_ms
void setup_op(Op& o) {
  const auto th0 = std::chrono::steady_clock::now();
  build_structure(o);
  o.info.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - th0).count();
}
}  // namespace

extern "C++" {
namespace bembel {
void destroy_op(Op* o) { free_op(o); }

// The dense operator (q = 0, FP64) of o's kernel, wavenumber, degree and quadrature
// orders on another level of the same geometry: the coarse Galerkin matrix of the
// two-level preconditioner.
Op* assemble_level(const Op& o, int level) {
  GeomHandle gh;
  gh.g = o.geom;  // shares the geometry's buffers; gh owns nothing
  bembel_opts opts = o.opts;
  opts.leaf_level = -1;
  opts.precision = BEMBEL_PREC_FP64;
  opts.coarse_level = 0;
  Op* c = make_op(reinterpret_cast<bembel_geom*>(&gh), o.op, o.kre, o.kim, level, o.d, 0, &opts);
  try {
    setup_op(*c);
    run_assembly_kernels(*c);
  } catch (...) {
    free_op(c);
    throw;
  }
  return c;
}
}  // namespace bembel
}

int bembel_assemble(bembel_geom* g, int op, double k_re, double k_im, int level, int p, int q, const bembel_opts* o,
                    bembel_op** out) {
  Op* res = nullptr;
  const int rc = guarded([&] {
    if (!g || !out) fail(BEMBEL_EINVAL, "assemble: NULL argument");
    res = make_op(g, op, k_re, k_im, level, p, q, o);
    int dev = 0;
    cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    cudaEvent_t e0, e1;
    cuda_check(cudaEventCreate(&e0), "event");
    cuda_check(cudaEventCreate(&e1), "event");
    setup_op(*res);
    noalloc_prepare();
    cuda_check(cudaEventRecord(e0, res->stream), "event record");
    run_assembly_kernels(*res);
    cuda_check(cudaEventRecord(e1, res->stream), "event record");
    cuda_check(cudaEventSynchronize(e1), "assembly sync");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    res->info.assemble_ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *out = reinterpret_cast<bembel_op*>(res);
    return BEMBEL_OK;
  });
  if (rc != BEMBEL_OK && res) {
    free_op(res);
    if (out) *out = nullptr;
  }
  return rc;
}

int bembel_assemble_batch(int op, int p, int q, const bembel_batch_item* items, int n, const bembel_opts* o,
                          bembel_op** out) {
  std::vector<Op*> ops;
  const int rc = guarded([&] {
    if (!items || !out) fail(BEMBEL_EINVAL, "assemble_batch: NULL argument");
    if (n < 1 || n > kMaxBatch) fail(BEMBEL_EINVAL, "assemble_batch: n must be in [1, 64]");
    for (int i = 0; i < n; ++i) out[i] = nullptr;
    if (op == BEMBEL_MAXWELL_SL) fail(BEMBEL_EUNSUPPORTED, "assemble_batch: single-layer scalar operators only");
    if (o && o->knot_repetition > 1) fail(BEMBEL_EUNSUPPORTED, "assemble_batch: knot_repetition 1 only");
    for (int i = 0; i < n; ++i) {
      if (!items[i].geom) fail(BEMBEL_EINVAL, "assemble_batch: NULL geometry in an item");
      ops.push_back(make_op(items[i].geom, op, items[i].k_re, items[i].k_im, items[i].level, p, q, o));
    }
    for (Op* r : ops) setup_op(*r);
    noalloc_prepare();
    cudaEvent_t e0, e1;
    cuda_check(cudaEventCreate(&e0), "event");
    cuda_check(cudaEventCreate(&e1), "event");
    cuda_check(cudaEventRecord(e0, ops[0]->stream), "event record");
    run_assembly_batch(ops);
    cuda_check(cudaEventRecord(e1, ops[0]->stream), "event record");
    cuda_check(cudaEventSynchronize(e1), "assembly sync");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int i = 0; i < n; ++i) {
      ops[i]->info.assemble_ms = ms;  // the whole batch's device time
      out[i] = reinterpret_cast<bembel_op*>(ops[i]);
    }
    return BEMBEL_OK;
  });
  if (rc != BEMBEL_OK) {
    for (Op* r : ops) free_op(r);
    if (out && items && n >= 1 && n <= kMaxBatch)
      for (int i = 0; i < n; ++i) out[i] = nullptr;
  }
  return rc;
}

int bembel_op_destroy(bembel_op* op) {
  Op* o = reinterpret_cast<Op*>(op);
  if (o) cudaStreamSynchronize(o->stream);
  free_op(o);
  return BEMBEL_OK;
}

int bembel_ndofs(const bembel_op* op, int64_t* n) {
  return guarded([&] {
    if (!op || !n) fail(BEMBEL_EINVAL, "ndofs: NULL argument");
    *n = reinterpret_cast<const Op*>(op)->ndofs;
    return BEMBEL_OK;
  });
}

int bembel_near_block(const bembel_op* op, int e_patch, int e_i1, int e_i2, int f_patch, int f_i1, int f_i2,
                      double* out) {
  return guarded([&] {
    if (!op || !out) fail(BEMBEL_EINVAL, "near_block: NULL argument");
    const Op* o = reinterpret_cast<const Op*>(op);
    if (o->efie) fail(BEMBEL_EUNSUPPORTED, "near_block: S^2 operators only");
    const int np = 6, nel = 1 << o->L;  // six patches (cube layout)
    auto elem = [&](int pa, int i1, int i2) -> int64_t {
      if (pa < 0 || pa >= np || i1 < 0 || i1 >= nel || i2 < 0 || i2 >= nel)
        fail(BEMBEL_EINVAL, "near_block: element out of range");
      return (int64_t)pa * nel * nel + morton_encode(uint32_t(i1), uint32_t(i2));
    };
    const int64_t ge = elem(e_patch, e_i1, e_i2), gf = elem(f_patch, f_i1, f_i2);
    const int shift = 2 * (o->L - o->leaf);
    const int64_t le = ge >> shift, lf = gf >> shift;
    const int64_t pe = ge - (le << shift), pf = gf - (lf << shift);
    cuda_check(cudaStreamSynchronize(o->stream), "near_block: sync");
    long long rng[2];
    cuda_check(cudaMemcpy(rng, o->d_near_ptr + le, sizeof(rng), cudaMemcpyDeviceToHost), "near_block: row range");
    std::vector<int> cols(size_t(rng[1] - rng[0]));
    if (!cols.empty())
      cuda_check(cudaMemcpy(cols.data(), o->d_near_col + rng[0], sizeof(int) * cols.size(), cudaMemcpyDeviceToHost),
                 "near_block: columns");
    const auto it = std::find(cols.begin(), cols.end(), int(lf));
    if (it == cols.end()) fail(BEMBEL_EINVAL, "near_block: the pair is not in the near field");
    const int64_t blk = rng[0] + (it - cols.begin());
    const int C = o->cplx ? 2 : 1;
    const size_t pitch = sizeof(double) * C * o->nld;
    const double* src = o->d_N + (size_t)blk * o->nld * o->nld * C + (size_t)(pe * o->nloc) * o->nld * C +
                        (size_t)(pf * o->nloc) * C;
    cuda_check(cudaMemcpy2D(out, sizeof(double) * C * o->nloc, src, pitch, sizeof(double) * C * o->nloc, o->nloc,
                            cudaMemcpyDeviceToHost),
               "near_block: copy");
    return BEMBEL_OK;
  });
}

int bembel_op_info_get(const bembel_op* op, bembel_op_info* info) {
  return guarded([&] {
    if (!op || !info) fail(BEMBEL_EINVAL, "op_info: NULL argument");
    *info = reinterpret_cast<const Op*>(op)->info;
    return BEMBEL_OK;
  });
}

int bembel_matvec(const bembel_op* op, const void* x_dev, void* y_dev, int nrhs, int fp32) {
  return guarded([&] {
    if (!op || !x_dev || !y_dev) fail(BEMBEL_EINVAL, "matvec: NULL argument");
    if (nrhs < 1) fail(BEMBEL_EINVAL, "matvec: nrhs must be >= 1");
    if (x_dev == y_dev) fail(BEMBEL_EINVAL, "matvec: x and y must not overlap");
    const Op* o = reinterpret_cast<const Op*>(op);
    tc_check(*o);
    matvec_device(*o, x_dev, y_dev, nrhs, fp32 != 0, o->stream);
    return BEMBEL_OK;
  });
}

int bembel_matvec_noalloc(const bembel_op* op, const void* x_dev, void* y_dev, int nrhs, int fp32) {
  return guarded([&] {
    if (!op || !x_dev || !y_dev) fail(BEMBEL_EINVAL, "matvec_noalloc: NULL argument");
    if (nrhs < 1) fail(BEMBEL_EINVAL, "matvec_noalloc: nrhs must be >= 1");
    if (x_dev == y_dev) fail(BEMBEL_EINVAL, "matvec_noalloc: x and y must not overlap");
    const Op* o = reinterpret_cast<const Op*>(op);
    tc_check(*o);
    matvec_noalloc(*o, x_dev, y_dev, nrhs, fp32 != 0, o->stream);
    return BEMBEL_OK;
  });
}

int bembel_autotune(bembel_geom* g, int op, double k_re, double k_im, int level, int p, double quad_tol,
                    double far_tol, int q_max, bembel_opts* inout, bembel_tune_report* rep) {
  return guarded([&] {
    if (op == BEMBEL_MAXWELL_SL) fail(BEMBEL_EUNSUPPORTED, "autotune: scalar operators only");
    return autotune_impl(g, op, k_re, k_im, level, p, quad_tol, far_tol, q_max, inout, rep);
  });
}

int bembel_learned_collect(bembel_op* op, int nsamples, uint64_t seed, bembel_learned_set** out) {
  return guarded([&] {
    if (!op || !out || nsamples < 1 || nsamples > 64) fail(BEMBEL_EINVAL, "learned_collect: bad argument");
    if (reinterpret_cast<Op*>(op)->efie) fail(BEMBEL_EUNSUPPORTED, "learned_collect: scalar operators only");
    *out = reinterpret_cast<bembel_learned_set*>(learned_collect(*reinterpret_cast<Op*>(op), nsamples, seed));
    return BEMBEL_OK;
  });
}

int bembel_learned_set_destroy(bembel_learned_set* s) {
  learned_set_free(reinterpret_cast<LearnedSet*>(s));
  return BEMBEL_OK;
}

int bembel_learned_train(bembel_learned_set* const* sets, int nsets, int epochs, double lr, float* params,
                         double* loss_history) {
  return guarded([&] {
    if (!sets || nsets < 1 || epochs < 1 || !params || !(lr > 0)) fail(BEMBEL_EINVAL, "learned_train: bad argument");
    for (int i = 0; i < nsets; ++i)
      if (!sets[i]) fail(BEMBEL_EINVAL, "learned_train: NULL set");
    learned_train(reinterpret_cast<LearnedSet* const*>(sets), nsets, epochs, lr, params, loss_history);
    return BEMBEL_OK;
  });
}

int bembel_learned_attach(bembel_op* op, const float* params) {
  return guarded([&] {
    if (!op || !params) fail(BEMBEL_EINVAL, "learned_attach: NULL argument");
    learned_attach(*reinterpret_cast<Op*>(op), params);
    return BEMBEL_OK;
  });
}

int bembel_mlp_eval(const float* params, const float* feat_dev, int64_t n, const float* gw_dev, float* w_dev,
                    float* grad_host) {
  return guarded([&] {
    if (!params || !feat_dev || !w_dev || n < 1) fail(BEMBEL_EINVAL, "mlp_eval: bad argument");
    mlp_eval_dev(params, feat_dev, n, gw_dev, w_dev, grad_host);
    return BEMBEL_OK;
  });
}

int bembel_tc_selftest(int n, double* max_abs_err) {
  return guarded([&] {
    if (!max_abs_err) fail(BEMBEL_EINVAL, "tc_selftest: NULL argument");
    if (n == 0) {  // the bounded-wait time-out path
      *max_abs_err = 0.0;
      if (tc_timeout_probe()) fail(BEMBEL_ETIMEOUT, "tc_selftest: the bounded wait on an unsignalled barrier ran out");
      return BEMBEL_OK;
    }
    *max_abs_err = tc_selftest(n);
    return BEMBEL_OK;
  });
}

int bembel_rhs(const bembel_op* op, int kind, const double* params, int nrhs, int g, void* b_dev) {
  return guarded([&] {
    if (!op || !params || !b_dev) fail(BEMBEL_EINVAL, "rhs: NULL argument");
    if (nrhs < 1) fail(BEMBEL_EINVAL, "rhs: nrhs must be >= 1");
    const Op* o = reinterpret_cast<const Op*>(op);
    if (o->efie ? kind != BEMBEL_RHS_EFIE_PLANE_WAVE
                : (kind != BEMBEL_RHS_POINT_SOURCE && kind != BEMBEL_RHS_PLANE_WAVE))
      fail(BEMBEL_EINVAL, "rhs: unknown kind for this operator");
    if (g < 1 || g > kMaxG) fail(BEMBEL_EINVAL, "rhs: g must be in [1, 10]");
    rhs_device(*o, kind, params, nrhs, g, b_dev);
    return BEMBEL_OK;
  });
}

int bembel_solve(const bembel_op* op, const void* b_dev, void* x_dev, int nrhs, const bembel_solve_opts* so,
                 bembel_solve_info* info) {
  return guarded([&] {
    if (!op || !b_dev || !x_dev) fail(BEMBEL_EINVAL, "solve: NULL argument");
    if (nrhs < 1) fail(BEMBEL_EINVAL, "solve: nrhs must be >= 1");
    bembel_solve_opts o;
    bembel_solve_opts_default(&o);
    if (so) o = *so;
    if (o.restart < 1 || o.restart > 200 || o.max_iter < 1 || !(o.tol > 0))
      fail(BEMBEL_EINVAL, "solve: restart in [1, 200], max_iter >= 1, tol > 0 required");
    if (o.precond != BEMBEL_PRECOND_NONE && o.precond != BEMBEL_PRECOND_BLOCK_JACOBI &&
        o.precond != BEMBEL_PRECOND_LEARNED && o.precond != BEMBEL_PRECOND_TWO_LEVEL)
      fail(BEMBEL_EINVAL, "solve: unknown preconditioner");
    tc_check(*reinterpret_cast<const Op*>(op));
    const int rc = solve_gmres(*reinterpret_cast<const Op*>(op), b_dev, x_dev, nrhs, o, info);
    tc_check(*reinterpret_cast<const Op*>(op));  // solve_gmres synchronised its stream
    if (rc == BEMBEL_ENOTCONV) g_last_error = "solve: GMRES reached max_iter before the tolerance";
    return rc;
  });
}

int bembel_precond_apply(const bembel_op* op, int precond, const void* x_dev, void* y_dev, int nrhs, int fp32) {
  return guarded([&] {
    if (!op || !x_dev || !y_dev) fail(BEMBEL_EINVAL, "precond_apply: NULL argument");
    if (nrhs < 1) fail(BEMBEL_EINVAL, "precond_apply: nrhs must be >= 1");
    if (x_dev == y_dev) fail(BEMBEL_EINVAL, "precond_apply: x and y must not overlap");
    if (precond < BEMBEL_PRECOND_NONE || precond > BEMBEL_PRECOND_TWO_LEVEL)
      fail(BEMBEL_EINVAL, "precond_apply: unknown preconditioner");
    Op& o = *const_cast<Op*>(reinterpret_cast<const Op*>(op));
    if (o.efie && precond != BEMBEL_PRECOND_NONE)
      fail(BEMBEL_EUNSUPPORTED, "precond_apply: S^2 operators only");
    const size_t el = fp32 ? sizeof(float) : sizeof(double);
    const size_t bytes = el * size_t(o.ndofs) * nrhs * (o.cplx ? 2 : 1);
    if (precond == BEMBEL_PRECOND_NONE) {
      cuda_check(cudaMemcpyAsync(y_dev, x_dev, bytes, cudaMemcpyDeviceToDevice, o.stream), "precond copy");
    } else {
      if (precond == BEMBEL_PRECOND_LEARNED && !o.d_lw)
        fail(BEMBEL_EINVAL, "precond_apply: the learned preconditioner needs bembel_learned_attach first");
      precond_setup(o);
      if (precond != BEMBEL_PRECOND_BLOCK_JACOBI) coarse_setup(o, nrhs);
      const int saved = o.active_precond;
      o.active_precond = precond;
      try {
        precond_apply(o, x_dev, y_dev, nrhs, fp32 != 0, o.stream);
      } catch (...) {
        o.active_precond = saved;
        throw;
      }
      o.active_precond = saved;
    }
    cuda_check(cudaStreamSynchronize(o.stream), "precond_apply sync");
    return BEMBEL_OK;
  });
}

int bembel_eval(const bembel_op* op, const double* pts_dev, int64_t npts, const void* rho_dev, int nrhs, int g,
                void* out_dev) {
  return guarded([&] {
    if (!op || !pts_dev || !rho_dev || !out_dev) fail(BEMBEL_EINVAL, "eval: NULL argument");
    if (npts < 1 || nrhs < 1) fail(BEMBEL_EINVAL, "eval: npts and nrhs must be >= 1");
    if (npts > (1LL << 31) - 1 || nrhs > 65535) fail(BEMBEL_EINVAL, "eval: npts or nrhs too large");
    if (g < 1 || g > kMaxG) fail(BEMBEL_EINVAL, "eval: g must be in [1, 10]");
    eval_device(*reinterpret_cast<const Op*>(op), pts_dev, npts, rho_dev, nrhs, g, out_dev);
    return BEMBEL_OK;
  });
}

int bembel_eval_h2(const bembel_op* op, const double* pts_dev, int64_t npts, const void* rho_dev, int nrhs, int g,
                   double eta, void* out_dev) {
  return guarded([&] {
    if (!op || !pts_dev || !rho_dev || !out_dev) fail(BEMBEL_EINVAL, "eval_h2: NULL argument");
    if (npts < 1 || nrhs < 1) fail(BEMBEL_EINVAL, "eval_h2: npts and nrhs must be >= 1");
    if (npts > (1LL << 31) - 1 || nrhs > 65535) fail(BEMBEL_EINVAL, "eval_h2: npts or nrhs too large");
    if (g < 1 || g > kMaxG) fail(BEMBEL_EINVAL, "eval_h2: g must be in [1, 10]");
    if (!(eta > 0.0)) fail(BEMBEL_EINVAL, "eval_h2: eta must be > 0");
    eval_h2_device(*reinterpret_cast<const Op*>(op), pts_dev, npts, rho_dev, nrhs, g, eta, out_dev);
    return BEMBEL_OK;
  });
}

int bembel_sphere_grid(double radius, int n, double* out_host) {
  return guarded([&] {
    if (!out_host) fail(BEMBEL_EINVAL, "sphere_grid: NULL argument");
    if (!(radius > 0.0) || n < 1 || n > 46340) fail(BEMBEL_EINVAL, "sphere_grid: radius > 0 and 1 <= n <= 46340");
    for (int i = 0; i < n; ++i) {
      const double th = M_PI * (i + 0.5) / n;
      for (int j = 0; j < n; ++j) {
        const double ph = 2.0 * M_PI * j / n;
        double* p = out_host + 3 * ((int64_t)i * n + j);
        p[0] = radius * std::sin(th) * std::cos(ph);
        p[1] = radius * std::sin(th) * std::sin(ph);
        p[2] = radius * std::cos(th);
      }
    }
    return BEMBEL_OK;
  });
}

}  // extern "C"
