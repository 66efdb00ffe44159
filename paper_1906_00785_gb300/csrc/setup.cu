// setup.cu - host-side structure of the compressed single-layer operator.
//
// * Element topology (App. D): elements touch iff they share physical corner
//   points; the shared corners select the Duffy rule (identical / common edge /
//   common vertex) and the canonical map of each element (Sec. 2, [SS97]).
// * Cluster tree and block tree (Sec. 2, embedded FMM / H^2 on the parameter
//   domain): per-patch quadtrees in Morton order; cluster balls with centre
//   gamma(midpoint) and radius max |gamma - centre| over a 9 x 9 grid of the
//   cluster square; a pair is admissible when max(diam) <= eta * dist.
// * Geometry-independent matrices: with the 2-form Piola lift of S^2 (App. E)
//   the leaf moments V[i,a] = int phi_hat_i L_a ds and the child-to-parent
//   transfers T_c[a',a] = L_a^parent(x_a'^child) are the same for every cluster.
// * Bezier extraction of the uniform open-knot B-splines of App. C onto the
//   element-local Bernstein basis.
#include <algorithm>
#include <array>
#include <map>
#include <cstring>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "op.h"

namespace bembel {

// Gauss-Legendre rule on [0,1] by Newton iteration on P_n.
void gauss01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) {
        p0 = 1.0;
        p1 = z;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    if (n == 1) {
      p0 = 1.0;
      p1 = z;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[n - 1 - i] = 0.5 * (1.0 - z);
    w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

double chebyshev01(int q, int a) { return 0.5 * (1.0 + std::cos((2 * a + 1) * M_PI / (2.0 * q))); }

double lagrange01(int q, int a, double x) {
  double r = 1.0;
  const double xa = chebyshev01(q, a);
  for (int b = 0; b < q; ++b)
    if (b != a) r *= (x - chebyshev01(q, b)) / (xa - chebyshev01(q, b));
  return r;
}

double bernstein_h(int d, int k, double u) {
  double c = 1.0;
  for (int i = 0; i < k; ++i) c = c * (d - i) / (i + 1);
  return c * std::pow(u, k) * std::pow(1.0 - u, d - k);
}

namespace {

// Cox-de Boor on the open knot vector of degree d with n_el uniform elements and
// every interior knot repeated rep times; value of B-spline j at x in [0,1]
// (x = 1 belongs to the last interval).
double bspline_h(int d, int n_el, int j, double x, int rep = 1) {
  const int nk = 2 * (d + 1) + (n_el - 1) * rep;
  std::vector<double> kn(nk);
  for (int i = 0; i < nk; ++i) {
    const int t = i - (d + 1);  // interior knot number t / rep + 1
    kn[i] = t < 0 ? 0.0 : (t >= (n_el - 1) * rep ? 1.0 : double(t / rep + 1) / n_el);
  }
  std::vector<double> b(nk - 1, 0.0);
  int last = 0;
  for (int i = 0; i < nk - 1; ++i)
    if (kn[i] < kn[i + 1]) last = i;
  for (int i = 0; i < nk - 1; ++i) b[i] = (kn[i] < kn[i + 1] && x >= kn[i] && x < kn[i + 1]) ? 1.0 : 0.0;
  if (x >= 1.0) {
    std::fill(b.begin(), b.end(), 0.0);
    b[last] = 1.0;
  }
  for (int p = 1; p <= d; ++p)
    for (int i = 0; i < nk - 1 - p; ++i) {
      const double d1 = kn[i + p] - kn[i], d2 = kn[i + p + 1] - kn[i + 1];
      const double t1 = d1 > 0 ? (x - kn[i]) / d1 * b[i] : 0.0;
      const double t2 = d2 > 0 ? (kn[i + p + 1] - x) / d2 * b[i + 1] : 0.0;
      b[i] = t1 + t2;
    }
  return b[j];
}

// Small dense solve (Gaussian elimination with partial pivoting), n <= 3.
void solve_small(int n, std::vector<double> A, std::vector<double>& x) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * (n + 1) + c]) > std::fabs(A[piv * (n + 1) + c])) piv = r;
    for (int k = 0; k <= n; ++k) std::swap(A[c * (n + 1) + k], A[piv * (n + 1) + k]);
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = A[r * (n + 1) + c] / A[c * (n + 1) + c];
      for (int k = c; k <= n; ++k) A[r * (n + 1) + k] -= f * A[c * (n + 1) + k];
    }
  }
  x.resize(n);
  for (int r = 0; r < n; ++r) x[r] = A[r * (n + 1) + n] / A[r * (n + 1) + r];
}

template <typename T>
T* upload(const std::vector<T>& v) {
  if (v.empty()) return nullptr;
  T* p = static_cast<T*>(dev_alloc(v.size() * sizeof(T)));
  cuda_check(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), "upload");
  return p;
}

// 1-D Bezier extraction of the open-knot B-splines of degree deg with nel1
// uniform elements and interior knots repeated rep times: B-spline (rep i + j)
// restricted to element i equals sum_k ex[(i (deg+1) + j) (deg+1) + k]
// Bern_k((x - x_i) nel1), found by interpolation at deg + 1 interior points of
// the element.
std::vector<double> extraction_1d(int deg, int nel1, int rep = 1) {
  const int n = deg + 1;
  std::vector<double> ex((size_t)nel1 * n * n);
  std::vector<double> A(n * (n + 1)), sol;
  for (int i = 0; i < nel1; ++i)
    for (int j = 0; j < n; ++j) {
      for (int r = 0; r < n; ++r) {
        const double u = (r + 0.5) / n;
        for (int k = 0; k < n; ++k) A[r * (n + 1) + k] = bernstein_h(deg, k, u);
        A[r * (n + 1) + n] = bspline_h(deg, nel1, rep * i + j, (i + u) / nel1, rep);
      }
      solve_small(n, A, sol);
      for (int k = 0; k < n; ++k) ex[((size_t)i * n + j) * n + k] = sol[k];
    }
  return ex;
}

// Leaf moments of the S^1 functions for the three EFIE channels (geometry
// independent): V[ch][i][a], ch 0: int phi_hat^1 L_a, 1: int phi_hat^2 L_a,
// 2: int div phi_hat L_a over the element, in patch parameters (measure h^2,
// d/ds = (1/h) d/du), i = (element in leaf, Morton) * nloc + local function.
void efie_moments(Op& o, const std::vector<double>& gx, const std::vector<double>& gw) {
  const int p = o.d, q = o.q, q2 = o.q2, m = o.m, nloc = o.nloc, nld = o.nld;
  auto bern_d = [](int deg, int k, double u) {  // d/du of the Bernstein polynomial
    if (deg == 0) return 0.0;
    const double lo = k >= 1 ? bernstein_h(deg - 1, k - 1, u) : 0.0;
    const double hi = k <= deg - 1 ? bernstein_h(deg - 1, k, u) : 0.0;
    return deg * (lo - hi);
  };
  // 1-D moments per element position me inside the leaf: degree p values,
  // degree p - 1 values, degree p derivatives
  std::vector<double> Mp((size_t)m * (p + 1) * q), Mq((size_t)m * p * q), Dp((size_t)m * (p + 1) * q);
  for (int me = 0; me < m; ++me)
    for (int a = 0; a < q; ++a) {
      for (int k = 0; k <= p; ++k) {
        double v = 0.0, dv = 0.0;
        for (size_t g = 0; g < gx.size(); ++g) {
          const double la = lagrange01(q, a, (me + gx[g]) / m);
          v += gw[g] * bernstein_h(p, k, gx[g]) * la;
          dv += gw[g] * bern_d(p, k, gx[g]) * la;
        }
        Mp[((size_t)me * (p + 1) + k) * q + a] = v;
        Dp[((size_t)me * (p + 1) + k) * q + a] = dv;
      }
      for (int k = 0; k < p; ++k) {
        double v = 0.0;
        for (size_t g = 0; g < gx.size(); ++g) v += gw[g] * bernstein_h(p - 1, k, gx[g]) * lagrange01(q, a, (me + gx[g]) / m);
        Mq[((size_t)me * p + k) * q + a] = v;
      }
    }
  const double h = o.h;
  std::vector<double> V((size_t)3 * nld * q2, 0.0);
  for (int pe = 0; pe < m * m; ++pe) {
    uint32_t e1, e2;
    morton_decode(pe, e1, e2);
    for (int k = 0; k < nloc; ++k) {
      const bool first = k < (p + 1) * p;
      const int kk = first ? k : k - (p + 1) * p;
      const int k1 = first ? kk % (p + 1) : kk % p, k2 = first ? kk / (p + 1) : kk / p;
      const int i = pe * nloc + k;
      for (int a2 = 0; a2 < q; ++a2)
        for (int a1 = 0; a1 < q; ++a1) {
          const int a = a1 + q * a2;
          if (first) {  // degree p in s, p - 1 in t
            const double ms = Mp[((size_t)e1 * (p + 1) + k1) * q + a1], mt = Mq[((size_t)e2 * p + k2) * q + a2];
            V[((size_t)0 * nld + i) * q2 + a] = h * h * ms * mt;
            V[((size_t)2 * nld + i) * q2 + a] = h * Dp[((size_t)e1 * (p + 1) + k1) * q + a1] * mt;
          } else {      // degree p - 1 in s, p in t
            const double ms = Mq[((size_t)e1 * p + k1) * q + a1], mt = Mp[((size_t)e2 * (p + 1) + k2) * q + a2];
            V[((size_t)1 * nld + i) * q2 + a] = h * h * ms * mt;
            V[((size_t)2 * nld + i) * q2 + a] = h * ms * Dp[((size_t)e2 * (p + 1) + k2) * q + a2];
          }
        }
    }
  }
  o.d_V = upload(V);
  o.d_V32 = upload(std::vector<float>(V.begin(), V.end()));
}

// S^1 space of App. E on the six patches: global numbering with the edge glue
// (normal continuity) and the signed extraction E (element-local Bernstein
// functions <- global dofs) as CSR, plus its transpose.
//  patch-local index: first component i1 + np j2 (i1 < np, j2 < nq), then
//  second component np nq + j1 + nq i2 (j1 < nq, i2 < np), np = 2^L + p, nq = np - 1;
//  global numbers follow patches and patch-local indices in order; an edge
//  function whose partner on the neighbouring patch already has a number takes
//  it with coefficient -sign_own * sign_partner (sign +1 on the sides s = 1,
//  t = 1 and -1 on s = 0, t = 0: equal and opposite outward fluxes);
//  element-local functions: first component k1 + (p+1) k2 (k1 <= p, k2 < p),
//  second p (p+1) + k1 + p k2 (k1 < p, k2 <= p).
void build_s1_space(Op& o) {
  const int p = o.d, nel1 = o.nel1;
  const int np = nel1 + p, nq = nel1 + p - 1;
  const int per_patch = 2 * np * nq;
  auto c1 = [&](int i1, int j2) { return i1 + np * j2; };
  auto c2 = [&](int j1, int i2) { return np * nq + j1 + nq * i2; };
  // sides: 0 s=0, 1 s=1, 2 t=0, 3 t=1; edge functions along the side and the flux sign
  auto side_fun = [&](int sd, std::vector<int>& f) {
    f.clear();
    for (int j = 0; j < nq; ++j)
      f.push_back(sd < 2 ? c1(sd == 0 ? 0 : np - 1, j) : c2(j, sd == 2 ? 0 : np - 1));
    return (sd == 1 || sd == 3) ? 1 : -1;
  };
  using Key = std::array<long long, 3>;
  auto key_of = [&](int patch, double s0, double t0) {
    double x[3];
    gamma_eval(o.geom, patch, s0, t0, x);
    return Key{llround(x[0] * 1e9), llround(x[1] * 1e9), llround(x[2] * 1e9)};
  };
  const double ends[4][4] = {{0, 0, 0, 1}, {1, 0, 1, 1}, {0, 0, 1, 0}, {0, 1, 1, 1}};
  std::map<std::pair<Key, Key>, std::vector<std::array<int, 3>>> sides;  // (min key, max key) -> (patch, side, forward)
  for (int P = 0; P < 6; ++P)
    for (int sd = 0; sd < 4; ++sd) {
      const Key a = key_of(P, ends[sd][0], ends[sd][1]), b = key_of(P, ends[sd][2], ends[sd][3]);
      const bool fwd = a < b;
      sides[fwd ? std::make_pair(a, b) : std::make_pair(b, a)].push_back({P, sd, fwd ? 1 : 0});
    }
  // partner of each edge function: (patch, local) -> (patch', local', coefficient)
  std::vector<std::array<int, 3>> partner((size_t)6 * per_patch, {-1, -1, 0});
  std::vector<int> fa, fb;
  for (auto& kv : sides) {
    if (kv.second.size() != 2) fail(BEMBEL_EINVAL, "S^1 space: every patch edge must be shared by two patches");
    const auto A = kv.second[0], B = kv.second[1];
    const int sa = side_fun(A[1], fa), sb = side_fun(B[1], fb);
    if (A[2] != B[2]) std::reverse(fb.begin(), fb.end());
    for (int j = 0; j < nq; ++j) {
      partner[(size_t)A[0] * per_patch + fa[j]] = {B[0], fb[j], -sa * sb};
      partner[(size_t)B[0] * per_patch + fb[j]] = {A[0], fa[j], -sa * sb};
    }
  }
  std::vector<long long> gid((size_t)6 * per_patch, -1);
  std::vector<double> gco((size_t)6 * per_patch, 0.0);
  long long n = 0;
  for (int P = 0; P < 6; ++P)
    for (int l = 0; l < per_patch; ++l) {
      const size_t at = (size_t)P * per_patch + l;
      if (gid[at] >= 0) continue;
      gid[at] = n;
      gco[at] = 1.0;
      const auto& pr = partner[at];
      if (pr[0] >= 0) {
        const size_t bt = (size_t)pr[0] * per_patch + pr[1];
        gid[bt] = n;
        gco[bt] = pr[2];
      }
      ++n;
    }
  o.ndofs = n;
  // extraction rows per element-local function
  const std::vector<double> exp_ = extraction_1d(p, nel1), exq = extraction_1d(p - 1, nel1);
  const int n1p = p + 1, n1q = p;
  const int64_t per = int64_t(nel1) * nel1;
  std::vector<int> rptr(o.nlocal + 1, 0), rcol;
  std::vector<double> rval;
  rcol.reserve(o.nlocal * n1p * n1q);
  rval.reserve(o.nlocal * n1p * n1q);
  for (int64_t e = 0; e < o.nelem; ++e) {
    const int P = int(e / per);
    uint32_t i1, i2;
    morton_decode(uint32_t(e % per), i1, i2);
    for (int k = 0; k < o.nloc; ++k) {
      const bool first = k < n1p * n1q;
      const int kk = first ? k : k - n1p * n1q;
      const int k1 = first ? kk % n1p : kk % n1q, k2 = first ? kk / n1p : kk / n1q;
      // first: degree p in s (n1p functions), p-1 in t; second: the reverse
      const int na = first ? n1p : n1q, nb = first ? n1q : n1p;
      const std::vector<double>& ea = first ? exp_ : exq;
      const std::vector<double>& eb = first ? exq : exp_;
      for (int b = 0; b < nb; ++b) {
        const double cb = eb[((size_t)i2 * nb + b) * nb + k2];
        if (cb == 0.0) continue;
        for (int a = 0; a < na; ++a) {
          const double ca = ea[((size_t)i1 * na + a) * na + k1];
          if (ca == 0.0) continue;
          const int loc = first ? c1(int(i1) + a, int(i2) + b) : c2(int(i1) + a, int(i2) + b);
          const size_t at = (size_t)P * per_patch + loc;
          rcol.push_back(int(gid[at]));
          rval.push_back(ca * cb * gco[at]);
        }
      }
      rptr[e * o.nloc + k + 1] = int(rcol.size());
    }
  }
  // transpose
  std::vector<int> tptr(n + 1, 0), tcol(rcol.size());
  std::vector<double> tval(rcol.size());
  for (int c : rcol) ++tptr[c + 1];
  for (long long g = 0; g < n; ++g) tptr[g + 1] += tptr[g];
  {
    std::vector<int> fill(tptr.begin(), tptr.end() - 1);
    for (int64_t r = 0; r < o.nlocal; ++r)
      for (int k = rptr[r]; k < rptr[r + 1]; ++k) {
        const int at = fill[rcol[k]]++;
        tcol[at] = int(r);
        tval[at] = rval[k];
      }
  }
  o.d_e_ptr = upload(rptr);
  o.d_e_col = upload(rcol);
  o.d_e_val = upload(rval);
  o.d_et_ptr = upload(tptr);
  o.d_et_col = upload(tcol);
  o.d_et_val = upload(tval);
}

struct Ball {
  double c[3];
  double r;
};

struct LevelTable {
  long long off[16];  // first cluster id of each level, then the total
};

// Bounding ball of each cluster: centre gamma(square midpoint), radius the
// largest distance to gamma on a 9 x 9 grid of the cluster square (corners
// included).  Output: (c0, c1, c2, r) per cluster.
__global__ void k_cluster_balls(Geom g, LevelTable lt, int64_t n, double* __restrict__ out) {
  const int64_t gc = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gc >= n) return;
  int l = 0;
  while (gc >= lt.off[l + 1]) ++l;
  const int64_t nper = int64_t(1) << (2 * l);
  const int64_t c = gc - lt.off[l];
  const double H = ldexp(1.0, -l);
  const int patch = int(c / nper);
  uint32_t j1, j2;
  morton_decode(uint32_t(c % nper), j1, j2);
  double ctr[3];
  gamma_eval(g, patch, (j1 + 0.5) * H, (j2 + 0.5) * H, ctr);
  double r = 0.0;
  for (int k2 = 0; k2 <= 8; ++k2)
    for (int k1 = 0; k1 <= 8; ++k1) {
      double x[3];
      gamma_eval(g, patch, (j1 + k1 / 8.0) * H, (j2 + k2 / 8.0) * H, x);
      const double dx = x[0] - ctr[0], dy = x[1] - ctr[1], dz = x[2] - ctr[2];
      r = fmax(r, sqrt(dx * dx + dy * dy + dz * dz));
    }
  out[gc * 4 + 0] = ctr[0];
  out[gc * 4 + 1] = ctr[1];
  out[gc * 4 + 2] = ctr[2];
  out[gc * 4 + 3] = r;
}

struct KeyHash {
  size_t operator()(const std::array<long long, 3>& k) const {
    return std::hash<long long>()(k[0] * 73856093LL ^ k[1] * 19349663LL ^ k[2] * 83492791LL);
  }
};

int num_threads(int64_t n) {
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  return int(std::max<int64_t>(1, std::min<int64_t>({(int64_t)hw, (int64_t)16, (n + 255) / 256})));
}

// Persistent host workers for the set-up loops (created on first use, kept for the process):
// creating a team of threads per loop cost more than the loops themselves.  One caller at a
// time uses the pool; a concurrent caller runs its ranges on its own thread.
class HostPool {
 public:
  static HostPool& get() {
    static HostPool pool;
    return pool;
  }
  // fn(t) for every t in [0, nth), taken one at a time by the workers and the caller
  void run(int nth, const std::function<void(int)>& fn) {
    std::unique_lock<std::mutex> busy(use_, std::try_to_lock);
    if (!busy.owns_lock() || nth <= 1 || workers_.empty()) {
      for (int t = 0; t < nth; ++t) fn(t);
      return;
    }
    {
      std::lock_guard<std::mutex> lk(m_);
      job_ = &fn;
      njob_ = nth;
      next_ = 0;
      left_ = nth;
    }
    cv_.notify_all();
    for (;;) {
      int t;
      {
        std::lock_guard<std::mutex> lk(m_);
        if (next_ >= njob_) break;
        t = next_++;
      }
      fn(t);
      std::lock_guard<std::mutex> lk(m_);
      if (--left_ == 0) done_.notify_all();
    }
    std::unique_lock<std::mutex> lk(m_);
    done_.wait(lk, [&] { return left_ == 0; });
    job_ = nullptr;
  }

 private:
  HostPool() {
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int n = int(std::min(15u, hw > 1 ? hw - 1 : 0u));
    for (int i = 0; i < n; ++i) workers_.emplace_back([this] { loop(); });
  }
  ~HostPool() {
    {
      std::lock_guard<std::mutex> lk(m_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& w : workers_) w.join();
  }
  void loop() {
    for (;;) {
      std::unique_lock<std::mutex> lk(m_);
      cv_.wait(lk, [&] { return stop_ || next_ < njob_; });
      if (stop_) return;
      const int t = next_++;
      const std::function<void(int)>* f = job_;
      lk.unlock();
      (*f)(t);
      lk.lock();
      if (--left_ == 0) done_.notify_all();
    }
  }
  std::vector<std::thread> workers_;
  std::mutex use_, m_;
  std::condition_variable cv_, done_;
  const std::function<void(int)>* job_ = nullptr;
  int njob_ = 0, next_ = 0, left_ = 0;
  bool stop_ = false;
};

// Run fn(thread, begin, end) on nth contiguous ranges of [0, n).
template <typename F>
void parallel_for_t(int64_t n, int nth, F fn) {
  if (nth <= 1) {
    fn(0, 0, n);
    return;
  }
  const std::function<void(int)> task = [&](int t) { fn(t, n * t / nth, n * (t + 1) / nth); };
  HostPool::get().run(nth, task);
}

template <typename F>
void parallel_for(int64_t n, F fn) {
  parallel_for_t(n, num_threads(n), [&](int, int64_t a, int64_t b) { fn(a, b); });
}

// Element pairs of the near field: thread per (near block, element slot) with
// target <= source (and pe <= pf on diagonal blocks).  Shared physical corners
// give the pair kind and the canonical map of each element (see apply_cmap):
// common edge: A, B = the two shared corners in the first element's corner
// order, D2 runs A -> B; common vertex: A = the shared corner, D1 along the
// first local axis.  Pass 0 counts per kind, pass 1 writes the records.
// ---- block tree on the device ------------------------------------------------------
// Level by level: the candidate sources of a target on level l are the children of the
// non-admissible sources of its parent (the six patches on level 0), visited in
// increasing order, so both lists come out sorted by target and source without a sort.
// Pass 0 counts far (admissible) and near (non-admissible) candidates per target, an
// exclusive scan turns counts into offsets, pass 1 writes the lists.
struct TreeParams {
  double eta, kdiam, kabs;  // kdiam > 0: Helmholtz limit |kappa| max(diam) <= kdiam
  int compress;             // q > 0: admissibility tested (else every pair is near)
};

// The same arithmetic as the reference order of operations, without contraction, so that
// borderline decisions do not depend on the compiler's FMA choices.
__device__ __forceinline__ bool tree_admissible(const Ball* __restrict__ balls, int t, int sc, const TreeParams& p) {
  if (!p.compress) return false;
  const Ball bt = balls[t], bs = balls[sc];
  const double dx = __dsub_rn(bt.c[0], bs.c[0]), dy = __dsub_rn(bt.c[1], bs.c[1]), dz = __dsub_rn(bt.c[2], bs.c[2]);
  const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  const double dist = fmax(0.0, __dsub_rn(__dsub_rn(__dsqrt_rn(d2), bt.r), bs.r));
  const double diam = __dmul_rn(2.0, fmax(bt.r, bs.r));
  if (p.kdiam > 0.0 && __dmul_rn(p.kabs, diam) > p.kdiam) return false;
  return diam <= __dmul_rn(p.eta, dist);
}

// One thread per target of level l (local index i, global id t0 + i).  pptr / pcol: CSR of the
// parent level's non-admissible sources (global ids).  Pass 0: cf[i], cn[i] = counts.  Pass 1:
// cf, cn hold exclusive offsets; far sources go to fout[cf[i]...], near ones to nout[cn[i]...].
__global__ void k_tree_level(int pass, int l, int64_t t0, int64_t nt, long long off_l, long long off_lm1,
                             const long long* __restrict__ pptr, const int* __restrict__ pcol,
                             const Ball* __restrict__ balls, TreeParams prm, long long* __restrict__ cf,
                             long long* __restrict__ cn, int* __restrict__ fout, int* __restrict__ nout) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nt) return;
  const int t = int(t0 + i);
  long long nf = 0, nn = 0;
  long long fo = pass ? cf[i] : 0, no = pass ? cn[i] : 0;
  auto visit = [&](int sc) {
    if (tree_admissible(balls, t, sc, prm)) {
      if (pass) fout[fo + nf] = sc;
      ++nf;
    } else {
      if (pass) nout[no + nn] = sc;
      ++nn;
    }
  };
  if (l == 0) {
    for (int p = 0; p < 6; ++p) visit(p);
  } else {
    const int64_t par = i >> 2;
    for (long long k = pptr[par]; k < pptr[par + 1]; ++k) {
      const long long sl = pcol[k] - off_lm1;
      for (int c = 0; c < 4; ++c) visit(int(off_l + 4 * sl + c));
    }
  }
  if (!pass) {
    cf[i] = nf;
    cn[i] = nn;
  }
}

// Exclusive scan of n counts in place for two arrays at once (blockIdx.y picks the array),
// in blocks of 1024: per-block scan + block totals, then one block per array scans the
// totals (sequentially over chunks of 1024) and writes the sum to a[n] and tot[y], then the
// offsets are added.  a0 / a1 hold n + 1 entries; bsum holds 2 x nbmax.
__global__ void k_scan_block(long long* __restrict__ a0, long long* __restrict__ a1, int64_t n,
                             long long* __restrict__ bsum, int64_t nbmax) {
  __shared__ long long sh[1024];
  long long* a = blockIdx.y ? a1 : a0;
  const int64_t i = blockIdx.x * 1024ll + threadIdx.x;
  const long long v = i < n ? a[i] : 0;
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const long long u = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += u;
    __syncthreads();
  }
  if (i < n) a[i] = sh[threadIdx.x] - v;  // exclusive
  if (threadIdx.x == 1023) bsum[blockIdx.y * nbmax + blockIdx.x] = sh[1023];
}

__global__ void k_scan_sums(long long* __restrict__ a0, long long* __restrict__ a1, int64_t n,
                            long long* __restrict__ bsum, int64_t nb, int64_t nbmax, long long* __restrict__ tot) {
  __shared__ long long sh[1024];
  __shared__ long long carry;
  long long* bs = bsum + blockIdx.x * nbmax;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t c0 = 0; c0 < nb; c0 += 1024) {
    const int64_t i = c0 + threadIdx.x;
    const long long v = i < nb ? bs[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const long long u = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += u;
      __syncthreads();
    }
    if (i < nb) bs[i] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += sh[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    (blockIdx.x ? a1 : a0)[n] = carry;
    tot[blockIdx.x] = carry;
  }
}

__global__ void k_scan_add(long long* __restrict__ a0, long long* __restrict__ a1, int64_t n,
                           const long long* __restrict__ bsum, int64_t nbmax) {
  long long* a = blockIdx.y ? a1 : a0;
  const int64_t i = blockIdx.x * 1024ll + threadIdx.x;
  if (i < n) a[i] += bsum[blockIdx.y * nbmax + blockIdx.x];
}

// fptr[t0 + i] = base + off[i]: the level's far offsets into the global CSR over clusters
__global__ void k_tree_fptr(long long* __restrict__ fptr, int64_t t0, int64_t nt, const long long* __restrict__ off,
                            long long base) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < nt) fptr[t0 + i] = base + off[i];
}

// target of every far entry (thread per cluster)
__global__ void k_tree_tgt(const long long* __restrict__ fptr, int64_t nclusters, int* __restrict__ tgt) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nclusters) return;
  for (long long k = fptr[c]; k < fptr[c + 1]; ++k) tgt[k] = int(c);
}

// leaf rows of the near field: leaf-local source ids, the diagonal block, the row of each
// block and the identity list of the block-diagonal products; err when a row lacks its
// diagonal block
__global__ void k_tree_rows(const long long* __restrict__ nptr, int* __restrict__ ncol, long long leaf_off,
                            int64_t nleaf, int* __restrict__ diag, int* __restrict__ ids, int* __restrict__ ntgt,
                            int* __restrict__ err) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nleaf) return;
  ids[t] = int(t);
  int dg = -1;
  for (long long k = nptr[t]; k < nptr[t + 1]; ++k) {
    const int c = int(ncol[k] - leaf_off);
    ncol[k] = c;
    ntgt[k] = int(t);
    if (c == t) dg = int(k);
  }
  diag[t] = dg;
  if (dg < 0) atomicExch(err, 1);
}

// Warp-aggregated slot of counter ctr[key]: one atomic per distinct key in the warp.
// Every lane of the warp calls it (active = false lanes take no slot).
__device__ __forceinline__ unsigned long long agg_slot(unsigned long long* ctr, int key, bool active) {
  const unsigned mask = __ballot_sync(0xffffffffu, active);
  if (!active) return 0ull;
  const unsigned same = __match_any_sync(mask, key);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(same) - 1;
  unsigned long long base = 0ull;
  if (lane == leader) base = atomicAdd(ctr + key, (unsigned long long)__popc(same));
  base = __shfl_sync(same, base, leader);
  return base + __popc(same & ((1u << lane) - 1u));
}

__global__ void k_build_pairs(const long long* __restrict__ nptr, const int* __restrict__ ncol,
                              const int* __restrict__ ntgt, int64_t nnear, const int* __restrict__ cid, int m2,
                              int nloc, int nld, int pass, unsigned long long* __restrict__ cnt, PairRec* out0,
                              PairRec* out1, PairRec* out2, PairRec* out3, const int* __restrict__ v2e) {
  // grid-stride over (near block, element pair) items; whole warps stay in the loop so that
  // the slot counters can be taken warp-aggregated
  const int64_t total = nnear * (int64_t)m2 * m2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < total; base += stride) {
    const int64_t id = base + threadIdx.x;
    bool valid = id < total;
    int64_t blk = 0, e = 0, f = 0;
    int pe = 0, pf = 0, t = 0, sc = 0;
    if (valid) {
      blk = id / ((int64_t)m2 * m2);
      const int slot = int(id % ((int64_t)m2 * m2));
      pe = slot / m2;
      pf = slot % m2;
      t = ntgt[blk];
      sc = ncol[blk];
      valid = !(t > sc || (t == sc && pf < pe));
      e = (int64_t)t * m2 + pe;
      f = (int64_t)sc * m2 + pf;
    }
    int kind = kRegular, me = 0, mf = 0;
    if (valid) {
      int se[4], sf[4], ns = 0;
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
          if (cid[e * 4 + a] == cid[f * 4 + b]) {
            se[ns] = a;
            sf[ns] = b;
            ++ns;
          }
      if (ns == 0) {
        kind = kRegular;
      } else if (ns == 4) {
        kind = kIdentical;
      } else if (ns == 2) {
        kind = kEdge;
        me = se[0] | ((((se[0] ^ se[1]) & 1) ? 1 : 0) << 2);
        mf = sf[0] | ((((sf[0] ^ sf[1]) & 1) ? 1 : 0) << 2);
      } else {
        kind = kVertex;  // ns == 1 (3 shared corners cannot occur on a conforming mesh)
        me = se[0];
        mf = sf[0];
      }
    }
    if (pass == 0) {
      agg_slot(cnt, kind, valid);
      continue;
    }
    // separated pairs: 0 if one element holds a corner of e and a corner of f
    // (the ring next to the touching pairs), 1 if they lie farther apart
    int far = 0;
    if (valid && kind == kRegular) {
      far = 1;
      for (int a = 0; a < 4 && far; ++a) {
        const int v = cid[e * 4 + a];
        for (int sl = 0; sl < 4 && far; ++sl) {
          const int g = v2e[v * 4 + sl];
          if (g < 0) continue;
          for (int c = 0; c < 4 && far; ++c)
            for (int b = 0; b < 4; ++b)
              if (cid[(int64_t)g * 4 + c] == cid[f * 4 + b]) {
                far = 0;
                break;
              }
        }
      }
    }
    agg_slot(cnt, 4, valid && far);
    const unsigned long long slot_out = agg_slot(cnt, kind, valid);
    if (!valid) continue;
    // mirror block (sc, t) by binary search in row sc
    long long lo = nptr[sc], hi = nptr[sc + 1] - 1;
    while (lo < hi) {
      const long long mid = (lo + hi) / 2;
      if (ncol[mid] < t)
        lo = mid + 1;
      else
        hi = mid;
    }
    const long long blk2 = (long long)nld * nld;
    PairRec pr;
    pr.e = int(e);
    pr.f = int(f);
    pr.code = kind | (me << 2) | (mf << 5);
    pr.pad = far;
    pr.off1 = blk * blk2 + (long long)(pe * nloc) * nld + pf * nloc;
    pr.off2 = (e == f) ? -1 : lo * blk2 + (long long)(pf * nloc) * nld + pe * nloc;
    PairRec* out = kind == 0 ? out0 : (kind == 1 ? out1 : (kind == 2 ? out2 : out3));
    out[slot_out] = pr;
  }
}

// S^2 with knot repetition r > 1: the tensor extraction as CSR, element-local
// function (e, k1 + (d+1) k2) <- global (patch, r i1 + j1, r i2 + j2) with
// coefficient ex[i1][j1][k1] ex[i2][j2][k2], and its transpose.
void build_s2_csr(Op& o) {
  const int d = o.d, D1 = d + 1, nel1 = 1 << o.L, n1 = o.n1, r = o.rep;
  const std::vector<double> ex = extraction_1d(d, nel1, r);
  const int64_t per = int64_t(nel1) * nel1;
  std::vector<int> rptr(o.nlocal + 1, 0), rcol;
  std::vector<double> rval;
  for (int64_t e = 0; e < o.nelem; ++e) {
    const int P = int(e / per);
    uint32_t i1, i2;
    morton_decode(uint32_t(e % per), i1, i2);
    for (int k = 0; k < o.nloc; ++k) {
      const int k1 = k % D1, k2 = k / D1;
      for (int j2 = 0; j2 < D1; ++j2) {
        const double c2 = ex[((size_t)i2 * D1 + j2) * D1 + k2];
        if (c2 == 0.0) continue;
        for (int j1 = 0; j1 < D1; ++j1) {
          const double c1 = ex[((size_t)i1 * D1 + j1) * D1 + k1];
          if (c1 == 0.0) continue;
          rcol.push_back(int((int64_t)P * n1 * n1 + (int64_t)(r * i2 + j2) * n1 + (r * i1 + j1)));
          rval.push_back(c1 * c2);
        }
      }
      rptr[e * o.nloc + k + 1] = int(rcol.size());
    }
  }
  const int64_t n = o.ndofs;
  std::vector<int> tptr(n + 1, 0), tcol(rcol.size());
  std::vector<double> tval(rcol.size());
  for (int c : rcol) ++tptr[c + 1];
  for (int64_t g = 0; g < n; ++g) tptr[g + 1] += tptr[g];
  std::vector<int> fill(tptr.begin(), tptr.end() - 1);
  for (int64_t row = 0; row < o.nlocal; ++row)
    for (int k = rptr[row]; k < rptr[row + 1]; ++k) {
      const int at = fill[rcol[k]]++;
      tcol[at] = int(row);
      tval[at] = rval[k];
    }
  o.d_e_ptr = upload(rptr);
  o.d_e_col = upload(rcol);
  o.d_e_val = upload(rval);
  o.d_et_ptr = upload(tptr);
  o.d_et_col = upload(tcol);
  o.d_et_val = upload(tval);
}

}  // namespace

void build_structure(Op& o) {
  const int L = o.L, d = o.d;
  const int nel1 = 1 << L;
  const int64_t per_patch = int64_t(nel1) * nel1;
  o.nel1 = nel1;
  o.h = 1.0 / nel1;
  // S^2: (d+1)^2 Bernstein functions per element; S^1 (EFIE): 2 p (p+1)
  o.nloc = o.efie ? 2 * d * (d + 1) : (d + 1) * (d + 1);
  o.n1 = d + 1 + (nel1 - 1) * o.rep;
  o.nelem = 6 * per_patch;
  o.ndofs = 6 * int64_t(o.n1) * o.n1;
  o.nlocal = o.nelem * o.nloc;
  if (o.efie) build_s1_space(o);  // sets ndofs (glued S^1 dofs) and the CSR extraction
  if (!o.efie && o.rep > 1) build_s2_csr(o);
  o.m = 1 << (L - o.leaf);
  o.nld = o.m * o.m * o.nloc;
  o.q2 = o.q * o.q;
  o.nleaf = 6 * (int64_t(1) << (2 * o.leaf));
  const int m2 = o.m * o.m;
  const int nld = o.nld, nloc = o.nloc;
  const long long blk2 = (long long)nld * nld;

  auto tstage = std::chrono::steady_clock::now();
  auto stage_done = [&](int k) {  // host time per set-up stage, into the operator's report
    const auto now = std::chrono::steady_clock::now();
    o.info.setup_phase_ms[k] += std::chrono::duration<double, std::milli>(now - tstage).count();
    tstage = now;
  };

  // ---- element corner ids (physical matching, App. D) --------------------------
  // A grid node inside a patch belongs to that patch alone; the nodes on patch
  // boundaries are matched across patches by rounded position.
  std::vector<long long> cid(o.nelem * 4);
  {
    const int64_t nn = int64_t(nel1 + 1) * (nel1 + 1);  // grid nodes per patch
    std::vector<long long> node(6 * nn, -1);
    std::unordered_map<std::array<long long, 3>, long long, KeyHash> table;
    table.reserve(6 * 4 * (size_t)nel1 * 2);
    long long next = 0;
    for (int patch = 0; patch < 6; ++patch)
      for (int i = 0; i <= nel1; ++i) {
        const int walk[4][2] = {{i, 0}, {i, nel1}, {0, i}, {nel1, i}};
        for (const auto& w : walk) {
          long long& id = node[patch * nn + w[0] + int64_t(nel1 + 1) * w[1]];
          if (id >= 0) continue;
          double x[3];
          gamma_eval(o.geom, patch, w[0] * o.h, w[1] * o.h, x);
          const std::array<long long, 3> key = {llround(x[0] * 1e9), llround(x[1] * 1e9), llround(x[2] * 1e9)};
          const auto it = table.emplace(key, next);
          if (it.second) ++next;
          id = it.first->second;
        }
      }
    for (int patch = 0; patch < 6; ++patch)
      for (int i2 = 1; i2 < nel1; ++i2)
        for (int i1 = 1; i1 < nel1; ++i1) node[patch * nn + i1 + int64_t(nel1 + 1) * i2] = next++;
    for (int64_t e = 0; e < o.nelem; ++e) {  // a table lookup per corner: cheaper than starting threads
      const int patch = int(e / per_patch);
      uint32_t i1, i2;
      morton_decode(uint32_t(e % per_patch), i1, i2);
      for (int c = 0; c < 4; ++c)
        cid[e * 4 + c] = node[patch * nn + (i1 + (c & 1)) + int64_t(nel1 + 1) * (i2 + (c >> 1))];
    }
  }

  stage_done(0);

  // ---- cluster balls on levels 0..leaf -----------------------------------------
  o.lvl_off.assign(o.leaf + 2, 0);
  for (int l = 0; l <= o.leaf; ++l) o.lvl_off[l + 1] = o.lvl_off[l] + 6 * (int64_t(1) << (2 * l));
  o.nclusters = o.lvl_off[o.leaf + 1];
  if (o.q > 0) {  // only the admissibility test uses them
    static_assert(sizeof(Ball) == 4 * sizeof(double), "Ball is four doubles");
    if (o.leaf > 14) fail(BEMBEL_EINVAL, "assemble: leaf level above 14");
    LevelTable lt{};
    for (int l = 0; l <= o.leaf + 1; ++l) lt.off[l] = o.lvl_off[l];
    // kept on the device for the compressed potential evaluation
    o.d_balls = static_cast<double*>(dev_alloc(sizeof(Ball) * o.nclusters));
    k_cluster_balls<<<int((o.nclusters + 127) / 128), 128>>>(o.geom, lt, o.nclusters, o.d_balls);
    launched("k_cluster_balls");
  }

  // ---- block tree, level by level, on the device (k_tree_level) --------------------
  // One host synchronisation per level (the two list lengths); the near lists of a level
  // are the next level's candidates (ping-pong buffers), the far lists of all levels are
  // appended to one buffer in target order.  Buffers grow when a level needs more.
  {
    const TreeParams prm{o.opts.eta, o.cplx ? o.opts.kdiam : 0.0, std::hypot(o.kre, o.kim), o.q > 0 ? 1 : 0};
    const Ball* balls = reinterpret_cast<const Ball*>(o.d_balls);
    const int64_t nt_max = o.lvl_off[o.leaf + 1] - o.lvl_off[o.leaf];
    const int64_t nb_max = (nt_max + 1023) / 1024;
    DevBuf cf_buf(sizeof(long long) * (nt_max + 1)), bsum_buf(sizeof(long long) * 2 * nb_max),
        tot_buf(sizeof(long long) * 2);
    long long* cf = static_cast<long long*>(cf_buf.p);
    long long* bsum = static_cast<long long*>(bsum_buf.p);
    long long* tot = static_cast<long long*>(tot_buf.p);
    struct Grow {  // device int array with a capacity
      int* p = nullptr;
      long long cap = 0;
      ~Grow() { dev_free(p); }
      void reserve(long long n, long long keep) {
        if (n <= cap) return;
        const long long c = std::max<long long>(n, 2 * cap);
        int* q = static_cast<int*>(dev_alloc(sizeof(int) * c));
        if (keep > 0) cuda_check(cudaMemcpy(q, p, sizeof(int) * keep, cudaMemcpyDeviceToDevice), "tree grow");
        dev_free(p);
        p = q;
        cap = c;
      }
    } far, near[2];
    far.reserve(64 * o.nclusters, 0);
    near[0].reserve(32 * nt_max, 0);
    near[1].reserve(32 * nt_max, 0);
    DevBuf cn_buf0(sizeof(long long) * (nt_max + 1)), cn_buf1(sizeof(long long) * (nt_max + 1));
    long long* cn[2] = {static_cast<long long*>(cn_buf0.p), static_cast<long long*>(cn_buf1.p)};
    o.d_far_ptr = static_cast<long long*>(dev_alloc(sizeof(long long) * (o.nclusters + 1)));
    long long far_base = 0, nnear_l = 0;
    int cur = 0;
    for (int l = 0; l <= o.leaf; ++l) {
      const int64_t t0 = o.lvl_off[l], nt = o.lvl_off[l + 1] - t0;
      const int grid = int((nt + 127) / 128);
      const long long off_lm1 = l > 0 ? o.lvl_off[l - 1] : 0;
      const long long* pptr = l > 0 ? cn[cur ^ 1] : nullptr;
      const int* pcol = l > 0 ? near[cur ^ 1].p : nullptr;
      k_tree_level<<<grid, 128>>>(0, l, t0, nt, o.lvl_off[l], off_lm1, pptr, pcol, balls, prm, cf, cn[cur], nullptr,
                                  nullptr);
      launched("k_tree_level");
      const int64_t nb = (nt + 1023) / 1024;
      k_scan_block<<<dim3(unsigned(nb), 2), 1024>>>(cf, cn[cur], nt, bsum, nb_max);
      k_scan_sums<<<2, 1024>>>(cf, cn[cur], nt, bsum, nb, nb_max, tot);
      k_scan_add<<<dim3(unsigned(nb), 2), 1024>>>(cf, cn[cur], nt, bsum, nb_max);
      launched("k_scan");
      long long h[2];
      cuda_check(cudaMemcpy(h, tot, sizeof(h), cudaMemcpyDeviceToHost), "tree counts");
      far.reserve(far_base + h[0], far_base);
      near[cur].reserve(std::max<long long>(1, h[1]), 0);
      k_tree_level<<<grid, 128>>>(1, l, t0, nt, o.lvl_off[l], off_lm1, pptr, pcol, balls, prm, cf, cn[cur],
                                  far.p + far_base, near[cur].p);
      launched("k_tree_level");
      k_tree_fptr<<<grid, 128>>>(o.d_far_ptr, t0, nt, cf, far_base);
      launched("k_tree_fptr");
      far_base += h[0];
      nnear_l = h[1];
      cur ^= 1;
    }
    cur ^= 1;  // the leaf level's lists
    cuda_check(cudaMemcpy(o.d_far_ptr + o.nclusters, &far_base, sizeof(long long), cudaMemcpyHostToDevice),
               "far total");
    o.nfar = far_base;
    if (o.nfar > 0) {
      o.d_far_src = static_cast<int*>(dev_alloc(sizeof(int) * o.nfar));
      cuda_check(cudaMemcpy(o.d_far_src, far.p, sizeof(int) * o.nfar, cudaMemcpyDeviceToDevice), "far lists");
      o.d_far_tgt = static_cast<int*>(dev_alloc(sizeof(int) * o.nfar));
      k_tree_tgt<<<int((o.nclusters + 127) / 128), 128>>>(o.d_far_ptr, o.nclusters, o.d_far_tgt);
      launched("k_tree_tgt");
    }
    // leaf-level non-admissible pairs are the near field (leaf-local ids)
    o.nnear = nnear_l;
    o.d_near_ptr = static_cast<long long*>(dev_alloc(sizeof(long long) * (o.nleaf + 1)));
    cuda_check(cudaMemcpy(o.d_near_ptr, cn[cur], sizeof(long long) * (o.nleaf + 1), cudaMemcpyDeviceToDevice),
               "near ptr");
    o.d_near_col = static_cast<int*>(dev_alloc(sizeof(int) * std::max<int64_t>(1, o.nnear)));
    if (o.nnear > 0)
      cuda_check(cudaMemcpy(o.d_near_col, near[cur].p, sizeof(int) * o.nnear, cudaMemcpyDeviceToDevice), "near col");
    o.d_diag_blk = static_cast<int*>(dev_alloc(sizeof(int) * o.nleaf));
    o.d_leaf_ids = static_cast<int*>(dev_alloc(sizeof(int) * o.nleaf));
    o.d_near_tgt = static_cast<int*>(dev_alloc(sizeof(int) * std::max<int64_t>(1, o.nnear)));
    cuda_check(cudaMemset(tot, 0, sizeof(long long)), "tree err");
    k_tree_rows<<<int((o.nleaf + 127) / 128), 128>>>(o.d_near_ptr, o.d_near_col, o.lvl_off[o.leaf], o.nleaf,
                                                     o.d_diag_blk, o.d_leaf_ids, o.d_near_tgt,
                                                     reinterpret_cast<int*>(tot));
    launched("k_tree_rows");
    int err = 0;
    cuda_check(cudaMemcpy(&err, tot, sizeof(int), cudaMemcpyDeviceToHost), "tree rows");
    if (err) fail(BEMBEL_EINVAL, "near field lacks a diagonal block");
  }

  stage_done(1);

  // ---- element pairs of the near field (classified on the device) -----------------
  {
    std::vector<int> cid32(cid.begin(), cid.end());
    int* d_cid = upload(cid32);
    // vertex -> the (at most 4) elements holding it, -1 padded
    int nvert = 0;
    for (int v : cid32) nvert = std::max(nvert, v + 1);
    std::vector<int> v2e((size_t)nvert * 4, -1);
    for (int64_t e = 0; e < o.nelem; ++e)
      for (int a = 0; a < 4; ++a) {
        int* slot = &v2e[(size_t)cid32[e * 4 + a] * 4];
        for (int k = 0; k < 4; ++k)
          if (slot[k] < 0) {
            slot[k] = int(e);
            break;
          }
      }
    int* d_v2e = upload(v2e);
    unsigned long long* d_cnt = static_cast<unsigned long long*>(dev_alloc(sizeof(unsigned long long) * 5));
    const int64_t work = o.nnear * (int64_t)m2 * m2;
    const int tb = 256;
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>((work + tb - 1) / tb, 152 * 64)));
    PairRec* outs[4] = {nullptr, nullptr, nullptr, nullptr};
    unsigned long long cnt[5];
    for (int pass = 0; pass < 2; ++pass) {
      cuda_check(cudaMemset(d_cnt, 0, sizeof(unsigned long long) * 5), "pair counters");
      k_build_pairs<<<grid, tb>>>(o.d_near_ptr, o.d_near_col, o.d_near_tgt, o.nnear, d_cid, m2, o.nloc, o.nld,
                                   pass, d_cnt, outs[0], outs[1], outs[2], outs[3], d_v2e);
      launched("k_build_pairs");
      cuda_check(cudaMemcpy(cnt, d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost), "pair counts");
      if (pass == 0)
        for (int k = 0; k < 4; ++k) {
          o.npairs[k] = (int64_t)cnt[k];
          outs[k] = static_cast<PairRec*>(dev_alloc(sizeof(PairRec) * std::max<int64_t>(1, o.npairs[k])));
        }
    }
    for (int k = 0; k < 4; ++k) {
      if (cnt[k] != (unsigned long long)o.npairs[k]) fail(BEMBEL_EINVAL, "pair list build is inconsistent");
      o.d_pairs[k] = outs[k];
    }
    o.npairs_regular_far = (int64_t)cnt[4];
    dev_free(d_v2e);
    dev_free(d_cid);
    dev_free(d_cnt);
  }

  stage_done(2);

  // ---- Bezier extraction (1-D, per element index); S^1: signed CSR with glue ------
  if (!o.efie) o.d_ex = upload(extraction_1d(d, nel1, o.rep));

  // ---- moments and transfers (geometry independent) --------------------------------
  if (o.q > 0) {
    const int q = o.q, q2 = o.q2;
    std::vector<double> gx, gw;
    gauss01(d + q, gx, gw);
    if (o.efie) efie_moments(o, gx, gw);
    // M1[me][k][a] = int_0^1 B_k(u) l_a((me + u)/m) du
    std::vector<double> M1((size_t)o.m * (d + 1) * q, 0.0);
    for (int me = 0; me < o.m; ++me)
      for (int k = 0; k <= d; ++k)
        for (int a = 0; a < q; ++a) {
          double acc = 0.0;
          for (size_t p = 0; p < gx.size(); ++p)
            acc += gw[p] * bernstein_h(d, k, gx[p]) * lagrange01(q, a, (me + gx[p]) / o.m);
          M1[((size_t)me * (d + 1) + k) * q + a] = acc;
        }
    std::vector<double> V((size_t)nld * q2);
    for (int pe = 0; pe < m2 && !o.efie; ++pe) {
      uint32_t e1, e2;
      morton_decode(pe, e1, e2);
      for (int k2 = 0; k2 <= d; ++k2)
        for (int k1 = 0; k1 <= d; ++k1)
          for (int a2 = 0; a2 < q; ++a2)
            for (int a1 = 0; a1 < q; ++a1) {
              const int i = pe * nloc + k1 + (d + 1) * k2;
              V[(size_t)i * q2 + a1 + q * a2] = o.h * o.h * M1[((size_t)e1 * (d + 1) + k1) * q + a1] *
                                                 M1[((size_t)e2 * (d + 1) + k2) * q + a2];
            }
    }
    std::vector<double> T1(2 * q * q);
    for (int cb = 0; cb < 2; ++cb)
      for (int ap = 0; ap < q; ++ap)
        for (int a = 0; a < q; ++a) T1[(cb * q + ap) * q + a] = lagrange01(q, a, 0.5 * (cb + chebyshev01(q, ap)));
    std::vector<double> T((size_t)4 * q2 * q2);
    for (int c = 0; c < 4; ++c)
      for (int ap2 = 0; ap2 < q; ++ap2)
        for (int ap1 = 0; ap1 < q; ++ap1)
          for (int a2 = 0; a2 < q; ++a2)
            for (int a1 = 0; a1 < q; ++a1)
              T[((size_t)c * q2 + ap1 + q * ap2) * q2 + a1 + q * a2] =
                  T1[((c & 1) * q + ap1) * q + a1] * T1[((c >> 1) * q + ap2) * q + a2];
    if (!o.efie) o.d_V = upload(V);
    o.d_T = upload(T);
    std::vector<float> V32(V.begin(), V.end()), T32(T.begin(), T.end());
    if (!o.efie) o.d_V32 = upload(V32);  // the EFIE's three channels are copied in efie_moments
    o.d_T32 = upload(T32);

    // cluster interpolation points in R^3
    std::vector<double> nodes((size_t)o.nclusters * q2 * 3);
    std::vector<double> cheb(q);
    for (int a = 0; a < q; ++a) cheb[a] = chebyshev01(q, a);
    parallel_for(o.nclusters, [&](int64_t c0, int64_t c1) {
      for (int64_t gc = c0; gc < c1; ++gc) {
        int l = 0;
        while (gc >= o.lvl_off[l + 1]) ++l;
        const int64_t nper = int64_t(1) << (2 * l);
        const int64_t c = gc - o.lvl_off[l];
        const double H = std::ldexp(1.0, -l);
        const int patch = int(c / nper);
        uint32_t j1, j2;
        morton_decode(uint32_t(c % nper), j1, j2);
        for (int a2 = 0; a2 < q; ++a2)
          for (int a1 = 0; a1 < q; ++a1)
            gamma_eval(o.geom, patch, (j1 + cheb[a1]) * H, (j2 + cheb[a2]) * H,
                       &nodes[((size_t)gc * q2 + a1 + q * a2) * 3]);
      }
    });
    o.d_nodes = upload(nodes);
    if (o.efie) {  // d_s gamma, d_t gamma at the cluster points (EFIE coupling)
      std::vector<double> jac((size_t)o.nclusters * q2 * 6);
      parallel_for(o.nclusters, [&](int64_t c0, int64_t c1) {
        for (int64_t gc = c0; gc < c1; ++gc) {
          int l = 0;
          while (gc >= o.lvl_off[l + 1]) ++l;
          const int64_t nper = int64_t(1) << (2 * l);
          const int64_t c = gc - o.lvl_off[l];
          const double H = std::ldexp(1.0, -l);
          uint32_t j1, j2;
          morton_decode(uint32_t(c % nper), j1, j2);
          for (int a2 = 0; a2 < q; ++a2)
            for (int a1 = 0; a1 < q; ++a1) {
              double x[3];
              double* J = &jac[((size_t)gc * q2 + a1 + q * a2) * 6];
              sphere6_jac(int(c / nper), (j1 + cheb[a1]) * H, (j2 + cheb[a2]) * H, x, J, J + 3);
            }
        }
      });
      o.d_nodes_jac = upload(jac);
    }
    std::vector<float> nodes32(nodes.size() / 3 * 4, 0.f);
    for (size_t k = 0; k < nodes.size() / 3; ++k)
      for (int c = 0; c < 3; ++c) nodes32[k * 4 + c] = float(nodes[k * 3 + c]);
    o.d_nodes32 = upload(nodes32);
    if (o.opts.precision == BEMBEL_PREC_MIXED && !o.efie) {
      // FP32 coupling entries of MIXED operators: cluster centres (mean of the cluster's
      // points, FP64) and the points as FP32 offsets from them
      std::vector<double> ccen((size_t)o.nclusters * 3, 0.0);
      std::vector<float> rel((size_t)o.nclusters * q2 * 4, 0.f);
      for (int64_t c = 0; c < o.nclusters; ++c) {
        double m[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < q2; ++a)
          for (int k = 0; k < 3; ++k) m[k] += nodes[((size_t)c * q2 + a) * 3 + k];
        for (int k = 0; k < 3; ++k) ccen[(size_t)c * 3 + k] = m[k] / q2;
        for (int a = 0; a < q2; ++a)
          for (int k = 0; k < 3; ++k)
            rel[((size_t)c * q2 + a) * 4 + k] = float(nodes[((size_t)c * q2 + a) * 3 + k] - ccen[(size_t)c * 3 + k]);
      }
      o.d_ccen = upload(ccen);
      o.d_nodes_rel32 = upload(rel);
    }
  }

  stage_done(3);

  // ---- quadrature tables -------------------------------------------------------------
  {
    std::vector<double> gx, gw;
    gauss01(o.g_reg, gx, gw);
    const int G = o.g_reg, G2 = G * G;
    std::vector<double> BW((size_t)G2 * nloc, 0.0);
    for (int p2 = 0; p2 < G && !o.efie; ++p2)
      for (int p1 = 0; p1 < G; ++p1)
        for (int k2 = 0; k2 <= d; ++k2)
          for (int k1 = 0; k1 <= d; ++k1)
            BW[(size_t)(p1 + G * p2) * nloc + k1 + (d + 1) * k2] =
                gw[p1] * gw[p2] * o.h * o.h * bernstein_h(d, k1, gx[p1]) * bernstein_h(d, k2, gx[p2]);
    o.d_BW = upload(BW);
    {
      // separated pairs farther than the ring next to the touching pairs: own order
      std::vector<double> fx, fw;
      gauss01(o.g_reg_far, fx, fw);
      const int F = o.g_reg_far, F2 = F * F;
      std::vector<double> BWf((size_t)F2 * nloc, 0.0);
      for (int p2 = 0; p2 < F && !o.efie; ++p2)
        for (int p1 = 0; p1 < F; ++p1)
          for (int k2 = 0; k2 <= d; ++k2)
            for (int k1 = 0; k1 <= d; ++k1)
              BWf[(size_t)(p1 + F * p2) * nloc + k1 + (d + 1) * k2] =
                  fw[p1] * fw[p2] * o.h * o.h * bernstein_h(d, k1, fx[p1]) * bernstein_h(d, k2, fx[p2]);
      o.d_BW_far = upload(BWf);
    }
    // per kind (regular first) and per variable: nodes then weights; the
    // regular kind repeats g_reg four times (its first nodes tabulate gamma)
    std::vector<double> rg;
    for (int k = kRegular; k <= kVertex; ++k) {
      o.gauss_off[k] = int(rg.size());
      for (int v = 0; v < 4; ++v) {
        gauss01(o.g_var[k][v], gx, gw);
        rg.insert(rg.end(), gx.begin(), gx.end());
        rg.insert(rg.end(), gw.begin(), gw.end());
      }
    }
    o.gauss_off_far = int(rg.size());  // nodes then weights of the far separated order
    gauss01(o.g_reg_far, gx, gw);
    rg.insert(rg.end(), gx.begin(), gx.end());
    rg.insert(rg.end(), gw.begin(), gw.end());
    o.d_gauss = upload(rg);
  }

  stage_done(4);

  // ---- report -------------------------------------------------------------------------
  bembel_op_info& in = o.info;
  in.ndofs = o.ndofs;
  in.nlocal = o.nlocal;
  in.nelements = o.nelem;
  in.n_clusters = o.nclusters;
  in.n_far_blocks = o.nfar;
  in.n_near_blocks = o.nnear;
  in.n_pairs_regular = o.npairs[kRegular];
  in.n_pairs_identical = o.npairs[kIdentical];
  in.n_pairs_edge = o.npairs[kEdge];
  in.n_pairs_vertex = o.npairs[kVertex];
  in.n_pairs_regular_far = o.npairs_regular_far;
  in.near_bytes = o.nnear * blk2 * 8 * (o.cplx ? 2 : 1);
  in.far_bytes = o.nfar * (int64_t)o.q2 * o.q2 * 8 * (o.cplx ? 2 : 1);
  in.leaf_level = o.leaf;
  in.q = o.q;
  in.degree = o.d;
  in.level = o.L;
}

}  // namespace bembel
