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
#include <cstring>
#include <unordered_map>

#include "op.h"

namespace bembel {

namespace {

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

// Cox-de Boor on the open knot vector of degree d with n_el uniform elements;
// value of B-spline j at x in [0,1] (x = 1 belongs to the last interval).
double bspline_h(int d, int n_el, int j, double x) {
  const int nk = n_el + 2 * d + 1;
  std::vector<double> kn(nk);
  for (int i = 0; i < nk; ++i) {
    const int t = i - d;
    kn[i] = t <= 0 ? 0.0 : (t >= n_el ? 1.0 : double(t) / n_el);
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

struct Ball {
  double c[3];
  double r;
};

template <typename T>
T* upload(const std::vector<T>& v) {
  if (v.empty()) return nullptr;
  T* p = static_cast<T*>(dev_alloc(v.size() * sizeof(T)));
  cuda_check(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), "upload");
  return p;
}

struct KeyHash {
  size_t operator()(const std::array<long long, 3>& k) const {
    return std::hash<long long>()(k[0] * 73856093LL ^ k[1] * 19349663LL ^ k[2] * 83492791LL);
  }
};

}  // namespace

void build_structure(Op& o) {
  const int L = o.L, d = o.d;
  const int nel1 = 1 << L;
  const int64_t per_patch = int64_t(nel1) * nel1;
  o.nel1 = nel1;
  o.h = 1.0 / nel1;
  o.nloc = (d + 1) * (d + 1);
  o.n1 = nel1 + d;
  o.nelem = 6 * per_patch;
  o.ndofs = 6 * int64_t(o.n1) * o.n1;
  o.nlocal = o.nelem * o.nloc;
  o.m = 1 << (L - o.leaf);
  o.nld = o.m * o.m * o.nloc;
  o.q2 = o.q * o.q;
  o.nleaf = 6 * (int64_t(1) << (2 * o.leaf));

  // ---- element corner ids (physical matching, App. D) --------------------------
  std::vector<long long> cid(o.nelem * 4);
  {
    std::unordered_map<std::array<long long, 3>, long long, KeyHash> table;
    table.reserve(o.nelem * 2);
    for (int64_t e = 0; e < o.nelem; ++e) {
      const int patch = int(e / per_patch);
      uint32_t i1, i2;
      morton_decode(uint32_t(e % per_patch), i1, i2);
      for (int c = 0; c < 4; ++c) {
        double x[3];
        gamma_eval(o.geom, patch, (i1 + (c & 1)) * o.h, (i2 + (c >> 1)) * o.h, x);
        std::array<long long, 3> key;
        for (int k = 0; k < 3; ++k) key[k] = llround(x[k] * 1e9);
        auto it = table.find(key);
        long long id;
        if (it == table.end()) {
          id = (long long)table.size();
          table.emplace(key, id);
        } else {
          id = it->second;
        }
        cid[e * 4 + c] = id;
      }
    }
  }

  debug_mark("setup: cluster balls on levels 0..leaf");
  // ---- cluster balls on levels 0..leaf -----------------------------------------
  o.lvl_off.assign(o.leaf + 2, 0);
  for (int l = 0; l <= o.leaf; ++l) o.lvl_off[l + 1] = o.lvl_off[l] + 6 * (int64_t(1) << (2 * l));
  o.nclusters = o.lvl_off[o.leaf + 1];
  std::vector<Ball> balls(o.nclusters);
  for (int l = 0; l <= o.leaf; ++l) {
    const int64_t nper = int64_t(1) << (2 * l);
    const double H = std::ldexp(1.0, -l);
    for (int64_t c = 0; c < 6 * nper; ++c) {
      const int patch = int(c / nper);
      uint32_t j1, j2;
      morton_decode(uint32_t(c % nper), j1, j2);
      Ball b;
      gamma_eval(o.geom, patch, (j1 + 0.5) * H, (j2 + 0.5) * H, b.c);
      double r = 0.0;
      for (int k2 = 0; k2 <= 8; ++k2)
        for (int k1 = 0; k1 <= 8; ++k1) {
          double x[3];
          gamma_eval(o.geom, patch, (j1 + k1 / 8.0) * H, (j2 + k2 / 8.0) * H, x);
          const double dx = x[0] - b.c[0], dy = x[1] - b.c[1], dz = x[2] - b.c[2];
          r = std::max(r, std::sqrt(dx * dx + dy * dy + dz * dz));
        }
      b.r = r;
      balls[o.lvl_off[l] + c] = b;
    }
  }

  debug_mark("setup: block tree");
  // ---- block tree ------------------------------------------------------------------
  std::vector<std::pair<int, int>> far, near;  // global cluster ids (target, source)
  {
    const bool compress = o.q > 0;
    std::vector<std::pair<int, int>> stack;
    for (int p = 0; p < 6; ++p)
      for (int r = 0; r < 6; ++r) stack.push_back({p, r});
    while (!stack.empty()) {
      auto [t, s] = stack.back();
      stack.pop_back();
      int lev = 0;
      while (t >= o.lvl_off[lev + 1]) ++lev;
      bool adm = false;
      if (compress) {
        const Ball &bt = balls[t], &bs = balls[s];
        const double dx = bt.c[0] - bs.c[0], dy = bt.c[1] - bs.c[1], dz = bt.c[2] - bs.c[2];
        const double dist = std::max(0.0, std::sqrt(dx * dx + dy * dy + dz * dz) - bt.r - bs.r);
        adm = 2.0 * std::max(bt.r, bs.r) <= o.opts.eta * dist;
      }
      if (adm) {
        far.push_back({t, s});
      } else if (lev == o.leaf) {
        near.push_back({t, s});
      } else {
        const int64_t tl = t - o.lvl_off[lev], sl = s - o.lvl_off[lev];
        for (int ct = 0; ct < 4; ++ct)
          for (int cs = 0; cs < 4; ++cs)
            stack.push_back({int(o.lvl_off[lev + 1] + 4 * tl + ct), int(o.lvl_off[lev + 1] + 4 * sl + cs)});
      }
    }
  }
  std::sort(far.begin(), far.end());
  std::sort(near.begin(), near.end());
  o.nfar = (int64_t)far.size();
  o.nnear = (int64_t)near.size();

  {
    std::vector<long long> ptr(o.nclusters + 1, 0);
    std::vector<int> src(o.nfar), tgt(o.nfar);
    for (int64_t i = 0; i < o.nfar; ++i) {
      ptr[far[i].first + 1]++;
      src[i] = far[i].second;
      tgt[i] = far[i].first;
    }
    for (int64_t c = 0; c < o.nclusters; ++c) ptr[c + 1] += ptr[c];
    o.d_far_ptr = upload(ptr);
    o.d_far_src = upload(src);
    o.d_far_tgt = upload(tgt);
  }
  std::vector<long long> nptr(o.nleaf + 1, 0);
  std::vector<int> ncol(o.nnear);
  const int64_t leaf_off = o.lvl_off[o.leaf];
  for (int64_t i = 0; i < o.nnear; ++i) {
    nptr[near[i].first - leaf_off + 1]++;
    ncol[i] = int(near[i].second - leaf_off);
  }
  for (int64_t c = 0; c < o.nleaf; ++c) nptr[c + 1] += nptr[c];
  o.d_near_ptr = upload(nptr);
  o.d_near_col = upload(ncol);

  debug_mark("setup: element pairs of the near field");
  // ---- element pairs of the near field --------------------------------------------
  auto block_index = [&](int64_t t, int64_t s) -> long long {
    const auto b = ncol.begin() + nptr[t], en = ncol.begin() + nptr[t + 1];
    auto it = std::lower_bound(b, en, int(s));
    if (it == en || *it != s) fail(BEMBEL_EINVAL, "block tree is not symmetric");
    return (long long)(it - ncol.begin());
  };
  const int m2 = o.m * o.m;
  const int nld = o.nld, nloc = o.nloc;
  const long long blk2 = (long long)nld * nld;
  std::vector<PairRec> lists[4];
  for (int64_t i = 0; i < o.nnear; ++i) {
    const int64_t t = near[i].first - leaf_off, s = near[i].second - leaf_off;
    if (t > s) continue;
    const long long b1 = i, b2 = block_index(s, t);
    for (int pe = 0; pe < m2; ++pe) {
      const int64_t e = t * m2 + pe;
      for (int pf = (t == s ? pe : 0); pf < m2; ++pf) {
        const int64_t f = s * m2 + pf;
        const long long* ce = &cid[e * 4];
        const long long* cf = &cid[f * 4];
        int shared_e[4], shared_f[4], ns = 0;
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b)
            if (ce[a] == cf[b]) {
              shared_e[ns] = a;
              shared_f[ns] = b;
              ++ns;
            }
        PairRec pr;
        pr.e = int(e);
        pr.f = int(f);
        pr.pad = 0;
        pr.off1 = b1 * blk2 + (long long)(pf * nloc) * nld + pe * nloc;
        pr.off2 = (e == f) ? -1 : b2 * blk2 + (long long)(pe * nloc) * nld + pf * nloc;
        int kind, me = 0, mf = 0;
        if (ns == 0) {
          kind = kRegular;
        } else if (ns == 4) {
          kind = kIdentical;
        } else if (ns == 2) {
          kind = kEdge;
          // A = first shared corner of e, B = second; D2 runs A -> B, D1 is the other axis.
          const int ae = shared_e[0], be = shared_e[1];
          const int af = shared_f[0], bf = shared_f[1];
          const int ax_e = ((ae ^ be) & 1) ? 1 : 0;  // A->B along axis 0 => D1 along axis 1
          const int ax_f = ((af ^ bf) & 1) ? 1 : 0;
          me = ae | (ax_e << 2);
          mf = af | (ax_f << 2);
        } else if (ns == 1) {
          kind = kVertex;
          me = shared_e[0];
          mf = shared_f[0];
        } else {
          fail(BEMBEL_EINVAL, "elements share 3 corners: mesh is not conforming (App. D)");
        }
        pr.code = kind | (me << 2) | (mf << 5);
        lists[kind].push_back(pr);
      }
    }
  }
  for (int k = 0; k < 4; ++k) {
    o.npairs[k] = (int64_t)lists[k].size();
    o.d_pairs[k] = upload(lists[k]);
  }

  debug_mark("setup: Bezier extraction");
  // ---- Bezier extraction (1-D, per element index) ----------------------------------
  {
    const int n = d + 1;
    std::vector<double> ex((size_t)nel1 * n * n);
    std::vector<double> A(n * (n + 1)), sol;
    for (int i = 0; i < nel1; ++i)
      for (int j = 0; j < n; ++j) {
        for (int r = 0; r < n; ++r) {
          const double u = (r + 0.5) / n;
          for (int k = 0; k < n; ++k) A[r * (n + 1) + k] = bernstein_h(d, k, u);
          A[r * (n + 1) + n] = bspline_h(d, nel1, i + j, (i + u) / nel1);
        }
        solve_small(n, A, sol);
        for (int k = 0; k < n; ++k) ex[((size_t)i * n + j) * n + k] = sol[k];
      }
    o.d_ex = upload(ex);
  }

  debug_mark("setup: moments and transfers");
  // ---- moments and transfers (geometry independent) --------------------------------
  if (o.q > 0) {
    const int q = o.q, q2 = o.q2;
    std::vector<double> gx, gw;
    gauss01(d + q, gx, gw);
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
    for (int pe = 0; pe < m2; ++pe) {
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
    o.d_V = upload(V);
    o.d_T = upload(T);
    std::vector<float> V32(V.begin(), V.end()), T32(T.begin(), T.end());
    o.d_V32 = upload(V32);
    o.d_T32 = upload(T32);

    // cluster interpolation points in R^3
    std::vector<double> nodes((size_t)o.nclusters * q2 * 3);
    for (int l = 0; l <= o.leaf; ++l) {
      const int64_t nper = int64_t(1) << (2 * l);
      const double H = std::ldexp(1.0, -l);
      for (int64_t c = 0; c < 6 * nper; ++c) {
        const int patch = int(c / nper);
        uint32_t j1, j2;
        morton_decode(uint32_t(c % nper), j1, j2);
        for (int a2 = 0; a2 < q; ++a2)
          for (int a1 = 0; a1 < q; ++a1)
            gamma_eval(o.geom, patch, (j1 + chebyshev01(q, a1)) * H, (j2 + chebyshev01(q, a2)) * H,
                       &nodes[(((size_t)(o.lvl_off[l] + c)) * q2 + a1 + q * a2) * 3]);
      }
    }
    o.d_nodes = upload(nodes);
  }

  debug_mark("setup: quadrature tables");
  // ---- quadrature tables -------------------------------------------------------------
  {
    std::vector<double> gx, gw;
    gauss01(o.g_reg, gx, gw);
    const int G = o.g_reg, G2 = G * G;
    std::vector<double> BW((size_t)G2 * nloc);
    for (int p2 = 0; p2 < G; ++p2)
      for (int p1 = 0; p1 < G; ++p1)
        for (int k2 = 0; k2 <= d; ++k2)
          for (int k1 = 0; k1 <= d; ++k1)
            BW[(size_t)(p1 + G * p2) * nloc + k1 + (d + 1) * k2] =
                gw[p1] * gw[p2] * o.h * o.h * bernstein_h(d, k1, gx[p1]) * bernstein_h(d, k2, gx[p2]);
    o.d_BW = upload(BW);
    std::vector<double> rg;
    gauss01(G, gx, gw);
    rg.insert(rg.end(), gx.begin(), gx.end());
    gauss01(o.g_sing, gx, gw);
    rg.insert(rg.end(), gx.begin(), gx.end());
    rg.insert(rg.end(), gw.begin(), gw.end());
    o.d_gauss = upload(rg);  // [g_reg nodes][g_sing nodes][g_sing weights]
  }

  debug_mark("setup: report");
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
  in.near_bytes = o.nnear * blk2 * 8 * (o.cplx ? 2 : 1);
  in.far_bytes = o.nfar * (int64_t)o.q2 * o.q2 * 8 * (o.cplx ? 2 : 1);
  in.leaf_level = o.leaf;
  in.q = o.q;
  in.degree = o.d;
  in.level = o.L;
}

}  // namespace bembel
