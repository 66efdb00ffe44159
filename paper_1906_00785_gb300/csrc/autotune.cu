// autotune.cu - choice of quadrature orders, interpolation order and block-
// sparse chunk size for a target accuracy (the paper states none of them).
//
// * Quadrature: for each pair kind (separated near, identical, common edge,
//   common vertex) a sample of that kind's element pairs is integrated on the
//   device at increasing Gauss orders and at a reference order; the smallest
//   order whose worst relative block difference is <= quad_tol is chosen.
// * Interpolation: leaf-level far blocks are sampled; the H^2 block V K V^T
//   (Sec. 2, kernel interpolated at q x q Chebyshev points per cluster) is
//   compared on the host with a converged tensor-Gauss integration of the same
//   element pairs; far blocks on the coarser levels (larger clusters) are sampled
//   too, by the pointwise error of the kernel interpolant; the smallest q whose
//   worst relative error is <= far_tol is chosen.
// * Chunk size of the block-sparse products: the fastest of a few by timing.
#include <algorithm>
#include <chrono>
#include <complex>
#include <vector>

#include "op.h"

namespace bembel {

namespace {

using cplx = std::complex<double>;

cplx green_h(const Op& o, const double* x, const double* y) {
  const double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
  const double r = std::sqrt(d0 * d0 + d1 * d1 + d2 * d2);
  if (!o.cplx) return cplx(kInv4Pi / r, 0.0);
  const cplx kap(o.kre, o.kim);
  return std::exp(cplx(0.0, -1.0) * kap * r) * (kInv4Pi / r);
}

// element e -> patch parameters of its local point u
void elem_point(const Op& o, int64_t e, double u1, double u2, double x[3]) {
  const int64_t per = int64_t(1) << (2 * o.L);
  uint32_t i1, i2;
  morton_decode(uint32_t(e % per), i1, i2);
  gamma_eval(o.geom, int(e / per), (i1 + u1) * o.h, (i2 + u2) * o.h, x);
}

// Relative Frobenius error of V K V^T against Gauss integration for sampled
// leaf-level far blocks, interpolation order q.
double far_error(const Op& o, int q, const std::vector<std::pair<int, int>>& blocks) {
  const int d = o.d, D1 = d + 1, nloc = o.nloc, m = o.m, m2 = m * m, nld = m2 * nloc, q2 = q * q;
  // leaf moments V (nld x q2), as in the operator set-up
  std::vector<double> gx, gw;
  gauss01(d + q, gx, gw);
  std::vector<double> M1((size_t)m * D1 * q);
  for (int me = 0; me < m; ++me)
    for (int k = 0; k <= d; ++k)
      for (int a = 0; a < q; ++a) {
        double acc = 0.0;
        for (size_t p = 0; p < gx.size(); ++p)
          acc += gw[p] * bernstein_h(d, k, gx[p]) * lagrange01(q, a, (me + gx[p]) / m);
        M1[((size_t)me * D1 + k) * q + a] = acc;
      }
  std::vector<double> V((size_t)nld * q2);
  for (int pe = 0; pe < m2; ++pe) {
    uint32_t e1, e2;
    morton_decode(pe, e1, e2);
    for (int k2 = 0; k2 <= d; ++k2)
      for (int k1 = 0; k1 <= d; ++k1)
        for (int a2 = 0; a2 < q; ++a2)
          for (int a1 = 0; a1 < q; ++a1)
            V[(size_t)(pe * nloc + k1 + D1 * k2) * q2 + a1 + q * a2] =
                o.h * o.h * M1[((size_t)e1 * D1 + k1) * q + a1] * M1[((size_t)e2 * D1 + k2) * q + a2];
  }
  // converged reference: tensor Gauss with 8 points per direction per element
  const int G = 8;
  std::vector<double> rx, rw;
  gauss01(G, rx, rw);
  const int64_t leaf_off = o.lvl_off[o.leaf];
  const int64_t nper = int64_t(1) << (2 * o.leaf);
  const double H = std::ldexp(1.0, -o.leaf);
  double worst = 0.0;
  for (const auto& bl : blocks) {
    const int64_t t = bl.first - leaf_off, sc = bl.second - leaf_off;
    // coupling K at the cluster Chebyshev points
    std::vector<double> xt((size_t)q2 * 3), xs((size_t)q2 * 3);
    for (int side = 0; side < 2; ++side) {
      const int64_t c = side == 0 ? t : sc;
      uint32_t j1, j2;
      morton_decode(uint32_t(c % nper), j1, j2);
      for (int a2 = 0; a2 < q; ++a2)
        for (int a1 = 0; a1 < q; ++a1)
          gamma_eval(o.geom, int(c / nper), (j1 + chebyshev01(q, a1)) * H, (j2 + chebyshev01(q, a2)) * H,
                     &(side == 0 ? xt : xs)[(size_t)(a1 + q * a2) * 3]);
    }
    std::vector<cplx> K((size_t)q2 * q2);
    for (int a = 0; a < q2; ++a)
      for (int b = 0; b < q2; ++b) K[(size_t)a * q2 + b] = green_h(o, &xt[a * 3], &xs[b * 3]);
    // approx = V K V^T
    std::vector<cplx> VK((size_t)nld * q2, cplx(0.0));
    for (int i = 0; i < nld; ++i)
      for (int a = 0; a < q2; ++a)
        for (int b = 0; b < q2; ++b) VK[(size_t)i * q2 + b] += V[(size_t)i * q2 + a] * K[(size_t)a * q2 + b];
    double num = 0.0, den = 0.0;
    for (int pe = 0; pe < m2; ++pe)
      for (int pf = 0; pf < m2; ++pf) {
        const int64_t e = t * m2 + pe, f = sc * m2 + pf;
        std::vector<double> X((size_t)G * G * 3), Y((size_t)G * G * 3), B((size_t)G * G * nloc);
        for (int p2 = 0; p2 < G; ++p2)
          for (int p1 = 0; p1 < G; ++p1) {
            elem_point(o, e, rx[p1], rx[p2], &X[(size_t)(p1 + G * p2) * 3]);
            elem_point(o, f, rx[p1], rx[p2], &Y[(size_t)(p1 + G * p2) * 3]);
            for (int k2 = 0; k2 <= d; ++k2)
              for (int k1 = 0; k1 <= d; ++k1)
                B[(size_t)(p1 + G * p2) * nloc + k1 + D1 * k2] = rw[p1] * rw[p2] * o.h * o.h *
                                                                  bernstein_h(d, k1, rx[p1]) *
                                                                  bernstein_h(d, k2, rx[p2]);
          }
        std::vector<cplx> ex((size_t)nloc * nloc, cplx(0.0));
        for (int pp = 0; pp < G * G; ++pp)
          for (int qq = 0; qq < G * G; ++qq) {
            const cplx gv = green_h(o, &X[(size_t)pp * 3], &Y[(size_t)qq * 3]);
            for (int i = 0; i < nloc; ++i)
              for (int j = 0; j < nloc; ++j)
                ex[(size_t)i * nloc + j] += gv * B[(size_t)pp * nloc + i] * B[(size_t)qq * nloc + j];
          }
        for (int i = 0; i < nloc; ++i)
          for (int j = 0; j < nloc; ++j) {
            cplx ap(0.0);
            const int ri = pe * nloc + i, cj = pf * nloc + j;
            for (int b = 0; b < q2; ++b) ap += VK[(size_t)ri * q2 + b] * V[(size_t)cj * q2 + b];
            num += std::norm(ap - ex[(size_t)i * nloc + j]);
            den += std::norm(ex[(size_t)i * nloc + j]);
          }
      }
    if (den > 0) worst = std::max(worst, std::sqrt(num / den));
  }
  return worst;
}

// Largest relative error of the kernel interpolant sum_ab L_a(s) K_ab L_b(t) against
// G(gamma(s), gamma(t)) over 64 seeded point pairs of each sampled far block (blocks of
// any level, global cluster ids): the coarse levels hold the largest clusters, where an
// oscillating Helmholtz kernel is hardest to interpolate.  Relative to the block's
// largest |G| at the samples.
double kernel_interp_error(const Op& o, int q, const std::vector<std::pair<int, int>>& blocks) {
  const int q2 = q * q;
  double worst = 0.0;
  unsigned long long state = 0x9E3779B97F4A7C15ull;
  auto unif = [&]() {  // splitmix64 -> [0, 1)
    state += 0x9E3779B97F4A7C15ull;
    unsigned long long z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return double((z ^ (z >> 31)) >> 11) * 0x1.0p-53;
  };
  for (const auto& bl : blocks) {
    double pts[2][kMaxQ * kMaxQ * 3];
    int patch[2], lev[2];
    uint32_t jj[2][2];
    for (int side = 0; side < 2; ++side) {
      const int64_t c = side == 0 ? bl.first : bl.second;
      int l = 0;
      while (c >= o.lvl_off[l + 1]) ++l;
      lev[side] = l;
      const int64_t nper = int64_t(1) << (2 * l), loc = c - o.lvl_off[l];
      patch[side] = int(loc / nper);
      morton_decode(uint32_t(loc % nper), jj[side][0], jj[side][1]);
      const double H = std::ldexp(1.0, -l);
      for (int a2 = 0; a2 < q; ++a2)
        for (int a1 = 0; a1 < q; ++a1)
          gamma_eval(o.geom, patch[side], (jj[side][0] + chebyshev01(q, a1)) * H,
                     (jj[side][1] + chebyshev01(q, a2)) * H, &pts[side][(a1 + q * a2) * 3]);
    }
    std::vector<cplx> K((size_t)q2 * q2);
    for (int a = 0; a < q2; ++a)
      for (int b = 0; b < q2; ++b) K[(size_t)a * q2 + b] = green_h(o, &pts[0][a * 3], &pts[1][b * 3]);
    double num = 0.0, den = 0.0;
    for (int smp = 0; smp < 64; ++smp) {
      double u[2][2], x[2][3];
      std::vector<double> La[2];
      for (int side = 0; side < 2; ++side) {
        u[side][0] = unif();
        u[side][1] = unif();
        const double H = std::ldexp(1.0, -lev[side]);
        gamma_eval(o.geom, patch[side], (jj[side][0] + u[side][0]) * H, (jj[side][1] + u[side][1]) * H, x[side]);
        La[side].resize(q2);
        for (int a2 = 0; a2 < q; ++a2)
          for (int a1 = 0; a1 < q; ++a1)
            La[side][a1 + q * a2] = lagrange01(q, a1, u[side][0]) * lagrange01(q, a2, u[side][1]);
      }
      cplx ap(0.0);
      for (int a = 0; a < q2; ++a)
        for (int b = 0; b < q2; ++b) ap += La[0][a] * K[(size_t)a * q2 + b] * La[1][b];
      const cplx ex = green_h(o, x[0], x[1]);
      num = std::max(num, std::abs(ap - ex));
      den = std::max(den, std::abs(ex));
    }
    if (den > 0) worst = std::max(worst, num / den);
  }
  return worst;
}

}  // namespace

}  // namespace bembel

namespace bembel {

namespace {

// Device time of one product (mean of 5 after a warm-up), FP32 or FP64, one column.
double product_ms(Op& o, bool fp32) {
  const int C = o.cplx ? 2 : 1;
  const size_t el = fp32 ? sizeof(float) : sizeof(double);
  DevBuf x(el * o.ndofs * C), y(el * o.ndofs * C);
  cuda_check(cudaMemsetAsync(x.p, 0, el * o.ndofs * C, o.stream), "x");
  cudaEvent_t e0, e1;
  cuda_check(cudaEventCreate(&e0), "event");
  cuda_check(cudaEventCreate(&e1), "event");
  matvec_device(o, x.p, y.p, 1, fp32, o.stream);
  cuda_check(cudaEventRecord(e0, o.stream), "event");
  for (int it = 0; it < 5; ++it) matvec_device(o, x.p, y.p, 1, fp32, o.stream);
  cuda_check(cudaEventRecord(e1, o.stream), "event");
  cuda_check(cudaEventSynchronize(e1), "event");
  float ms = 0.f;
  cuda_check(cudaEventElapsedTime(&ms, e0, e1), "event");
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms / 5.0;
}

}  // namespace

// Leaf level and FP32 coupling storage by timing (inout->leaf_level < 0 only): operators
// with the chosen orders and q at leaf levels L-1 and L-2 are assembled, each scored by
// host set-up + assembly + kTunedProducts products (FP32 for MIXED, else FP64), and the
// cheapest is kept.  For MIXED operators the FP32 product of the chosen layout is then
// timed with the coupling evaluated on the fly and with a stored FP32 copy.
constexpr int kTunedProducts = 100;

static void choose_layout(bembel_geom* g, int op, double k_re, double k_im, int level, int p, int q, bembel_opts* inout,
                   bembel_tune_report& r) {
  r.leaf_level = inout->leaf_level < 0 ? (level > 0 ? level - 1 : 0) : inout->leaf_level;
  r.far_fp32_stored = inout->far_fp32_stored;
  if (inout->leaf_level >= 0 || level < 2 || q == 0) return;
  const bool mixed = inout->precision == BEMBEL_PREC_MIXED;
  double best = 1e300;
  int best_leaf = r.leaf_level;
  for (int c = 0; c < 2; ++c) {
    const int leaf = level - 1 - c;
    if (leaf < 1) break;
    bembel_opts o = *inout;
    o.leaf_level = leaf;
    o.far_fp32_stored = 0;
    bembel_op* h = nullptr;
    const int rc = bembel_assemble(g, op, k_re, k_im, level, p, q, &o, &h);
    if (rc == BEMBEL_ENOMEM || rc == BEMBEL_EINVAL) {
      r.leaf_score_ms[c] = -1.0;  // does not fit (memory, or the leaf moments in shared memory)
      continue;
    }
    if (rc != BEMBEL_OK) fail(rc, std::string("autotune: ") + bembel_last_error());
    try {
      Op& oc = *reinterpret_cast<Op*>(h);
      const double score = oc.info.setup_ms + oc.info.assemble_ms + kTunedProducts * product_ms(oc, mixed);
      r.leaf_score_ms[c] = score;
      if (score < best) {
        best = score;
        best_leaf = leaf;
      }
    } catch (...) {
      bembel_op_destroy(h);
      throw;
    }
    bembel_op_destroy(h);
  }
  r.leaf_level = best_leaf;
  inout->leaf_level = best_leaf;
  if (!mixed) return;
  bembel_opts o = *inout;
  bembel_op* h = nullptr;
  const int rc = bembel_assemble(g, op, k_re, k_im, level, p, q, &o, &h);
  if (rc != BEMBEL_OK) fail(rc, std::string("autotune: ") + bembel_last_error());
  try {
    Op& oc = *reinterpret_cast<Op*>(h);
    r.fp32_product_ms[0] = product_ms(oc, true);
    oc.opts.far_fp32_stored = 1;
    coupling_f32_prepare(oc, 1);
    r.fp32_product_ms[1] = oc.d_K32 ? product_ms(oc, true) : -1.0;
  } catch (...) {
    bembel_op_destroy(h);
    throw;
  }
  bembel_op_destroy(h);
  r.far_fp32_stored = (r.fp32_product_ms[1] > 0 && r.fp32_product_ms[1] < r.fp32_product_ms[0]) ? 1 : 0;
  inout->far_fp32_stored = r.far_fp32_stored;
}

int autotune_impl(bembel_geom* g, int op, double k_re, double k_im, int level, int p, double quad_tol,
                               double far_tol, int q_max, bembel_opts* inout, bembel_tune_report* rep) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!g || !inout || !(quad_tol > 0) || !(far_tol > 0) || q_max < 2 || q_max > kMaxQ)
    fail(BEMBEL_EINVAL, "autotune: NULL argument, non-positive tolerance or q_max outside [2, 8]");
  bembel_opts o = *inout;
  o.precision = BEMBEL_PREC_FP64;
  bembel_op* handle = nullptr;
  // sampling operator: interpolation order 2 keeps the coupling store small;
  // the block partition does not depend on q
  const int rc = bembel_assemble(g, op, k_re, k_im, level, p, 2, &o, &handle);
  if (rc != BEMBEL_OK) fail(rc, std::string("autotune: ") + bembel_last_error());
  Op& opr = *reinterpret_cast<Op*>(handle);
  bembel_tune_report r{};
  try {
    // quadrature orders per kind
    const int kinds[4] = {kRegular, kIdentical, kEdge, kVertex};
    int chosen[4] = {o.g_regular, o.g_singular, o.g_singular, o.g_singular};
    int chosen_var[4][4] = {};
    double errs[4] = {0, 0, 0, 0};
    int chosen_far = o.g_regular;
    double err_far_reg = 0.0;
    // separated pairs beyond the ring next to the touching pairs: own order
    if (opr.npairs_regular_far > 0) {
      std::vector<double> ref;
      for (int gg = 2; gg < kMaxG; ++gg) {
        const int g4[4] = {gg, gg, gg, gg};
        const double e = sample_pair_error(opr, kRegular, g4, kMaxG, 4096, &ref, 1);
        chosen_far = gg;
        err_far_reg = e;
        if (e <= quad_tol) break;
      }
    }
    for (int ki = 0; ki < 4; ++ki) {
      const int kind = kinds[ki];
      if (opr.npairs[kind] == 0) continue;
      const int g_ref = kMaxG;
      const int max_pairs = kind == kRegular ? 4096 : 512;
      const int cls = kind == kRegular ? 0 : -1;  // separated: the ring next to the touching pairs
      std::vector<double> ref;  // reference blocks at order g_ref, computed once per kind
      int best = kMaxG - 1;
      double err_best = 0.0;
      for (int gg = 2; gg < g_ref; ++gg) {
        const int g4[4] = {gg, gg, gg, gg};
        const double e = sample_pair_error(opr, kind, g4, g_ref, max_pairs, &ref, cls);
        best = gg;
        err_best = e;
        if (e <= quad_tol) break;
      }
      int gv[4] = {best, best, best, best};
      // Duffy rules: lower the orders of groups of variables in turn (the
      // variables along the element first: they are the smoothest) while the
      // sample still meets the target.  Groups keep the rule symmetric under
      // exchanging the two elements: identical (u1 u2) (eta) (xi); edge (u)
      // (eta1 eta2) (xi); vertex (eta1 eta2 eta3) (xi).
      if (kind != kRegular && err_best <= quad_tol) {
        static const unsigned groups[4][3] = {{0, 0, 0}, {0xC, 0x2, 0x1}, {0x8, 0x6, 0x1}, {0xE, 0x1, 0}};
        for (unsigned mask : groups[kind]) {
          if (!mask) continue;
          for (;;) {
            int lo = kMaxG;
            for (int v = 0; v < 4; ++v)
              if (mask >> v & 1) lo = std::min(lo, gv[v]);
            if (lo <= 2) break;
            for (int v = 0; v < 4; ++v)
              if (mask >> v & 1) --gv[v];
            const double e = sample_pair_error(opr, kind, gv, g_ref, max_pairs, &ref, cls);
            if (e <= quad_tol) {
              err_best = e;
            } else {
              for (int v = 0; v < 4; ++v)
                if (mask >> v & 1) ++gv[v];
              break;
            }
          }
        }
      }
      chosen[ki] = std::max(std::max(gv[0], gv[1]), std::max(gv[2], gv[3]));
      for (int v = 0; v < 4; ++v) chosen_var[ki][v] = gv[v];
      errs[ki] = err_best;
    }
    // interpolation order from sampled leaf-level far blocks
    int q_best = q_max;
    double far_err = 0.0;
    {
      std::vector<long long> ptr(opr.nclusters + 1);
      cuda_check(cudaMemcpy(ptr.data(), opr.d_far_ptr, sizeof(long long) * ptr.size(), cudaMemcpyDeviceToHost),
                 "far ptr");
      std::vector<int> src(opr.nfar);
      if (opr.nfar > 0)
        cuda_check(cudaMemcpy(src.data(), opr.d_far_src, sizeof(int) * opr.nfar, cudaMemcpyDeviceToHost), "far src");
      std::vector<std::pair<int, int>> blocks;
      const int64_t leaf_off = opr.lvl_off[opr.leaf];
      const int64_t nleaf = opr.nleaf;
      for (int64_t k = 0; k < 32; ++k) {
        const int64_t t = leaf_off + (k * 7919) % nleaf;
        const long long n = ptr[t + 1] - ptr[t];
        if (n == 0) continue;
        blocks.push_back({int(t), src[ptr[t] + (k * 31) % n]});
      }
      // far blocks of every level above the leaves: a few targets per level
      std::vector<std::pair<int, int>> coarse;
      for (int l = 0; l < opr.leaf; ++l) {
        const int64_t n_l = opr.lvl_off[l + 1] - opr.lvl_off[l];
        for (int64_t k = 0; k < 4; ++k) {
          const int64_t t = opr.lvl_off[l] + (k * 7919) % n_l;
          const long long n = ptr[t + 1] - ptr[t];
          if (n > 0) coarse.push_back({int(t), src[ptr[t] + (k * 31) % n]});
        }
      }
      if (!blocks.empty() || !coarse.empty()) {
        for (int qq = 2; qq <= q_max; ++qq) {
          far_err = std::max(blocks.empty() ? 0.0 : far_error(opr, qq, blocks),
                             coarse.empty() ? 0.0 : kernel_interp_error(opr, qq, coarse));
          q_best = qq;
          if (far_err <= far_tol) break;
        }
      }
    }
    // chunk size of the block-sparse products, by timing FP64 matvecs
    int best_chunk = 32;
    {
      const int C = opr.cplx ? 2 : 1;
      double* x = static_cast<double*>(dev_alloc(sizeof(double) * opr.ndofs * C));
      double* y = static_cast<double*>(dev_alloc(sizeof(double) * opr.ndofs * C));
      cuda_check(cudaMemset(x, 0, sizeof(double) * opr.ndofs * C), "x");
      cudaEvent_t e0, e1;
      cuda_check(cudaEventCreate(&e0), "event");
      cuda_check(cudaEventCreate(&e1), "event");
      float best_ms = 1e30f;
      const int cands[5] = {8, 16, 32, 64, 128};
      for (int ci = 0; ci < 5; ++ci) {
        opr.bsr_chunk = cands[ci];
        matvec_device(opr, x, y, 1, false, opr.stream);
        cuda_check(cudaEventRecord(e0, opr.stream), "event");
        for (int it = 0; it < 5; ++it) matvec_device(opr, x, y, 1, false, opr.stream);
        cuda_check(cudaEventRecord(e1, opr.stream), "event");
        cuda_check(cudaEventSynchronize(e1), "event");
        float ms = 0.f;
        cuda_check(cudaEventElapsedTime(&ms, e0, e1), "event");
        r.chunk_ms[ci] = ms / 5;
        if (ms < best_ms) {
          best_ms = ms;
          best_chunk = cands[ci];
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      dev_free(x);
      dev_free(y);
    }
    inout->g_regular = chosen[0];
    inout->g_regular_far = chosen_far;
    r.g_regular_far = chosen_far;
    r.err_regular_far = err_far_reg;
    inout->g_identical = chosen[1];
    inout->g_edge = chosen[2];
    inout->g_vertex = chosen[3];
    for (int v = 0; v < 4; ++v) {
      inout->g_identical_var[v] = r.g_identical_var[v] = chosen_var[1][v];
      inout->g_edge_var[v] = r.g_edge_var[v] = chosen_var[2][v];
      inout->g_vertex_var[v] = r.g_vertex_var[v] = chosen_var[3][v];
    }
    inout->g_singular = std::max(chosen[1], std::max(chosen[2], chosen[3]));
    inout->bsr_chunk = best_chunk;
    r.g_regular = chosen[0];
    r.g_identical = chosen[1];
    r.g_edge = chosen[2];
    r.g_vertex = chosen[3];
    r.q = q_best;
    r.bsr_chunk = best_chunk;
    r.err_regular = errs[0];
    r.err_identical = errs[1];
    r.err_edge = errs[2];
    r.err_vertex = errs[3];
    r.err_far = far_err;
  } catch (...) {
    bembel_op_destroy(handle);  // release the sampling operator, then report the error
    throw;
  }
  bembel_op_destroy(handle);
  choose_layout(g, op, k_re, k_im, level, p, r.q, inout, r);
  r.tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (rep) *rep = r;
  return BEMBEL_OK;
}

}  // namespace bembel
