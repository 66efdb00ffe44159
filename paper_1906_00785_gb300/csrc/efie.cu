// efie.cu - electric field integral equation on the S^1 space (App. B (MS),
// App. E).
//
// Galerkin form (the kappa^-2 gradient term of (MS) moved onto the test
// function by surface integration by parts):
//   a(j, mu) = int int G(x,y) [ j(y) . mu(x) - kappa^-2 div j(y) div mu(x) ],
//   G = exp(-i kappa r) / (4 pi r),
// with the perfectly conducting boundary condition of (MP) as
//   a(j, mu) = -int E_inc . mu.
// The div-conforming Piola lift j = D gamma phi_hat / |d1 gamma x d2 gamma|,
// div j = div phi_hat / |...| cancels every surface measure, so an element pair
// contributes
//   h^4 sum_k W_k G(x_k, y_k) [ (d_alpha gamma(s_k) . d_beta gamma(t_k)) b_i(s_k) b_j(t_k)
//                               - kappa^-2 d_i(s_k) d_j(t_k) ]
// for element-local functions i of component alpha and j of component beta,
// b = the Bernstein product of the function, d = its parameter divergence.
// Quadrature: the same element-pair rules as the scalar operators (tensor
// Gauss on separated pairs, the Duffy-type rules on touching ones; identical
// pairs use all 8 sub-domains).  One warp per pair, lanes over rule points; the
// 2 x 2 component quadrants of the block are accumulated one after the other so
// the accumulators stay in registers.
//
// Geometry: the cube-face sphere (analytic Jacobian).
#include <vector>

#include "op.h"
#include "pairrules.cuh"

namespace bembel {

namespace {

constexpr int kEfieWarps = 4;

// Bernstein values and derivatives d/du of degree D at u
template <int D>
__device__ __forceinline__ void bern_d(double u, double b[D + 1], double db[D + 1]) {
  const double v = 1.0 - u;
  if (D == 0) {
    b[0] = 1.0;
    db[0] = 0.0;
  } else if (D == 1) {
    b[0] = v;
    b[1] = u;
    db[0] = -1.0;
    db[1] = 1.0;
  } else if (D == 2) {
    b[0] = v * v;
    b[1] = 2.0 * u * v;
    b[2] = u * u;
    db[0] = -2.0 * v;
    db[1] = 2.0 * (v - u);
    db[2] = 2.0 * u;
  } else {
    // degree D from degree D - 1 (de Casteljau's recursion b_k = u b'_{k-1} + v b'_k of the
    // degree-(D-1) values b'); derivative D (b'_{k-1} - b'_k)
    double lo[D + 1];
    lo[0] = 1.0;
    for (int r = 1; r < D; ++r) {
      lo[r] = u * lo[r - 1];
      for (int k = r - 1; k >= 1; --k) lo[k] = u * lo[k - 1] + v * lo[k];
      lo[0] = v * lo[0];
    }
    for (int k = 0; k <= D; ++k) {
      const double left = k >= 1 ? lo[k - 1] : 0.0, right = k <= D - 1 ? lo[k] : 0.0;
      b[k] = u * left + v * right;
      db[k] = D * (left - right);
    }
  }
}

// 1-D factors of component comp (0: degree P in the first parameter, P-1 in
// the second; 1: the reverse) at local (u, v):
//   values fa (first parameter) x fb (second), divergence factor dfa x fb or fa x dfb.
template <int P>
struct Comp1D {
  double a[P + 1], da[P + 1], b[P + 1], db[P + 1];
};

template <int P>
__device__ __forceinline__ void comp_factors(int comp, double u, double v, Comp1D<P>& f) {
  // component 0: a = degree P in u, b = degree P-1 in v; component 1: a = degree P-1 in u, b = degree P in v
  double hb[P + 1], hd[P + 1], lb[P], ld[P];
  if (comp == 0) {
    bern_d<P>(u, hb, hd);
    bern_d<P - 1>(v, lb, ld);
    for (int k = 0; k <= P; ++k) {
      f.a[k] = hb[k];
      f.da[k] = hd[k];
    }
    for (int k = 0; k < P; ++k) {
      f.b[k] = lb[k];
      f.db[k] = 0.0;
    }
  } else {
    bern_d<P - 1>(u, lb, ld);
    bern_d<P>(v, hb, hd);
    for (int k = 0; k < P; ++k) {
      f.a[k] = lb[k];
      f.da[k] = 0.0;
    }
    for (int k = 0; k <= P; ++k) {
      f.b[k] = hb[k];
      f.db[k] = hd[k];
    }
  }
}

// value b and divergence factor d (d/du or d/dv on the local square) of local
// function n (0 <= n < P (P+1)) of component comp
template <int P>
__device__ __forceinline__ void comp_fun(int comp, int n, const Comp1D<P>& f, double& b, double& d) {
  if (comp == 0) {  // k1 <= P (first), k2 < P (second)
    const int k1 = n % (P + 1), k2 = n / (P + 1);
    b = f.a[k1] * f.b[k2];
    d = f.da[k1] * f.b[k2];
  } else {  // k1 < P, k2 <= P
    const int k1 = n % P, k2 = n / P;
    b = f.a[k1] * f.b[k2];
    d = f.a[k1] * f.db[k2];
  }
}

template <int P, int KIND>
__global__ void __launch_bounds__(32 * kEfieWarps) k_efie_pairs(const PairRec* __restrict__ pairs, int64_t npairs,
                                                                int L, int4 G, const double* __restrict__ gauss,
                                                                double kre, double kim, double* __restrict__ N,
                                                                int nld) {
  constexpr int NH = P * (P + 1);  // local functions per component
  constexpr int NSUB = KIND == kIdentical ? 8 : (KIND == kEdge ? 6 : (KIND == kVertex ? 4 : 1));
  __shared__ double gx[4][kMaxG], gw[4][kMaxG];
  load_rule_tables(gauss, G, gx, gw);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int npts = NSUB * G.x * G.y * G.z * G.w;
  const int64_t per = int64_t(1) << (2 * L);
  const double h = ldexp(1.0, -L);
  const double hinv = 1.0 / h;
  // -kappa^-2
  const double kk_r = kre * kre - kim * kim, kk_i = 2.0 * kre * kim;
  const double kk_n = kk_r * kk_r + kk_i * kk_i;
  const double cr = -kk_r / kk_n, ci = kk_i / kk_n;
  for (int64_t w = blockIdx.x * (int64_t)kEfieWarps + (threadIdx.x >> 5); w < npairs;
       w += (int64_t)gridDim.x * kEfieWarps) {
    const PairRec pr = pairs[w];
    const int pe = int(pr.e / per), pf = int(pr.f / per);
    uint32_t e1, e2, f1, f2;
    morton_decode(uint32_t(pr.e % per), e1, e2);
    morton_decode(uint32_t(pr.f % per), f1, f2);
    const int ce = (pr.code >> 2) & 7, cf = (pr.code >> 5) & 7;
    // rows of the (NH x NH) quadrant block in passes of IB rows: the accumulators
    // stay in registers for P = 3 (NH = 12) at the price of re-evaluating the kernel
    constexpr int IB = P <= 2 ? NH : 4;
    for (int pass = 0; pass < 4 * (NH / IB); ++pass) {
      const int quad = pass % 4, ib0 = (pass / 4) * IB;
      const int al = quad & 1, be = quad >> 1;
      double ar[IB * NH], ai[IB * NH];
#pragma unroll
      for (int k = 0; k < IB * NH; ++k) ar[k] = ai[k] = 0.0;
      for (int idx = lane; idx < npts; idx += 32) {
        int sub, i0, i1, i2, i3;
        rule_index(idx, G, sub, i0, i1, i2, i3);
        double ls1, ls2, lt1, lt2, wt;
        const double w4 = gw[0][i0] * gw[1][i1] * gw[2][i2] * gw[3][i3];
        if (KIND == kRegular) {
          ls1 = gx[0][i0];
          ls2 = gx[1][i1];
          lt1 = gx[2][i2];
          lt2 = gx[3][i3];
          wt = w4;
        } else {
          double s1, s2, t1, t2;
          const double jac = duffy_point<KIND == kRegular ? kIdentical : KIND>(sub, gx[0][i0], gx[1][i1], gx[2][i2],
                                                                                gx[3][i3], s1, s2, t1, t2);
          wt = jac * w4;
          apply_cmap(ce, s1, s2, ls1, ls2);
          apply_cmap(cf, t1, t2, lt1, lt2);
        }
        double x[3], xs[3], xt[3], y[3], ys[3], yt[3];
        sphere6_jac(pe, (e1 + ls1) * h, (e2 + ls2) * h, x, xs, xt);
        sphere6_jac(pf, (f1 + lt1) * h, (f2 + lt2) * h, y, ys, yt);
        const double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
        double gr, gi;
        kernel_value(true, d0 * d0 + d1 * d1 + d2 * d2, kre, kim, gr, gi);
        gr *= wt;
        gi *= wt;
        const double* ja = al == 0 ? xs : xt;
        const double* jb = be == 0 ? ys : yt;
        const double g = ja[0] * jb[0] + ja[1] * jb[1] + ja[2] * jb[2];
        // P = G g (vector part), Q = -kappa^-2 G / h^2 (divergence part; d/du -> d/ds)
        const double Pr = gr * g, Pi = gi * g;
        const double Qr = (gr * cr - gi * ci) * hinv * hinv, Qi = (gr * ci + gi * cr) * hinv * hinv;
        Comp1D<P> fs, ft;
        comp_factors<P>(al, ls1, ls2, fs);
        comp_factors<P>(be, lt1, lt2, ft);
#pragma unroll
        for (int ii = 0; ii < IB; ++ii) {
          double bi, di;
          comp_fun<P>(al, ib0 + ii, fs, bi, di);
#pragma unroll
          for (int j = 0; j < NH; ++j) {
            double bj, dj;
            comp_fun<P>(be, j, ft, bj, dj);
            const double bb = bi * bj, dd = di * dj;
            ar[ii * NH + j] = fma(Pr, bb, fma(Qr, dd, ar[ii * NH + j]));
            ai[ii * NH + j] = fma(Pi, bb, fma(Qi, dd, ai[ii * NH + j]));
          }
        }
      }
#pragma unroll
      for (int k = 0; k < IB * NH; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          ar[k] += __shfl_xor_sync(0xffffffffu, ar[k], o);
          ai[k] += __shfl_xor_sync(0xffffffffu, ai[k], o);
        }
      }
      const double sc = kInv4Pi * h * h * h * h;
      const int io = al * NH + ib0, jo = be * NH;
#pragma unroll
      for (int k = 0; k < IB * NH; ++k) {
        if ((k & 31) != lane) continue;
        const int i = io + k / NH, j = jo + k % NH;
        const long long o1 = pr.off1 + (long long)i * nld + j;
        N[o1 * 2] = ar[k] * sc;
        N[o1 * 2 + 1] = ai[k] * sc;
        if (pr.off2 >= 0) {
          const long long o2 = pr.off2 + (long long)j * nld + i;
          N[o2 * 2] = ar[k] * sc;
          N[o2 * 2 + 1] = ai[k] * sc;
        }
      }
    }
  }
}

// Load vectors b_loc[e, i][rhs] = -h^2 sum_q w_q E_inc(x_q) . (d_alpha gamma(q) b_i(q)),
// E_inc = pol exp(-i kappa dir . x).  One thread per (element, rhs).
template <int P>
__global__ void k_efie_rhs_local(int L, int64_t nelem, int G, const double* __restrict__ gx,
                                 const double* __restrict__ gw, const double* __restrict__ prm, int nrhs, double kre,
                                 double kim, double* __restrict__ bl) {
  constexpr int NH = P * (P + 1), NLOC = 2 * NH;
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= nelem * nrhs) return;
  const int64_t e = id / nrhs;
  const int r = int(id % nrhs);
  const int64_t per = int64_t(1) << (2 * L);
  const int patch = int(e / per);
  uint32_t i1, i2;
  morton_decode(uint32_t(e % per), i1, i2);
  const double h = ldexp(1.0, -L);
  const double* pp = prm + 6 * r;
  double accr[NLOC], acci[NLOC];
  for (int k = 0; k < NLOC; ++k) accr[k] = acci[k] = 0.0;
  for (int b = 0; b < G; ++b)
    for (int a = 0; a < G; ++a) {
      const double u = gx[a], v = gx[b];
      double x[3], xs[3], xt[3];
      sphere6_jac(patch, (i1 + u) * h, (i2 + v) * h, x, xs, xt);
      // exp(-i kappa d.x) = exp(kim d.x) (cos(kre d.x) - i sin(kre d.x))
      const double dx = pp[0] * x[0] + pp[1] * x[1] + pp[2] * x[2];
      double sn, cs;
      sincos(kre * dx, &sn, &cs);
      const double am = exp(kim * dx) * gw[a] * gw[b] * h * h;
      const double er = am * cs, ei = -am * sn;
      const double ps = pp[3] * xs[0] + pp[4] * xs[1] + pp[5] * xs[2];  // pol . d_s gamma
      const double pt = pp[3] * xt[0] + pp[4] * xt[1] + pp[5] * xt[2];
      for (int comp = 0; comp < 2; ++comp) {
        Comp1D<P> f;
        comp_factors<P>(comp, u, v, f);
        const double pj = comp == 0 ? ps : pt;
        for (int n = 0; n < NH; ++n) {
          double bv, dv;
          comp_fun<P>(comp, n, f, bv, dv);
          accr[comp * NH + n] -= er * pj * bv;
          acci[comp * NH + n] -= ei * pj * bv;
        }
      }
    }
  const int ncol = 2 * nrhs;
  for (int k = 0; k < NLOC; ++k) {
    bl[(e * NLOC + k) * ncol + 2 * r] = accr[k];
    bl[(e * NLOC + k) * ncol + 2 * r + 1] = acci[k];
  }
}

// Per element quadrature point: position, the current D gamma phi (3 complex)
// and the divergence (1 complex), weights included, for every rhs.
template <int P>
__global__ void k_efie_density(const double* __restrict__ rl, int L, int64_t nelem, int G,
                               const double* __restrict__ gx, const double* __restrict__ gw, int nrhs,
                               double* __restrict__ Y, double* __restrict__ J) {
  constexpr int NH = P * (P + 1), NLOC = 2 * NH;
  const int G2 = G * G;
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= nelem * G2) return;
  const int64_t e = id / G2;
  const int q = int(id % G2);
  const int64_t per = int64_t(1) << (2 * L);
  const int patch = int(e / per);
  uint32_t i1, i2;
  morton_decode(uint32_t(e % per), i1, i2);
  const double h = ldexp(1.0, -L);
  const double u = gx[q % G], v = gx[q / G];
  double x[3], xs[3], xt[3];
  sphere6_jac(patch, (i1 + u) * h, (i2 + v) * h, x, xs, xt);
  Y[id * 3] = x[0];
  Y[id * 3 + 1] = x[1];
  Y[id * 3 + 2] = x[2];
  const double wq = gw[q % G] * gw[q / G] * h * h;
  const int ncol = 2 * nrhs;
  Comp1D<P> f0, f1;
  comp_factors<P>(0, u, v, f0);
  comp_factors<P>(1, u, v, f1);
  for (int r = 0; r < nrhs; ++r) {
    double js_r = 0, js_i = 0, jt_r = 0, jt_i = 0, dv_r = 0, dv_i = 0;
    for (int k = 0; k < NLOC; ++k) {
      const int comp = k / NH, n = k % NH;
      double bv, dvv;
      comp_fun<P>(comp, n, comp == 0 ? f0 : f1, bv, dvv);
      const double cr = rl[(e * NLOC + k) * ncol + 2 * r], ci = rl[(e * NLOC + k) * ncol + 2 * r + 1];
      if (comp == 0) {
        js_r += bv * cr;
        js_i += bv * ci;
      } else {
        jt_r += bv * cr;
        jt_i += bv * ci;
      }
      dv_r += dvv * cr;
      dv_i += dvv * ci;
    }
    double* out = J + (id * nrhs + r) * 8;
    for (int c = 0; c < 3; ++c) {
      out[2 * c] = wq * (xs[c] * js_r + xt[c] * jt_r);
      out[2 * c + 1] = wq * (xs[c] * js_i + xt[c] * jt_i);
    }
    out[6] = wq * dv_r / h;  // divergence in patch parameters (d/du = h d/ds)
    out[7] = wq * dv_i / h;
  }
}

// Block per (evaluation point, rhs): E(x) = sum_k G (D gamma phi)_k + kappa^-2 grad_x G (div phi)_k,
// grad_x G = G (-i kappa - 1/r) (x - y) / r.
__global__ void k_efie_field(const double* __restrict__ pts, const double* __restrict__ Y,
                             const double* __restrict__ J, int64_t nsrc, int nrhs, double kre, double kim,
                             double* __restrict__ out, int64_t npts) {
  const int64_t ip = blockIdx.x;
  const int r = blockIdx.y;
  const double x0 = pts[ip * 3], x1 = pts[ip * 3 + 1], x2 = pts[ip * 3 + 2];
  // 1 / kappa^2
  const double kk_r = kre * kre - kim * kim, kk_i = 2.0 * kre * kim;
  const double kk_n = kk_r * kk_r + kk_i * kk_i;
  const double ikr = kk_r / kk_n, iki = -kk_i / kk_n;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t k = threadIdx.x; k < nsrc; k += blockDim.x) {
    const double d[3] = {x0 - Y[k * 3], x1 - Y[k * 3 + 1], x2 - Y[k * 3 + 2]};
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double rinv = rsqrt(r2);
    const double rr = r2 * rinv;
    double sn, cs;
    sincos(kre * rr, &sn, &cs);
    const double am = exp(kim * rr) * rinv * kInv4Pi;
    const double gr = am * cs, gi = -am * sn;
    // factor (-i kappa - 1/r) / r
    const double fr = (kim - rinv) * rinv, fi = -kre * rinv;
    const double hr = gr * fr - gi * fi, hi = gr * fi + gi * fr;  // G (-i kappa - 1/r) / r
    const double* jj = J + (k * nrhs + r) * 8;
    // kappa^-2 * div
    const double qr = ikr * jj[6] - iki * jj[7], qi = ikr * jj[7] + iki * jj[6];
    const double tr = hr * qr - hi * qi, ti = hr * qi + hi * qr;
    for (int c = 0; c < 3; ++c) {
      acc[2 * c] += gr * jj[2 * c] - gi * jj[2 * c + 1] + tr * d[c];
      acc[2 * c + 1] += gr * jj[2 * c + 1] + gi * jj[2 * c] + ti * d[c];
    }
  }
  __shared__ double red[6][32];
  for (int c = 0; c < 6; ++c)
    for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
    for (int c = 0; c < 6; ++c) red[c][wid] = acc[c];
  __syncthreads();
  if (threadIdx.x < 6) {
    double s = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
    out[((int64_t)r * npts + ip) * 6 + threadIdx.x] = s;
  }
}

int4 orders(const Op& o, int kind) {
  return make_int4(o.g_var[kind][0], o.g_var[kind][1], o.g_var[kind][2], o.g_var[kind][3]);
}

// Far-field coupling of the compressed EFIE, per far block and cluster points
// (a, b): K[blk][c][b][a] = G(x_a, y_b) d_alpha gamma(x_a) . d_beta gamma(y_b)
// for c = 2 alpha + beta (alpha, beta: 0 = d_s, 1 = d_t) and K[blk][4][b][a] =
// -kappa^-2 G(x_a, y_b); complex interleaved, G with its 1/(4 pi).  Stored with the
// target point a fastest, so the product's threads (one per a) read consecutive words.
__global__ void k_efie_coupling(const int* __restrict__ tgt, const int* __restrict__ src, int64_t nfar,
                                const double* __restrict__ nodes, const double* __restrict__ jac, int q2, double kre,
                                double kim, double* __restrict__ K) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)q2 * q2;
  if (id >= nfar * per) return;
  const int64_t blk = id / per;
  const int b = int(id % per) / q2, a = int(id % per) % q2;
  const int64_t pa = (int64_t)tgt[blk] * q2 + a, pb = (int64_t)src[blk] * q2 + b;
  const double* xa = nodes + pa * 3;
  const double* xb = nodes + pb * 3;
  const double* Ja = jac + pa * 6;
  const double* Jb = jac + pb * 6;
  const double d0 = xa[0] - xb[0], d1 = xa[1] - xb[1], d2 = xa[2] - xb[2];
  double gr, gi;
  kernel_value(true, d0 * d0 + d1 * d1 + d2 * d2, kre, kim, gr, gi);
  gr *= kInv4Pi;
  gi *= kInv4Pi;
  const double kk_r = kre * kre - kim * kim, kk_i = 2.0 * kre * kim, kk_n = kk_r * kk_r + kk_i * kk_i;
  const double cr = -kk_r / kk_n, ci = kk_i / kk_n;  // -kappa^-2
  double* out = K + ((blk * 5) * per + (int64_t)b * q2 + a) * 2;
  for (int al = 0; al < 2; ++al)
    for (int be = 0; be < 2; ++be) {
      const double g = Ja[3 * al] * Jb[3 * be] + Ja[3 * al + 1] * Jb[3 * be + 1] + Ja[3 * al + 2] * Jb[3 * be + 2];
      out[(2 * al + be) * per * 2] = gr * g;
      out[(2 * al + be) * per * 2 + 1] = gi * g;
    }
  out[4 * per * 2] = gr * cr - gi * ci;
  out[4 * per * 2 + 1] = gr * ci + gi * cr;
}

// yh[t][a][co ncol + 2r] += sum over far blocks (t, s), points b and input channels:
// output channels 0, 1 (the two components) couple with input channels 0, 1 through
// K[0..3], channel 2 (the divergence) with channel 2 through K[4].  One thread per
// (chunk of kEfieChunk consecutive far blocks, rhs, a), a fastest: the coupling words of
// consecutive threads are consecutive (K[blk][c][b][a]) and the source moments are the
// same for the whole group.  The far list is ordered by target: partial sums are flushed
// with atomics when the target changes inside a chunk and at its end (yh cleared before).
constexpr int kEfieChunk = 8;

template <typename T>
__global__ void k_efie_coupling_mv(const int* __restrict__ ftgt, const int* __restrict__ fsrc, int64_t nfar,
                                   const T* __restrict__ K, int q2, const T* __restrict__ xh, T* __restrict__ yh,
                                   int nrhs) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nchunk = (nfar + kEfieChunk - 1) / kEfieChunk;
  if (id >= nchunk * q2 * nrhs) return;
  const int a = int(id % q2);
  const int r = int((id / q2) % nrhs);
  const int64_t c = id / ((int64_t)q2 * nrhs);
  const int ncol = 2 * nrhs, ncolh = 3 * ncol;
  const int64_t per = (int64_t)q2 * q2;
  T acc[6] = {0, 0, 0, 0, 0, 0};  // (re, im) of the three output channels
  int cur = -1;
  auto flush = [&]() {
    T* y = yh + ((int64_t)cur * q2 + a) * ncolh + 2 * r;
#pragma unroll
    for (int co = 0; co < 3; ++co) {
      atomicAdd(y + co * ncol, acc[2 * co]);
      atomicAdd(y + co * ncol + 1, acc[2 * co + 1]);
      acc[2 * co] = acc[2 * co + 1] = 0;
    }
  };
  const int64_t k1 = min(nfar, (c + 1) * kEfieChunk);
  for (int64_t k = c * kEfieChunk; k < k1; ++k) {
    const int t = ftgt[k];
    if (t != cur) {
      if (cur >= 0) flush();
      cur = t;
    }
    const int64_t sc = fsrc[k];
    const T* Kb = K + k * 5 * per * 2 + (int64_t)a * 2;
    const T* xs = xh + sc * q2 * ncolh + 2 * r;
    for (int b = 0; b < q2; ++b) {
      const T* xb = xs + (int64_t)b * ncolh;
      const T x0r = xb[0], x0i = xb[1], x1r = xb[ncol], x1i = xb[ncol + 1], x2r = xb[2 * ncol], x2i = xb[2 * ncol + 1];
      const T* kb = Kb + (int64_t)b * q2 * 2;
#pragma unroll
      for (int co = 0; co < 2; ++co) {
        const T* k0 = kb + (int64_t)(2 * co) * per * 2;
        const T* k1p = kb + (int64_t)(2 * co + 1) * per * 2;
        acc[2 * co] += k0[0] * x0r - k0[1] * x0i + k1p[0] * x1r - k1p[1] * x1i;
        acc[2 * co + 1] += k0[0] * x0i + k0[1] * x0r + k1p[0] * x1i + k1p[1] * x1r;
      }
      const T* k4 = kb + (int64_t)4 * per * 2;
      acc[4] += k4[0] * x2r - k4[1] * x2i;
      acc[5] += k4[0] * x2i + k4[1] * x2r;
    }
  }
  if (cur >= 0) flush();
}

template <int P>
void launch_efie_pairs(Op& o, cudaEvent_t* ev) {
  const cudaStream_t s = o.stream;
  const int threads = 32 * kEfieWarps;
  auto grid_of = [](int64_t n) { return int(std::max<int64_t>(1, std::min<int64_t>((n + kEfieWarps - 1) / kEfieWarps, 152 * 64))); };
  if (o.npairs[kRegular] > 0) {
    k_efie_pairs<P, kRegular><<<grid_of(o.npairs[kRegular]), threads, 0, s>>>(
        o.d_pairs[kRegular], o.npairs[kRegular], o.L, orders(o, kRegular), o.d_gauss + o.gauss_off[kRegular], o.kre, o.kim, o.d_N, o.nld);
    launched("k_efie_pairs regular");
  }
  cuda_check(cudaEventRecord(ev[2], s), "event");
  if (o.npairs[kIdentical] > 0) {
    k_efie_pairs<P, kIdentical><<<grid_of(o.npairs[kIdentical]), threads, 0, s>>>(
        o.d_pairs[kIdentical], o.npairs[kIdentical], o.L, orders(o, kIdentical), o.d_gauss + o.gauss_off[kIdentical],
        o.kre, o.kim, o.d_N, o.nld);
    launched("k_efie_pairs identical");
  }
  cuda_check(cudaEventRecord(ev[3], s), "event");
  if (o.npairs[kEdge] > 0) {
    k_efie_pairs<P, kEdge><<<grid_of(o.npairs[kEdge]), threads, 0, s>>>(
        o.d_pairs[kEdge], o.npairs[kEdge], o.L, orders(o, kEdge), o.d_gauss + o.gauss_off[kEdge], o.kre, o.kim,
        o.d_N, o.nld);
    launched("k_efie_pairs edge");
  }
  cuda_check(cudaEventRecord(ev[4], s), "event");
  if (o.npairs[kVertex] > 0) {
    k_efie_pairs<P, kVertex><<<grid_of(o.npairs[kVertex]), threads, 0, s>>>(
        o.d_pairs[kVertex], o.npairs[kVertex], o.L, orders(o, kVertex), o.d_gauss + o.gauss_off[kVertex], o.kre,
        o.kim, o.d_N, o.nld);
    launched("k_efie_pairs vertex");
  }
  cuda_check(cudaEventRecord(ev[5], s), "event");
}

}  // namespace

void efie_pair_kernels(Op& o, cudaEvent_t* ev) {
  if (o.d == 1)
    launch_efie_pairs<1>(o, ev);
  else if (o.d == 2)
    launch_efie_pairs<2>(o, ev);
  else
    launch_efie_pairs<3>(o, ev);
}

void efie_coupling_assemble(Op& o) {
  const int64_t n = o.nfar * (int64_t)o.q2 * o.q2;
  if (n == 0) return;
  k_efie_coupling<<<int((n + 255) / 256), 256, 0, o.stream>>>(o.d_far_tgt, o.d_far_src, o.nfar, o.d_nodes,
                                                              o.d_nodes_jac, o.q2, o.kre, o.kim, o.d_K);
  launched("k_efie_coupling");
}

void efie_coupling_apply(const Op& o, const double* xh, double* yh, int nrhs, cudaStream_t s) {
  cuda_check(cudaMemsetAsync(yh, 0, sizeof(double) * o.nclusters * o.q2 * 6 * nrhs, s), "efie yh clear");
  const int64_t n = (o.nfar + kEfieChunk - 1) / kEfieChunk * o.q2 * nrhs;
  if (n == 0) return;
  k_efie_coupling_mv<double><<<int((n + 127) / 128), 128, 0, s>>>(o.d_far_tgt, o.d_far_src, o.nfar, o.d_K, o.q2, xh,
                                                                  yh, nrhs);
  launched("k_efie_coupling_mv");
}

void efie_coupling_apply(const Op& o, const float* xh, float* yh, int nrhs, cudaStream_t s) {
  if (!o.d_K32) fail(BEMBEL_EINVAL, "compressed EFIE: the FP32 product needs an operator assembled MIXED");
  cuda_check(cudaMemsetAsync(yh, 0, sizeof(float) * o.nclusters * o.q2 * 6 * nrhs, s), "efie yh clear");
  const int64_t n = (o.nfar + kEfieChunk - 1) / kEfieChunk * o.q2 * nrhs;
  if (n == 0) return;
  k_efie_coupling_mv<float><<<int((n + 127) / 128), 128, 0, s>>>(o.d_far_tgt, o.d_far_src, o.nfar, o.d_K32, o.q2, xh,
                                                                 yh, nrhs);
  launched("k_efie_coupling_mv");
}

void efie_rhs_local(const Op& o, const double* gx, const double* gw, int G, const double* prm_dev, int nrhs,
                    double* bl, cudaStream_t s) {
  const int64_t n = o.nelem * nrhs;
  const int grid = int((n + 127) / 128);
  if (o.d == 1)
    k_efie_rhs_local<1><<<grid, 128, 0, s>>>(o.L, o.nelem, G, gx, gw, prm_dev, nrhs, o.kre, o.kim, bl);
  else if (o.d == 2)
    k_efie_rhs_local<2><<<grid, 128, 0, s>>>(o.L, o.nelem, G, gx, gw, prm_dev, nrhs, o.kre, o.kim, bl);
  else
    k_efie_rhs_local<3><<<grid, 128, 0, s>>>(o.L, o.nelem, G, gx, gw, prm_dev, nrhs, o.kre, o.kim, bl);
  launched("k_efie_rhs_local");
}

void efie_field(const Op& o, const double* rl, const double* gx, const double* gw, int G, const double* pts,
                int64_t npts, int nrhs, double* out, cudaStream_t s) {
  const int64_t nq = o.nelem * G * G;
  DevBuf Y(sizeof(double) * nq * 3), J(sizeof(double) * nq * nrhs * 8);
  const int grid = int((nq + 127) / 128);
  if (o.d == 1)
    k_efie_density<1><<<grid, 128, 0, s>>>(rl, o.L, o.nelem, G, gx, gw, nrhs, static_cast<double*>(Y.p),
                                           static_cast<double*>(J.p));
  else if (o.d == 2)
    k_efie_density<2><<<grid, 128, 0, s>>>(rl, o.L, o.nelem, G, gx, gw, nrhs, static_cast<double*>(Y.p),
                                           static_cast<double*>(J.p));
  else
    k_efie_density<3><<<grid, 128, 0, s>>>(rl, o.L, o.nelem, G, gx, gw, nrhs, static_cast<double*>(Y.p),
                                           static_cast<double*>(J.p));
  launched("k_efie_density");
  if (npts > 0) {
    k_efie_field<<<dim3(unsigned(npts), unsigned(nrhs)), 256, 0, s>>>(
        pts, static_cast<double*>(Y.p), static_cast<double*>(J.p), nq, nrhs, o.kre, o.kim, out, npts);
    launched("k_efie_field");
  }
  cuda_check(cudaStreamSynchronize(s), "efie field sync");
}

}  // namespace bembel
