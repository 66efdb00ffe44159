// pairkernels.cuh - per-pair device functions of the near-field and coupling
// assembly, shared by the single-mesh kernels (quad.cu) and the persistent
// multi-mesh kernel (quad_batch.cu).
#pragma once

#include <algorithm>

#include "op.h"
#include "pairrules.cuh"

namespace bembel {

namespace {

constexpr int kWarps = 4;  // warps per block in the pair kernels

// gamma at regular point id = e * G^2 + p of element e
__device__ __forceinline__ void tabulate_point(const Geom& g, int L, int G, const double* __restrict__ gx, double h,
                                               int64_t id, double* __restrict__ Xq) {
  const int G2 = G * G;
  const int64_t e = id / G2;
  const int p = int(id % G2);
  const int64_t per = int64_t(1) << (2 * L);
  uint32_t i1, i2;
  morton_decode(uint32_t(e % per), i1, i2);
  double x[3];
  gamma_eval(g, int(e / per), (i1 + gx[p % G]) * h, (i2 + gx[p / G]) * h, x);
  Xq[id * 3 + 0] = x[0];
  Xq[id * 3 + 1] = x[1];
  Xq[id * 3 + 2] = x[2];
}

// One separated pair per warp: u_p[j] = sum_q G(x_p, y_q) BW[q][j] per point p
// of e, then block[i][j] = sum_p BW[p][i] u_p[j] / (4 pi).  BW: G2 x NL table
// (basis x weight at the regular points), ubuf: this warp's G2 * NL * C scratch.
template <int D, bool CPLX>
__device__ __forceinline__ void regular_pair(const PairRec& pr, const double* __restrict__ Xq,
                                             const double* __restrict__ BW, double* __restrict__ ubuf, int G2,
                                             double kre, double kim, double* __restrict__ N, int nld, int lane) {
  constexpr int NL = (D + 1) * (D + 1);
  constexpr int C = CPLX ? 2 : 1;
  const int S = G2 <= 16 ? 2 : 1;      // lanes per point p
  const int P = 32 / S;                // points handled per sweep
  const int half = lane / P;
  const int qlen = (G2 + S - 1) / S;
  const double* xe = Xq + (int64_t)pr.e * G2 * 3;
  const double* xf = Xq + (int64_t)pr.f * G2 * 3;
  for (int p0 = 0; p0 < G2; p0 += P) {
    const int p = p0 + (lane % P);
    double ur[NL], ui[NL];
#pragma unroll
    for (int j = 0; j < NL; ++j) ur[j] = ui[j] = 0.0;
    if (p < G2) {
      const double x0 = xe[p * 3], x1 = xe[p * 3 + 1], x2 = xe[p * 3 + 2];
      const int qb = half * qlen, qe = min(G2, qb + qlen);
      for (int qq = qb; qq < qe; ++qq) {
        const double d0 = x0 - xf[qq * 3], d1 = x1 - xf[qq * 3 + 1], d2 = x2 - xf[qq * 3 + 2];
        double gr, gi;
        kernel_value(CPLX, d0 * d0 + d1 * d1 + d2 * d2, kre, kim, gr, gi);
#pragma unroll
        for (int j = 0; j < NL; ++j) {
          ur[j] = fma(gr, BW[qq * NL + j], ur[j]);
          if (CPLX) ui[j] = fma(gi, BW[qq * NL + j], ui[j]);
        }
      }
    }
    if (S == 2) {
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        ur[j] += __shfl_down_sync(0xffffffffu, ur[j], P);
        if (CPLX) ui[j] += __shfl_down_sync(0xffffffffu, ui[j], P);
      }
    }
    if (lane < P && p < G2) {
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        ubuf[(p * NL + j) * C] = ur[j];
        if (CPLX) ubuf[(p * NL + j) * C + 1] = ui[j];
      }
    }
  }
  __syncwarp();
  for (int ij = lane; ij < NL * NL; ij += 32) {
    const int i = ij % NL, j = ij / NL;
    double ar = 0.0, ai = 0.0;
    for (int p = 0; p < G2; ++p) {
      ar = fma(BW[p * NL + i], ubuf[(p * NL + j) * C], ar);
      if (CPLX) ai = fma(BW[p * NL + i], ubuf[(p * NL + j) * C + 1], ai);
    }
    ar *= kInv4Pi;
    ai *= kInv4Pi;
    const long long o1 = pr.off1 + (long long)i * nld + j;
    N[o1 * C] = ar;
    if (CPLX) N[o1 * C + 1] = ai;
    if (pr.off2 >= 0) {
      const long long o2 = pr.off2 + (long long)j * nld + i;
      N[o2 * C] = ar;
      if (CPLX) N[o2 * C + 1] = ai;
    }
  }
  __syncwarp();
}

// Separated pair beyond the ring with the kernel in FP32 (MIXED operators):
// points are stored as FP32 offsets from their element's centre, the centre
// difference is taken in FP64 once per pair, so each distance is formed from
// numbers of the size of the distance itself (relative error ~1e-7); the sum
// over f's points runs in FP32 per point of e and everything after it in FP64,
// as in regular_pair.  Block error ~3e-7 relative, below the quadrature target.
template <int D, bool CPLX>
__device__ __forceinline__ void regular_pair_f32(const PairRec& pr, const float4* __restrict__ Xq32,
                                                 const double* __restrict__ cen, const float* __restrict__ BW32,
                                                 const double* __restrict__ BW, double* __restrict__ ubuf, int G2,
                                                 float kre, float kim, double* __restrict__ N, int nld, int lane) {
  constexpr int NL = (D + 1) * (D + 1);
  constexpr int C = CPLX ? 2 : 1;
  const int S = G2 <= 16 ? 2 : 1;  // lanes per point p
  const int P = 32 / S;
  const int half = lane / P;
  const int qlen = (G2 + S - 1) / S;
  const float4* xe = Xq32 + (int64_t)pr.e * G2;
  const float4* xf = Xq32 + (int64_t)pr.f * G2;
  const float c0 = float(cen[pr.e * 4] - cen[pr.f * 4]);
  const float c1 = float(cen[pr.e * 4 + 1] - cen[pr.f * 4 + 1]);
  const float c2 = float(cen[pr.e * 4 + 2] - cen[pr.f * 4 + 2]);
  for (int p0 = 0; p0 < G2; p0 += P) {
    const int p = p0 + (lane % P);
    float ur[NL], ui[NL];
#pragma unroll
    for (int j = 0; j < NL; ++j) ur[j] = ui[j] = 0.f;
    if (p < G2) {
      const float4 a = xe[p];
      const float a0 = c0 + a.x, a1 = c1 + a.y, a2 = c2 + a.z;
      const int qb = half * qlen, qe = min(G2, qb + qlen);
      for (int qq = qb; qq < qe; ++qq) {
        const float4 b = xf[qq];
        const float d0 = a0 - b.x, d1 = a1 - b.y, d2 = a2 - b.z;
        float gr, gi;
        kernel_value_f(CPLX, fmaf(d0, d0, fmaf(d1, d1, d2 * d2)), kre, kim, gr, gi);
#pragma unroll
        for (int j = 0; j < NL; ++j) {
          ur[j] = fmaf(gr, BW32[qq * NL + j], ur[j]);
          if (CPLX) ui[j] = fmaf(gi, BW32[qq * NL + j], ui[j]);
        }
      }
    }
    if (S == 2) {
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        ur[j] += __shfl_down_sync(0xffffffffu, ur[j], P);
        if (CPLX) ui[j] += __shfl_down_sync(0xffffffffu, ui[j], P);
      }
    }
    if (lane < P && p < G2) {
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        ubuf[(p * NL + j) * C] = double(ur[j]);
        if (CPLX) ubuf[(p * NL + j) * C + 1] = double(ui[j]);
      }
    }
  }
  __syncwarp();
  for (int ij = lane; ij < NL * NL; ij += 32) {
    const int i = ij % NL, j = ij / NL;
    double ar = 0.0, ai = 0.0;
    for (int p = 0; p < G2; ++p) {
      ar = fma(BW[p * NL + i], ubuf[(p * NL + j) * C], ar);
      if (CPLX) ai = fma(BW[p * NL + i], ubuf[(p * NL + j) * C + 1], ai);
    }
    ar *= kInv4Pi;
    ai *= kInv4Pi;
    const long long o1 = pr.off1 + (long long)i * nld + j;
    N[o1 * C] = ar;
    if (CPLX) N[o1 * C + 1] = ai;
    if (pr.off2 >= 0) {
      const long long o2 = pr.off2 + (long long)j * nld + i;
      N[o2 * C] = ar;
      if (CPLX) N[o2 * C + 1] = ai;
    }
  }
  __syncwarp();
}

// shared memory of k_near_regular: both FP64 tables, the FP32 copy of the far
// table (FP32 path only), per-warp inner sums
inline size_t regular_smem(int G2, int G2f, int NL, int C, bool f32 = false) {
  return sizeof(double) * ((size_t)G2 * NL + (size_t)G2f * NL + (size_t)kWarps * std::max(G2, G2f) * NL * C) +
         (f32 ? sizeof(float) * (size_t)G2f * NL : 0);
}

// Separable Duffy rules.  In the common-vertex and common-edge rules (see
// duffy_point) one element's point depends on fewer Gauss variables than the
// other's: vertex sub-domains 0, 1 put s on (xi, eta1) and t on (xi, eta2,
// eta3), sub-domains 2, 3 the reverse with eta3; edge sub-domains with xi on |z|
// put s on (xi, u, eta1) and t on (xi, u, eta2), the others fix one point per
// (xi, eta2, u) and move the other with eta1.  The rule sum then factorises:
//   block[i][j] += sum_o W_o[i] sum_a G(x_o, y_a) W_a[j]      (outer point on s)
// with W the Bernstein values times the weights, so each patch map is taken
// once per distinct point and the (d+1)^4 block products once per outer point.
constexpr int kStageCap = 128;  // inner points staged per warp

// doubles of shared memory per warp for the staged inner points
__host__ __device__ constexpr int stage_doubles(int kind, int NL) { return kind == kIdentical ? 0 : kStageCap * (3 + NL); }

// one element of a touching pair: patch, corner (units of h) and the map from
// the rule's canonical coordinates to element-local ones
struct PairSide {
  int patch;
  double o1, o2;
  int cmap;
};

// gamma and the weighted local Bernstein values at canonical point (u1, u2)
template <int D>
__device__ __forceinline__ void side_point(const Geom& geom, const PairSide& sd, double h, double u1, double u2,
                                           double wt, double* __restrict__ x, double* __restrict__ W) {
  constexpr int D1 = D + 1;
  double l1, l2;
  apply_cmap(sd.cmap, u1, u2, l1, l2);
  gamma_eval(geom, sd.patch, (sd.o1 + l1) * h, (sd.o2 + l2) * h, x);
  double b1[D1], b2[D1];
  bernstein<D>(l1, b1);
  bernstein<D>(l2, b2);
#pragma unroll
  for (int k = 0; k < D1 * D1; ++k) W[k] = wt * b1[k % D1] * b2[k / D1];
}

// v += G(x, y) W
template <int NL, bool CPLX>
__device__ __forceinline__ void add_kernel_row(const double* __restrict__ x, const double* __restrict__ y,
                                               const double* __restrict__ W, double kre, double kim,
                                               double* __restrict__ vr, double* __restrict__ vi) {
  const double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
  double gr, gi;
  kernel_value(CPLX, d0 * d0 + d1 * d1 + d2 * d2, kre, kim, gr, gi);
#pragma unroll
  for (int k = 0; k < NL; ++k) {
    vr[k] = fma(gr, W[k], vr[k]);
    if (CPLX) vi[k] = fma(gi, W[k], vi[k]);
  }
}

// acc[i][j] += Wo[i] v[j] (outer point on s) or v[i] Wo[j] (outer point on t)
template <int NL, bool CPLX>
__device__ __forceinline__ void add_outer(bool outer_s, const double* __restrict__ Wo, const double* __restrict__ vr,
                                          const double* __restrict__ vi, double* __restrict__ ar,
                                          double* __restrict__ ai) {
  if (outer_s) {
#pragma unroll
    for (int i = 0; i < NL; ++i)
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        ar[i * NL + j] = fma(Wo[i], vr[j], ar[i * NL + j]);
        if (CPLX) ai[i * NL + j] = fma(Wo[i], vi[j], ai[i * NL + j]);
      }
  } else {
#pragma unroll
    for (int i = 0; i < NL; ++i)
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        ar[i * NL + j] = fma(vr[i], Wo[j], ar[i * NL + j]);
        if (CPLX) ai[i * NL + j] = fma(vi[i], Wo[j], ai[i * NL + j]);
      }
  }
}

// nG groups of nI inner points (computed once into this warp's stage) and nO
// outer points; lanes take (group, outer point) items.
template <int D, bool CPLX, bool OUTER_S, typename InnerF, typename OuterF>
__device__ __forceinline__ void staged_phase(int nG, int nI, int nO, InnerF inner, OuterF outer, double kre,
                                             double kim, double* __restrict__ stage, int lane, double* ar,
                                             double* ai) {
  constexpr int NL = (D + 1) * (D + 1);
  constexpr int SP = 3 + NL;
  const int gchunk = kStageCap / nI;  // nI <= kMaxG < kStageCap
  for (int gb = 0; gb < nG; gb += gchunk) {
    const int ng = min(gchunk, nG - gb);
    for (int p = lane; p < ng * nI; p += 32) {
      const int g = p / nI;
      inner(gb + g, p - g * nI, stage + p * SP, stage + p * SP + 3);
    }
    __syncwarp();
    for (int it = lane; it < ng * nO; it += 32) {
      const int g = it / nO;
      double x[3], Wo[NL], vr[NL], vi[NL];
      outer(gb + g, it - g * nO, x, Wo);
#pragma unroll
      for (int k = 0; k < NL; ++k) vr[k] = vi[k] = 0.0;
      const double* sp = stage + g * nI * SP;
      for (int a = 0; a < nI; ++a, sp += SP) add_kernel_row<NL, CPLX>(x, sp, sp + 3, kre, kim, vr, vi);
      add_outer<NL, CPLX>(OUTER_S, Wo, vr, vi, ar, ai);
    }
    __syncwarp();
  }
}

// Common-vertex pair (both corners at the canonical origin).
template <int D, bool CPLX>
__device__ __forceinline__ void vertex_pair(const Geom& geom, const PairSide& S, const PairSide& T, double h, int4 G,
                                            const double (*gx)[kMaxG], const double (*gw)[kMaxG], double kre,
                                            double kim, double* stage, int lane, double* ar, double* ai) {
  // sub-domains 0, 1 (xi on s1 / s2): s over eta1 staged, t over (eta2, eta3)
  staged_phase<D, CPLX, false>(
      2 * G.x, G.y, G.z * G.w,
      [&](int g, int a, double* x, double* W) {
        const int sub = g / G.x;
        const double xi = gx[0][g % G.x], e = xi * gx[1][a];
        side_point<D>(geom, S, h, sub == 0 ? xi : e, sub == 0 ? e : xi, gw[1][a], x, W);
      },
      [&](int g, int o, double* x, double* W) {
        const int i0 = g % G.x, i2 = o % G.z, i3 = o / G.z;
        const double xi = gx[0][i0];
        side_point<D>(geom, T, h, xi * gx[2][i2], xi * gx[3][i3], xi * xi * xi * gw[0][i0] * gw[2][i2] * gw[3][i3],
                      x, W);
      },
      kre, kim, stage, lane, ar, ai);
  // sub-domains 2, 3 (xi on t1 / t2): t over eta3 staged, s over (eta1, eta2)
  staged_phase<D, CPLX, true>(
      2 * G.x, G.w, G.y * G.z,
      [&](int g, int a, double* x, double* W) {
        const int sub = 2 + g / G.x;
        const double xi = gx[0][g % G.x], e = xi * gx[3][a];
        side_point<D>(geom, T, h, sub == 2 ? xi : e, sub == 2 ? e : xi, gw[3][a], x, W);
      },
      [&](int g, int o, double* x, double* W) {
        const int i0 = g % G.x, i1 = o % G.y, i2 = o / G.y;
        const double xi = gx[0][i0];
        side_point<D>(geom, S, h, xi * gx[1][i1], xi * gx[2][i2], xi * xi * xi * gw[0][i0] * gw[1][i1] * gw[2][i2],
                      x, W);
      },
      kre, kim, stage, lane, ar, ai);
}

// Common-edge pair (shared edge {s1 = 0} = {t1 = 0} in canonical position).
template <int D, bool CPLX>
__device__ __forceinline__ void edge_pair(const Geom& geom, const PairSide& S, const PairSide& T, double h, int4 G,
                                          const double (*gx)[kMaxG], const double (*gw)[kMaxG], double kre,
                                          double kim, double* stage, int lane, double* ar, double* ai) {
  constexpr int NL = (D + 1) * (D + 1);
  // xi on |z| (sub-domains 2, 5): per (sign of z, xi, u) s over eta1 staged,
  // t over eta2; group g = (sign * G.w + i3) * G.x + i0
  const int nxu = G.x * G.w;
  staged_phase<D, CPLX, false>(
      2 * nxu, G.y, G.z,
      [&](int g, int a, double* x, double* W) {
        const int r = g % nxu;
        const double xi = gx[0][r % G.x], z = g < nxu ? xi : -xi;
        const double s2 = fmax(0.0, -z) + gx[3][r / G.x] * (1.0 - xi);
        side_point<D>(geom, S, h, xi * gx[1][a], s2, gw[1][a], x, W);
      },
      [&](int g, int o, double* x, double* W) {
        const int r = g % nxu, i0 = r % G.x, i3 = r / G.x;
        const double xi = gx[0][i0], z = g < nxu ? xi : -xi;
        const double t2 = fmax(0.0, -z) + gx[3][i3] * (1.0 - xi) + z;
        side_point<D>(geom, T, h, xi * gx[2][o], t2, xi * xi * (1.0 - xi) * gw[0][i0] * gw[3][i3] * gw[2][o], x, W);
      },
      kre, kim, stage, lane, ar, ai);
  // xi on s1 (sub-domains 0, 3) or t1 (1, 4): per (c, sign, u, eta2, xi) the
  // point on the xi side is fixed and the other moves with eta1
  const int nB = 4 * G.x * G.z * G.w;
  for (int it = lane; it < nB; it += 32) {
    int r = it;
    const int i0 = r % G.x;
    r /= G.x;
    const int i2 = r % G.z;
    r /= G.z;
    const int i3 = r % G.w;
    r /= G.w;
    const bool fixed_s = (r >> 1) == 0;
    const double xi = gx[0][i0], az = xi * gx[2][i2];
    const double z = (r & 1) ? -az : az;
    const double s2 = fmax(0.0, -z) + gx[3][i3] * (1.0 - az), t2 = s2 + z;
    double xo[3], Wo[NL], vr[NL], vi[NL];
    side_point<D>(geom, fixed_s ? S : T, h, xi, fixed_s ? s2 : t2,
                  xi * xi * (1.0 - az) * gw[0][i0] * gw[2][i2] * gw[3][i3], xo, Wo);
#pragma unroll
    for (int k = 0; k < NL; ++k) vr[k] = vi[k] = 0.0;
    for (int a = 0; a < G.y; ++a) {
      double xm[3], Wm[NL];
      side_point<D>(geom, fixed_s ? T : S, h, xi * gx[1][a], fixed_s ? t2 : s2, gw[1][a], xm, Wm);
      add_kernel_row<NL, CPLX>(xo, xm, Wm, kre, kim, vr, vi);
    }
    add_outer<NL, CPLX>(fixed_s, Wo, vr, vi, ar, ai);
  }
}

// One touching pair per warp, block accumulated in registers and reduced over
// the warp.  Identical pairs: lanes stride over the rule points.  Edge and
// vertex pairs: the separable forms above (stage: this warp's shared buffer).
template <int D, bool CPLX, int KIND>
__device__ __forceinline__ void singular_pair(const PairRec& pr, const Geom& geom, int L, int4 G,
                                              const double (*gx)[kMaxG], const double (*gw)[kMaxG],
                                              double kre, double kim, double* __restrict__ N, int nld, int lane,
                                              double* __restrict__ stage) {
  constexpr int D1 = D + 1;
  constexpr int NL = D1 * D1;
  constexpr int C = CPLX ? 2 : 1;
  const int64_t per = int64_t(1) << (2 * L);
  const double h = ldexp(1.0, -L);
  const int pe = int(pr.e / per), pf = int(pr.f / per);
  uint32_t e1, e2, f1, f2;
  morton_decode(uint32_t(pr.e % per), e1, e2);
  morton_decode(uint32_t(pr.f % per), f1, f2);
  const int ce = (pr.code >> 2) & 7, cf = (pr.code >> 5) & 7;
  double ar[NL * NL], ai[NL * NL];
#pragma unroll
  for (int k = 0; k < NL * NL; ++k) ar[k] = ai[k] = 0.0;
  if constexpr (KIND == kIdentical) {
    // The rule is symmetric under s <-> t (quadrant sigma maps to -sigma with the same
    // weight), so half the sub-domains are integrated and the block is symmetrised at the
    // end: A = M + M^T.  Identical pairs use the identity map (pair code 0), and for fixed
    // (sub, xi, eta, u1) only the second coordinates s2, t2 move with u2 (s1, t1 and the
    // Jacobian are fixed), so the sum factorises along these u lines:
    //   M[i1 i2][j1 j2] += w B_i1(s1) B_j1(t1) sum_u2 w2 G(gamma(s), gamma(t)) B_i2(s2) B_j2(t2)
    // with (d+1)^2 products per rule point and (d+1)^4 per line instead of (d+1)^4 per point.
    (void)ce;
    (void)cf;
    const int nline = 4 * G.x * G.y * G.z;
    for (int idx = lane; idx < nline; idx += 32) {
      int r = idx;
      const int i0 = r % G.x;
      r /= G.x;
      const int i1 = r % G.y;
      r /= G.y;
      const int i2 = r % G.z;
      r /= G.z;
      // sub-domains with sigma_1 = +1 only (quadrants (+,+), (+,-)), both triangles
      const int sub = ((r & 1) << 1) | ((r >> 1) << 2);
      double Sr[D1 * D1], Si[D1 * D1];
#pragma unroll
      for (int k = 0; k < D1 * D1; ++k) Sr[k] = Si[k] = 0.0;
      double s1 = 0.0, t1 = 0.0, jac = 0.0;
      for (int i3 = 0; i3 < G.w; ++i3) {
        double s2, t2;
        jac = duffy_point<KIND>(sub, gx[0][i0], gx[1][i1], gx[2][i2], gx[3][i3], s1, s2, t1, t2);
        double x[3], y[3];
        gamma_eval(geom, pe, (e1 + s1) * h, (e2 + s2) * h, x);
        gamma_eval(geom, pf, (f1 + t1) * h, (f2 + t2) * h, y);
        const double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
        double gr, gi;
        kernel_value(CPLX, d0 * d0 + d1 * d1 + d2 * d2, kre, kim, gr, gi);
        gr *= gw[3][i3];
        gi *= gw[3][i3];
        double bs2[D1], bt2[D1];
        bernstein<D>(s2, bs2);
        bernstein<D>(t2, bt2);
#pragma unroll
        for (int a = 0; a < D1; ++a) {
          const double wr = gr * bs2[a], wi = gi * bs2[a];
#pragma unroll
          for (int c = 0; c < D1; ++c) {
            Sr[a * D1 + c] = fma(wr, bt2[c], Sr[a * D1 + c]);
            if (CPLX) Si[a * D1 + c] = fma(wi, bt2[c], Si[a * D1 + c]);
          }
        }
      }
      const double wl = jac * gw[0][i0] * gw[1][i1] * gw[2][i2];
      double bs1[D1], bt1[D1];
      bernstein<D>(s1, bs1);
      bernstein<D>(t1, bt1);
#pragma unroll
      for (int i = 0; i < NL; ++i) {
        const double wi1 = wl * bs1[i % D1];
#pragma unroll
        for (int j = 0; j < NL; ++j) {
          const double f = wi1 * bt1[j % D1];
          const int k = (i / D1) * D1 + j / D1;
          ar[i * NL + j] = fma(f, Sr[k], ar[i * NL + j]);
          if (CPLX) ai[i * NL + j] = fma(f, Si[k], ai[i * NL + j]);
        }
      }
    }
  } else {
    const PairSide S{pe, double(e1), double(e2), ce}, T{pf, double(f1), double(f2), cf};
    if constexpr (KIND == kEdge)
      edge_pair<D, CPLX>(geom, S, T, h, G, gx, gw, kre, kim, stage, lane, ar, ai);
    else
      vertex_pair<D, CPLX>(geom, S, T, h, G, gx, gw, kre, kim, stage, lane, ar, ai);
  }
#pragma unroll
  for (int k = 0; k < NL * NL; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ar[k] += __shfl_xor_sync(0xffffffffu, ar[k], o);
      if (CPLX) ai[k] += __shfl_xor_sync(0xffffffffu, ai[k], o);
    }
  }
  const double sc = kInv4Pi * h * h * h * h;
  if (KIND == kIdentical) {
    double tr[NL * NL], ti[NL * NL];
#pragma unroll
    for (int k = 0; k < NL * NL; ++k) {
      tr[k] = ar[k] + ar[(k % NL) * NL + k / NL];
      if (CPLX) ti[k] = ai[k] + ai[(k % NL) * NL + k / NL];
    }
#pragma unroll
    for (int k = 0; k < NL * NL; ++k) {
      ar[k] = tr[k];
      if (CPLX) ai[k] = ti[k];
    }
  }
#pragma unroll
  for (int k = 0; k < NL * NL; ++k) {
    if ((k & 31) != lane) continue;
    const int i = k / NL, j = k % NL;
    const long long o1 = pr.off1 + (long long)i * nld + j;
    N[o1 * C] = ar[k] * sc;
    if (CPLX) N[o1 * C + 1] = ai[k] * sc;
    if (pr.off2 >= 0) {
      const long long o2 = pr.off2 + (long long)j * nld + i;
      N[o2 * C] = ar[k] * sc;
      if (CPLX) N[o2 * C + 1] = ai[k] * sc;
    }
  }
}

// Coupling entry id = blk * q2^2 + a * q2 + b (row-major block):
// K[blk][a][b] = G(node_a(target), node_b(source)) / (4 pi) for entry r = a q2 + b of far
// block blk (32-bit index arithmetic: no 64-bit division per entry).  f32k: the difference and
// r^2 in FP64, the kernel value in FP32, stored in FP64 (used where the FP32 point offsets
// of coupling_entry_f32 are not available).
template <bool CPLX>
__device__ __forceinline__ void coupling_entry(int64_t blk, int r, const int* __restrict__ tgt,
                                               const int* __restrict__ src, const double* __restrict__ nodes, int q2,
                                               double kre, double kim, double* __restrict__ K, bool f32k = false) {
  const int a = r / q2, b = r - (r / q2) * q2;
  const double* xa = nodes + ((int64_t)tgt[blk] * q2 + a) * 3;
  const double* xb = nodes + ((int64_t)src[blk] * q2 + b) * 3;
  const double d0 = xa[0] - xb[0], d1 = xa[1] - xb[1], d2 = xa[2] - xb[2];
  double gr, gi;
  if (f32k) {
    float fr, fi;
    kernel_value_f(CPLX, float(d0 * d0 + d1 * d1 + d2 * d2), float(kre), float(kim), fr, fi);
    gr = fr;
    gi = fi;
  } else {
    kernel_value(CPLX, d0 * d0 + d1 * d1 + d2 * d2, kre, kim, gr, gi);
  }
  const int64_t id = blk * (int64_t)q2 * q2 + r;
  if (CPLX) {
    K[id * 2] = gr * kInv4Pi;
    K[id * 2 + 1] = gi * kInv4Pi;
  } else {
    K[id] = gr * kInv4Pi;
  }
}

// MIXED coupling entry without FP64 arithmetic per entry: the difference of the two cluster
// centres (FP64, rounded to FP32 once per block: relative error ~6e-8 of the distance) plus
// the FP32 offsets of the two points from their centres (errors ~6e-8 of a cluster
// diameter), kernel value in FP32 (relative error ~1e-7, far below the interpolation error
// of the far field), stored in FP64 so that the FP64 residual products of the refinement
// apply one fixed operator.  The single-operator and the multi-mesh kernels both evaluate
// entries with this function, so their operators agree bit for bit.
__device__ __forceinline__ float3 centre_difference(const double* __restrict__ ccen, int t, int sc) {
  return make_float3(float(ccen[(int64_t)t * 3] - ccen[(int64_t)sc * 3]),
                     float(ccen[(int64_t)t * 3 + 1] - ccen[(int64_t)sc * 3 + 1]),
                     float(ccen[(int64_t)t * 3 + 2] - ccen[(int64_t)sc * 3 + 2]));
}

template <bool CPLX>
__device__ __forceinline__ void coupling_entry_f32(int64_t blk, int r, int t, int sc, float3 dc,
                                                   const float4* __restrict__ rel, int q2, float kre, float kim,
                                                   double* __restrict__ K) {
  const int a = r / q2, b = r - (r / q2) * q2;
  const float4 u = rel[(int64_t)t * q2 + a], v = rel[(int64_t)sc * q2 + b];
  const float d0 = dc.x + (u.x - v.x), d1 = dc.y + (u.y - v.y), d2 = dc.z + (u.z - v.z);
  float fr, fi;
  kernel_value_f(CPLX, fmaf(d0, d0, fmaf(d1, d1, d2 * d2)), kre, kim, fr, fi);
  // scaled in FP32, one conversion per stored value
  const float s4 = float(kInv4Pi);
  const int64_t id = blk * (int64_t)q2 * q2 + r;
  if (CPLX) {
    K[id * 2] = double(fr * s4);
    K[id * 2 + 1] = double(fi * s4);
  } else {
    K[id] = double(fr * s4);
  }
}

inline int4 rule_orders(const Op& o, int kind) {
  return make_int4(o.g_var[kind][0], o.g_var[kind][1], o.g_var[kind][2], o.g_var[kind][3]);
}

inline int grid_for(int64_t work, int per_block) {
  int64_t g = (work + per_block - 1) / per_block;
  return int(std::min<int64_t>(std::max<int64_t>(g, 1), 1 << 30));
}

}  // namespace

}  // namespace bembel
