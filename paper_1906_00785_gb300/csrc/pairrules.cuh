// pairrules.cuh - pointwise pieces shared by the element-pair quadrature
// kernels: the single-layer kernel value and the Duffy-type rule points.
#pragma once

#include "op.h"

namespace bembel {

// exp(-i kappa r) / r (App. B, (HS)); 1/r for Laplace.  The 1/(4 pi) is applied
// by the callers.
__device__ __forceinline__ void kernel_value(bool cplx, double r2, double kre, double kim, double& gr, double& gi) {
  const double rinv = rsqrt(r2);
  if (!cplx) {
    gr = rinv;
    gi = 0.0;
  } else {
    // exp(-i kappa r) = exp(kim r) (cos(kre r) - i sin(kre r))
    const double r = r2 * rinv;
    double sn, cs;
    sincos(kre * r, &sn, &cs);
    const double a = (kim != 0.0 ? exp(kim * r) : 1.0) * rinv;
    gr = a * cs;
    gi = -a * sn;
  }
}

// Point of a Duffy rule in canonical position.  x = (x0, x1, x2, x3) are the
// Gauss variables in [0,1]^4, sub the sub-domain.  Returns (s1, s2, t1, t2) and
// the Jacobian factor.
//  KIND 1 (identical): z = t - s in quadrant (sg1, sg2) = (+-1, +-1) from sub & 3,
//     triangle sub >> 2: (a, b) = (xi, xi eta) or (xi eta, xi); |z| = (a, b);
//     s_k = max(0, -z_k) + u_k (1 - |z_k|), t = s + z; Jacobian xi (1-a)(1-b).
//  KIND 2 (common edge {s1 = 0} = {t1 = 0}): sign of z = t2 - s2 from sub / 3,
//     pyramid c = sub % 3 puts xi on coordinate c of (s1, t1, |z|), the others
//     xi eta1, xi eta2; s2 = max(0, -z) + u (1 - |z|); Jacobian xi^2 (1 - |z|).
//  KIND 3 (common vertex s = t = 0): pyramid c = sub puts xi on coordinate c of
//     (s1, s2, t1, t2), the others xi eta1..3; Jacobian xi^3.
template <int KIND>
__device__ __forceinline__ double duffy_point(int sub, double x0, double x1, double x2, double x3, double& s1,
                                              double& s2, double& t1, double& t2) {
  const double xi = x0;
  if (KIND == kIdentical) {
    const double a = (sub >> 2) == 0 ? xi : xi * x1;
    const double b = (sub >> 2) == 0 ? xi * x1 : xi;
    const double z1 = (sub & 1) ? -a : a;
    const double z2 = (sub & 2) ? -b : b;
    s1 = fmax(0.0, -z1) + x2 * (1.0 - a);
    s2 = fmax(0.0, -z2) + x3 * (1.0 - b);
    t1 = s1 + z1;
    t2 = s2 + z2;
    return xi * (1.0 - a) * (1.0 - b);
  } else if (KIND == kEdge) {
    // (s1, t1, |z|) = xi at position c, (xi eta1, xi eta2) in order elsewhere
    const int c = sub % 3;
    const double e1 = xi * x1, e2 = xi * x2;
    s1 = c == 0 ? xi : e1;
    t1 = c == 0 ? e1 : (c == 1 ? xi : e2);
    const double az = c == 2 ? xi : e2;
    const double z = (sub < 3) ? az : -az;
    s2 = fmax(0.0, -z) + x3 * (1.0 - az);
    t2 = s2 + z;
    return xi * xi * (1.0 - az);
  } else {
    const double e1 = xi * x1, e2 = xi * x2, e3 = xi * x3;
    s1 = sub == 0 ? xi : e1;
    s2 = sub == 0 ? e1 : (sub == 1 ? xi : e2);
    t1 = sub <= 1 ? e2 : (sub == 2 ? xi : e3);
    t2 = sub <= 2 ? e3 : xi;
    return xi * xi * xi;
  }
}

// Gauss tables of a rule with per-variable orders g = (g0, g1, g2, g3): at tab,
// for v = 0..3, the g_v nodes then the g_v weights on [0,1].  Block-cooperative
// (needs blockDim.x >= 4 kMaxG); the caller synchronises afterwards.
__device__ __forceinline__ void load_rule_tables(const double* __restrict__ tab, int4 g, double (*gx)[kMaxG],
                                                 double (*gw)[kMaxG]) {
  const int t = threadIdx.x;
  if (t < 4 * kMaxG) {
    const int v = t / kMaxG, i = t % kMaxG;
    const int gv[4] = {g.x, g.y, g.z, g.w};
    int off = 0;
    for (int u = 0; u < v; ++u) off += 2 * gv[u];
    if (i < gv[v]) {
      gx[v][i] = tab[off + i];
      gw[v][i] = tab[off + gv[v] + i];
    }
  }
}

// rule point idx of NSUB sub-domains x g0 g1 g2 g3 tensor points:
// sub-domain and the four Gauss indices (variable 0 fastest)
__device__ __forceinline__ void rule_index(int idx, int4 g, int& sub, int& i0, int& i1, int& i2, int& i3) {
  const int g4 = g.x * g.y * g.z * g.w;
  sub = idx / g4;
  int rem = idx - sub * g4;
  i0 = rem % g.x;
  rem /= g.x;
  i1 = rem % g.y;
  rem /= g.y;
  i2 = rem % g.z;
  i3 = rem / g.z;
}

}  // namespace bembel
