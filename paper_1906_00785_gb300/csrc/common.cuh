// common.cuh - shared device/host helpers of the GB300 single-layer BEM library.
//
// Geometry (Sec. 4.1, App. D): patch maps gamma_i: [0,1]^2 -> R^3 evaluated in
// FP64 on host and device.  Basis (App. E): element-local tensor Bernstein
// polynomials of degree d; global S^2 B-splines are reached through the 1-D
// Bezier extraction built in setup.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>

#define BEMBEL_HD __host__ __device__ __forceinline__

namespace bembel {

constexpr double kInv4Pi = 0.079577471545947667884441881686257181;  // 1/(4 pi)
constexpr int kMaxDeg = 2;                                           // ansatz degree d <= 2
constexpr int kMaxEfieDeg = 3;                                       // S^1 degree p <= 3 (EFIE)
constexpr int kMaxQ = 8;                                             // interpolation points per direction
constexpr int kMaxG = 10;                                            // Gauss points per variable
constexpr int kMaxBatch = 64;                                        // meshes per batched assembly

// ---------------------------------------------------------------------------
// Geometry
// ---------------------------------------------------------------------------
enum GeomKind { kSphere6 = 0, kPerturbedSphere = 1, kNurbs = 2 };
constexpr int kMaxNurbsDeg = 4;

struct Geom {
  int kind;
  double w[24];  // amp * a_lm * N_l|m| for the perturbed sphere (see sph_sum)
  // NURBS patches: one buffer, host and device copies (owned by the geometry
  // handle).  doubles [0..5]: offset of patch P's record; record: p1, p2, k1,
  // k2, the k1 + p1 + 1 knots in s, the k2 + p2 + 1 knots in t, then k1 k2
  // control points (x, y, z, weight), index i1 + k1 i2.
  const double* nurbs_host;
  const double* nurbs_dev;
};

// The p + 1 B-splines of degree p (open knot vector kn of n = k + p + 1 knots)
// that are non-zero at x, by the two-term recursion of App. C restricted to the
// knot span holding x (x = 1 in the last non-empty span): T[j][r] holds the
// degree-j function with index span - j + r.  Returns the index of the first.
BEMBEL_HD int nurbs_basis(const double* kn, int k, int p, double x, double* N) {
  int span = p;  // kn[span] <= x < kn[span + 1]
  while (span < k - 1 && x >= kn[span + 1]) ++span;
  double T[kMaxNurbsDeg + 1][kMaxNurbsDeg + 1];
  T[0][0] = 1.0;
  for (int j = 1; j <= p; ++j)
    for (int r = 0; r <= j; ++r) {
      const int i = span - j + r;
      double v = 0.0;
      if (r >= 1) {  // (x - kn_i) / (kn_{i+j} - kn_i) B_{i, j-1}
        const double den = kn[i + j] - kn[i];
        if (den > 0.0) v += (x - kn[i]) / den * T[j - 1][r - 1];
      }
      if (r <= j - 1) {  // (kn_{i+j+1} - x) / (kn_{i+j+1} - kn_{i+1}) B_{i+1, j-1}
        const double den = kn[i + j + 1] - kn[i + 1];
        if (den > 0.0) v += (kn[i + j + 1] - x) / den * T[j - 1][r];
      }
      T[j][r] = v;
    }
  for (int r = 0; r <= p; ++r) N[r] = T[p][r];
  return span - p;
}

// Rational tensor-product patch: x = sum N_a(s) N_b(t) w_ab P_ab / sum N_a N_b w_ab.
BEMBEL_HD void nurbs_eval(const double* buf, int patch, double s, double t, double x[3]) {
  const double* r = buf + (long long)buf[patch];
  const int p1 = int(r[0]), p2 = int(r[1]), k1 = int(r[2]), k2 = int(r[3]);
  const double* kn1 = r + 4;
  const double* kn2 = kn1 + k1 + p1 + 1;
  const double* cp = kn2 + k2 + p2 + 1;
  double N1[kMaxNurbsDeg + 1], N2[kMaxNurbsDeg + 1];
  const int a0 = nurbs_basis(kn1, k1, p1, s, N1);
  const int b0 = nurbs_basis(kn2, k2, p2, t, N2);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = 0; b <= p2; ++b)
    for (int a = 0; a <= p1; ++a) {
      const double* P = cp + 4 * ((long long)(a0 + a) + (long long)k1 * (b0 + b));
      const double c = N1[a] * N2[b] * P[3];
      acc[0] += c * P[0];
      acc[1] += c * P[1];
      acc[2] += c * P[2];
      acc[3] += c;
    }
  x[0] = acc[0] / acc[3];
  x[1] = acc[1] / acc[3];
  x[2] = acc[2] / acc[3];
}

// Cube face of patch p: c(s,t) = o + (2s-1) e1 + (2t-1) e2 with e1 x e2 = o.
// Patch order +x, -x, +y, -y, +z, -z.  Each axis vector is +-1 on a single
// coordinate, encoded as (coordinate, sign).
BEMBEL_HD void cube_point(int p, double s, double t, double c[3]) {
  const double u = 2.0 * s - 1.0, v = 2.0 * t - 1.0;
  switch (p) {
    case 0: c[0] = 1.0;  c[1] = u;    c[2] = v;    break;  // o=+x e1=+y e2=+z
    case 1: c[0] = -1.0; c[1] = v;    c[2] = u;    break;  // o=-x e1=+z e2=+y
    case 2: c[0] = v;    c[1] = 1.0;  c[2] = u;    break;  // o=+y e1=+z e2=+x
    case 3: c[0] = u;    c[1] = -1.0; c[2] = v;    break;  // o=-y e1=+x e2=+z
    case 4: c[0] = u;    c[1] = v;    c[2] = 1.0;  break;  // o=+z e1=+x e2=+y
    default: c[0] = v;   c[1] = u;    c[2] = -1.0; break;  // o=-z e1=+y e2=+x
  }
}

// Radial perturbation sum_lm w_lm Y_lm at a unit vector (x, y, z) for 1 <= l <= 4.
// Real orthonormal harmonics without the Condon-Shortley phase:
//   Y_lm = N_l|m| * (d^|m| P_l / dz^|m|)(z) * {Re (x+iy)^m  (m > 0) | 1 (m = 0) | Im (x+iy)^|m| (m < 0)}
// with N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) * (sqrt 2 if m != 0), using
// sin^m(theta) e^{i m phi} = (x + i y)^m on the unit sphere.  The host folds
// amp * a_lm * N_l|m| into w (index (l, m = -l..l) -> l*l - 1 + l + m).
BEMBEL_HD double sph_sum(const double* w, double x, double y, double z) {
  double re[5], im[5];
  re[0] = 1.0;
  im[0] = 0.0;
  for (int m = 1; m <= 4; ++m) {
    re[m] = x * re[m - 1] - y * im[m - 1];
    im[m] = x * im[m - 1] + y * re[m - 1];
  }
  const double z2 = z * z;
  // dP[l][m] = d^m P_l / dz^m
  double dP[5][5] = {};
  dP[1][0] = z;                                   dP[1][1] = 1.0;
  dP[2][0] = 0.5 * (3.0 * z2 - 1.0);              dP[2][1] = 3.0 * z;
  dP[2][2] = 3.0;
  dP[3][0] = 0.5 * (5.0 * z2 - 3.0) * z;          dP[3][1] = 0.5 * (15.0 * z2 - 3.0);
  dP[3][2] = 15.0 * z;                            dP[3][3] = 15.0;
  dP[4][0] = (35.0 * z2 * z2 - 30.0 * z2 + 3.0) / 8.0;
  dP[4][1] = (140.0 * z2 - 60.0) * z / 8.0;
  dP[4][2] = (420.0 * z2 - 60.0) / 8.0;
  dP[4][3] = 105.0 * z;                           dP[4][4] = 105.0;
  double r = 0.0;
  for (int l = 1; l <= 4; ++l) {
    const int base = l * l - 1 + l;
    r += w[base] * dP[l][0];
    for (int m = 1; m <= l; ++m) r += dP[l][m] * (w[base + m] * re[m] + w[base - m] * im[m]);
  }
  return r;
}

// gamma and its parameter derivatives on the cube-face sphere: gamma = c / |c|,
// d gamma = (dc - gamma (gamma . dc)) / |c| with dc/ds, dc/dt constant per patch.
BEMBEL_HD void sphere6_jac(int patch, double s, double t, double x[3], double ds[3], double dt[3]) {
  double c[3], c00[3], c10[3], c01[3];
  cube_point(patch, s, t, c);
  cube_point(patch, 0.0, 0.0, c00);
  cube_point(patch, 1.0, 0.0, c10);
  cube_point(patch, 0.0, 1.0, c01);
#ifdef __CUDA_ARCH__
  const double inv = rsqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
#else
  const double inv = 1.0 / std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
#endif
  double gs = 0.0, gt = 0.0;
  for (int k = 0; k < 3; ++k) {
    x[k] = c[k] * inv;
    gs += x[k] * (c10[k] - c00[k]);
    gt += x[k] * (c01[k] - c00[k]);
  }
  for (int k = 0; k < 3; ++k) {
    ds[k] = ((c10[k] - c00[k]) - x[k] * gs) * inv;
    dt[k] = ((c01[k] - c00[k]) - x[k] * gt) * inv;
  }
}

// gamma_p(s, t) in FP64.
BEMBEL_HD void gamma_eval(const Geom& g, int p, double s, double t, double x[3]) {
  if (g.kind == kNurbs) {
#ifdef __CUDA_ARCH__
    nurbs_eval(g.nurbs_dev, p, s, t, x);
#else
    nurbs_eval(g.nurbs_host, p, s, t, x);
#endif
    return;
  }
  double c[3];
  cube_point(p, s, t, c);
  const double n2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
#ifdef __CUDA_ARCH__
  double inv = rsqrt(n2);
#else
  double inv = 1.0 / std::sqrt(n2);
#endif
  x[0] = c[0] * inv;
  x[1] = c[1] * inv;
  x[2] = c[2] * inv;
  if (g.kind == kPerturbedSphere) {
    const double r = 1.0 + sph_sum(g.w, x[0], x[1], x[2]);
    x[0] *= r;
    x[1] *= r;
    x[2] *= r;
  }
}

// ---------------------------------------------------------------------------
// Bernstein basis of degree D on [0,1]: B_k(u) = C(D,k) u^k (1-u)^(D-k).
// ---------------------------------------------------------------------------
template <int D>
BEMBEL_HD void bernstein(double u, double b[D + 1]) {
  const double v = 1.0 - u;
  if (D == 0) {
    b[0] = 1.0;
  } else if (D == 1) {
    b[0] = v;
    b[1] = u;
  } else {
    b[0] = v * v;
    b[1] = 2.0 * u * v;
    b[2] = u * u;
  }
}

// ---------------------------------------------------------------------------
// Morton order inside a patch: the bits of i1 (first parameter) take the even
// positions, so children of cluster c at the next level are 4c + (c1 | c2 << 1).
// ---------------------------------------------------------------------------
BEMBEL_HD uint32_t morton_encode(uint32_t i1, uint32_t i2) {
  uint32_t m = 0;
  for (int b = 0; b < 16; ++b) m |= (((i1 >> b) & 1u) << (2 * b)) | (((i2 >> b) & 1u) << (2 * b + 1));
  return m;
}
BEMBEL_HD void morton_decode(uint32_t m, uint32_t& i1, uint32_t& i2) {
  i1 = 0;
  i2 = 0;
  for (int b = 0; b < 16; ++b) {
    i1 |= ((m >> (2 * b)) & 1u) << b;
    i2 |= ((m >> (2 * b + 1)) & 1u) << b;
  }
}

// Canonical map of a Duffy rule onto an element's local square:
// T(u) = A + u1 * D1 + u2 * D2 with A the corner (code & 3) = (a1, a2) =
// (code & 1, (code >> 1) & 1), D1 the inward unit vector along local axis
// ax = (code >> 2) & 1 and D2 the inward unit vector along the other axis.
BEMBEL_HD void apply_cmap(int code, double u1, double u2, double& s1, double& s2) {
  const int a1 = code & 1, a2 = (code >> 1) & 1, ax = (code >> 2) & 1;
  const double d_first = ax == 0 ? u1 : u2;   // displacement along local axis 0
  const double d_second = ax == 0 ? u2 : u1;  // displacement along local axis 1
  s1 = a1 ? 1.0 - d_first : d_first;
  s2 = a2 ? 1.0 - d_second : d_second;
}

#ifdef __CUDACC__
// Single-layer kernel in FP32: 1/r and, for Helmholtz, exp(-i kappa r) / r (the 1/(4 pi)
// factor is applied by the caller).
__device__ __forceinline__ void kernel_value_f(bool cplx, float r2, float kre, float kim, float& gr, float& gi) {
  const float rinv = rsqrtf(r2);
  if (!cplx) {
    gr = rinv;
    gi = 0.f;
  } else {
    const float r = r2 * rinv;
    float sn, cs;
    sincosf(kre * r, &sn, &cs);
    const float a = (kim != 0.f ? expf(kim * r) : 1.f) * rinv;
    gr = a * cs;
    gi = -a * sn;
  }
}
#endif

}  // namespace bembel
