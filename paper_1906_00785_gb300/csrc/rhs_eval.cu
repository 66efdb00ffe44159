// rhs_eval.cu - load vectors (Sec. 4.4) and potential evaluation (Sec. 4.7).
//
// Load vector: b_i = int_Gamma g phi_i = int_square g(gamma(s)) phi_hat_i(s) ds
// (2-form Piola lift of App. E), tensor Gauss with g x g points per element,
// accumulated per element in the Bernstein basis and mapped to the B-spline
// dofs with the transposed Bezier extraction.
// Potential: u(x) = sum_j rho_j int_square G(x, gamma(t)) phi_hat_j(t) dt with
// G of (LS) / (HS); the density is gathered to the elements, its values at the
// Gauss points (times weights) formed once, then a direct sum over all
// element points per evaluation point.
#include <vector>

#include "op.h"

namespace bembel {

namespace {

// b_loc[(e*nloc + k)*ncol + r*C + comp] = sum_p w_p h^2 B_k(u_p) g_r(gamma(s_p))
template <int D, bool CPLX>
__global__ void k_rhs_local(Geom geom, int L, int64_t nelem, int G, const double* __restrict__ gx,
                            const double* __restrict__ gw, int kind, const double* __restrict__ params, int nrhs,
                            double kre, double kim, double* __restrict__ bl) {
  constexpr int D1 = D + 1, NL = D1 * D1;
  const int C = CPLX ? 2 : 1;
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= nelem * nrhs) return;
  const int64_t e = id / nrhs;
  const int r = int(id % nrhs);
  const int64_t per = int64_t(1) << (2 * L);
  const int patch = int(e / per);
  uint32_t i1, i2;
  morton_decode(uint32_t(e % per), i1, i2);
  const double h = ldexp(1.0, -L);
  const double p0 = params[3 * r], p1 = params[3 * r + 1], p2 = params[3 * r + 2];
  double ar[NL], ai[NL];
  for (int k = 0; k < NL; ++k) ar[k] = ai[k] = 0.0;
  for (int b = 0; b < G; ++b)
    for (int a = 0; a < G; ++a) {
      double x[3];
      gamma_eval(geom, patch, (i1 + gx[a]) * h, (i2 + gx[b]) * h, x);
      double vr, vi;
      if (kind == BEMBEL_RHS_POINT_SOURCE) {
        const double d0 = x[0] - p0, d1 = x[1] - p1, d2 = x[2] - p2;
        const double rr = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        if (CPLX) {
          double sn, cs;
          sincos(kre * rr, &sn, &cs);
          const double am = exp(kim * rr) / rr;
          vr = am * cs;
          vi = -am * sn;
        } else {
          vr = 1.0 / rr;
          vi = 0.0;
        }
      } else {
        const double ph = p0 * x[0] + p1 * x[1] + p2 * x[2];
        double sn, cs;
        sincos(kre * ph, &sn, &cs);
        const double am = exp(kim * ph);
        vr = am * cs;
        vi = -am * sn;
      }
      double b1[D1], b2[D1];
      bernstein<D>(gx[a], b1);
      bernstein<D>(gx[b], b2);
      const double w = gw[a] * gw[b] * h * h;
      for (int k = 0; k < NL; ++k) {
        const double bk = w * b1[k % D1] * b2[k / D1];
        ar[k] += bk * vr;
        ai[k] += bk * vi;
      }
    }
  const int ncol = nrhs * C;
  for (int k = 0; k < NL; ++k) {
    bl[(e * NL + k) * ncol + r * C] = ar[k];
    if (CPLX) bl[(e * NL + k) * ncol + r * C + 1] = ai[k];
  }
}

// rq[(e*G2 + p)*ncol + col] = w_p h^2 sum_k B_k(u_p) rho_loc[(e*nloc + k)*ncol + col]
template <int D>
__global__ void k_density_points(const double* __restrict__ rl, int64_t nelem, int G, const double* __restrict__ gx,
                                 const double* __restrict__ gw, double h, int ncol, double* __restrict__ rq) {
  constexpr int D1 = D + 1, NL = D1 * D1;
  const int G2 = G * G;
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= nelem * G2 * ncol) return;
  const int col = int(id % ncol);
  const int p = int((id / ncol) % G2);
  const int64_t e = id / ((int64_t)ncol * G2);
  double b1[D1], b2[D1];
  bernstein<D>(gx[p % G], b1);
  bernstein<D>(gx[p / G], b2);
  double acc = 0.0;
  for (int k = 0; k < NL; ++k) acc += b1[k % D1] * b2[k / D1] * rl[(e * NL + k) * ncol + col];
  rq[id] = acc * gw[p % G] * gw[p / G] * h * h;
}

// Block per (evaluation point, rhs, source chunk): u = sum over element points G(x, y) rq /
// (4 pi), in FP64 (FP64 operators; MIXED operators use k_potential_elem).
template <bool CPLX>
__global__ void k_potential(const double* __restrict__ pts, int64_t npts, const double* __restrict__ Y,
                            const double* __restrict__ rq, int64_t nsrc, int nrhs, double kre, double kim,
                            double* __restrict__ out) {
  // block (point, column, source chunk): the chunk's partial sum is added to out
  const int64_t ip = blockIdx.x;
  const int r = blockIdx.y;
  const int C = CPLX ? 2 : 1;
  const int ncol = nrhs * C;
  const int64_t chunk = (nsrc + gridDim.z - 1) / gridDim.z;
  const int64_t k0 = blockIdx.z * chunk, k1 = min(nsrc, k0 + chunk);
  const double x0 = pts[ip * 3], x1 = pts[ip * 3 + 1], x2 = pts[ip * 3 + 2];
  double sr = 0.0, si = 0.0;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const double d0 = x0 - Y[k * 3], d1 = x1 - Y[k * 3 + 1], d2 = x2 - Y[k * 3 + 2];
    const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
    const double rhr = rq[k * ncol + r * C];
    double gr, gi = 0.0;
    const double rinv = rsqrt(r2);
    if (CPLX) {
      const double rr = r2 * rinv;
      double sn, cs;
      sincos(kre * rr, &sn, &cs);
      const double am = exp(kim * rr) * rinv;
      gr = am * cs;
      gi = -am * sn;
    } else {
      gr = rinv;
    }
    if (CPLX) {
      const double rhi = rq[k * ncol + r * C + 1];
      sr += gr * rhr - gi * rhi;
      si += gr * rhi + gi * rhr;
    } else {
      sr += gr * rhr;
    }
  }
  __shared__ double red[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sr;
    red[1][threadIdx.x >> 5] = si;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a += red[0][k];
      b += red[1][k];
    }
    atomicAdd(out + ((int64_t)r * npts + ip) * C, a * kInv4Pi);
    if (CPLX) atomicAdd(out + ((int64_t)r * npts + ip) * C + 1, b * kInv4Pi);
  }
}

// Element centres (mean of the element's G2 points) and the points as FP32 offsets from them,
// for the element-wise FP32 potential of MIXED operators.
__global__ void k_eval_offsets(const double* __restrict__ Y, int64_t nelem, int G2, double* __restrict__ cen,
                               float4* __restrict__ rel) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nelem) return;
  double c[3] = {0.0, 0.0, 0.0};
  for (int p = 0; p < G2; ++p)
    for (int k = 0; k < 3; ++k) c[k] += Y[(e * G2 + p) * 3 + k];
  for (int k = 0; k < 3; ++k) {
    c[k] /= G2;
    cen[e * 3 + k] = c[k];
  }
  for (int p = 0; p < G2; ++p) {
    const double* y = Y + (e * G2 + p) * 3;
    rel[e * G2 + p] = make_float4(float(y[0] - c[0]), float(y[1] - c[1]), float(y[2] - c[2]), 0.f);
  }
}

// MIXED operators: thread per element of the block's chunk.  An element whose centre lies
// farther than sqrt(far2e) from the point is summed in FP32 from the FP64 centre difference
// (rounded once) and the FP32 point offsets, its sum added in FP64; nearer elements take the
// FP64 sum of k_potential.  rq32 is the FP32 copy of the weighted density.
template <bool CPLX>
__global__ void k_potential_elem(const double* __restrict__ pts, int64_t npts, const double* __restrict__ Y,
                                 const double* __restrict__ cen, const float4* __restrict__ rel,
                                 const double* __restrict__ rq, const float* __restrict__ rq32, int64_t nelem,
                                 int G2, int nrhs, double kre, double kim, double far2e, double* __restrict__ out) {
  const int64_t ip = blockIdx.x;
  const int r = blockIdx.y;
  const int C = CPLX ? 2 : 1;
  const int ncol = nrhs * C;
  const int64_t chunk = (nelem + gridDim.z - 1) / gridDim.z;
  const int64_t e0 = blockIdx.z * chunk, e1 = min(nelem, e0 + chunk);
  const double x0 = pts[ip * 3], x1 = pts[ip * 3 + 1], x2 = pts[ip * 3 + 2];
  double sr = 0.0, si = 0.0;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const double c0 = x0 - cen[e * 3], c1 = x1 - cen[e * 3 + 1], c2 = x2 - cen[e * 3 + 2];
    if (c0 * c0 + c1 * c1 + c2 * c2 > far2e) {
      const float f0 = float(c0), f1 = float(c1), f2 = float(c2);
      float ar = 0.f, ai = 0.f;
      for (int p = 0; p < G2; ++p) {
        const int64_t k = e * G2 + p;
        const float4 v = rel[k];
        const float d0 = f0 - v.x, d1 = f1 - v.y, d2 = f2 - v.z;
        float gr, gi;
        kernel_value_f(CPLX, fmaf(d0, d0, fmaf(d1, d1, d2 * d2)), float(kre), float(kim), gr, gi);
        const float rhr = rq32[k * ncol + r * C];
        if (CPLX) {
          const float rhi = rq32[k * ncol + r * C + 1];
          ar = fmaf(gr, rhr, fmaf(-gi, rhi, ar));
          ai = fmaf(gr, rhi, fmaf(gi, rhr, ai));
        } else {
          ar = fmaf(gr, rhr, ar);
        }
      }
      sr += double(ar);
      si += double(ai);
    } else {
      for (int p = 0; p < G2; ++p) {
        const int64_t k = e * G2 + p;
        const double d0 = x0 - Y[k * 3], d1 = x1 - Y[k * 3 + 1], d2 = x2 - Y[k * 3 + 2];
        const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
        const double rinv = rsqrt(r2);
        const double rhr = rq[k * ncol + r * C];
        if (CPLX) {
          const double rhi = rq[k * ncol + r * C + 1];
          const double rr = r2 * rinv;
          double sn, cs;
          sincos(kre * rr, &sn, &cs);
          const double am = exp(kim * rr) * rinv;
          const double gr = am * cs, gi = -am * sn;
          sr += gr * rhr - gi * rhi;
          si += gr * rhi + gi * rhr;
        } else {
          sr += rinv * rhr;
        }
      }
    }
  }
  __shared__ double red[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sr;
    red[1][threadIdx.x >> 5] = si;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a += red[0][k];
      b += red[1][k];
    }
    atomicAdd(out + ((int64_t)r * npts + ip) * C, a * kInv4Pi);
    if (CPLX) atomicAdd(out + ((int64_t)r * npts + ip) * C + 1, b * kInv4Pi);
  }
}

__global__ void k_d2f(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = float(a[i]);
}

// Compressed evaluation, one warp per (evaluation point, rhs column): a level-by-level
// descent of the cluster tree from the six patch clusters.  A cluster admissible for
// the point (2 r <= eta max(0, |x - c| - r), and |kappa| 2 r <= kdiam when the
// operator sets that Helmholtz limit) adds sum_b G(x, y_b) xh[b] over its q^2
// interpolation points y_b and moments xh; a non-admissible leaf adds its elements'
// Gauss points directly; any other non-admissible cluster passes on its four children.
// The frontier of one level lives in shared memory; a frontier that would exceed
// kFront sets *err and the point is left unfinished (the host reports it).
constexpr int kTreeWarps = 4;
constexpr int kFront = 1024;

struct TreeLevels {
  long long off[16];
};

template <bool CPLX>
__device__ __forceinline__ void add_kernel_sum(double x0, double x1, double x2, const double* __restrict__ Y,
                                               const double* __restrict__ w, int64_t wstride, int n, double kre,
                                               double kim, double& sr, double& si) {
  for (int k = 0; k < n; ++k) {
    const double d0 = x0 - Y[k * 3], d1 = x1 - Y[k * 3 + 1], d2 = x2 - Y[k * 3 + 2];
    const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
    const double rinv = rsqrt(r2);
    const double wr = w[k * wstride];
    if (CPLX) {
      const double wi = w[k * wstride + 1];
      const double rr = r2 * rinv;
      double sn, cs;
      sincos(kre * rr, &sn, &cs);
      const double am = exp(kim * rr) * rinv;
      const double gr = am * cs, gi = -am * sn;
      sr += gr * wr - gi * wi;
      si += gr * wi + gi * wr;
    } else {
      sr += rinv * wr;
    }
  }
}

template <bool CPLX>
__global__ void __launch_bounds__(32 * kTreeWarps)
    k_potential_tree(const double* __restrict__ pts, int64_t npts, const double* __restrict__ balls,
                     const double* __restrict__ nodes, const double* __restrict__ xh, int q2, TreeLevels lv,
                     int leaf, int L, const double* __restrict__ Y, const double* __restrict__ rq, int G2, int ncol,
                     double eta, double kdiam, double kre, double kim, int* __restrict__ err,
                     double* __restrict__ out) {
  __shared__ int front[kTreeWarps][2][kFront];
  __shared__ int count[kTreeWarps][2];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ip = blockIdx.x * (int64_t)kTreeWarps + wid;
  if (ip >= npts) return;  // whole warps leave together
  const int C = CPLX ? 2 : 1;
  const int col = blockIdx.y * C;  // first real column of this rhs
  const double x0 = pts[ip * 3], x1 = pts[ip * 3 + 1], x2 = pts[ip * 3 + 2];
  if (lane < 6) front[wid][0][lane] = int(lv.off[0]) + lane;
  if (lane == 0) count[wid][0] = 6;
  __syncwarp();
  double sr = 0.0, si = 0.0;
  int cur = 0;
  bool overflow = false;
  for (int l = 0; l <= leaf; ++l) {
    const int n = count[wid][cur];
    if (lane == 0) count[wid][cur ^ 1] = 0;
    __syncwarp();
    for (int idx = lane; idx < n; idx += 32) {
      const int c = front[wid][cur][idx];
      const double* b = balls + (int64_t)c * 4;
      const double e0 = x0 - b[0], e1 = x1 - b[1], e2 = x2 - b[2];
      const double dist = fmax(0.0, sqrt(e0 * e0 + e1 * e1 + e2 * e2) - b[3]);
      const bool osc_ok = !(CPLX && kdiam > 0.0) || hypot(kre, kim) * 2.0 * b[3] <= kdiam;
      if (osc_ok && 2.0 * b[3] <= eta * dist) {
        add_kernel_sum<CPLX>(x0, x1, x2, nodes + (int64_t)c * q2 * 3, xh + (int64_t)c * q2 * ncol + col, ncol, q2,
                             kre, kim, sr, si);
      } else if (l == leaf) {
        const int sh = 2 * (L - leaf);
        const int64_t e0i = (int64_t(c) - lv.off[leaf]) << sh;
        const int ne = 1 << sh;
        add_kernel_sum<CPLX>(x0, x1, x2, Y + e0i * G2 * 3, rq + e0i * G2 * ncol + col, ncol, ne * G2, kre, kim, sr,
                             si);
      } else {
        const int k = atomicAdd(&count[wid][cur ^ 1], 4);
        if (k + 4 <= kFront) {
          const int first = int(lv.off[l + 1] + 4 * (int64_t(c) - lv.off[l]));
          for (int j = 0; j < 4; ++j) front[wid][cur ^ 1][k + j] = first + j;
        } else {
          overflow = true;
        }
      }
    }
    __syncwarp();
    if (__any_sync(0xffffffffu, overflow)) {
      if (lane == 0) atomicExch(err, 1);
      return;
    }
    cur ^= 1;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  if (lane == 0) {
    out[((int64_t)blockIdx.y * npts + ip) * C] = sr * kInv4Pi;
    if (CPLX) out[((int64_t)blockIdx.y * npts + ip) * C + 1] = si * kInv4Pi;
  }
}

__global__ void k_tab_points(Geom g, int L, int64_t nelem, int G, const double* __restrict__ gx, double h,
                             double* __restrict__ Y) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int G2 = G * G;
  if (id >= nelem * G2) return;
  const int64_t e = id / G2;
  const int p = int(id % G2);
  const int64_t per = int64_t(1) << (2 * L);
  uint32_t i1, i2;
  morton_decode(uint32_t(e % per), i1, i2);
  gamma_eval(g, int(e / per), (i1 + gx[p % G]) * h, (i2 + gx[p / G]) * h, &Y[id * 3]);
}

void gauss_table(int G, double* d_buf, cudaStream_t s) {
  // Gauss-Legendre nodes/weights on [0,1] by Newton on P_G, uploaded as [x..., w...]
  std::vector<double> t(2 * G);
  for (int i = 0; i < G; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (G + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= G; ++k) {
        const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (G == 1) p0 = 1.0;
      dp = G * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= G; ++k) {
      const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    if (G == 1) p0 = 1.0;
    dp = G * (z * p1 - p0) / (z * z - 1.0);
    t[G - 1 - i] = 0.5 * (1.0 - z);
    t[G + G - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
  cuda_check(cudaMemcpyAsync(d_buf, t.data(), sizeof(double) * 2 * G, cudaMemcpyHostToDevice, s), "gauss upload");
  cuda_check(cudaStreamSynchronize(s), "gauss sync");
}

struct Buf {
  void* p;
  explicit Buf(size_t n) : p(dev_alloc(n)) {}
  ~Buf() { dev_free(p); }
};

}  // namespace

void rhs_device(const Op& o, int kind, const double* params, int nrhs, int G, void* b) {
  const cudaStream_t s = o.stream;
  const int C = o.cplx ? 2 : 1;
  if (o.efie) {
    // EFIE: plane waves E_inc = pol exp(-i kappa dir . x), 6 parameters per column
    Buf gt(sizeof(double) * 2 * G), pr(sizeof(double) * 6 * nrhs), bl(sizeof(double) * o.nlocal * nrhs * 2);
    gauss_table(G, static_cast<double*>(gt.p), s);
    cuda_check(cudaMemcpyAsync(pr.p, params, sizeof(double) * 6 * nrhs, cudaMemcpyHostToDevice, s), "params");
    const double* gx = static_cast<double*>(gt.p);
    efie_rhs_local(o, gx, gx + G, G, static_cast<const double*>(pr.p), nrhs, static_cast<double*>(bl.p), s);
    scatter_to_global(o, static_cast<double*>(bl.p), static_cast<double*>(b), nrhs, s);
    cuda_check(cudaStreamSynchronize(s), "rhs sync");
    return;
  }
  Buf gt(sizeof(double) * 2 * G), pr(sizeof(double) * 3 * nrhs), bl(sizeof(double) * o.nlocal * nrhs * C);
  gauss_table(G, static_cast<double*>(gt.p), s);
  cuda_check(cudaMemcpyAsync(pr.p, params, sizeof(double) * 3 * nrhs, cudaMemcpyHostToDevice, s), "params");
  const double* gx = static_cast<double*>(gt.p);
  const double* gw = gx + G;
  const int64_t n = o.nelem * nrhs;
  const int tb = 128;
  const int grid = int((n + tb - 1) / tb);
  double* blp = static_cast<double*>(bl.p);
  const double* pp = static_cast<double*>(pr.p);
#define BEMBEL_RHS(D, CP) \
  k_rhs_local<D, CP><<<grid, tb, 0, s>>>(o.geom, o.L, o.nelem, G, gx, gw, kind, pp, nrhs, o.kre, o.kim, blp)
  switch (o.d * 2 + (o.cplx ? 1 : 0)) {
    case 0: BEMBEL_RHS(0, false); break;
    case 1: BEMBEL_RHS(0, true); break;
    case 2: BEMBEL_RHS(1, false); break;
    case 3: BEMBEL_RHS(1, true); break;
    case 4: BEMBEL_RHS(2, false); break;
    default: BEMBEL_RHS(2, true); break;
  }
#undef BEMBEL_RHS
  launched("k_rhs_local");
  scatter_to_global(o, blp, static_cast<double*>(b), nrhs, s);
  cuda_check(cudaStreamSynchronize(s), "rhs sync");
}

void eval_device(const Op& o, const double* pts, int64_t npts, const void* rho, int nrhs, int G, void* out) {
  const cudaStream_t s = o.stream;
  const int C = o.cplx ? 2 : 1;
  const int ncol = nrhs * C;
  const int G2 = G * G;
  Buf gt(sizeof(double) * 2 * G), rl(sizeof(double) * o.nlocal * ncol), rq(sizeof(double) * o.nelem * G2 * ncol);
  gauss_table(G, static_cast<double*>(gt.p), s);
  const double* gx = static_cast<double*>(gt.p);
  const double* gw = gx + G;
  gather_to_local(o, static_cast<const double*>(rho), static_cast<double*>(rl.p), nrhs, s);
  if (o.efie) {
    efie_field(o, static_cast<double*>(rl.p), gx, gw, G, pts, npts, nrhs, static_cast<double*>(out), s);
    return;
  }
  const int64_t nq = o.nelem * G2;
  // the quadrature points of every element for this G, kept with the operator
  Op& om = const_cast<Op&>(o);
  const bool elem32 = o.opts.precision == BEMBEL_PREC_MIXED;
  if (!om.d_evalY || om.evalG != G || (elem32 && !om.d_evalC)) {
    for (void* p : {(void*)om.d_evalY, (void*)om.d_evalC, (void*)om.d_evalRel}) dev_free(p);
    om.d_evalY = nullptr;
    om.d_evalC = nullptr;
    om.d_evalRel = nullptr;
    om.d_evalY = static_cast<double*>(dev_alloc(sizeof(double) * nq * 3));
    om.evalG = G;
    k_tab_points<<<int((nq + 255) / 256), 256, 0, s>>>(o.geom, o.L, o.nelem, G, gx, o.h, om.d_evalY);
    launched("kernel");
    if (elem32) {
      om.d_evalC = static_cast<double*>(dev_alloc(sizeof(double) * o.nelem * 3));
      om.d_evalRel = static_cast<float*>(dev_alloc(sizeof(float) * 4 * nq));
      k_eval_offsets<<<int((o.nelem + 127) / 128), 128, 0, s>>>(om.d_evalY, o.nelem, G2, om.d_evalC,
                                                                reinterpret_cast<float4*>(om.d_evalRel));
      launched("k_eval_offsets");
    }
  }
  struct {
    void* p;
  } Y{om.d_evalY};
  const int64_t nd = nq * ncol;
  switch (o.d) {
    case 0:
      k_density_points<0><<<int((nd + 255) / 256), 256, 0, s>>>(static_cast<double*>(rl.p), o.nelem, G, gx, gw, o.h,
                                                                 ncol, static_cast<double*>(rq.p));
      launched("kernel");
      break;
    case 1:
      k_density_points<1><<<int((nd + 255) / 256), 256, 0, s>>>(static_cast<double*>(rl.p), o.nelem, G, gx, gw, o.h,
                                                                 ncol, static_cast<double*>(rq.p));
      launched("kernel");
      break;
    default:
      k_density_points<2><<<int((nd + 255) / 256), 256, 0, s>>>(static_cast<double*>(rl.p), o.nelem, G, gx, gw, o.h,
                                                                 ncol, static_cast<double*>(rq.p));
      launched("kernel");
      break;
  }
  // source chunks: about eight blocks per SM over all (point, column) pairs, chunks of at
  // least 4,096 quadrature points
  const int64_t pairs = npts * nrhs;
  const int64_t chunks = std::max<int64_t>(1, std::min<int64_t>((152 * 8 + pairs - 1) / pairs, nq / 4096));
  dim3 grid((unsigned)npts, (unsigned)nrhs, (unsigned)chunks);
  cuda_check(cudaMemsetAsync(out, 0, sizeof(double) * npts * nrhs * C, s), "eval clear");
  if (elem32) {
    // MIXED: element-wise sums, FP32 for elements whose centre is farther than 10 h
    Buf rq32(sizeof(float) * nd);
    k_d2f<<<int((nd + 255) / 256), 256, 0, s>>>(static_cast<double*>(rq.p), static_cast<float*>(rq32.p), nd);
    launched("k_d2f");
    const int64_t echunks = std::max<int64_t>(1, std::min<int64_t>((152 * 8 + pairs - 1) / pairs, o.nelem / 256));
    dim3 egrid((unsigned)npts, (unsigned)nrhs, (unsigned)echunks);
    const double far2e = 100.0 * o.h * o.h;
    if (o.cplx)
      k_potential_elem<true><<<egrid, 128, 0, s>>>(pts, npts, om.d_evalY, om.d_evalC,
                                                   reinterpret_cast<const float4*>(om.d_evalRel),
                                                   static_cast<double*>(rq.p), static_cast<float*>(rq32.p), o.nelem,
                                                   G2, nrhs, o.kre, o.kim, far2e, static_cast<double*>(out));
    else
      k_potential_elem<false><<<egrid, 128, 0, s>>>(pts, npts, om.d_evalY, om.d_evalC,
                                                    reinterpret_cast<const float4*>(om.d_evalRel),
                                                    static_cast<double*>(rq.p), static_cast<float*>(rq32.p), o.nelem,
                                                    G2, nrhs, o.kre, o.kim, far2e, static_cast<double*>(out));
    launched("k_potential_elem");
    cuda_check(cudaStreamSynchronize(s), "eval sync");
    return;
  }
  if (o.cplx)
    k_potential<true><<<grid, 256, 0, s>>>(pts, npts, static_cast<double*>(Y.p), static_cast<double*>(rq.p), nq,
                                           nrhs, o.kre, o.kim, static_cast<double*>(out));
  else
    k_potential<false><<<grid, 256, 0, s>>>(pts, npts, static_cast<double*>(Y.p), static_cast<double*>(rq.p), nq,
                                            nrhs, o.kre, o.kim, static_cast<double*>(out));
  launched("eval kernels");
  cuda_check(cudaStreamSynchronize(s), "eval sync");
}

void eval_h2_device(const Op& o, const double* pts, int64_t npts, const void* rho, int nrhs, int G, double eta,
                    void* out) {
  if (o.efie || o.q2 == 0) fail(BEMBEL_EUNSUPPORTED, "eval_h2: compressed S^2 operators only");
  const cudaStream_t s = o.stream;
  const int C = o.cplx ? 2 : 1;
  const int ncol = nrhs * C;
  const int G2 = G * G;
  Buf gt(sizeof(double) * 2 * G), rl(sizeof(double) * o.nlocal * ncol), rq(sizeof(double) * o.nelem * G2 * ncol),
      Y(sizeof(double) * o.nelem * G2 * 3), xh(sizeof(double) * o.nclusters * o.q2 * ncol), err(sizeof(int));
  gauss_table(G, static_cast<double*>(gt.p), s);
  const double* gx = static_cast<double*>(gt.p);
  const double* gw = gx + G;
  cluster_moments(o, static_cast<const double*>(rho), static_cast<double*>(rl.p), static_cast<double*>(xh.p), nrhs,
                  s);
  const int64_t nq = o.nelem * G2;
  k_tab_points<<<int((nq + 255) / 256), 256, 0, s>>>(o.geom, o.L, o.nelem, G, gx, o.h, static_cast<double*>(Y.p));
  launched("k_tab_points");
  const int64_t nd = nq * ncol;
  switch (o.d) {
    case 0:
      k_density_points<0><<<int((nd + 255) / 256), 256, 0, s>>>(static_cast<double*>(rl.p), o.nelem, G, gx, gw, o.h,
                                                                 ncol, static_cast<double*>(rq.p));
      break;
    case 1:
      k_density_points<1><<<int((nd + 255) / 256), 256, 0, s>>>(static_cast<double*>(rl.p), o.nelem, G, gx, gw, o.h,
                                                                 ncol, static_cast<double*>(rq.p));
      break;
    default:
      k_density_points<2><<<int((nd + 255) / 256), 256, 0, s>>>(static_cast<double*>(rl.p), o.nelem, G, gx, gw, o.h,
                                                                 ncol, static_cast<double*>(rq.p));
      break;
  }
  launched("k_density_points");
  cuda_check(cudaMemsetAsync(err.p, 0, sizeof(int), s), "err clear");
  TreeLevels lv{};
  for (int l = 0; l <= o.leaf + 1 && l < 16; ++l) lv.off[l] = o.lvl_off[l];
  dim3 grid(unsigned((npts + kTreeWarps - 1) / kTreeWarps), unsigned(nrhs));
  if (o.cplx)
    k_potential_tree<true><<<grid, 32 * kTreeWarps, 0, s>>>(
        pts, npts, o.d_balls, o.d_nodes, static_cast<double*>(xh.p), o.q2, lv, o.leaf, o.L, static_cast<double*>(Y.p),
        static_cast<double*>(rq.p), G2, ncol, eta, o.opts.kdiam, o.kre, o.kim, static_cast<int*>(err.p),
        static_cast<double*>(out));
  else
    k_potential_tree<false><<<grid, 32 * kTreeWarps, 0, s>>>(
        pts, npts, o.d_balls, o.d_nodes, static_cast<double*>(xh.p), o.q2, lv, o.leaf, o.L, static_cast<double*>(Y.p),
        static_cast<double*>(rq.p), G2, ncol, eta, o.opts.kdiam, o.kre, o.kim, static_cast<int*>(err.p),
        static_cast<double*>(out));
  launched("k_potential_tree");
  int h_err = 0;
  cuda_check(cudaMemcpyAsync(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost, s), "err read");
  cuda_check(cudaStreamSynchronize(s), "eval_h2 sync");
  if (h_err) fail(BEMBEL_EINVAL, "eval_h2: cluster frontier of a point exceeds its capacity (eta too small?)");
}

}  // namespace bembel
