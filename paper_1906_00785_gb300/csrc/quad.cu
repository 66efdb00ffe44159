// quad.cu - assembly kernels (FP64).
//
// A_ij = int int G(gamma(s), gamma(t)) phi_hat_i(s) phi_hat_j(t) ds dt on element
// pairs (Sec. 2 conforming Galerkin scheme; App. E 2-form Piola lift, so no
// surface measure appears), with
//   Laplace   G = 1/(4 pi r)                 (App. B, LS)
//   Helmholtz G = exp(-i kappa r)/(4 pi r)    (App. B, HS), kappa complex.
// * k_tabulate: gamma at the tensor Gauss points of every element.
// * k_near_regular: separated near-field pairs, tensor Gauss g x g per element.
// * k_near_singular<KIND>: identical / common-edge / common-vertex pairs with the
//   Duffy-type regularising transforms (Sec. 2, [SS97]): 8 / 6 / 4 sub-domains
//   of g^4 Gauss points each, sub-domains and variables as described per KIND
//   in duffy_point().
// * k_coupling: far-field coupling K_ab = G(gamma(x_a^tau), gamma(x_b^sigma))
//   at the cluster Chebyshev points (Sec. 2, interpolation on the unit square).
#include <algorithm>
#include <vector>

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

__global__ void k_tabulate(Geom g, int L, int64_t nelem, int G, const double* __restrict__ gx, double h,
                           double* __restrict__ Xq) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= nelem * G * G) return;
  tabulate_point(g, L, G, gx, h, id, Xq);
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

// Separated pairs: the ring next to the touching pairs (pad 0) at order G2 =
// g^2 points per element, farther pairs (pad 1) at their own order G2f.
template <int D, bool CPLX>
__global__ void __launch_bounds__(32 * kWarps) k_near_regular(const PairRec* __restrict__ pairs, int64_t npairs,
                                                              const double* __restrict__ Xq,
                                                              const double* __restrict__ BWg, int G2,
                                                              const double* __restrict__ Xqf,
                                                              const double* __restrict__ BWfg, int G2f, double kre,
                                                              double kim, double* __restrict__ N, int nld) {
  constexpr int NL = (D + 1) * (D + 1);
  constexpr int C = CPLX ? 2 : 1;
  extern __shared__ double sh[];
  const int gmax = max(G2, G2f);
  double* BW = sh;                                                      // G2 * NL
  double* BWf = sh + G2 * NL;                                           // G2f * NL
  double* ubuf = BWf + G2f * NL + (threadIdx.x >> 5) * gmax * NL * C;  // per warp
  for (int i = threadIdx.x; i < G2 * NL; i += blockDim.x) BW[i] = BWg[i];
  for (int i = threadIdx.x; i < G2f * NL; i += blockDim.x) BWf[i] = BWfg[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (int64_t w = blockIdx.x * (int64_t)kWarps + (threadIdx.x >> 5); w < npairs; w += (int64_t)gridDim.x * kWarps) {
    const PairRec& pr = pairs[w];
    if (pr.pad)
      regular_pair<D, CPLX>(pr, Xqf, BWf, ubuf, G2f, kre, kim, N, nld, lane);
    else
      regular_pair<D, CPLX>(pr, Xq, BW, ubuf, G2, kre, kim, N, nld, lane);
  }
}

size_t regular_smem(int G2, int G2f, int NL, int C) {
  return sizeof(double) * ((size_t)G2 * NL + (size_t)G2f * NL + (size_t)kWarps * std::max(G2, G2f) * NL * C);
}

// One touching pair per warp; lanes stride over the nsub * g^4 rule points and
// accumulate the (D+1)^2 x (D+1)^2 block in registers, reduced over the warp.
template <int D, bool CPLX, int KIND>
__device__ __forceinline__ void singular_pair(const PairRec& pr, const Geom& geom, int L, int4 G,
                                              const double (*gx)[kMaxG], const double (*gw)[kMaxG],
                                              double kre, double kim, double* __restrict__ N, int nld, int lane) {
  constexpr int D1 = D + 1;
  constexpr int NL = D1 * D1;
  constexpr int C = CPLX ? 2 : 1;
  // identical pairs: the rule is symmetric under s <-> t (quadrant sigma maps to
  // -sigma with the same weight), so half the sub-domains are integrated and
  // the block is symmetrised at the end: A = M + M^T.
  constexpr int NSUB = KIND == kIdentical ? 4 : (KIND == kEdge ? 6 : 4);
  const int npts = NSUB * G.x * G.y * G.z * G.w;
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
  for (int idx = lane; idx < npts; idx += 32) {
    int sub0, i0, i1, i2, i3;
    rule_index(idx, G, sub0, i0, i1, i2, i3);
    // identical: sub-domains with sigma_1 = +1 only (sub & 1 == 0 -> quadrants (+,+), (+,-))
    const int sub = KIND == kIdentical ? (((sub0 & 1) << 1) | ((sub0 >> 1) << 2)) : sub0;
    double s1, s2, t1, t2;
    const double jac = duffy_point<KIND>(sub, gx[0][i0], gx[1][i1], gx[2][i2], gx[3][i3], s1, s2, t1, t2);
    const double wt = jac * gw[0][i0] * gw[1][i1] * gw[2][i2] * gw[3][i3];
    double ls1, ls2, lt1, lt2;
    apply_cmap(ce, s1, s2, ls1, ls2);
    apply_cmap(cf, t1, t2, lt1, lt2);
    double x[3], y[3];
    gamma_eval(geom, pe, (e1 + ls1) * h, (e2 + ls2) * h, x);
    gamma_eval(geom, pf, (f1 + lt1) * h, (f2 + lt2) * h, y);
    const double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
    double gr, gi;
    kernel_value(CPLX, d0 * d0 + d1 * d1 + d2 * d2, kre, kim, gr, gi);
    gr *= wt;
    gi *= wt;
    double bs1[D1], bs2[D1], bt1[D1], bt2[D1];
    bernstein<D>(ls1, bs1);
    bernstein<D>(ls2, bs2);
    bernstein<D>(lt1, bt1);
    bernstein<D>(lt2, bt2);
#pragma unroll
    for (int i = 0; i < NL; ++i) {
      const double bi = bs1[i % D1] * bs2[i / D1];
      const double wr = gr * bi, wi = gi * bi;
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        const double bj = bt1[j % D1] * bt2[j / D1];
        ar[i * NL + j] = fma(wr, bj, ar[i * NL + j]);
        if (CPLX) ai[i * NL + j] = fma(wi, bj, ai[i * NL + j]);
      }
    }
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

template <int D, bool CPLX, int KIND>
__global__ void __launch_bounds__(32 * kWarps) k_near_singular(const PairRec* __restrict__ pairs, int64_t npairs,
                                                               Geom geom, int L, int4 G,
                                                               const double* __restrict__ gauss, double kre,
                                                               double kim, double* __restrict__ N, int nld) {
  __shared__ double gx[4][kMaxG], gw[4][kMaxG];
  load_rule_tables(gauss, G, gx, gw);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (int64_t w = blockIdx.x * (int64_t)kWarps + (threadIdx.x >> 5); w < npairs; w += (int64_t)gridDim.x * kWarps)
    singular_pair<D, CPLX, KIND>(pairs[w], geom, L, G, gx, gw, kre, kim, N, nld, lane);
}

// Coupling entry id = blk * q2^2 + a * q2 + b (row-major block):
// K[blk][a][b] = G(node_a(target), node_b(source)) / (4 pi).
template <bool CPLX>
__device__ __forceinline__ void coupling_entry(int64_t id, const int* __restrict__ tgt, const int* __restrict__ src,
                                               const double* __restrict__ nodes, int q2, double kre, double kim,
                                               double* __restrict__ K) {
  const int64_t per = (int64_t)q2 * q2;
  const int64_t blk = id / per;
  const int r = int(id % per);
  const int a = r / q2, b = r % q2;
  const double* xa = nodes + ((int64_t)tgt[blk] * q2 + a) * 3;
  const double* xb = nodes + ((int64_t)src[blk] * q2 + b) * 3;
  const double d0 = xa[0] - xb[0], d1 = xa[1] - xb[1], d2 = xa[2] - xb[2];
  double gr, gi;
  kernel_value(CPLX, d0 * d0 + d1 * d1 + d2 * d2, kre, kim, gr, gi);
  if (CPLX) {
    K[id * 2] = gr * kInv4Pi;
    K[id * 2 + 1] = gi * kInv4Pi;
  } else {
    K[id] = gr * kInv4Pi;
  }
}

// Thread per coupling entry.
template <bool CPLX>
__global__ void k_coupling(const int* __restrict__ tgt, const int* __restrict__ src, int64_t nfar,
                           const double* __restrict__ nodes, int q2, double kre, double kim, double* __restrict__ K) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= nfar * (int64_t)q2 * q2) return;
  coupling_entry<CPLX>(id, tgt, src, nodes, q2, kre, kim, K);
}

template <typename T>
__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = float(a[i]);
}

int4 rule_orders(const Op& o, int kind) {
  return make_int4(o.g_var[kind][0], o.g_var[kind][1], o.g_var[kind][2], o.g_var[kind][3]);
}

int grid_for(int64_t work, int per_block) {
  int64_t g = (work + per_block - 1) / per_block;
  return int(std::min<int64_t>(std::max<int64_t>(g, 1), 1 << 30));
}

template <int D, bool CPLX>
void launch_pairs(Op& o, cudaEvent_t* ev) {
  const cudaStream_t s = o.stream;
  const int G2 = o.g_reg * o.g_reg;
  const int NL = (D + 1) * (D + 1);
  const int threads = 32 * kWarps;
  if (o.npairs[kRegular] > 0) {
    const int G2f = o.g_reg_far * o.g_reg_far;
    const size_t shm = regular_smem(G2, G2f, NL, CPLX ? 2 : 1);
    if (shm > 48 * 1024)
      cuda_check(cudaFuncSetAttribute(k_near_regular<D, CPLX>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(shm)),
                 "smem attr");
    const int grid = int(std::min<int64_t>((o.npairs[kRegular] + kWarps - 1) / kWarps, 152 * 64));
    k_near_regular<D, CPLX><<<grid, threads, shm, s>>>(o.d_pairs[kRegular], o.npairs[kRegular], o.d_Xq, o.d_BW,
                                                       G2, o.d_Xq_far, o.d_BW_far, G2f, o.kre, o.kim, o.d_N, o.nld);
    launched("k_near_regular");
  }
  cuda_check(cudaEventRecord(ev[2], s), "event");

  auto grid_of = [](int64_t n) { return int(std::min<int64_t>((n + kWarps - 1) / kWarps, 152 * 64)); };
  if (o.npairs[kIdentical] > 0) {
    k_near_singular<D, CPLX, kIdentical><<<grid_of(o.npairs[kIdentical]), threads, 0, s>>>(
        o.d_pairs[kIdentical], o.npairs[kIdentical], o.geom, o.L, rule_orders(o, kIdentical), o.d_gauss + o.gauss_off[kIdentical], o.kre,
        o.kim, o.d_N, o.nld);
    launched("k_near_singular identical");
  }
  cuda_check(cudaEventRecord(ev[3], s), "event");
  if (o.npairs[kEdge] > 0) {
    k_near_singular<D, CPLX, kEdge><<<grid_of(o.npairs[kEdge]), threads, 0, s>>>(
        o.d_pairs[kEdge], o.npairs[kEdge], o.geom, o.L, rule_orders(o, kEdge), o.d_gauss + o.gauss_off[kEdge], o.kre,
        o.kim, o.d_N, o.nld);
    launched("k_near_singular edge");
  }
  cuda_check(cudaEventRecord(ev[4], s), "event");
  if (o.npairs[kVertex] > 0) {
    k_near_singular<D, CPLX, kVertex><<<grid_of(o.npairs[kVertex]), threads, 0, s>>>(
        o.d_pairs[kVertex], o.npairs[kVertex], o.geom, o.L, rule_orders(o, kVertex), o.d_gauss + o.gauss_off[kVertex], o.kre,
        o.kim, o.d_N, o.nld);
    launched("k_near_singular vertex");
  }
  cuda_check(cudaEventRecord(ev[5], s), "event");
}

}  // namespace

void alloc_assembly_outputs(Op& o) {
  const int C = o.cplx ? 2 : 1;
  const int64_t nN = o.nnear * (int64_t)o.nld * o.nld * C;
  const int64_t nK = o.nfar * (int64_t)o.q2 * o.q2 * (o.efie ? 5 : 1);  // EFIE: five coupling matrices
  o.d_Xq = static_cast<double*>(dev_alloc(sizeof(double) * o.nelem * o.g_reg * o.g_reg * 3));
  o.d_Xq_far = static_cast<double*>(dev_alloc(sizeof(double) * o.nelem * o.g_reg_far * o.g_reg_far * 3));
  o.d_N = static_cast<double*>(dev_alloc(sizeof(double) * std::max<int64_t>(nN, 1)));
  if (nK > 0) o.d_K = static_cast<double*>(dev_alloc(sizeof(double) * nK * C));
  if (o.opts.precision == BEMBEL_PREC_MIXED) {
    o.d_N32 = static_cast<float*>(dev_alloc(sizeof(float) * std::max<int64_t>(nN, 1)));
  }
}

void run_assembly_kernels(Op& o) {
  const cudaStream_t s = o.stream;
  const int C = o.cplx ? 2 : 1;
  // phase events: 0 tabulation, 1 regular, 2 identical, 3 edge, 4 vertex, 5 coupling, 6 FP32 copies
  cudaEvent_t ev[8];
  for (auto& e : ev) cuda_check(cudaEventCreate(&e), "event");
  // outputs first, so that no allocation falls between the phase events
  const int64_t nN = o.nnear * (int64_t)o.nld * o.nld * C;
  const int64_t nK = o.nfar * (int64_t)o.q2 * o.q2;
  alloc_assembly_outputs(o);
  cuda_check(cudaEventRecord(ev[0], s), "event");
  // A1: tabulation of gamma at the regular Gauss points
  {
    const int64_t n = o.nelem * o.g_reg * o.g_reg;
    k_tabulate<<<grid_for(n, 256), 256, 0, s>>>(o.geom, o.L, o.nelem, o.g_reg, o.d_gauss, o.h, o.d_Xq);
    launched("k_tabulate");
    const int64_t nf = o.nelem * o.g_reg_far * o.g_reg_far;
    k_tabulate<<<grid_for(nf, 256), 256, 0, s>>>(o.geom, o.L, o.nelem, o.g_reg_far, o.d_gauss + o.gauss_off_far, o.h,
                                                 o.d_Xq_far);
    launched("k_tabulate");
  }
  cuda_check(cudaEventRecord(ev[1], s), "event");
  // A4 + A5: near field (S^1 functions for the EFIE)
  if (o.efie) {
    efie_pair_kernels(o, ev);
  } else {
    switch (o.d * 2 + (o.cplx ? 1 : 0)) {
      case 0: launch_pairs<0, false>(o, ev); break;
      case 1: launch_pairs<0, true>(o, ev); break;
      case 2: launch_pairs<1, false>(o, ev); break;
      case 3: launch_pairs<1, true>(o, ev); break;
      case 4: launch_pairs<2, false>(o, ev); break;
      default: launch_pairs<2, true>(o, ev); break;
    }
  }
  // A6: coupling
  if (o.nfar > 0 && o.efie) {
    efie_coupling_assemble(o);
  } else if (o.nfar > 0) {
    const int64_t n = nK;
    if (o.cplx)
      k_coupling<true><<<grid_for(n, 256), 256, 0, s>>>(o.d_far_tgt, o.d_far_src, o.nfar, o.d_nodes, o.q2, o.kre,
                                                        o.kim, o.d_K);
    else
      k_coupling<false><<<grid_for(n, 256), 256, 0, s>>>(o.d_far_tgt, o.d_far_src, o.nfar, o.d_nodes, o.q2, o.kre,
                                                         o.kim, o.d_K);
    launched("k_coupling");
  }
  cuda_check(cudaEventRecord(ev[6], s), "event");
  // FP32 copies for the mixed-precision inner solves
  if (o.opts.precision == BEMBEL_PREC_MIXED) {
    k_to_f32<float><<<1024, 256, 0, s>>>(o.d_N, o.d_N32, nN);
    launched("k_to_f32");
  }
  cuda_check(cudaEventRecord(ev[7], s), "event");
  cuda_check(cudaEventSynchronize(ev[7]), "assembly sync");
  for (int i = 0; i < 7; ++i) {
    float ms = 0.f;
    cuda_check(cudaEventElapsedTime(&ms, ev[i], ev[i + 1]), "event time");
    o.info.phase_ms[i] = ms;
  }
  o.info.phase_ms[7] = 0.0;
  for (auto& e : ev) cudaEventDestroy(e);
}

// ---------------------------------------------------------------------------
// Several meshes in one persistent launch.  The near field (regular and the
// three touching classes) and the coupling of all meshes form one global work
// list: a table of segments (mesh, phase, units, units per item) in shared
// memory; warps take item numbers from one atomic counter, most expensive
// phases first, and run the same per-pair device functions as the single-mesh
// kernels (so each block is bit-identical to a single-mesh assembly).
// Tabulation runs before, the FP32 copies after, as separate launches: no
// kernel waits on another.
// ---------------------------------------------------------------------------
namespace {

constexpr int kPhaseCoupling = 4;
constexpr int kMaxSegments = 5 * kMaxBatch;

struct MeshWork {
  Geom geom;
  int L, nld;
  const double* BW;  // regular basis x weight table (holds h^2: per level)
  const double* BWf; // the same for the far separated order
  double* Xqf;
  double kre, kim, h;
  int64_t nelem;
  double* Xq;
  double* N;
  float* N32;
  int64_t nN;  // near-field reals
  const PairRec* pairs[4];
  const int* far_tgt;
  const int* far_src;
  const double* nodes;
  double* K;
};

struct Segment {
  int mesh, phase, chunk, pad;
  long long units, item0;  // units (pairs or blocks) and first global item number
};

__global__ void k_tabulate_multi(const MeshWork* __restrict__ ms, const long long* __restrict__ off, int nmesh, int G,
                                 const double* __restrict__ gx, bool far) {
  const long long total = off[nmesh];
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    int m = 0;
    while (id >= off[m + 1]) ++m;
    tabulate_point(ms[m].geom, ms[m].L, G, gx, ms[m].h, id - off[m], far ? ms[m].Xqf : ms[m].Xq);
  }
}

__global__ void k_to_f32_multi(const MeshWork* __restrict__ ms, const long long* __restrict__ off, int nmesh) {
  const long long total = off[nmesh];
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    int m = 0;
    while (id >= off[m + 1]) ++m;
    ms[m].N32[id - off[m]] = float(ms[m].N[id - off[m]]);
  }
}

template <int D, bool CPLX>
__global__ void __launch_bounds__(32 * kWarps) k_assemble_multi(const MeshWork* __restrict__ ms,
                                                                const Segment* __restrict__ segs_g, int nseg,
                                                                long long nitems, unsigned long long* __restrict__ next,
                                                                int G2, int G2f,
                                                                const double* __restrict__ gauss, int4 gi, int4 ge,
                                                                int4 gv, int3 goff, int q2) {
  constexpr int NL = (D + 1) * (D + 1);
  constexpr int C = CPLX ? 2 : 1;
  extern __shared__ double sh[];
  double* ubuf = sh + (threadIdx.x >> 5) * max(G2, G2f) * NL * C;
  __shared__ double gx[3][4][kMaxG], gw[3][4][kMaxG];
  __shared__ Segment segs[kMaxSegments];
  for (int i = threadIdx.x; i < nseg; i += blockDim.x) segs[i] = segs_g[i];
  load_rule_tables(gauss + goff.x, gi, gx[0], gw[0]);
  load_rule_tables(gauss + goff.y, ge, gx[1], gw[1]);
  load_rule_tables(gauss + goff.z, gv, gx[2], gw[2]);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long it = 0;
    if (lane == 0) it = atomicAdd(next, 1ull);
    it = __shfl_sync(0xffffffffu, it, 0);
    if ((long long)it >= nitems) break;
    int si = 0;
    while (si + 1 < nseg && (long long)it >= segs[si + 1].item0) ++si;
    const Segment sg = segs[si];
    const MeshWork& m = ms[sg.mesh];
    const long long first = ((long long)it - sg.item0) * sg.chunk;
    const long long last = min(sg.units, first + sg.chunk);
    switch (sg.phase) {
      case kRegular:
        for (long long w = first; w < last; ++w)
          if (m.pairs[kRegular][w].pad)
            regular_pair<D, CPLX>(m.pairs[kRegular][w], m.Xqf, m.BWf, ubuf, G2f, m.kre, m.kim, m.N, m.nld, lane);
          else
            regular_pair<D, CPLX>(m.pairs[kRegular][w], m.Xq, m.BW, ubuf, G2, m.kre, m.kim, m.N, m.nld, lane);
        break;
      case kIdentical:
        for (long long w = first; w < last; ++w)
          singular_pair<D, CPLX, kIdentical>(m.pairs[kIdentical][w], m.geom, m.L, gi, gx[0], gw[0], m.kre, m.kim,
                                             m.N, m.nld, lane);
        break;
      case kEdge:
        for (long long w = first; w < last; ++w)
          singular_pair<D, CPLX, kEdge>(m.pairs[kEdge][w], m.geom, m.L, ge, gx[1], gw[1], m.kre, m.kim, m.N,
                                        m.nld, lane);
        break;
      case kVertex:
        for (long long w = first; w < last; ++w)
          singular_pair<D, CPLX, kVertex>(m.pairs[kVertex][w], m.geom, m.L, gv, gx[2], gw[2], m.kre, m.kim, m.N,
                                          m.nld, lane);
        break;
      default: {
        const long long per = (long long)q2 * q2;
        for (long long id = first * per + lane; id < last * per; id += 32)
          coupling_entry<CPLX>(id, m.far_tgt, m.far_src, m.nodes, q2, m.kre, m.kim, m.K);
        break;
      }
    }
  }
}

template <int D, bool CPLX>
void launch_multi(const std::vector<Op*>& ops, const MeshWork* d_ms, const Segment* d_seg, int nseg, long long nitems,
                  unsigned long long* d_next, cudaStream_t s) {
  const Op& o = *ops[0];
  const int G2 = o.g_reg * o.g_reg;
  const int NL = (D + 1) * (D + 1);
  const int G2f = o.g_reg_far * o.g_reg_far;
  const size_t shm = sizeof(double) * (kWarps * std::max(G2, G2f) * NL * (CPLX ? 2 : 1));
  if (shm > 48 * 1024)
    cuda_check(cudaFuncSetAttribute(k_assemble_multi<D, CPLX>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(shm)),
               "smem attr");
  int per_sm = 0;
  cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_assemble_multi<D, CPLX>, 32 * kWarps, shm),
             "occupancy");
  int dev = 0, nsm = 0;
  cuda_check(cudaGetDevice(&dev), "device");
  cuda_check(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "sm count");
  const long long want = (nitems + kWarps - 1) / kWarps;
  const int grid = int(std::max<long long>(1, std::min<long long>(want, (long long)std::max(1, per_sm) * nsm)));
  const int3 goff = make_int3(int(o.gauss_off[kIdentical]), int(o.gauss_off[kEdge]), int(o.gauss_off[kVertex]));
  k_assemble_multi<D, CPLX><<<grid, 32 * kWarps, shm, s>>>(d_ms, d_seg, nseg, nitems, d_next, G2, G2f, o.d_gauss,
                                                           rule_orders(o, kIdentical), rule_orders(o, kEdge),
                                                           rule_orders(o, kVertex), goff, o.q2);
  launched("k_assemble_multi");
}

}  // namespace

void run_assembly_batch(const std::vector<Op*>& ops) {
  const int nmesh = int(ops.size());
  if (nmesh < 1 || nmesh > kMaxBatch) fail(BEMBEL_EINVAL, "assemble_batch: 1..64 meshes");
  const Op& o0 = *ops[0];
  const cudaStream_t s = o0.stream;
  const int C = o0.cplx ? 2 : 1;
  const bool mixed = o0.opts.precision == BEMBEL_PREC_MIXED;
  for (Op* o : ops) alloc_assembly_outputs(*o);
  // per-mesh descriptors and offsets of the tabulation and copy ranges
  std::vector<MeshWork> mw(nmesh);
  std::vector<long long> tab_off(nmesh + 1, 0), tabf_off(nmesh + 1, 0), cpy_off(nmesh + 1, 0);
  for (int m = 0; m < nmesh; ++m) {
    const Op& o = *ops[m];
    MeshWork& w = mw[m];
    w.geom = o.geom;
    w.L = o.L;
    w.nld = o.nld;
    w.BW = o.d_BW;
    w.BWf = o.d_BW_far;
    w.Xqf = o.d_Xq_far;
    w.kre = o.kre;
    w.kim = o.kim;
    w.h = o.h;
    w.nelem = o.nelem;
    w.Xq = o.d_Xq;
    w.N = o.d_N;
    w.N32 = o.d_N32;
    w.nN = o.nnear * (int64_t)o.nld * o.nld * C;
    for (int k = 0; k < 4; ++k) w.pairs[k] = o.d_pairs[k];
    w.far_tgt = o.d_far_tgt;
    w.far_src = o.d_far_src;
    w.nodes = o.d_nodes;
    w.K = o.d_K;
    tab_off[m + 1] = tab_off[m] + o.nelem * (long long)o.g_reg * o.g_reg;
    tabf_off[m + 1] = tabf_off[m] + o.nelem * (long long)o.g_reg_far * o.g_reg_far;
    cpy_off[m + 1] = cpy_off[m] + (mixed ? w.nN : 0);
  }
  // segments: most expensive phases first (edge, identical, vertex, regular, coupling)
  std::vector<Segment> seg;
  long long nitems = 0;
  const int order[5] = {kEdge, kIdentical, kVertex, kRegular, kPhaseCoupling};
  const int chunk_of[5] = {4, 1, 1, 1, 8};  // units per item, indexed by phase
  for (int ph : order)
    for (int m = 0; m < nmesh; ++m) {
      const Op& o = *ops[m];
      const long long units = ph == kPhaseCoupling ? o.nfar : o.npairs[ph];
      if (units <= 0) continue;
      Segment sg{};
      sg.mesh = m;
      sg.phase = ph;
      sg.chunk = chunk_of[ph];
      sg.units = units;
      sg.item0 = nitems;
      nitems += (units + sg.chunk - 1) / sg.chunk;
      seg.push_back(sg);
    }
  DevBuf dms(sizeof(MeshWork) * nmesh), dseg(sizeof(Segment) * std::max<size_t>(1, seg.size())),
      dtab(sizeof(long long) * (nmesh + 1)), dtabf(sizeof(long long) * (nmesh + 1)),
      dcpy(sizeof(long long) * (nmesh + 1)), dnext(sizeof(unsigned long long));
  cuda_check(cudaMemcpyAsync(dms.p, mw.data(), sizeof(MeshWork) * nmesh, cudaMemcpyHostToDevice, s), "mesh upload");
  if (!seg.empty())
    cuda_check(cudaMemcpyAsync(dseg.p, seg.data(), sizeof(Segment) * seg.size(), cudaMemcpyHostToDevice, s),
               "segments");
  cuda_check(cudaMemcpyAsync(dtab.p, tab_off.data(), sizeof(long long) * (nmesh + 1), cudaMemcpyHostToDevice, s),
             "offsets");
  cuda_check(cudaMemcpyAsync(dcpy.p, cpy_off.data(), sizeof(long long) * (nmesh + 1), cudaMemcpyHostToDevice, s),
             "offsets");
  cuda_check(cudaMemcpyAsync(dtabf.p, tabf_off.data(), sizeof(long long) * (nmesh + 1), cudaMemcpyHostToDevice, s),
             "offsets");
  cuda_check(cudaMemsetAsync(dnext.p, 0, sizeof(unsigned long long), s), "counter");
  const MeshWork* d_ms = static_cast<const MeshWork*>(dms.p);
  cudaEvent_t ev[4];
  for (auto& e : ev) cuda_check(cudaEventCreate(&e), "event");
  cuda_check(cudaEventRecord(ev[0], s), "event");
  k_tabulate_multi<<<grid_for(tab_off[nmesh], 256), 256, 0, s>>>(d_ms, static_cast<const long long*>(dtab.p), nmesh,
                                                                  o0.g_reg, o0.d_gauss, false);
  launched("k_tabulate_multi");
  k_tabulate_multi<<<grid_for(tabf_off[nmesh], 256), 256, 0, s>>>(d_ms, static_cast<const long long*>(dtabf.p),
                                                                   nmesh, o0.g_reg_far, o0.d_gauss + o0.gauss_off_far,
                                                                   true);
  launched("k_tabulate_multi");
  cuda_check(cudaEventRecord(ev[1], s), "event");
  if (nitems > 0) {
    const Segment* d_seg = static_cast<const Segment*>(dseg.p);
    auto* d_next = static_cast<unsigned long long*>(dnext.p);
    const int nseg = int(seg.size());
    switch (o0.d * 2 + (o0.cplx ? 1 : 0)) {
      case 0: launch_multi<0, false>(ops, d_ms, d_seg, nseg, nitems, d_next, s); break;
      case 1: launch_multi<0, true>(ops, d_ms, d_seg, nseg, nitems, d_next, s); break;
      case 2: launch_multi<1, false>(ops, d_ms, d_seg, nseg, nitems, d_next, s); break;
      case 3: launch_multi<1, true>(ops, d_ms, d_seg, nseg, nitems, d_next, s); break;
      case 4: launch_multi<2, false>(ops, d_ms, d_seg, nseg, nitems, d_next, s); break;
      default: launch_multi<2, true>(ops, d_ms, d_seg, nseg, nitems, d_next, s); break;
    }
  }
  cuda_check(cudaEventRecord(ev[2], s), "event");
  if (mixed && cpy_off[nmesh] > 0) {
    k_to_f32_multi<<<1024, 256, 0, s>>>(d_ms, static_cast<const long long*>(dcpy.p), nmesh);
    launched("k_to_f32_multi");
  }
  cuda_check(cudaEventRecord(ev[3], s), "event");
  cuda_check(cudaEventSynchronize(ev[3]), "batch sync");
  float t[3] = {0.f, 0.f, 0.f};
  for (int i = 0; i < 3; ++i) cuda_check(cudaEventElapsedTime(&t[i], ev[i], ev[i + 1]), "event time");
  for (Op* o : ops) {
    for (double& v : o->info.phase_ms) v = 0.0;
    o->info.phase_ms[0] = t[0];
    o->info.phase_ms[6] = t[2];
    o->info.phase_ms[7] = t[1];
  }
  for (auto& e : ev) cudaEventDestroy(e);
}

// ---------------------------------------------------------------------------
// Autotuner support: integrate a sample of pairs of one kind at order g and at a
// reference order g_ref into compact blocks and return the largest relative
// Frobenius difference over the sample.
// ---------------------------------------------------------------------------
namespace {

template <int D, bool CPLX>
void run_sample(Op& o, int kind, const PairRec* d_sample, int64_t ns, const int gv[4], double* out) {
  const cudaStream_t s = o.stream;
  const int nloc = (D + 1) * (D + 1);
  const int g = gv[0];  // regular pairs: one order
  std::vector<double> gx, gw;
  gauss01(g, gx, gw);
  // per-variable tables (nodes, weights) for the Duffy rules
  std::vector<double> tab;
  for (int v = 0; v < 4; ++v) {
    std::vector<double> x, w;
    gauss01(kind == kRegular ? g : gv[v], x, w);
    tab.insert(tab.end(), x.begin(), x.end());
    tab.insert(tab.end(), w.begin(), w.end());
  }
  const int4 g4 = make_int4(gv[0], gv[1], gv[2], gv[3]);
  double* d_tab = static_cast<double*>(dev_alloc(sizeof(double) * tab.size()));
  cuda_check(cudaMemcpy(d_tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice), "tab");
  const int threads = 32 * kWarps;
  const int grid = int(std::min<int64_t>((ns + kWarps - 1) / kWarps, 152 * 64));
  if (kind == kRegular) {
    const int G2 = g * g;
    double* Xq = static_cast<double*>(dev_alloc(sizeof(double) * o.nelem * G2 * 3));
    std::vector<double> BW((size_t)G2 * nloc);
    for (int p2 = 0; p2 < g; ++p2)
      for (int p1 = 0; p1 < g; ++p1)
        for (int k2 = 0; k2 <= D; ++k2)
          for (int k1 = 0; k1 <= D; ++k1)
            BW[(size_t)(p1 + g * p2) * nloc + k1 + (D + 1) * k2] =
                gw[p1] * gw[p2] * o.h * o.h * bernstein_h(D, k1, gx[p1]) * bernstein_h(D, k2, gx[p2]);
    double* d_BW = static_cast<double*>(dev_alloc(sizeof(double) * BW.size()));
    cuda_check(cudaMemcpy(d_BW, BW.data(), sizeof(double) * BW.size(), cudaMemcpyHostToDevice), "BW");
    k_tabulate<<<grid_for(o.nelem * G2, 256), 256, 0, s>>>(o.geom, o.L, o.nelem, g, d_tab, o.h, Xq);
    launched("k_tabulate");
    const size_t shm = regular_smem(G2, G2, nloc, CPLX ? 2 : 1);
    if (shm > 48 * 1024)
      cuda_check(cudaFuncSetAttribute(k_near_regular<D, CPLX>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(shm)),
                 "smem attr");
    k_near_regular<D, CPLX><<<grid, threads, shm, s>>>(d_sample, ns, Xq, d_BW, G2, Xq, d_BW, G2, o.kre, o.kim, out,
                                                       nloc);
    launched("k_near_regular");
    cuda_check(cudaStreamSynchronize(s), "sample sync");
    dev_free(Xq);
    dev_free(d_BW);
  } else if (kind == kIdentical) {
    k_near_singular<D, CPLX, kIdentical><<<grid, threads, 0, s>>>(d_sample, ns, o.geom, o.L, g4, d_tab, o.kre, o.kim,
                                                                  out, nloc);
    launched("k_near_singular");
  } else if (kind == kEdge) {
    k_near_singular<D, CPLX, kEdge><<<grid, threads, 0, s>>>(d_sample, ns, o.geom, o.L, g4, d_tab, o.kre, o.kim, out,
                                                             nloc);
    launched("k_near_singular");
  } else {
    k_near_singular<D, CPLX, kVertex><<<grid, threads, 0, s>>>(d_sample, ns, o.geom, o.L, g4, d_tab, o.kre, o.kim,
                                                               out, nloc);
    launched("k_near_singular");
  }
  cuda_check(cudaStreamSynchronize(s), "sample sync");
  dev_free(d_tab);
}

}  // namespace

double sample_pair_error(Op& o, int kind, const int g[4], int g_ref, int max_pairs, std::vector<double>* ref_cache,
                         int cls) {
  const int C = o.cplx ? 2 : 1;
  const int nloc = o.nloc;
  // up to max_pairs pairs from the start of the list (built in parallel, so not
  // ordered by position), of the given separation class (separated pairs; -1:
  // any), each given a compact output block
  const int64_t look = std::min<int64_t>(o.npairs[kind], cls < 0 ? max_pairs : 16 * (int64_t)max_pairs);
  std::vector<PairRec> all(look);
  if (look > 0)
    cuda_check(cudaMemcpy(all.data(), o.d_pairs[kind], sizeof(PairRec) * look, cudaMemcpyDeviceToHost), "sample");
  if (cls >= 0)
    all.erase(std::remove_if(all.begin(), all.end(), [&](const PairRec& p) { return p.pad != cls; }), all.end());
  if ((int64_t)all.size() > max_pairs) all.resize(max_pairs);
  const int64_t ns = (int64_t)all.size();
  if (ns == 0) return 0.0;
  for (int64_t i = 0; i < ns; ++i) {
    all[i].off1 = i * (long long)nloc * nloc;
    all[i].off2 = -1;
  }
  PairRec* d_sample = static_cast<PairRec*>(dev_alloc(sizeof(PairRec) * ns));
  cuda_check(cudaMemcpy(d_sample, all.data(), sizeof(PairRec) * ns, cudaMemcpyHostToDevice), "sample up");
  const size_t nb = (size_t)ns * nloc * nloc * C;
  double* d_a = static_cast<double*>(dev_alloc(sizeof(double) * nb));
  double* d_b = static_cast<double*>(dev_alloc(sizeof(double) * nb));
  auto run = [&](const int* gg, double* out) {
    switch (o.d * 2 + (o.cplx ? 1 : 0)) {
      case 0: run_sample<0, false>(o, kind, d_sample, ns, gg, out); break;
      case 1: run_sample<0, true>(o, kind, d_sample, ns, gg, out); break;
      case 2: run_sample<1, false>(o, kind, d_sample, ns, gg, out); break;
      case 3: run_sample<1, true>(o, kind, d_sample, ns, gg, out); break;
      case 4: run_sample<2, false>(o, kind, d_sample, ns, gg, out); break;
      default: run_sample<2, true>(o, kind, d_sample, ns, gg, out); break;
    }
  };
  run(g, d_a);
  std::vector<double> a(nb), b;
  cuda_check(cudaMemcpy(a.data(), d_a, sizeof(double) * nb, cudaMemcpyDeviceToHost), "sample down");
  if (ref_cache && ref_cache->size() == nb) {
    b = *ref_cache;  // reference blocks of this sample at g_ref, computed earlier
  } else {
    const int gr[4] = {g_ref, g_ref, g_ref, g_ref};
    run(gr, d_b);
    b.resize(nb);
    cuda_check(cudaMemcpy(b.data(), d_b, sizeof(double) * nb, cudaMemcpyDeviceToHost), "sample down");
    if (ref_cache) *ref_cache = b;
  }
  dev_free(d_sample);
  dev_free(d_a);
  dev_free(d_b);
  double worst = 0.0;
  const size_t per = (size_t)nloc * nloc * C;
  for (int64_t i = 0; i < ns; ++i) {
    double num = 0.0, den = 0.0;
    for (size_t k = 0; k < per; ++k) {
      const double dd = a[i * per + k] - b[i * per + k];
      num += dd * dd;
      den += b[i * per + k] * b[i * per + k];
    }
    if (den > 0) worst = std::max(worst, std::sqrt(num / den));
  }
  return worst;
}

}  // namespace bembel
