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
//   in duffy_point(); edge and vertex rule sums taken in factorised form
//   (pairkernels.cuh).
// * k_coupling: far-field coupling K_ab = G(gamma(x_a^tau), gamma(x_b^sigma))
//   at the cluster Chebyshev points (Sec. 2, interpolation on the unit square).
#include <algorithm>
#include <vector>

#include "op.h"
#include "pairkernels.cuh"

namespace bembel {

namespace {

__global__ void k_tabulate(Geom g, int L, int64_t nelem, int G, const double* __restrict__ gx, double h,
                           double* __restrict__ Xq) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= nelem * G * G) return;
  tabulate_point(g, L, G, gx, h, id, Xq);
}

// Separated pairs: the ring next to the touching pairs (pad 0) at order G2 =
// g^2 points per element, farther pairs (pad 1) at their own order G2f, with
// the kernel in FP32 when Xqf32 is given (MIXED operators; regular_pair_f32).
template <int D, bool CPLX>
__global__ void __launch_bounds__(32 * kWarps) k_near_regular(const PairRec* __restrict__ pairs, int64_t npairs,
                                                              const double* __restrict__ Xq,
                                                              const double* __restrict__ BWg, int G2,
                                                              const double* __restrict__ Xqf,
                                                              const double* __restrict__ BWfg, int G2f, double kre,
                                                              double kim, double* __restrict__ N, int nld,
                                                              const float4* __restrict__ Xqf32,
                                                              const double* __restrict__ cen) {
  constexpr int NL = (D + 1) * (D + 1);
  constexpr int C = CPLX ? 2 : 1;
  extern __shared__ double sh[];
  const int gmax = max(G2, G2f);
  double* BW = sh;                                                      // G2 * NL
  double* BWf = sh + G2 * NL;                                           // G2f * NL
  double* ubuf = BWf + G2f * NL + (threadIdx.x >> 5) * gmax * NL * C;  // per warp
  float* BWf32 = reinterpret_cast<float*>(BWf + G2f * NL + kWarps * gmax * NL * C);  // G2f * NL (FP32 path)
  for (int i = threadIdx.x; i < G2 * NL; i += blockDim.x) BW[i] = BWg[i];
  for (int i = threadIdx.x; i < G2f * NL; i += blockDim.x) {
    BWf[i] = BWfg[i];
    if (Xqf32) BWf32[i] = float(BWfg[i]);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (int64_t w = blockIdx.x * (int64_t)kWarps + (threadIdx.x >> 5); w < npairs; w += (int64_t)gridDim.x * kWarps) {
    const PairRec& pr = pairs[w];
    if (pr.pad && Xqf32)
      regular_pair_f32<D, CPLX>(pr, Xqf32, cen, BWf32, BWf, ubuf, G2f, float(kre), float(kim), N, nld, lane);
    else if (pr.pad)
      regular_pair<D, CPLX>(pr, Xqf, BWf, ubuf, G2f, kre, kim, N, nld, lane);
    else
      regular_pair<D, CPLX>(pr, Xq, BW, ubuf, G2, kre, kim, N, nld, lane);
  }
}

// FP32 copy of the far-order points for regular_pair_f32: per element the mean
// of its G2 points (FP64) and each point as an FP32 offset from it.
__global__ void k_points_f32(const double* __restrict__ Xq, int64_t nelem, int G2, float4* __restrict__ X32,
                             double* __restrict__ cen) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nelem) return;
  const double* x = Xq + e * G2 * 3;
  double c[3] = {0.0, 0.0, 0.0};
  for (int p = 0; p < G2; ++p)
    for (int k = 0; k < 3; ++k) c[k] += x[p * 3 + k];
  for (int k = 0; k < 3; ++k) c[k] /= G2;
  for (int p = 0; p < G2; ++p)
    X32[e * G2 + p] = make_float4(float(x[p * 3] - c[0]), float(x[p * 3 + 1] - c[1]), float(x[p * 3 + 2] - c[2]), 0.f);
  for (int k = 0; k < 3; ++k) cen[e * 4 + k] = c[k];
  cen[e * 4 + 3] = 0.0;
}

template <int D, bool CPLX, int KIND>
__global__ void __launch_bounds__(32 * kWarps) k_near_singular(const PairRec* __restrict__ pairs, int64_t npairs,
                                                               Geom geom, int L, int4 G,
                                                               const double* __restrict__ gauss, double kre,
                                                               double kim, double* __restrict__ N, int nld) {
  __shared__ double gx[4][kMaxG], gw[4][kMaxG];
  extern __shared__ double stage_all[];
  load_rule_tables(gauss, G, gx, gw);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  double* stage = stage_all + (threadIdx.x >> 5) * stage_doubles(KIND, (D + 1) * (D + 1));
  for (int64_t w = blockIdx.x * (int64_t)kWarps + (threadIdx.x >> 5); w < npairs; w += (int64_t)gridDim.x * kWarps)
    singular_pair<D, CPLX, KIND>(pairs[w], geom, L, G, gx, gw, kre, kim, N, nld, lane, stage);
}

// launch of k_near_singular with its staging buffers
template <int D, bool CPLX, int KIND>
void launch_singular(int grid, cudaStream_t s, const PairRec* pairs, int64_t npairs, const Geom& geom, int L, int4 G,
                     const double* gauss, double kre, double kim, double* N, int nld) {
  const size_t shm = sizeof(double) * kWarps * stage_doubles(KIND, (D + 1) * (D + 1));
  if (shm > 0)  // opt in: the static rule tables come on top of shm
    cuda_check(cudaFuncSetAttribute(k_near_singular<D, CPLX, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    int(shm)),
               "smem attr");
  k_near_singular<D, CPLX, KIND><<<grid, 32 * kWarps, shm, s>>>(pairs, npairs, geom, L, G, gauss, kre, kim, N, nld);
  launched("k_near_singular");
}

// CTA per far block (grid-stride over the blocks), the block's q2 x q2 entries over its
// threads.  MIXED operators with FP32 point offsets: entries by coupling_entry_f32.
template <bool CPLX>
__global__ void k_coupling(const int* __restrict__ tgt, const int* __restrict__ src, int64_t nfar,
                           const double* __restrict__ nodes, int q2, double kre, double kim, double* __restrict__ K,
                           bool f32k, const double* __restrict__ ccen, const float4* __restrict__ rel) {
  const int per = q2 * q2;
  if (f32k && rel) {
    // the block's centre difference once per CTA (FP64 work per block, not per entry)
    __shared__ float3 sdc;
    __shared__ int st, ssc;
    for (int64_t blk = blockIdx.x; blk < nfar; blk += gridDim.x) {
      if (threadIdx.x == 0) {
        st = tgt[blk];
        ssc = src[blk];
        sdc = centre_difference(ccen, st, ssc);
      }
      __syncthreads();
      const int t = st, sc = ssc;
      const float3 dc = sdc;
      for (int r = threadIdx.x; r < per; r += blockDim.x)
        coupling_entry_f32<CPLX>(blk, r, t, sc, dc, rel, q2, float(kre), float(kim), K);
      __syncthreads();
    }
    return;
  }
  for (int64_t blk = blockIdx.x; blk < nfar; blk += gridDim.x)
    for (int r = threadIdx.x; r < per; r += blockDim.x)
      coupling_entry<CPLX>(blk, r, tgt, src, nodes, q2, kre, kim, K, f32k);
}

template <typename T>
__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = float(a[i]);
}

template <int D, bool CPLX>
void launch_pairs(Op& o, cudaEvent_t* ev) {
  const cudaStream_t s = o.stream;
  const int G2 = o.g_reg * o.g_reg;
  const int NL = (D + 1) * (D + 1);
  const int threads = 32 * kWarps;
  if (o.npairs[kRegular] > 0) {
    const int G2f = o.g_reg_far * o.g_reg_far;
    const size_t shm = regular_smem(G2, G2f, NL, CPLX ? 2 : 1, o.d_Xq_far32 != nullptr);
    if (shm > 48 * 1024)
      cuda_check(cudaFuncSetAttribute(k_near_regular<D, CPLX>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(shm)),
                 "smem attr");
    const int grid = int(std::min<int64_t>((o.npairs[kRegular] + kWarps - 1) / kWarps, 152 * 64));
    k_near_regular<D, CPLX><<<grid, threads, shm, s>>>(o.d_pairs[kRegular], o.npairs[kRegular], o.d_Xq, o.d_BW,
                                                       G2, o.d_Xq_far, o.d_BW_far, G2f, o.kre, o.kim, o.d_N, o.nld,
                                                       reinterpret_cast<const float4*>(o.d_Xq_far32), o.d_cen);
    launched("k_near_regular");
  }
  cuda_check(cudaEventRecord(ev[2], s), "event");

  auto grid_of = [](int64_t n) { return int(std::min<int64_t>((n + kWarps - 1) / kWarps, 152 * 64)); };
  if (o.npairs[kIdentical] > 0)
    launch_singular<D, CPLX, kIdentical>(grid_of(o.npairs[kIdentical]), s, o.d_pairs[kIdentical], o.npairs[kIdentical],
                                         o.geom, o.L, rule_orders(o, kIdentical), o.d_gauss + o.gauss_off[kIdentical],
                                         o.kre, o.kim, o.d_N, o.nld);
  cuda_check(cudaEventRecord(ev[3], s), "event");
  if (o.npairs[kEdge] > 0)
    launch_singular<D, CPLX, kEdge>(grid_of(o.npairs[kEdge]), s, o.d_pairs[kEdge], o.npairs[kEdge], o.geom, o.L,
                                    rule_orders(o, kEdge), o.d_gauss + o.gauss_off[kEdge], o.kre, o.kim, o.d_N,
                                    o.nld);
  cuda_check(cudaEventRecord(ev[4], s), "event");
  if (o.npairs[kVertex] > 0)
    launch_singular<D, CPLX, kVertex>(grid_of(o.npairs[kVertex]), s, o.d_pairs[kVertex], o.npairs[kVertex], o.geom,
                                      o.L, rule_orders(o, kVertex), o.d_gauss + o.gauss_off[kVertex], o.kre, o.kim,
                                      o.d_N, o.nld);
  cuda_check(cudaEventRecord(ev[5], s), "event");
}

}  // namespace

void points_f32(Op& o, cudaStream_t s) {
  if (!o.d_Xq_far32) return;
  const int G2f = o.g_reg_far * o.g_reg_far;
  k_points_f32<<<grid_for(o.nelem, 128), 128, 0, s>>>(o.d_Xq_far, o.nelem, G2f,
                                                      reinterpret_cast<float4*>(o.d_Xq_far32), o.d_cen);
  launched("k_points_f32");
  k_to_f32<float><<<1, 256, 0, s>>>(o.d_BW_far, o.d_BW_far32, int64_t(G2f) * o.nloc);
  launched("k_to_f32");
}

void coupling_f32(Op& o, cudaStream_t s) {
  if (!o.d_K32) return;
  const int C = o.cplx ? 2 : 1;
  k_to_f32<float><<<1024, 256, 0, s>>>(o.d_K, o.d_K32, o.nfar * (int64_t)o.q2 * o.q2 * (o.efie ? 5 : 1) * C);
  launched("k_to_f32");
}

void coupling_f32_prepare(Op& o, int nrhs) {
  const int C = o.cplx ? 2 : 1;
  if (o.d_K32 || o.efie || o.nfar == 0 || !o.d_K || o.opts.precision != BEMBEL_PREC_MIXED ||
      (nrhs * C < 8 && !o.opts.far_fp32_stored) || capturing())
    return;
  o.d_K32 = static_cast<float*>(dev_alloc(sizeof(float) * o.nfar * (int64_t)o.q2 * o.q2 * C));
  coupling_f32(o, o.stream);
}

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
    // FP32 copy of the compressed EFIE's stored coupling (it has no on-the-fly form); S^2
    // operators make theirs at the first wide product (coupling_f32_prepare)
    if (o.efie && nK > 0) o.d_K32 = static_cast<float*>(dev_alloc(sizeof(float) * nK * C));
    // FP32 kernel evaluation for separated pairs beyond the ring (S^2 operators)
    if (!o.efie && o.npairs_regular_far > 0) {
      const int64_t G2f = int64_t(o.g_reg_far) * o.g_reg_far;
      o.d_Xq_far32 = static_cast<float*>(dev_alloc(sizeof(float) * 4 * o.nelem * G2f));
      o.d_cen = static_cast<double*>(dev_alloc(sizeof(double) * 4 * o.nelem));
      o.d_BW_far32 = static_cast<float*>(dev_alloc(sizeof(float) * G2f * o.nloc));
    }
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
    points_f32(o, s);
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
    const bool f32k = o.opts.precision == BEMBEL_PREC_MIXED;
    // CTA of q2 x q2 threads rounded to warps (at most 1024), grid-stride over the blocks
    const int cthreads = std::min(1024, ((o.q2 * o.q2 + 31) / 32) * 32);
    const int cgrid = int(std::max<int64_t>(1, std::min<int64_t>(o.nfar, int64_t(152) * 2048 / cthreads * 4)));
    const float4* rel = reinterpret_cast<const float4*>(o.d_nodes_rel32);
    if (o.cplx)
      k_coupling<true><<<cgrid, cthreads, 0, s>>>(o.d_far_tgt, o.d_far_src, o.nfar, o.d_nodes, o.q2, o.kre, o.kim,
                                                  o.d_K, f32k, o.d_ccen, rel);
    else
      k_coupling<false><<<cgrid, cthreads, 0, s>>>(o.d_far_tgt, o.d_far_src, o.nfar, o.d_nodes, o.q2, o.kre, o.kim,
                                                   o.d_K, f32k, o.d_ccen, rel);
    launched("k_coupling");
  }
  cuda_check(cudaEventRecord(ev[6], s), "event");
  // FP32 copies for the mixed-precision inner solves
  if (o.opts.precision == BEMBEL_PREC_MIXED) {
    k_to_f32<float><<<1024, 256, 0, s>>>(o.d_N, o.d_N32, nN);
    launched("k_to_f32");
    coupling_f32(o, s);
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
                                                       nloc, nullptr, nullptr);
    launched("k_near_regular");
    cuda_check(cudaStreamSynchronize(s), "sample sync");
    dev_free(Xq);
    dev_free(d_BW);
  } else if (kind == kIdentical) {
    launch_singular<D, CPLX, kIdentical>(grid, s, d_sample, ns, o.geom, o.L, g4, d_tab, o.kre, o.kim, out, nloc);
  } else if (kind == kEdge) {
    launch_singular<D, CPLX, kEdge>(grid, s, d_sample, ns, o.geom, o.L, g4, d_tab, o.kre, o.kim, out, nloc);
  } else {
    launch_singular<D, CPLX, kVertex>(grid, s, d_sample, ns, o.geom, o.L, g4, d_tab, o.kre, o.kim, out, nloc);
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
