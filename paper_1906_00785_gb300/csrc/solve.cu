// solve.cu - restarted GMRES (Sec. 4.6), load vectors (Sec. 4.4) and potential
// evaluation (Sec. 4.7).
//
// GMRES(m) runs nrhs independent systems side by side: one matvec per Arnoldi
// step for all columns, classical Gram-Schmidt applied twice (CGS2) on the
// device, and the (m+1) x m Hessenberg least-squares problem with Givens
// rotations on the host, one small device-to-host copy per step.  FP64
// operators solve in FP64; MIXED operators run FP32 inner GMRES on the FP32
// copies of the near and coupling matrices inside FP64 iterative refinement
// (r = b - A x with the FP64 matvec, x += correction), which restores FP64
// residual accuracy.
#include <chrono>
#include <complex>
#include <vector>

#include "op.h"

namespace bembel {

namespace {

using cd = std::complex<double>;

inline int nblk(int64_t n, int t) { return int(std::max<int64_t>(1, std::min<int64_t>((n + t - 1) / t, 65535 * 16))); }

// h[i*nrhs + r] = sum_n conj(V_i[n, r]) w[n, r] for i < nv (V_i stride vstride).
template <typename T, bool CPLX>
__global__ void k_dots(const T* __restrict__ V, int64_t vstride, int nv, const T* __restrict__ w, int64_t n,
                       int nrhs, double* __restrict__ h) {
  const int pair = blockIdx.x;  // i * nrhs + r
  const int i = pair / nrhs, r = pair % nrhs;
  if (i >= nv) return;
  const int C = CPLX ? 2 : 1;
  const T* v = V + (int64_t)i * vstride + (int64_t)r * n * C;
  const T* x = w + (int64_t)r * n * C;
  double sr = 0.0, si = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
    if (CPLX) {
      const double vr = v[2 * k], vi = v[2 * k + 1], xr = x[2 * k], xi = x[2 * k + 1];
      sr += vr * xr + vi * xi;
      si += vr * xi - vi * xr;
    } else {
      sr += (double)v[k] * (double)x[k];
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
    h[pair * 2] = a;
    h[pair * 2 + 1] = b;
  }
}

// w[n, r] -= sum_i V_i[n, r] h[i, r]   (h complex, stored as pairs)
template <typename T, bool CPLX>
__global__ void k_orth_update(const T* __restrict__ V, int64_t vstride, int nv, T* __restrict__ w, int64_t n,
                              int nrhs, const double* __restrict__ h) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= n * nrhs) return;
  const int r = int(id / n);
  const int64_t k = id % n;
  const int C = CPLX ? 2 : 1;
  double ar = CPLX ? (double)w[(r * n + k) * 2] : (double)w[r * n + k];
  double ai = CPLX ? (double)w[(r * n + k) * 2 + 1] : 0.0;
  for (int i = 0; i < nv; ++i) {
    const T* v = V + (int64_t)i * vstride + ((int64_t)r * n + k) * C;
    const double hr = h[(i * nrhs + r) * 2], hi = h[(i * nrhs + r) * 2 + 1];
    if (CPLX) {
      ar -= hr * (double)v[0] - hi * (double)v[1];
      ai -= hr * (double)v[1] + hi * (double)v[0];
    } else {
      ar -= hr * (double)v[0];
    }
  }
  if (CPLX) {
    w[(r * n + k) * 2] = T(ar);
    w[(r * n + k) * 2 + 1] = T(ai);
  } else {
    w[r * n + k] = T(ar);
  }
}

// y[n, r] = alpha_r * x[n, r]  (real per-column scale)
template <typename T>
__global__ void k_scale(const T* __restrict__ x, T* __restrict__ y, int64_t nper, int nrhs,
                        const double* __restrict__ alpha) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= nper * nrhs) return;
  y[id] = T(alpha[id / nper] * (double)x[id]);
}

// x[n, r] += sum_i V_i[n, r] c[i, r]  (x FP64; c complex pairs)
template <typename T, bool CPLX>
__global__ void k_combine(const T* __restrict__ V, int64_t vstride, int nv, double* __restrict__ x, int64_t n,
                          int nrhs, const double* __restrict__ c, double scale) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= n * nrhs) return;
  const int r = int(id / n);
  const int64_t k = id % n;
  const int C = CPLX ? 2 : 1;
  double ar = 0.0, ai = 0.0;
  for (int i = 0; i < nv; ++i) {
    const T* v = V + (int64_t)i * vstride + ((int64_t)r * n + k) * C;
    const double cr = c[(i * nrhs + r) * 2], ci = c[(i * nrhs + r) * 2 + 1];
    if (CPLX) {
      ar += cr * (double)v[0] - ci * (double)v[1];
      ai += cr * (double)v[1] + ci * (double)v[0];
    } else {
      ar += cr * (double)v[0];
    }
  }
  if (CPLX) {
    x[(r * n + k) * 2] += scale * ar;
    x[(r * n + k) * 2 + 1] += scale * ai;
  } else {
    x[r * n + k] += scale * ar;
  }
}

template <typename T>
__global__ void k_to_type(const double* __restrict__ a, T* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = T(a[i]);
}

__global__ void k_add_inplace(double* __restrict__ x, const double* __restrict__ d, int64_t n) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id < n) x[id] += d[id];
}

__global__ void k_sub(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ c, int64_t n) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id < n) c[id] = a[id] - b[id];
}

struct DevVec {
  void* p = nullptr;
  explicit DevVec(size_t bytes) { p = dev_alloc(bytes); }
  ~DevVec() { dev_free(p); }
  DevVec(const DevVec&) = delete;
  DevVec& operator=(const DevVec&) = delete;
};

// Column norms ||x_r|| of an n x nrhs (complex) FP64-or-FP32 block, on the host.
template <typename T, bool CPLX>
void col_norms(const T* x, int64_t n, int nrhs, double* d_h, std::vector<double>& out, cudaStream_t s) {
  k_dots<T, CPLX><<<nrhs, 256, 0, s>>>(x, 0, 1, x, n, nrhs, d_h);
  launched("k_dots");
  std::vector<double> h(2 * nrhs);
  cuda_check(cudaMemcpyAsync(h.data(), d_h, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, s), "norm copy");
  cuda_check(cudaStreamSynchronize(s), "norm sync");
  out.resize(nrhs);
  for (int r = 0; r < nrhs; ++r) out[r] = std::sqrt(std::max(0.0, h[2 * r]));
}

// One GMRES(m) run on A x = b (x0 = 0), T = vector type of the Krylov basis.
// b, x: FP64 device blocks (n x nrhs).  For T = float the basis and matvec are
// FP32.  Returns the number of Arnoldi steps of the slowest column; fills
// relres (estimates) per column.
template <typename T, bool CPLX>
int gmres_run(const Op& o, const double* b, double* x, int nrhs, double tol, int restart, int max_iter, bool fp32,
              std::vector<double>& relres, cudaStream_t s) {
  const int C = CPLX ? 2 : 1;
  const int64_t n = o.ndofs;
  const int64_t vstride = n * nrhs * C;
  const int m = restart;
  DevVec Vbuf(sizeof(T) * vstride * (m + 1));
  DevVec wbuf(sizeof(T) * vstride);
  DevVec rbuf(sizeof(double) * vstride);
  DevVec hbuf(sizeof(double) * 2 * (m + 2) * nrhs * 2);
  DevVec abuf(sizeof(double) * nrhs);
  T* V = static_cast<T*>(Vbuf.p);
  T* w = static_cast<T*>(wbuf.p);
  double* r = static_cast<double*>(rbuf.p);
  double* d_h = static_cast<double*>(hbuf.p);
  double* d_h2 = d_h + 2 * (m + 2) * nrhs;
  double* d_alpha = static_cast<double*>(abuf.p);
  const int tb = 256;
  cuda_check(cudaMemsetAsync(x, 0, sizeof(double) * vstride, s), "x0");

  std::vector<double> bnorm;
  col_norms<double, CPLX>(b, n, nrhs, d_h, bnorm, s);
  relres.assign(nrhs, 0.0);
  std::vector<char> done(nrhs, 0);
  for (int rr = 0; rr < nrhs; ++rr)
    if (bnorm[rr] == 0.0) done[rr] = 1;
  int iters = 0;
  std::vector<cd> H((size_t)(m + 1) * m * nrhs), g((size_t)(m + 1) * nrhs), cs((size_t)m * nrhs),
      sn((size_t)m * nrhs);
  std::vector<double> hh(2 * (m + 2) * nrhs), hh2(2 * (m + 2) * nrhs), alpha(nrhs);
  std::vector<int> jend(nrhs, 0);
  bool first = true;
  while (iters < max_iter) {
    // residual r = b - A x
    if (first) {
      cuda_check(cudaMemcpyAsync(r, b, sizeof(double) * vstride, cudaMemcpyDeviceToDevice, s), "r0");
    } else {
      matvec_device(o, x, r, nrhs, false, s);
      k_sub<<<nblk(vstride, tb), tb, 0, s>>>(b, r, r, vstride);
      launched("kernel");
    }
    first = false;
    std::vector<double> rn;
    col_norms<double, CPLX>(r, n, nrhs, d_h, rn, s);
    bool all = true;
    for (int rr = 0; rr < nrhs; ++rr) {
      relres[rr] = bnorm[rr] > 0 ? rn[rr] / bnorm[rr] : 0.0;
      if (relres[rr] <= tol) done[rr] = 1;
      all = all && done[rr];
    }
    if (all) break;
    for (int rr = 0; rr < nrhs; ++rr) alpha[rr] = rn[rr] > 0 ? 1.0 / rn[rr] : 0.0;
    cuda_check(cudaMemcpyAsync(d_alpha, alpha.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s), "alpha");
    if (fp32) {
      // V_0 = r / ||r|| in FP32
      DevVec tmp(sizeof(double) * vstride);
      k_scale<double><<<nblk(vstride, tb), tb, 0, s>>>(r, static_cast<double*>(tmp.p), n * C, nrhs, d_alpha);
      launched("kernel");
      k_to_type<T><<<nblk(vstride, tb), tb, 0, s>>>(static_cast<double*>(tmp.p), V, vstride);
      launched("kernel");
      cuda_check(cudaStreamSynchronize(s), "v0 sync");
    } else {
      k_scale<T><<<nblk(vstride, tb), tb, 0, s>>>(reinterpret_cast<const T*>(r), V, n * C, nrhs, d_alpha);
      launched("kernel");
    }
    for (int rr = 0; rr < nrhs; ++rr) {
      g[(size_t)rr * (m + 1)] = rn[rr];
      for (int k = 1; k <= m; ++k) g[(size_t)rr * (m + 1) + k] = 0.0;
      jend[rr] = 0;
    }
    std::vector<char> active(nrhs);
    for (int rr = 0; rr < nrhs; ++rr) active[rr] = !done[rr];
    int j = 0;
    for (; j < m && iters < max_iter; ++j) {
      T* vj = V + (int64_t)j * vstride;
      matvec_device(o, vj, w, nrhs, fp32, s);
      // CGS2
      k_dots<T, CPLX><<<(j + 1) * nrhs, 256, 0, s>>>(V, vstride, j + 1, w, n, nrhs, d_h);
      launched("kernel");
      k_orth_update<T, CPLX><<<nblk(n * nrhs, tb), tb, 0, s>>>(V, vstride, j + 1, w, n, nrhs, d_h);
      launched("kernel");
      k_dots<T, CPLX><<<(j + 1) * nrhs, 256, 0, s>>>(V, vstride, j + 1, w, n, nrhs, d_h2);
      launched("kernel");
      k_orth_update<T, CPLX><<<nblk(n * nrhs, tb), tb, 0, s>>>(V, vstride, j + 1, w, n, nrhs, d_h2);
      launched("kernel");
      k_dots<T, CPLX><<<nrhs, 256, 0, s>>>(w, 0, 1, w, n, nrhs, d_h2 + 2 * (j + 1) * nrhs);
      launched("arnoldi kernels");
      cuda_check(cudaMemcpyAsync(hh.data(), d_h, sizeof(double) * 2 * (j + 1) * nrhs, cudaMemcpyDeviceToHost, s),
                 "h copy");
      cuda_check(cudaMemcpyAsync(hh2.data(), d_h2, sizeof(double) * 2 * (j + 2) * nrhs, cudaMemcpyDeviceToHost, s),
                 "h2 copy");
      cuda_check(cudaStreamSynchronize(s), "arnoldi sync");
      ++iters;
      bool all_conv = true;
      for (int rr = 0; rr < nrhs; ++rr) {
        const double hn = std::sqrt(std::max(0.0, hh2[2 * ((j + 1) * nrhs + rr)]));
        alpha[rr] = hn > 0 ? 1.0 / hn : 0.0;
        if (!active[rr]) continue;
        cd* Hc = &H[(size_t)rr * (m + 1) * m];
        for (int i = 0; i <= j; ++i)
          Hc[i * m + j] = cd(hh[2 * (i * nrhs + rr)] + hh2[2 * (i * nrhs + rr)],
                             hh[2 * (i * nrhs + rr) + 1] + hh2[2 * (i * nrhs + rr) + 1]);
        Hc[(j + 1) * m + j] = hn;
        for (int i = 0; i < j; ++i) {
          const cd c = cs[(size_t)rr * m + i], sg = sn[(size_t)rr * m + i];
          const cd t = c * Hc[i * m + j] + sg * Hc[(i + 1) * m + j];
          Hc[(i + 1) * m + j] = -std::conj(sg) * Hc[i * m + j] + c * Hc[(i + 1) * m + j];
          Hc[i * m + j] = t;
        }
        const cd a = Hc[j * m + j], bb = Hc[(j + 1) * m + j];
        const double den = std::sqrt(std::norm(a) + std::norm(bb));
        cd c, sg;
        if (den == 0.0) {
          c = 1.0;
          sg = 0.0;
        } else if (std::abs(a) == 0.0) {
          c = 0.0;
          sg = std::conj(bb) / std::abs(bb);
        } else {
          c = std::abs(a) / den;
          sg = (a / std::abs(a)) * std::conj(bb) / den;
        }
        cs[(size_t)rr * m + j] = c;
        sn[(size_t)rr * m + j] = sg;
        Hc[j * m + j] = c * a + sg * bb;
        Hc[(j + 1) * m + j] = 0.0;
        cd* gc = &g[(size_t)rr * (m + 1)];
        gc[j + 1] = -std::conj(sg) * gc[j];
        gc[j] = c * gc[j];
        jend[rr] = j + 1;
        relres[rr] = std::abs(gc[j + 1]) / bnorm[rr];
        if (relres[rr] <= tol || hn == 0.0) active[rr] = 0;
        all_conv = all_conv && !active[rr];
      }
      cuda_check(cudaMemcpyAsync(d_alpha, alpha.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s), "alpha");
      k_scale<T><<<nblk(vstride, tb), tb, 0, s>>>(w, V + (int64_t)(j + 1) * vstride, n * C, nrhs, d_alpha);
      launched("kernel");
      if (all_conv) {
        ++j;
        break;
      }
    }
    // y = R^{-1} g per column; x += V y
    std::vector<double> ybuf(2 * (size_t)(m + 1) * nrhs, 0.0);
    int nv = 0;
    for (int rr = 0; rr < nrhs; ++rr) {
      const int k = jend[rr];
      nv = std::max(nv, k);
      if (k == 0) continue;
      const cd* Hc = &H[(size_t)rr * (m + 1) * m];
      const cd* gc = &g[(size_t)rr * (m + 1)];
      std::vector<cd> y(k);
      for (int i = k - 1; i >= 0; --i) {
        cd acc = gc[i];
        for (int l = i + 1; l < k; ++l) acc -= Hc[i * m + l] * y[l];
        y[i] = acc / Hc[i * m + i];
      }
      for (int i = 0; i < k; ++i) {
        ybuf[2 * (i * nrhs + rr)] = y[i].real();
        ybuf[2 * (i * nrhs + rr) + 1] = y[i].imag();
      }
    }
    if (nv > 0) {
      cuda_check(cudaMemcpyAsync(d_h, ybuf.data(), sizeof(double) * 2 * nv * nrhs, cudaMemcpyHostToDevice, s),
                 "y copy");
      k_combine<T, CPLX><<<nblk(n * nrhs, tb), tb, 0, s>>>(V, vstride, nv, x, n, nrhs, d_h, 1.0);
      launched("k_combine");
      cuda_check(cudaStreamSynchronize(s), "combine sync");
    }
  }
  return iters;
}

}  // namespace

int solve_gmres(const Op& o, const void* bv, void* xv, int nrhs, const bembel_solve_opts& so,
                bembel_solve_info* info) {
  const auto t0 = std::chrono::steady_clock::now();
  const cudaStream_t s = o.stream;
  const double* b = static_cast<const double*>(bv);
  double* x = static_cast<double*>(xv);
  const int C = o.cplx ? 2 : 1;
  const int64_t vn = o.ndofs * nrhs * C;
  std::vector<double> relres;
  int iters = 0, refinements = 0;
  const bool mixed = o.opts.precision == BEMBEL_PREC_MIXED && so.refine;
  if (!mixed) {
    iters = o.cplx ? gmres_run<double, true>(o, b, x, nrhs, so.tol, so.restart, so.max_iter, false, relres, s)
                   : gmres_run<double, false>(o, b, x, nrhs, so.tol, so.restart, so.max_iter, false, relres, s);
  } else {
    // FP64 iterative refinement around FP32 GMRES
    DevVec rbuf(sizeof(double) * vn), dbuf(sizeof(double) * vn), hbuf(sizeof(double) * 2 * nrhs);
    double* r = static_cast<double*>(rbuf.p);
    double* dx = static_cast<double*>(dbuf.p);
    cuda_check(cudaMemsetAsync(x, 0, sizeof(double) * vn, s), "x0");
    std::vector<double> bn, rn;
    if (o.cplx)
      col_norms<double, true>(b, o.ndofs, nrhs, static_cast<double*>(hbuf.p), bn, s);
    else
      col_norms<double, false>(b, o.ndofs, nrhs, static_cast<double*>(hbuf.p), bn, s);
    relres.assign(nrhs, 1.0);
    for (int outer = 0; outer < 30 && iters < so.max_iter; ++outer) {
      if (outer == 0) {
        cuda_check(cudaMemcpyAsync(r, b, sizeof(double) * vn, cudaMemcpyDeviceToDevice, s), "r");
      } else {
        matvec_device(o, x, r, nrhs, false, s);
        k_sub<<<nblk(vn, 256), 256, 0, s>>>(b, r, r, vn);
        launched("kernel");
      }
      if (o.cplx)
        col_norms<double, true>(r, o.ndofs, nrhs, static_cast<double*>(hbuf.p), rn, s);
      else
        col_norms<double, false>(r, o.ndofs, nrhs, static_cast<double*>(hbuf.p), rn, s);
      double worst = 0.0, ratio = 0.0;
      for (int rr = 0; rr < nrhs; ++rr) {
        relres[rr] = bn[rr] > 0 ? rn[rr] / bn[rr] : 0.0;
        worst = std::max(worst, relres[rr]);
        if (rn[rr] > 0) ratio = std::max(ratio, bn[rr] / rn[rr]);
      }
      if (worst <= so.tol) break;
      ++refinements;
      // inner tolerance relative to the current residual: what is still
      // missing to reach tol, but not below what FP32 Krylov vectors resolve
      const double inner = std::min(0.5, std::max(1e-5, 0.3 * so.tol / worst));
      (void)ratio;
      std::vector<double> rel_inner;
      iters += o.cplx ? gmres_run<float, true>(o, r, dx, nrhs, inner, so.restart, so.max_iter - iters, true,
                                               rel_inner, s)
                      : gmres_run<float, false>(o, r, dx, nrhs, inner, so.restart, so.max_iter - iters, true,
                                                rel_inner, s);
      k_add_inplace<<<nblk(vn, 256), 256, 0, s>>>(x, dx, vn);
      launched("refine update");
    }
  }
  cuda_check(cudaStreamSynchronize(s), "solve sync");
  double worst = 0.0;
  for (double v : relres) worst = std::max(worst, v);
  if (info) {
    info->iterations = iters;
    info->refinements = refinements;
    info->rel_residual = worst;
    info->solve_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return worst <= so.tol ? BEMBEL_OK : BEMBEL_ENOTCONV;
}

}  // namespace bembel
