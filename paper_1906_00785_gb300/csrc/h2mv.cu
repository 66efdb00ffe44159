// h2mv.cu - the H^2 matrix-vector product y = A~ x (Sec. 2 embedded FMM on the
// parameter domain; Sec. 4.5 "H * x").
//
// A~ = E^T (N + sum_levels U_l^T ... ) E in element-local Bernstein coordinates:
//   1. gather   x_loc = E x                 (Bezier extraction, App. C/E)
//   2. leaf up  xh_leaf = V^T x_loc          (leaf moments, geometry independent)
//   3. up       xh_parent = sum_c T_c^T xh_c (interpolation transfers)
//   4. coupling yh_tau = sum_sigma K_tau,sigma xh_sigma over far blocks
//   5. down     yh_c += T_c yh_parent
//   6. leaf     y_loc = V yh_leaf + sum_sigma N_tau,sigma x_loc,sigma (near field)
//   7. scatter  y = E^T y_loc
// Internal vectors are dof-major with the nrhs (x2 for complex) real columns
// contiguous; real moment/transfer/extraction matrices act on complex vectors
// as on pairs of real columns.  Instantiated for double (FP64 path) and float
// (inner solves of the mixed-precision path).
#include <mutex>
#include <string>

#include "op.h"

namespace bembel {

namespace {

inline int blocks_for(int64_t n, int t) { return int(std::max<int64_t>(1, std::min<int64_t>((n + t - 1) / t, 1 << 30))); }

template <typename T>
__global__ void k_gather(const T* __restrict__ x, T* __restrict__ xl, const double* __restrict__ ex, int L, int d,
                         int n1, int64_t ndofs, int64_t nlocal, int ncol, int C) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= nlocal * ncol) return;
  const int64_t ld = id / ncol;
  const int col = int(id % ncol);
  const int r = col / C, comp = col % C;
  const int D1 = d + 1, nloc = D1 * D1;
  const int64_t e = ld / nloc;
  const int k = int(ld % nloc), k1 = k % D1, k2 = k / D1;
  const int64_t per = int64_t(1) << (2 * L);
  const int patch = int(e / per);
  uint32_t i1, i2;
  morton_decode(uint32_t(e % per), i1, i2);
  const T* xr = x + (int64_t)r * ndofs * C + comp;
  double acc = 0.0;
  for (int j2 = 0; j2 < D1; ++j2) {
    const double c2 = ex[((int64_t)i2 * D1 + j2) * D1 + k2];
    if (c2 == 0.0) continue;
    for (int j1 = 0; j1 < D1; ++j1) {
      const double c1 = ex[((int64_t)i1 * D1 + j1) * D1 + k1];
      if (c1 == 0.0) continue;
      const int64_t g = (int64_t)patch * n1 * n1 + (int64_t)(i2 + j2) * n1 + (i1 + j1);
      acc += c1 * c2 * (double)xr[g * C];
    }
  }
  xl[id] = T(acc);
}

template <typename T>
__global__ void k_scatter(const T* __restrict__ yl, T* __restrict__ y, const double* __restrict__ ex, int L, int d,
                          int n1, int64_t ndofs, int ncol, int C) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= ndofs * ncol) return;
  const int64_t g = id / ncol;
  const int col = int(id % ncol);
  const int r = col / C, comp = col % C;
  const int D1 = d + 1, nloc = D1 * D1;
  const int nel1 = 1 << L;
  const int patch = int(g / ((int64_t)n1 * n1));
  const int rem = int(g % ((int64_t)n1 * n1));
  const int j2 = rem / n1, j1 = rem % n1;
  const int64_t per = int64_t(1) << (2 * L);
  double acc = 0.0;
  for (int i2 = max(0, j2 - d); i2 <= min(nel1 - 1, j2); ++i2)
    for (int i1 = max(0, j1 - d); i1 <= min(nel1 - 1, j1); ++i1) {
      const int64_t e = (int64_t)patch * per + morton_encode(i1, i2);
      for (int k2 = 0; k2 < D1; ++k2) {
        const double c2 = ex[((int64_t)i2 * D1 + (j2 - i2)) * D1 + k2];
        if (c2 == 0.0) continue;
        for (int k1 = 0; k1 < D1; ++k1) {
          const double c1 = ex[((int64_t)i1 * D1 + (j1 - i1)) * D1 + k1];
          if (c1 == 0.0) continue;
          acc += c1 * c2 * (double)yl[(e * nloc + k1 + D1 * k2) * ncol + col];
        }
      }
    }
  y[((int64_t)r * ndofs + g) * C + comp] = T(acc);
}

// xh[leaf][a][col] = sum_i V[i][a] xl[leaf*nld + i][col]
template <typename T>
__global__ void k_leaf_up(const T* __restrict__ xl, T* __restrict__ xh, const T* __restrict__ V, int64_t nleaf,
                          int nld, int q2, int ncol) {
  extern __shared__ unsigned char smem_raw[];
  T* Vs = reinterpret_cast<T*>(smem_raw);
  for (int i = threadIdx.x; i < nld * q2; i += blockDim.x) Vs[i] = V[i];
  __syncthreads();
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= nleaf * q2 * ncol) return;
  const int col = int(id % ncol);
  const int a = int((id / ncol) % q2);
  const int64_t t = id / ((int64_t)ncol * q2);
  const T* x = xl + t * nld * ncol + col;
  T acc = 0;
  for (int i = 0; i < nld; ++i) acc = fma(Vs[i * q2 + a], x[(int64_t)i * ncol], acc);
  xh[id] = acc;
}

// parents P on one level: xh[P][a][col] = sum_c sum_a' T[c][a'][a] xh[4P+c][a'][col]
template <typename T>
__global__ void k_up(T* __restrict__ xh_par, const T* __restrict__ xh_ch, const T* __restrict__ Tm, int64_t npar,
                     int q2, int ncol) {
  extern __shared__ unsigned char smem_raw[];
  T* Ts = reinterpret_cast<T*>(smem_raw);
  for (int i = threadIdx.x; i < 4 * q2 * q2; i += blockDim.x) Ts[i] = Tm[i];
  __syncthreads();
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= npar * q2 * ncol) return;
  const int col = int(id % ncol);
  const int a = int((id / ncol) % q2);
  const int64_t P = id / ((int64_t)ncol * q2);
  T acc = 0;
  for (int c = 0; c < 4; ++c) {
    const T* x = xh_ch + ((4 * P + c) * q2) * ncol + col;
    const T* Tc = Ts + c * q2 * q2;
    for (int ap = 0; ap < q2; ++ap) acc = fma(Tc[ap * q2 + a], x[(int64_t)ap * ncol], acc);
  }
  xh_par[id] = acc;
}

// children c on one level: yh[c][a'][col] += sum_a T[c%4][a'][a] yh[c/4][a][col]
template <typename T>
__global__ void k_down(T* __restrict__ yh_ch, const T* __restrict__ yh_par, const T* __restrict__ Tm, int64_t nch,
                       int q2, int ncol) {
  extern __shared__ unsigned char smem_raw[];
  T* Ts = reinterpret_cast<T*>(smem_raw);
  for (int i = threadIdx.x; i < 4 * q2 * q2; i += blockDim.x) Ts[i] = Tm[i];
  __syncthreads();
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= nch * q2 * ncol) return;
  const int col = int(id % ncol);
  const int ap = int((id / ncol) % q2);
  const int64_t c = id / ((int64_t)ncol * q2);
  const T* Tc = Ts + (c & 3) * q2 * q2 + ap * q2;
  const T* y = yh_par + ((c >> 2) * q2) * ncol + col;
  T acc = yh_ch[id];
  for (int a = 0; a < q2; ++a) acc = fma(Tc[a], y[(int64_t)a * ncol], acc);
  yh_ch[id] = acc;
}

// yh[t][a][r] = sum over far blocks of t: K[blk][b][a] xh[s][b][r]  (complex r: 2 reals)
template <typename T, bool CPLX>
__global__ void k_coupling_mv(const long long* __restrict__ ptr, const int* __restrict__ src,
                              const T* __restrict__ K, const T* __restrict__ xh, T* __restrict__ yh, int64_t nclus,
                              int q2, int nrhs) {
  const int C = CPLX ? 2 : 1;
  const int ncol = nrhs * C;
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= nclus * q2 * nrhs) return;
  const int r = int(id % nrhs);
  const int a = int((id / nrhs) % q2);
  const int64_t t = id / ((int64_t)nrhs * q2);
  T ar = 0, ai = 0;
  for (long long blk = ptr[t]; blk < ptr[t + 1]; ++blk) {
    const T* Kb = K + (blk * q2 * q2) * C;
    const T* x = xh + ((int64_t)src[blk] * q2) * ncol + r * C;
    for (int b = 0; b < q2; ++b) {
      if (CPLX) {
        const T kr = Kb[(b * q2 + a) * 2], ki = Kb[(b * q2 + a) * 2 + 1];
        const T xr = x[(int64_t)b * ncol], xi = x[(int64_t)b * ncol + 1];
        ar = fma(kr, xr, fma(-ki, xi, ar));
        ai = fma(kr, xi, fma(ki, xr, ai));
      } else {
        ar = fma(Kb[b * q2 + a], x[(int64_t)b * ncol], ar);
      }
    }
  }
  T* y = yh + (t * q2 + a) * ncol + r * C;
  y[0] = ar;
  if (CPLX) y[1] = ai;
}

// y_loc[t*nld + i][r] = sum_a V[i][a] yh[t][a][r] + sum_near N[blk][j][i] x_loc[s*nld + j][r]
template <typename T, bool CPLX>
__global__ void k_leaf_near(const long long* __restrict__ ptr, const int* __restrict__ col,
                            const T* __restrict__ N, const T* __restrict__ xl, const T* __restrict__ V,
                            const T* __restrict__ yh, T* __restrict__ yl, int64_t nleaf, int nld, int q2, int nrhs) {
  const int C = CPLX ? 2 : 1;
  const int ncol = nrhs * C;
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= nleaf * nld * nrhs) return;
  const int r = int(id % nrhs);
  const int i = int((id / nrhs) % nld);
  const int64_t t = id / ((int64_t)nrhs * nld);
  T ar = 0, ai = 0;
  if (q2 > 0) {
    const T* y = yh + (t * q2) * ncol + r * C;
    for (int a = 0; a < q2; ++a) {
      const T v = V[i * q2 + a];
      ar = fma(v, y[(int64_t)a * ncol], ar);
      if (CPLX) ai = fma(v, y[(int64_t)a * ncol + 1], ai);
    }
  }
  for (long long blk = ptr[t]; blk < ptr[t + 1]; ++blk) {
    const T* Nb = N + (blk * nld * nld) * C;
    const T* x = xl + ((int64_t)col[blk] * nld) * ncol + r * C;
    for (int j = 0; j < nld; ++j) {
      if (CPLX) {
        const T nr = Nb[(j * nld + i) * 2], ni = Nb[(j * nld + i) * 2 + 1];
        const T xr = x[(int64_t)j * ncol], xi = x[(int64_t)j * ncol + 1];
        ar = fma(nr, xr, fma(-ni, xi, ar));
        ai = fma(nr, xi, fma(ni, xr, ai));
      } else {
        ar = fma(Nb[j * nld + i], x[(int64_t)j * ncol], ar);
      }
    }
  }
  T* y = yl + (t * nld + i) * ncol + r * C;
  y[0] = ar;
  if (CPLX) y[1] = ai;
}

template <typename T>
void matvec_impl(const Op& o, const T* x, T* y, int nrhs, cudaStream_t s, const T* K, const T* N, const T* V,
                 const T* Tm, void* scratch) {
  const int C = o.cplx ? 2 : 1;
  const int ncol = nrhs * C;
  const int q2 = o.q2;
  T* base = static_cast<T*>(scratch);
  T* xl = base;
  T* yl = xl + o.nlocal * ncol;
  T* xh = yl + o.nlocal * ncol;
  T* yh = xh + o.nclusters * q2 * ncol;
  const int tb = 256;
  k_gather<T><<<blocks_for(o.nlocal * ncol, tb), tb, 0, s>>>(x, xl, o.d_ex, o.L, o.d, o.n1, o.ndofs, o.nlocal, ncol, C);
  launched("kernel");
  if (q2 > 0) {
    const int64_t leaf_off = o.lvl_off[o.leaf];
    k_leaf_up<T><<<blocks_for(o.nleaf * q2 * ncol, tb), tb, sizeof(T) * o.nld * q2, s>>>(
        xl, xh + leaf_off * q2 * ncol, V, o.nleaf, o.nld, q2, ncol);
    launched("kernel");
    const size_t tsh = sizeof(T) * 4 * q2 * q2;
    for (int l = o.leaf - 1; l >= 0; --l) {
      const int64_t np = o.lvl_off[l + 1] - o.lvl_off[l];
      k_up<T><<<blocks_for(np * q2 * ncol, tb), tb, tsh, s>>>(xh + o.lvl_off[l] * q2 * ncol,
                                                               xh + o.lvl_off[l + 1] * q2 * ncol, Tm, np, q2, ncol);
      launched("kernel");
    }
    if (o.cplx)
      k_coupling_mv<T, true><<<blocks_for(o.nclusters * q2 * nrhs, tb), tb, 0, s>>>(o.d_far_ptr, o.d_far_src, K, xh,
                                                                                    yh, o.nclusters, q2, nrhs);
    else
      k_coupling_mv<T, false><<<blocks_for(o.nclusters * q2 * nrhs, tb), tb, 0, s>>>(o.d_far_ptr, o.d_far_src, K,
                                                                                     xh, yh, o.nclusters, q2, nrhs);
      launched("kernel");
    for (int l = 1; l <= o.leaf; ++l) {
      const int64_t nc = o.lvl_off[l + 1] - o.lvl_off[l];
      k_down<T><<<blocks_for(nc * q2 * ncol, tb), tb, tsh, s>>>(yh + o.lvl_off[l] * q2 * ncol,
                                                                 yh + o.lvl_off[l - 1] * q2 * ncol, Tm, nc, q2, ncol);
      launched("kernel");
    }
  }
  const T* yh_leaf = q2 > 0 ? yh + o.lvl_off[o.leaf] * q2 * ncol : nullptr;
  if (o.cplx)
    k_leaf_near<T, true><<<blocks_for(o.nleaf * o.nld * nrhs, tb), tb, 0, s>>>(
        o.d_near_ptr, o.d_near_col, N, xl, V, yh_leaf, yl, o.nleaf, o.nld, q2, nrhs);
  else
    k_leaf_near<T, false><<<blocks_for(o.nleaf * o.nld * nrhs, tb), tb, 0, s>>>(
        o.d_near_ptr, o.d_near_col, N, xl, V, yh_leaf, yl, o.nleaf, o.nld, q2, nrhs);
    launched("kernel");
  k_scatter<T><<<blocks_for(o.ndofs * ncol, tb), tb, 0, s>>>(yl, y, o.d_ex, o.L, o.d, o.n1, o.ndofs, ncol, C);
  launched("matvec kernels");
}

}  // namespace

void gather_to_local(const Op& o, const double* x, double* xl, int nrhs, cudaStream_t s) {
  const int C = o.cplx ? 2 : 1;
  const int ncol = nrhs * C;
  k_gather<double><<<blocks_for(o.nlocal * ncol, 256), 256, 0, s>>>(x, xl, o.d_ex, o.L, o.d, o.n1, o.ndofs, o.nlocal,
                                                                    ncol, C);
  launched("k_gather");
}

void scatter_to_global(const Op& o, const double* yl, double* y, int nrhs, cudaStream_t s) {
  const int C = o.cplx ? 2 : 1;
  const int ncol = nrhs * C;
  k_scatter<double><<<blocks_for(o.ndofs * ncol, 256), 256, 0, s>>>(yl, y, o.d_ex, o.L, o.d, o.n1, o.ndofs, ncol, C);
  launched("k_scatter");
}

size_t matvec_scratch_bytes(const Op& o, int nrhs, bool fp32) {
  const int C = o.cplx ? 2 : 1;
  const size_t el = fp32 ? sizeof(float) : sizeof(double);
  return el * (size_t)nrhs * C * (2 * (size_t)o.nlocal + 2 * (size_t)o.nclusters * o.q2);
}

void matvec_device(const Op& o, const void* x, void* y, int nrhs, bool fp32, cudaStream_t s) {
  ensure_scratch(const_cast<Op&>(o), matvec_scratch_bytes(o, nrhs, fp32));
  if (fp32) {
    if (!o.d_N32) fail(BEMBEL_EINVAL, "FP32 matvec needs an operator assembled with precision MIXED");
    matvec_impl<float>(o, static_cast<const float*>(x), static_cast<float*>(y), nrhs, s, o.d_K32, o.d_N32, o.d_V32,
                       o.d_T32, o.d_scratch);
  } else {
    matvec_impl<double>(o, static_cast<const double*>(x), static_cast<double*>(y), nrhs, s, o.d_K, o.d_N, o.d_V,
                        o.d_T, o.d_scratch);
  }
}

// ---------------------------------------------------------------------------
// Matvec without allocation.  The scratch lives in this file-scope device
// array instead of operator-owned cudaMalloc memory; every GPU that loads the
// library holds it until the process exits.  Host code cannot use the array's
// name as a device address, so its address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and cached.
// ---------------------------------------------------------------------------
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // 8 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

void* noalloc_scratch_address() {
  int dev = 0;
  cuda_check(cudaGetDevice(&dev), "matvec_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) fail(BEMBEL_EINVAL, "matvec_noalloc: device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cuda_check(cudaGetSymbolAddress(&p, g_noalloc_scratch), "matvec_noalloc: cudaGetSymbolAddress");
    g_noalloc_ptr[dev] = p;
  }
  return g_noalloc_ptr[dev];
}
}  // namespace

size_t matvec_noalloc_limit() { return kNoAllocScratchBytes; }

void matvec_noalloc(const Op& o, const void* x, void* y, int nrhs, bool fp32, cudaStream_t s) {
  const size_t need = matvec_scratch_bytes(o, nrhs, fp32);
  if (need > kNoAllocScratchBytes)
    fail(BEMBEL_EINVAL, "matvec_noalloc: this operator and nrhs need " + std::to_string(need) +
                            " bytes of scratch; the fixed buffer holds " + std::to_string(kNoAllocScratchBytes) +
                            " bytes (use bembel_matvec)");
  if (fp32 && !o.d_N32) fail(BEMBEL_EINVAL, "FP32 matvec needs an operator assembled with precision MIXED");
  // every scratch element is written before it is read, so nothing is cleared
  void* scratch = noalloc_scratch_address();
  if (fp32)
    matvec_impl<float>(o, static_cast<const float*>(x), static_cast<float*>(y), nrhs, s, o.d_K32, o.d_N32, o.d_V32,
                       o.d_T32, scratch);
  else
    matvec_impl<double>(o, static_cast<const double*>(x), static_cast<double*>(y), nrhs, s, o.d_K, o.d_N, o.d_V,
                        o.d_T, scratch);
}

void ensure_scratch(Op& o, size_t bytes) {
  if (bytes <= o.scratch_bytes) return;
  if (o.d_scratch) {
    cuda_check(cudaStreamSynchronize(o.stream), "scratch sync");
    dev_free(o.d_scratch);
    o.d_scratch = nullptr;
    o.scratch_bytes = 0;
  }
  o.d_scratch = dev_alloc(bytes);
  o.scratch_bytes = bytes;
}

}  // namespace bembel
