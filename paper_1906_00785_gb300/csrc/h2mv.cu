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
#include <type_traits>
#include <string>

#include "op.h"

namespace bembel {

namespace {

template <typename K>
void set_smem_limit(K kernel, size_t bytes) {
  if (bytes > 48 * 1024)
    cuda_check(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)), "smem attr");
}

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

// S^1 (EFIE): extraction as CSR.  Gather: xl[row][col] = sum val * x[col_k][col];
// scatter with the transposed CSR (rows = global dofs).  API vectors are
// column-major (ndofs x nrhs, C reals per entry); local vectors dof-major.
template <typename T>
__global__ void k_csr_gather(const int* __restrict__ ptr, const int* __restrict__ cols,
                             const double* __restrict__ val, const T* __restrict__ x, T* __restrict__ xl,
                             int64_t ndofs, int64_t nlocal, int ncol, int C) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= nlocal * ncol) return;
  const int64_t row = id / ncol;
  const int col = int(id % ncol);
  const int r = col / C, comp = col % C;
  const T* xr = x + (int64_t)r * ndofs * C + comp;
  double acc = 0.0;
  for (int k = ptr[row]; k < ptr[row + 1]; ++k) acc += val[k] * (double)xr[(int64_t)cols[k] * C];
  xl[id] = T(acc);
}

template <typename T>
__global__ void k_csr_scatter(const int* __restrict__ ptr, const int* __restrict__ rows,
                              const double* __restrict__ val, const T* __restrict__ yl, T* __restrict__ y,
                              int64_t ndofs, int ncol, int C) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= ndofs * ncol) return;
  const int64_t g = id / ncol;
  const int col = int(id % ncol);
  const int r = col / C, comp = col % C;
  double acc = 0.0;
  for (int k = ptr[g]; k < ptr[g + 1]; ++k) acc += val[k] * (double)yl[(int64_t)rows[k] * ncol + col];
  y[((int64_t)r * ndofs + g) * C + comp] = T(acc);
}

// Wide products: the API vectors (one contiguous vector per column) are first
// transposed to dof-major (ndofs x ncol, 32 x 32 shared-memory tiles), so the
// gather and scatter read and write whole rows of columns.
template <typename T>
__global__ void k_to_dofmajor(const T* __restrict__ x, T* __restrict__ xt, int64_t ndofs, int ncol, int C) {
  __shared__ T tile[32][33];
  const int64_t g0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  // read: consecutive threads along dofs of one column (column c = r * C + comp)
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i;
    const int64_t g = g0 + threadIdx.x;
    if (c < ncol && g < ndofs) tile[i][threadIdx.x] = x[((int64_t)(c / C) * ndofs + g) * C + c % C];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t g = g0 + i;
    const int c = c0 + threadIdx.x;
    if (c < ncol && g < ndofs) xt[g * ncol + c] = tile[threadIdx.x][i];
  }
}

template <typename T>
__global__ void k_from_dofmajor(const T* __restrict__ yt, T* __restrict__ y, int64_t ndofs, int ncol, int C) {
  __shared__ T tile[32][33];
  const int64_t g0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t g = g0 + i;
    const int c = c0 + threadIdx.x;
    if (c < ncol && g < ndofs) tile[i][threadIdx.x] = yt[g * ncol + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i;
    const int64_t g = g0 + threadIdx.x;
    if (c < ncol && g < ndofs) y[((int64_t)(c / C) * ndofs + g) * C + c % C] = tile[threadIdx.x][i];
  }
}

// S^2 gather from dof-major x: warp per local dof, lanes over columns.  The extraction
// coefficient of each term is formed once per block of kCb columns per lane and the sums run
// in T (FP32 products accumulate in FP32).
constexpr int kCb = 4;

template <typename T>
__global__ void k_gather_dm(const T* __restrict__ xt, T* __restrict__ xl, const double* __restrict__ ex, int L, int d,
                            int n1, int64_t nlocal, int ncol) {
  const int64_t ld = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (ld >= nlocal) return;
  const int D1 = d + 1, nloc = D1 * D1;
  const int64_t e = ld / nloc;
  const int k = int(ld % nloc), k1 = k % D1, k2 = k / D1;
  const int64_t per = int64_t(1) << (2 * L);
  const int patch = int(e / per);
  uint32_t i1, i2;
  morton_decode(uint32_t(e % per), i1, i2);
  for (int c0 = 0; c0 < ncol; c0 += 32 * kCb) {
    T acc[kCb];
#pragma unroll
    for (int b = 0; b < kCb; ++b) acc[b] = T(0);
    for (int j2 = 0; j2 < D1; ++j2) {
      const double c2 = ex[((int64_t)i2 * D1 + j2) * D1 + k2];
      if (c2 == 0.0) continue;
      for (int j1 = 0; j1 < D1; ++j1) {
        const double c1 = ex[((int64_t)i1 * D1 + j1) * D1 + k1];
        if (c1 == 0.0) continue;
        const T w = T(c1 * c2);
        const T* xr = xt + ((int64_t)patch * n1 * n1 + (int64_t)(i2 + j2) * n1 + (i1 + j1)) * ncol;
#pragma unroll
        for (int b = 0; b < kCb; ++b) {
          const int c = c0 + b * 32 + lane;
          if (c < ncol) acc[b] = fma(w, xr[c], acc[b]);
        }
      }
    }
#pragma unroll
    for (int b = 0; b < kCb; ++b) {
      const int c = c0 + b * 32 + lane;
      if (c < ncol) xl[ld * ncol + c] = acc[b];
    }
  }
}

// S^2 scatter to dof-major y: warp per global dof, lanes over columns (as k_gather_dm).
template <typename T>
__global__ void k_scatter_dm(const T* __restrict__ yl, T* __restrict__ yt, const double* __restrict__ ex, int L,
                             int d, int n1, int64_t ndofs, int ncol) {
  const int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= ndofs) return;
  const int D1 = d + 1, nloc = D1 * D1;
  const int nel1 = 1 << L;
  const int patch = int(g / ((int64_t)n1 * n1));
  const int rem = int(g % ((int64_t)n1 * n1));
  const int j2 = rem / n1, j1 = rem % n1;
  const int64_t per = int64_t(1) << (2 * L);
  for (int c0 = 0; c0 < ncol; c0 += 32 * kCb) {
    T acc[kCb];
#pragma unroll
    for (int b = 0; b < kCb; ++b) acc[b] = T(0);
    for (int i2 = max(0, j2 - d); i2 <= min(nel1 - 1, j2); ++i2)
      for (int i1 = max(0, j1 - d); i1 <= min(nel1 - 1, j1); ++i1) {
        const int64_t e = (int64_t)patch * per + morton_encode(i1, i2);
        for (int k2 = 0; k2 < D1; ++k2) {
          const double c2 = ex[((int64_t)i2 * D1 + (j2 - i2)) * D1 + k2];
          if (c2 == 0.0) continue;
          for (int k1 = 0; k1 < D1; ++k1) {
            const double c1 = ex[((int64_t)i1 * D1 + (j1 - i1)) * D1 + k1];
            if (c1 == 0.0) continue;
            const T w = T(c1 * c2);
            const T* yr = yl + (e * nloc + k1 + D1 * k2) * ncol;
#pragma unroll
            for (int b = 0; b < kCb; ++b) {
              const int c = c0 + b * 32 + lane;
              if (c < ncol) acc[b] = fma(w, yr[c], acc[b]);
            }
          }
        }
      }
#pragma unroll
    for (int b = 0; b < kCb; ++b) {
      const int c = c0 + b * 32 + lane;
      if (c < ncol) yt[g * ncol + c] = acc[b];
    }
  }
}

// element-local <-> global for either space
// matvec_noalloc sets this: nothing may be allocated on its path
static thread_local bool t_no_alloc = false;

// dof-major staging buffer for wide S^2 products (ndofs x ncol): used when it
// is already large enough, or grown when allocating is allowed here (not under
// graph capture, not on the no-allocation path); otherwise the strided kernels run
template <typename T>
T* dofmajor_buffer(const Op& o, int ncol) {
  const size_t bytes = sizeof(T) * (size_t)o.ndofs * ncol;
  if (o.d_e_ptr || ncol < 32) return nullptr;  // CSR extraction: no dof-major path
  if (o.dofmajor_bytes < bytes) {
    if (capturing() || t_no_alloc) return nullptr;
    ensure_dofmajor(const_cast<Op&>(o), bytes);
  }
  return static_cast<T*>(o.d_dofmajor);
}

template <typename T>
void gather_l(const Op& o, const T* x, T* xl, int ncol, int C, cudaStream_t s) {
  if (T* xt = dofmajor_buffer<T>(o, ncol)) {
    k_to_dofmajor<T><<<dim3(unsigned((o.ndofs + 31) / 32), unsigned((ncol + 31) / 32)), dim3(32, 8), 0, s>>>(
        x, xt, o.ndofs, ncol, C);
    launched("k_to_dofmajor");
    k_gather_dm<T><<<blocks_for(o.nlocal * 32, 256), 256, 0, s>>>(xt, xl, o.d_ex, o.L, o.d, o.n1, o.nlocal, ncol);
    launched("k_gather_dm");
    return;
  }
  if (o.d_e_ptr)
    k_csr_gather<T><<<blocks_for(o.nlocal * ncol, 256), 256, 0, s>>>(o.d_e_ptr, o.d_e_col, o.d_e_val, x, xl,
                                                                      o.ndofs, o.nlocal, ncol, C);
  else
    k_gather<T><<<blocks_for(o.nlocal * ncol, 256), 256, 0, s>>>(x, xl, o.d_ex, o.L, o.d, o.n1, o.ndofs, o.nlocal,
                                                                  ncol, C);
  launched("k_gather");
}

template <typename T>
void scatter_l(const Op& o, const T* yl, T* y, int ncol, int C, cudaStream_t s) {
  if (T* yt = dofmajor_buffer<T>(o, ncol)) {
    k_scatter_dm<T><<<blocks_for(o.ndofs * 32, 256), 256, 0, s>>>(yl, yt, o.d_ex, o.L, o.d, o.n1, o.ndofs, ncol);
    launched("k_scatter_dm");
    k_from_dofmajor<T><<<dim3(unsigned((o.ndofs + 31) / 32), unsigned((ncol + 31) / 32)), dim3(32, 8), 0, s>>>(
        yt, y, o.ndofs, ncol, C);
    launched("k_from_dofmajor");
    return;
  }
  if (o.d_e_ptr)
    k_csr_scatter<T><<<blocks_for(o.ndofs * ncol, 256), 256, 0, s>>>(o.d_et_ptr, o.d_et_col, o.d_et_val, yl, y,
                                                                      o.ndofs, ncol, C);
  else
    k_scatter<T><<<blocks_for(o.ndofs * ncol, 256), 256, 0, s>>>(yl, y, o.d_ex, o.L, o.d, o.n1, o.ndofs, ncol, C);
  launched("k_scatter");
}

// Compressed EFIE, three moment channels stored as extra columns of the
// cluster vectors: xh[leaf][a][ch ncol + col] = sum_i V[ch][i][a] xl[leaf nld + i][col]
template <typename T>
__global__ void k_leaf_up_ch(const T* __restrict__ xl, T* __restrict__ xh, const T* __restrict__ V, int64_t nleaf,
                             int nld, int q2, int ncol) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= nleaf * q2 * 3 * ncol) return;
  const int col = int(id % ncol);
  const int ch = int((id / ncol) % 3);
  const int a = int((id / (3 * ncol)) % q2);
  const int64_t lf = id / ((int64_t)3 * ncol * q2);
  const T* Vc = V + (int64_t)ch * nld * q2;
  const T* x = xl + lf * nld * ncol + col;
  T acc = 0;
  for (int i = 0; i < nld; ++i) acc += Vc[(int64_t)i * q2 + a] * x[(int64_t)i * ncol];
  xh[(lf * q2 + a) * 3 * ncol + ch * ncol + col] = acc;
}

// yl[leaf nld + i][col] = sum_ch sum_a V[ch][i][a] yh[leaf][a][ch ncol + col]
template <typename T>
__global__ void k_leaf_down_ch(const T* __restrict__ yh, const T* __restrict__ V, T* __restrict__ yl, int64_t nleaf,
                               int nld, int q2, int ncol) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= nleaf * nld * ncol) return;
  const int col = int(id % ncol);
  const int i = int((id / ncol) % nld);
  const int64_t lf = id / ((int64_t)ncol * nld);
  T acc = 0;
  for (int ch = 0; ch < 3; ++ch) {
    const T* Vc = V + (int64_t)ch * nld * q2 + (int64_t)i * q2;
    const T* y = yh + lf * q2 * 3 * ncol + ch * ncol + col;
    for (int a = 0; a < q2; ++a) acc += Vc[a] * y[(int64_t)a * 3 * ncol];
  }
  yl[id] = acc;
}

// xh[leaf][a][col] = sum_i V[i][a] xl[leaf*nld + i][col]
template <typename T>
__global__ void k_leaf_up(const T* __restrict__ xl, T* __restrict__ xh, const T* __restrict__ V, int64_t nleaf,
                          int nld, int q2, int ncol) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
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
  extern __shared__ __align__(16) unsigned char smem_raw[];
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
  extern __shared__ __align__(16) unsigned char smem_raw[];
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

// Block-sparse product y[tgt(blk)] += M_blk x[src(blk)] over all blocks (bs x bs
// blocks stored row-major, entry (a, b) at a*bs + b; vectors block-major
// with nrhs (x2 complex) real columns contiguous).  With ONFLY the block is
// not read from memory but evaluated in FP32 from the cluster interpolation
// points: M_blk[a][b] = G(p[tgt][a], p[src][b]) / (4 pi).
// Blocks are split in equal chunks over warps; a slot of SW lanes (the power of
// two >= bs, at most 32) handles one block, one row a per lane (two for bs > 32).
// Row sums stay in registers while consecutive blocks of a slot share a target
// and are added to y with atomicAdd when it changes, so every block is read
// exactly once with coalesced loads and every SM gets an equal share.
template <typename T, bool CPLX, bool ONFLY, int RT>
__global__ void __launch_bounds__(256) k_bsr_mv(const int* __restrict__ tgt, const int* __restrict__ src,
                                                int64_t nblk, const T* __restrict__ M, const float* __restrict__ pts,
                                                float kre, float kim, const T* __restrict__ x, T* __restrict__ y,
                                                int bs, int nrhs, int chunk) {
  const int C = CPLX ? 2 : 1;
  const int ncol = nrhs * C;
  const int lane = threadIdx.x & 31;
  const int SW = bs <= 1 ? 1 : (bs <= 2 ? 2 : (bs <= 4 ? 4 : (bs <= 8 ? 8 : (bs <= 16 ? 16 : 32))));
  const int nslot = 32 / SW;
  const int slot = lane / SW, sl = lane % SW;
  const int rows = (bs + SW - 1) / SW;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t b0 = warp * chunk;
  if (b0 >= nblk) return;
  const int64_t b1 = min(nblk, b0 + chunk);
  const int64_t bs2 = (int64_t)bs * bs;
  for (int r0 = 0; r0 < nrhs; r0 += RT) {
    const int nr = min(RT, nrhs - r0);
    for (int ri = 0; ri < rows; ++ri) {
      const int a = sl + ri * SW;
      if (a >= bs) continue;
      T ar[RT], ai[RT];
#pragma unroll
      for (int k = 0; k < RT; ++k) ar[k] = ai[k] = T(0);
      int cur = -1;
      for (int64_t blk = b0 + slot; blk < b1; blk += nslot) {
        const int t = tgt[blk];
        if (t != cur) {
          if (cur >= 0) {
            T* yo = y + ((int64_t)cur * bs + a) * ncol + r0 * C;
#pragma unroll
            for (int k = 0; k < RT; ++k)
              if (k < nr) {
                atomicAdd(yo + k * C, ar[k]);
                if (CPLX) atomicAdd(yo + k * C + 1, ai[k]);
                ar[k] = ai[k] = T(0);
              }
          }
          cur = t;
        }
        const int sidx = src[blk];
        const T* xs = x + ((int64_t)sidx * bs) * ncol + r0 * C;
        float pa0 = 0.f, pa1 = 0.f, pa2 = 0.f;
        if (ONFLY) {
          const float* pa = pts + ((int64_t)t * bs + a) * 4;
          pa0 = pa[0];
          pa1 = pa[1];
          pa2 = pa[2];
        }
        for (int bb = 0; bb < bs; ++bb) {
          T mr, mi = T(0);
          if (ONFLY) {
            const float* pb = pts + ((int64_t)sidx * bs + bb) * 4;
            const float d0 = pa0 - pb[0], d1 = pa1 - pb[1], d2 = pa2 - pb[2];
            const float r2 = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
            const float rinv = rsqrtf(r2) * float(kInv4Pi);
            if (CPLX) {
              const float rr = r2 * rsqrtf(r2);
              float sn, cs;
              sincosf(kre * rr, &sn, &cs);
              const float am = (kim != 0.f ? expf(kim * rr) : 1.f) * rinv;
              mr = T(am * cs);
              mi = T(-am * sn);
            } else {
              mr = T(rinv);
            }
          } else {
            const T* mp = M + (blk * bs2 + (int64_t)a * bs + bb) * C;
            mr = mp[0];
            if (CPLX) mi = mp[1];
          }
          const T* xb = xs + (int64_t)bb * ncol;
#pragma unroll
          for (int k = 0; k < RT; ++k)
            if (k < nr) {
              if (CPLX) {
                const T xr = xb[k * 2], xi = xb[k * 2 + 1];
                ar[k] = fma(mr, xr, fma(-mi, xi, ar[k]));
                ai[k] = fma(mr, xi, fma(mi, xr, ai[k]));
              } else {
                ar[k] = fma(mr, xb[k], ar[k]);
              }
            }
        }
      }
      if (cur >= 0) {
        T* yo = y + ((int64_t)cur * bs + a) * ncol + r0 * C;
#pragma unroll
        for (int k = 0; k < RT; ++k)
          if (k < nr) {
            atomicAdd(yo + k * C, ar[k]);
            if (CPLX) atomicAdd(yo + k * C + 1, ai[k]);
          }
      }
    }
  }
}

// Single right-hand side form of k_bsr_mv: a lane reads its whole block row
// with 16-byte vector loads (row-major blocks), and the source vector segment
// (or the source points when ONFLY) with broadcast vector loads.
template <typename T, bool CPLX, bool ONFLY>
__global__ void __launch_bounds__(256) k_bsr_mv1(const int* __restrict__ tgt, const int* __restrict__ src,
                                                 int64_t nblk, const T* __restrict__ M,
                                                 const float4* __restrict__ pts, float kre, float kim,
                                                 const T* __restrict__ x, T* __restrict__ y, int bs, int chunk) {
  constexpr int C = CPLX ? 2 : 1;
  constexpr int V = 16 / sizeof(T);  // scalars per 16-byte load
  using VT = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  const int lane = threadIdx.x & 31;
  const int SW = bs <= 4 ? 4 : (bs <= 8 ? 8 : (bs <= 16 ? 16 : 32));
  const int nslot = 32 / SW;
  const int slot = lane / SW, sl = lane % SW;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t b0 = warp * chunk;
  if (b0 >= nblk) return;
  const int64_t b1 = min(nblk, b0 + chunk);
  const int rowlen = bs * C;  // scalars per block row
  const int nvec = rowlen / V;
  const T fscale = ONFLY ? T(kInv4Pi) : T(1);
  for (int a = sl; a < bs; a += SW) {
    T ar = T(0), ai = T(0);
    int cur = -1;
    for (int64_t blk = b0 + slot; blk < b1; blk += nslot) {
      const int t = tgt[blk];
      if (t != cur) {
        if (cur >= 0) {
          atomicAdd(y + ((int64_t)cur * bs + a) * C, ar * fscale);
          if (CPLX) atomicAdd(y + ((int64_t)cur * bs + a) * C + 1, ai * fscale);
          ar = ai = T(0);
        }
        cur = t;
      }
      const int sidx = src[blk];
      const VT* xv = reinterpret_cast<const VT*>(x + (int64_t)sidx * rowlen);
      if (!ONFLY) {
        const VT* mv = reinterpret_cast<const VT*>(M + ((int64_t)blk * bs + a) * rowlen);
#pragma unroll 4
        for (int k = 0; k < nvec; ++k) {
          const VT m4 = mv[k], x4 = xv[k];
          const T* mm = reinterpret_cast<const T*>(&m4);
          const T* xx = reinterpret_cast<const T*>(&x4);
#pragma unroll
          for (int u = 0; u < V; u += C) {
            if (CPLX) {
              ar = fma(mm[u], xx[u], fma(-mm[u + 1], xx[u + 1], ar));
              ai = fma(mm[u], xx[u + 1], fma(mm[u + 1], xx[u], ai));
            } else {
              ar = fma(mm[u], xx[u], ar);
            }
          }
        }
      } else {
        const float4 pa = pts[(int64_t)t * bs + a];
        const float4* pb = pts + (int64_t)sidx * bs;
#pragma unroll 4
        for (int k = 0; k < nvec; ++k) {
          const VT x4 = xv[k];
          const T* xx = reinterpret_cast<const T*>(&x4);
#pragma unroll
          for (int u = 0; u < V; u += C) {
            const float4 p = pb[(k * V + u) / C];
            const float d0 = pa.x - p.x, d1 = pa.y - p.y, d2 = pa.z - p.z;
            const float r2 = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
            const float rinv = rsqrtf(r2);  // 1/(4 pi) applied when the row sum is flushed
            if (CPLX) {
              const float rr = r2 * rinv;
              float sn, cs;
              sincosf(kre * rr, &sn, &cs);  // full range reduction: kappa r reaches tens
              const float am = (kim != 0.f ? expf(kim * rr) : 1.f) * rinv;
              const float mr = am * cs, mi = -am * sn;
              ar = fma(T(mr), xx[u], fma(T(-mi), xx[u + 1], ar));
              ai = fma(T(mr), xx[u + 1], fma(T(mi), xx[u], ai));
            } else {
              ar = fma(T(rinv), xx[u], ar);
            }
          }
        }
      }
    }
    if (cur >= 0) {
      atomicAdd(y + ((int64_t)cur * bs + a) * C, ar * fscale);
      if (CPLX) atomicAdd(y + ((int64_t)cur * bs + a) * C + 1, ai * fscale);
    }
  }
}

// FP32 far-field coupling evaluated on the fly for one right-hand side and q = 4 (16
// interpolation points per cluster): four lanes per far block, each with four target
// points in registers and all 16 source points, eight blocks of a warp's chunk at a time.
// A source point is loaded once per four kernel evaluations (the generic kernel above
// loads one per evaluation) and a target's points once per run of blocks with that
// target (the far list is ordered by target); row sums are flushed with atomics when the
// target changes.  y must be cleared by the caller.
template <bool CPLX>
__global__ void __launch_bounds__(256) k_onfly_q4(const int* __restrict__ tgt, const int* __restrict__ src,
                                                  int64_t nblk, const float4* __restrict__ pts, float kre, float kim,
                                                  const float* __restrict__ x, float* __restrict__ y, int chunk) {
  constexpr int C = CPLX ? 2 : 1;
  const int lane = threadIdx.x & 31;
  const int grp = lane >> 2, sl = lane & 3;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t b0 = warp * chunk;
  if (b0 >= nblk) return;
  const int64_t b1 = min(nblk, b0 + chunk);
  float ar[4] = {0.f, 0.f, 0.f, 0.f}, ai[4] = {0.f, 0.f, 0.f, 0.f};
  float4 pa[4];
  int cur = -1;
  auto flush = [&]() {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t row = (int64_t)cur * 16 + sl + 4 * k;
      atomicAdd(y + row * C, ar[k] * float(kInv4Pi));
      if (CPLX) atomicAdd(y + row * C + 1, ai[k] * float(kInv4Pi));
      ar[k] = ai[k] = 0.f;
    }
  };
  for (int64_t blk = b0 + grp; blk < b1; blk += 8) {
    const int t = tgt[blk];
    if (t != cur) {
      if (cur >= 0) flush();
      cur = t;
#pragma unroll
      for (int k = 0; k < 4; ++k) pa[k] = pts[(int64_t)t * 16 + sl + 4 * k];
    }
    const int sidx = src[blk];
    const float4* pb = pts + (int64_t)sidx * 16;
    const float* xs = x + (int64_t)sidx * 16 * C;
#pragma unroll 4
    for (int b = 0; b < 16; ++b) {
      const float4 p = pb[b];
      const float xr = xs[b * C], xi = CPLX ? xs[b * C + 1] : 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float d0 = pa[k].x - p.x, d1 = pa[k].y - p.y, d2 = pa[k].z - p.z;
        const float r2 = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
        const float rinv = rsqrtf(r2);
        if (CPLX) {
          const float rr = r2 * rinv;
          float sn, cs;
          sincosf(kre * rr, &sn, &cs);
          const float am = (kim != 0.f ? expf(kim * rr) : 1.f) * rinv;
          const float mr = am * cs, mi = -am * sn;
          ar[k] = fmaf(mr, xr, fmaf(-mi, xi, ar[k]));
          ai[k] = fmaf(mr, xi, fmaf(mi, xr, ai[k]));
        } else {
          ar[k] = fmaf(rinv, xr, ar[k]);
        }
      }
    }
  }
  if (cur >= 0) flush();
}

// y_loc[t*nld + i][col] = sum_a V[i][a] yh_leaf[t][a][col]  (real V, any columns)
template <typename T>
__global__ void k_leaf_down(const T* __restrict__ yh, const T* __restrict__ V, T* __restrict__ yl, int64_t nleaf,
                            int nld, int q2, int ncol) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Vs = reinterpret_cast<T*>(smem_raw);
  for (int i = threadIdx.x; i < nld * q2; i += blockDim.x) Vs[i] = V[i];
  __syncthreads();
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= nleaf * nld * ncol) return;
  const int col = int(id % ncol);
  const int i = int((id / ncol) % nld);
  const int64_t t = id / ((int64_t)ncol * nld);
  const T* yt = yh + (t * q2) * ncol + col;
  T acc = 0;
  for (int a = 0; a < q2; ++a) acc = fma(Vs[i * q2 + a], yt[(int64_t)a * ncol], acc);
  yl[id] = acc;
}

// ---------------------------------------------------------------------------
// Fused transfer passes.  Levels ls = max(0, leaf - 3) .. leaf are handled per
// subtree (one thread block per level-ls cluster, the subtree's values kept in
// shared memory); the few levels below ls by one small kernel per level.
// ---------------------------------------------------------------------------
struct LevelOffsets {
  long long off[16];
};

// Up: leaf moments xh_leaf = V^T x_loc and transfers up to level ls, one block
// per level-ls cluster P; writes xh on every level of the subtree.
template <typename T>
__global__ void k_up_subtree(const T* __restrict__ xl, T* __restrict__ xh, const T* __restrict__ V,
                             const T* __restrict__ Tm, LevelOffsets lo, int leaf, int ls, int q2, int nld, int ncol) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Vs = reinterpret_cast<T*>(smem_raw);
  T* Ts = Vs + nld * q2;
  T* bufA = Ts + 4 * q2 * q2;
  const int D = leaf - ls;
  const int nsub = 1 << (2 * D);
  T* bufB = bufA + nsub * q2 * ncol;
  for (int i = threadIdx.x; i < nld * q2; i += blockDim.x) Vs[i] = V[i];
  for (int i = threadIdx.x; i < 4 * q2 * q2; i += blockDim.x) Ts[i] = Tm[i];
  __syncthreads();
  const int64_t P = blockIdx.x;
  const int per = q2 * ncol;
  for (int idx = threadIdx.x; idx < nsub * per; idx += blockDim.x) {
    const int col = idx % ncol, a = (idx / ncol) % q2, li = idx / per;
    const int64_t leafid = P * nsub + li;
    const T* x = xl + leafid * nld * ncol + col;
    T acc = 0;
    for (int i = 0; i < nld; ++i) acc = fma(Vs[i * q2 + a], x[(int64_t)i * ncol], acc);
    bufA[idx] = acc;
    xh[(lo.off[leaf] + leafid) * per + a * ncol + col] = acc;
  }
  __syncthreads();
  T* cur = bufA;
  T* nxt = bufB;
  int ncur = nsub;
  for (int l = leaf - 1; l >= ls; --l) {
    const int npar = ncur >> 2;
    for (int idx = threadIdx.x; idx < npar * per; idx += blockDim.x) {
      const int col = idx % ncol, a = (idx / ncol) % q2, pi = idx / per;
      T acc = 0;
      for (int c = 0; c < 4; ++c) {
        const T* xc = cur + (4 * pi + c) * per + col;
        const T* Tc = Ts + c * q2 * q2;
        for (int ap = 0; ap < q2; ++ap) acc = fma(Tc[ap * q2 + a], xc[ap * ncol], acc);
      }
      nxt[idx] = acc;
      xh[(lo.off[l] + P * npar + pi) * per + a * ncol + col] = acc;
    }
    __syncthreads();
    T* t = cur;
    cur = nxt;
    nxt = t;
    ncur = npar;
  }
}

// Down from level ls to the leaves and the leaf evaluation y_loc = V yh_leaf,
// one block per level-ls cluster (intermediate levels stay in shared memory).
template <typename T>
__global__ void k_down_subtree(const T* __restrict__ yh, T* __restrict__ yl, const T* __restrict__ V,
                               const T* __restrict__ Tm, LevelOffsets lo, int leaf, int ls, int q2, int nld,
                               int ncol) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Vs = reinterpret_cast<T*>(smem_raw);
  T* Ts = Vs + nld * q2;
  T* bufA = Ts + 4 * q2 * q2;
  const int D = leaf - ls;
  const int nsub = 1 << (2 * D);
  T* bufB = bufA + nsub * q2 * ncol;
  for (int i = threadIdx.x; i < nld * q2; i += blockDim.x) Vs[i] = V[i];
  for (int i = threadIdx.x; i < 4 * q2 * q2; i += blockDim.x) Ts[i] = Tm[i];
  const int64_t P = blockIdx.x;
  const int per = q2 * ncol;
  for (int idx = threadIdx.x; idx < per; idx += blockDim.x) bufA[idx] = yh[(lo.off[ls] + P) * per + idx];
  __syncthreads();
  T* cur = bufA;
  T* nxt = bufB;
  int ncur = 1;
  for (int l = ls + 1; l <= leaf; ++l) {
    const int nch = ncur * 4;
    for (int idx = threadIdx.x; idx < nch * per; idx += blockDim.x) {
      const int col = idx % ncol, ap = (idx / ncol) % q2, ci = idx / per;
      const T* Tc = Ts + (ci & 3) * q2 * q2 + ap * q2;
      const T* y = cur + (ci >> 2) * per + col;
      T acc = yh[(lo.off[l] + P * nch + ci) * per + ap * ncol + col];
      for (int a = 0; a < q2; ++a) acc = fma(Tc[a], y[a * ncol], acc);
      nxt[idx] = acc;
    }
    __syncthreads();
    T* t = cur;
    cur = nxt;
    nxt = t;
    ncur = nch;
  }
  // leaves of this subtree: y_loc = V yh_leaf
  for (int idx = threadIdx.x; idx < nsub * nld * ncol; idx += blockDim.x) {
    const int col = idx % ncol, i = (idx / ncol) % nld, li = idx / (nld * ncol);
    const T* y = cur + li * per + col;
    T acc = 0;
    for (int a = 0; a < q2; ++a) acc = fma(Vs[i * q2 + a], y[a * ncol], acc);
    yl[((P * nsub + li) * nld + i) * (int64_t)ncol + col] = acc;
  }
}

// Block-sparse product for many right-hand sides, one CTA per target block
// row: y[t] += sum_{k in row t} M_k x[col_k].  Each block (bs x bs, row-major)
// and its source slice (bs x ncol) are staged in shared memory (two buffers),
// every thread accumulates up to rows_for(JB) rows for JB columns (complex pairs
// for CPLX) in registers and adds them into its own outputs: the block matrix is
// read once per product and no atomics are needed.  JB = 2 serves two columns
// from each block entry read from shared memory (half the loads per FMA).
constexpr int kRowOut = 16;
constexpr int kRowThreads = 256;
__host__ __device__ constexpr int rows_for(int jb) { return jb == 1 ? kRowOut : 10; }

template <typename T>
struct Pair;
template <>
struct Pair<float> {
  using type = float2;
};
template <>
struct Pair<double> {
  using type = double2;
};

template <typename T, bool CPLX, int JB>
__global__ void __launch_bounds__(kRowThreads) k_bsr_rows(const long long* __restrict__ ptr,
                                                          const int* __restrict__ col, int64_t nrows,
                                                          const T* __restrict__ M, const T* __restrict__ x,
                                                          T* __restrict__ y, int bs, int nrhs) {
  constexpr int C = CPLX ? 2 : 1;
  constexpr int RO = rows_for(JB);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ncol = nrhs * C;
  const int mstride = bs * bs * C, xstride = bs * ncol;
  T* Ms = reinterpret_cast<T*>(smem_raw);  // [2][bs*bs*C]
  T* Xs = Ms + 2 * mstride;                // [2][bs*ncol]
  const int64_t t = blockIdx.x;
  if (t >= nrows) return;
  // thread (row group rg, column slot js): columns js + nj q (q < JB), rows rg + ng o
  const int nj = nrhs / JB;
  const int js = threadIdx.x % nj, rg = threadIdx.x / nj, ng = kRowThreads / nj;
  T accr[RO][JB], acci[RO][JB];
#pragma unroll
  for (int o = 0; o < RO; ++o)
#pragma unroll
    for (int q = 0; q < JB; ++q) accr[o][q] = acci[o][q] = T(0);
  const long long k0 = ptr[t], k1 = ptr[t + 1];
  // staging: asynchronous 16-byte copies (cp.async) when every piece is 16-byte
  // aligned, so the next block streams in while the current one is used
  const bool async = ((mstride * sizeof(T)) % 16 == 0) && ((xstride * sizeof(T)) % 16 == 0) &&
                     ((reinterpret_cast<uintptr_t>(M) | reinterpret_cast<uintptr_t>(x)) % 16 == 0);
  auto stage = [&](long long k, int buf) {
    const T* mk = M + k * (int64_t)mstride;
    const T* xk = x + (int64_t)col[k] * xstride;
    if (async) {
      const int mchunks = int(mstride * sizeof(T) / 16), xchunks = int(xstride * sizeof(T) / 16);
      const char* msrc = reinterpret_cast<const char*>(mk);
      const char* xsrc = reinterpret_cast<const char*>(xk);
      const uint32_t mdst = static_cast<uint32_t>(__cvta_generic_to_shared(Ms + buf * mstride));
      const uint32_t xdst = static_cast<uint32_t>(__cvta_generic_to_shared(Xs + buf * xstride));
      for (int i = threadIdx.x; i < mchunks; i += blockDim.x)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(mdst + 16 * i), "l"(msrc + 16 * i)
                     : "memory");
      for (int i = threadIdx.x; i < xchunks; i += blockDim.x)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(xdst + 16 * i), "l"(xsrc + 16 * i)
                     : "memory");
      asm volatile("cp.async.commit_group;" ::: "memory");
    } else {
      for (int i = threadIdx.x; i < mstride; i += blockDim.x) Ms[buf * mstride + i] = mk[i];
      for (int i = threadIdx.x; i < xstride; i += blockDim.x) Xs[buf * xstride + i] = xk[i];
    }
  };
  if (k0 < k1) stage(k0, 0);
  for (long long k = k0; k < k1; ++k) {
    const int buf = int((k - k0) & 1);
    if (k + 1 < k1) stage(k + 1, buf ^ 1);  // buf ^ 1 was released by the previous iteration's barrier
    if (async) {
      if (k + 1 < k1)
        asm volatile("cp.async.wait_group 1;" ::: "memory");  // block k has landed (k + 1 may be in flight)
      else
        asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    const T* Mb = Ms + buf * mstride;
    const T* Xb = Xs + buf * xstride;
    if (rg < ng) {
      for (int b = 0; b < bs; ++b) {
        T xr[JB], xi[JB];
#pragma unroll
        for (int q = 0; q < JB; ++q) {
          const T* xv = Xb + (int64_t)b * ncol + (js + nj * q) * C;
          if (CPLX) {  // complex pairs as one 8- or 16-byte shared load
            const auto x2 = *reinterpret_cast<const typename Pair<T>::type*>(xv);
            xr[q] = x2.x;
            xi[q] = x2.y;
          } else {
            xr[q] = xv[0];
            xi[q] = T(0);
          }
        }
#pragma unroll
        for (int o = 0; o < RO; ++o) {
          const int a = rg + ng * o;
          if (a >= bs) break;
          const T* m = Mb + ((int64_t)a * bs + b) * C;
          if (CPLX) {
            const auto m2 = *reinterpret_cast<const typename Pair<T>::type*>(m);
#pragma unroll
            for (int q = 0; q < JB; ++q) {
              accr[o][q] = fma(m2.x, xr[q], fma(-m2.y, xi[q], accr[o][q]));
              acci[o][q] = fma(m2.x, xi[q], fma(m2.y, xr[q], acci[o][q]));
            }
          } else {
            const T mv = m[0];
#pragma unroll
            for (int q = 0; q < JB; ++q) accr[o][q] = fma(mv, xr[q], accr[o][q]);
          }
        }
      }
    }
    __syncthreads();
  }
  if (rg >= ng) return;
#pragma unroll
  for (int o = 0; o < RO; ++o) {
    const int a = rg + ng * o;
    if (a >= bs) break;
#pragma unroll
    for (int q = 0; q < JB; ++q) {
      T* yo = y + (t * bs + a) * (int64_t)ncol + (js + nj * q) * C;
      yo[0] += accr[o][q];
      if (CPLX) yo[1] += acci[o][q];
    }
  }
}

// the row kernel applies when the product is wide, nrhs divides the thread
// count and every thread's rows fit its registers
bool rows_kernel_fits(int bs, int nrhs, int C, size_t el) {
  const size_t shm = el * 2 * ((size_t)bs * bs * C + (size_t)bs * nrhs * C);
  if (nrhs * C < 8 || nrhs > kRowThreads || kRowThreads % nrhs != 0) return false;
  const int ng = kRowThreads / nrhs;
  return (bs + ng - 1) / ng <= kRowOut && shm <= 160 * 1024;
}

// two columns per thread when nrhs is even and the rows of a thread fit its registers
static bool rows_two_columns(int bs, int nrhs) {
  if (nrhs % 2 != 0) return false;
  const int ng = kRowThreads / (nrhs / 2);
  return ng > 0 && (bs + ng - 1) / ng <= rows_for(2);
}

template <typename T, bool CPLX>
void launch_bsr_rows(const long long* ptr, const int* col, int64_t nrows, const T* M, const T* x, T* y, int bs,
                     int nrhs, cudaStream_t s) {
  const int C = CPLX ? 2 : 1;
  const size_t shm = sizeof(T) * 2 * ((size_t)bs * bs * C + (size_t)bs * nrhs * C);
  if (rows_two_columns(bs, nrhs)) {
    set_smem_limit(k_bsr_rows<T, CPLX, 2>, shm);
    k_bsr_rows<T, CPLX, 2><<<int(nrows), kRowThreads, shm, s>>>(ptr, col, nrows, M, x, y, bs, nrhs);
  } else {
    set_smem_limit(k_bsr_rows<T, CPLX, 1>, shm);
    k_bsr_rows<T, CPLX, 1><<<int(nrows), kRowThreads, shm, s>>>(ptr, col, nrows, M, x, y, bs, nrhs);
  }
  launched("k_bsr_rows");
}

template <typename T, bool CPLX, bool ONFLY>
void launch_bsr(const int* tgt, const int* src, int64_t nblk, const T* M, const float* pts, float kre, float kim,
                const T* x, T* y, int bs, int nrhs, cudaStream_t s, int chunk) {
  if (nblk == 0) return;
  const int64_t warps = (nblk + chunk - 1) / chunk;
  const int threads = 256;
  const int grid = int((warps * 32 + threads - 1) / threads);
  const int C = CPLX ? 2 : 1;
  const bool vec_ok = (bs * C * sizeof(T)) % 16 == 0 && bs >= 4 && bs <= 64;
  if constexpr (ONFLY && sizeof(T) == 4) {
    if (nrhs == 1 && bs == 16) {  // q = 4: register-blocked on-the-fly coupling
      constexpr int kChunk = 64;
      const int64_t w4 = (nblk + kChunk - 1) / kChunk;
      k_onfly_q4<CPLX><<<int((w4 * 32 + threads - 1) / threads), threads, 0, s>>>(
          tgt, src, nblk, reinterpret_cast<const float4*>(pts), kre, kim, reinterpret_cast<const float*>(x),
          reinterpret_cast<float*>(y), kChunk);
      launched("k_onfly_q4");
      return;
    }
  }
  if (nrhs == 1 && vec_ok)
    k_bsr_mv1<T, CPLX, ONFLY><<<grid, threads, 0, s>>>(tgt, src, nblk, M, reinterpret_cast<const float4*>(pts), kre,
                                                        kim, x, y, bs, chunk);
  else if (nrhs == 1)
    k_bsr_mv<T, CPLX, ONFLY, 1><<<grid, threads, 0, s>>>(tgt, src, nblk, M, pts, kre, kim, x, y, bs, nrhs, chunk);
  else
    k_bsr_mv<T, CPLX, ONFLY, 4><<<grid, threads, 0, s>>>(tgt, src, nblk, M, pts, kre, kim, x, y, bs, nrhs, chunk);
  launched("k_bsr_mv");
}

template <typename T>
void matvec_impl(const Op& o, const T* x, T* y, int nrhs, cudaStream_t s, const T* K, const T* N, const T* V,
                 const T* Tm, void* scratch) {
  const int C = o.cplx ? 2 : 1;
  const int ncol = nrhs * C;
  const int q2 = o.q2;
  const bool fp32 = sizeof(T) == 4;
  T* base = static_cast<T*>(scratch);
  T* xl = base;
  T* yl = xl + o.nlocal * ncol;
  T* xh = yl + o.nlocal * ncol;
  T* yh = xh + o.nclusters * q2 * ncol;
  const int tb = 256;
  gather_l<T>(o, x, xl, ncol, C, s);
  if (q2 > 0 && o.efie) {
    // compressed EFIE: channel moments, transfers on 3 ncol columns, coupling, back
    const int nch = 3 * ncol;
    T* xhe = xh;
    T* yhe = xh + o.nclusters * q2 * nch;
    const int64_t leaf_off = o.lvl_off[o.leaf];
    const size_t tsh = sizeof(T) * 4 * q2 * q2;
    set_smem_limit(k_up<T>, tsh);  // q >= 7: the four transfer matrices exceed 48 KiB
    set_smem_limit(k_down<T>, tsh);
    k_leaf_up_ch<T><<<blocks_for(o.nleaf * q2 * nch, tb), tb, 0, s>>>(xl, xhe + leaf_off * q2 * nch, V, o.nleaf,
                                                                       o.nld, q2, ncol);
    launched("k_leaf_up_ch");
    for (int l = o.leaf - 1; l >= 0; --l) {
      const int64_t np = o.lvl_off[l + 1] - o.lvl_off[l];
      k_up<T><<<blocks_for(np * q2 * nch, tb), tb, tsh, s>>>(xhe + o.lvl_off[l] * q2 * nch,
                                                             xhe + o.lvl_off[l + 1] * q2 * nch, Tm, np, q2, nch);
      launched("k_up");
    }
    efie_coupling_apply(o, xhe, yhe, nrhs, s);
    for (int l = 1; l <= o.leaf; ++l) {
      const int64_t nc = o.lvl_off[l + 1] - o.lvl_off[l];
      k_down<T><<<blocks_for(nc * q2 * nch, tb), tb, tsh, s>>>(yhe + o.lvl_off[l] * q2 * nch,
                                                               yhe + o.lvl_off[l - 1] * q2 * nch, Tm, nc, q2, nch);
      launched("k_down");
    }
    k_leaf_down_ch<T><<<blocks_for(o.nleaf * o.nld * ncol, tb), tb, 0, s>>>(yhe + leaf_off * q2 * nch, V, yl,
                                                                             o.nleaf, o.nld, q2, ncol);
    launched("k_leaf_down_ch");
  } else if (q2 > 0) {
    const int64_t leaf_off = o.lvl_off[o.leaf];
    const int ls = std::max(0, o.leaf - 3);
    const int nsub = 1 << (2 * (o.leaf - ls));
    const size_t sub_shm = sizeof(T) * ((size_t)o.nld * q2 + 4 * q2 * q2 + 2 * (size_t)nsub * q2 * ncol);
    const size_t tsh = sizeof(T) * 4 * q2 * q2;
    set_smem_limit(k_up<T>, tsh);  // q >= 7: the four transfer matrices exceed 48 KiB
    set_smem_limit(k_down<T>, tsh);
    const bool fused = sub_shm <= 96 * 1024 && o.leaf < 15;
    LevelOffsets lo{};
    for (int l = 0; l <= std::min(o.leaf, 14); ++l) lo.off[l] = o.lvl_off[l];
    if (fused) {
      set_smem_limit(k_up_subtree<T>, sub_shm);
      set_smem_limit(k_down_subtree<T>, sub_shm);
      const int nsubtrees = int(o.lvl_off[ls + 1] - o.lvl_off[ls]);
      k_up_subtree<T><<<nsubtrees, 256, sub_shm, s>>>(xl, xh, V, Tm, lo, o.leaf, ls, q2, o.nld, ncol);
      launched("k_up_subtree");
      for (int l = ls - 1; l >= 0; --l) {
        const int64_t np = o.lvl_off[l + 1] - o.lvl_off[l];
        k_up<T><<<blocks_for(np * q2 * ncol, 128), 128, tsh, s>>>(xh + o.lvl_off[l] * q2 * ncol,
                                                                   xh + o.lvl_off[l + 1] * q2 * ncol, Tm, np, q2,
                                                                   ncol);
        launched("k_up");
      }
    } else {
      set_smem_limit(k_leaf_up<T>, sizeof(T) * o.nld * q2);  // coarse leaves: moment matrix above 48 KiB
      k_leaf_up<T><<<blocks_for(o.nleaf * q2 * ncol, tb), tb, sizeof(T) * o.nld * q2, s>>>(
          xl, xh + leaf_off * q2 * ncol, V, o.nleaf, o.nld, q2, ncol);
      launched("k_leaf_up");
      for (int l = o.leaf - 1; l >= 0; --l) {
        const int64_t np = o.lvl_off[l + 1] - o.lvl_off[l];
        k_up<T><<<blocks_for(np * q2 * ncol, tb), tb, tsh, s>>>(xh + o.lvl_off[l] * q2 * ncol,
                                                                 xh + o.lvl_off[l + 1] * q2 * ncol, Tm, np, q2, ncol);
        launched("k_up");
      }
    }
    cuda_check(cudaMemsetAsync(yh, 0, sizeof(T) * o.nclusters * q2 * ncol, s), "yh clear");
    // FP32: coupling evaluated on the fly from the cluster points; FP64: stored coupling
    if (fp32 && tc_coupling_usable(o, nrhs)) {
      // many right-hand sides: sibling-grouped coupling on the tensor cores
      tc_coupling(o, reinterpret_cast<const float*>(xh), reinterpret_cast<float*>(yh), nrhs, s);
    } else if (fp32 && K && ncol >= 8 && rows_kernel_fits(q2, nrhs, C, sizeof(T))) {
      // many right-hand sides on the CUDA cores: stream the stored FP32 coupling
      if (o.cplx)
        launch_bsr_rows<T, true>(o.d_far_ptr, o.d_far_src, o.nclusters, K, xh, yh, q2, nrhs, s);
      else
        launch_bsr_rows<T, false>(o.d_far_ptr, o.d_far_src, o.nclusters, K, xh, yh, q2, nrhs, s);
    } else if (fp32 && K && o.opts.far_fp32_stored) {
      // narrow products streaming the stored FP32 coupling (chosen by the autotuner)
      if (o.cplx)
        launch_bsr<T, true, false>(o.d_far_tgt, o.d_far_src, o.nfar, K, nullptr, 0.f, 0.f, xh, yh, q2, nrhs, s,
                                   o.bsr_chunk);
      else
        launch_bsr<T, false, false>(o.d_far_tgt, o.d_far_src, o.nfar, K, nullptr, 0.f, 0.f, xh, yh, q2, nrhs, s,
                                    o.bsr_chunk);
    } else if (o.cplx) {
      if (fp32)
        launch_bsr<T, true, true>(o.d_far_tgt, o.d_far_src, o.nfar, nullptr, o.d_nodes32, float(o.kre),
                                  float(o.kim), xh, yh, q2, nrhs, s, o.bsr_chunk);
      else if (rows_kernel_fits(q2, nrhs, C, sizeof(T)))
        launch_bsr_rows<T, true>(o.d_far_ptr, o.d_far_src, o.nclusters, K, xh, yh, q2, nrhs, s);
      else
        launch_bsr<T, true, false>(o.d_far_tgt, o.d_far_src, o.nfar, K, nullptr, 0.f, 0.f, xh, yh, q2, nrhs, s, o.bsr_chunk);
    } else {
      if (fp32)
        launch_bsr<T, false, true>(o.d_far_tgt, o.d_far_src, o.nfar, nullptr, o.d_nodes32, 0.f, 0.f, xh, yh, q2,
                                   nrhs, s, o.bsr_chunk);
      else if (rows_kernel_fits(q2, nrhs, C, sizeof(T)))
        launch_bsr_rows<T, false>(o.d_far_ptr, o.d_far_src, o.nclusters, K, xh, yh, q2, nrhs, s);
      else
        launch_bsr<T, false, false>(o.d_far_tgt, o.d_far_src, o.nfar, K, nullptr, 0.f, 0.f, xh, yh, q2, nrhs, s, o.bsr_chunk);
    }
    if (fused) {
      for (int l = 1; l <= ls; ++l) {
        const int64_t nc = o.lvl_off[l + 1] - o.lvl_off[l];
        k_down<T><<<blocks_for(nc * q2 * ncol, 128), 128, tsh, s>>>(yh + o.lvl_off[l] * q2 * ncol,
                                                                     yh + o.lvl_off[l - 1] * q2 * ncol, Tm, nc, q2,
                                                                     ncol);
        launched("k_down");
      }
      const int nsubtrees = int(o.lvl_off[ls + 1] - o.lvl_off[ls]);
      k_down_subtree<T><<<nsubtrees, 256, sub_shm, s>>>(yh, yl, V, Tm, lo, o.leaf, ls, q2, o.nld, ncol);
      launched("k_down_subtree");
    } else {
      for (int l = 1; l <= o.leaf; ++l) {
        const int64_t nc = o.lvl_off[l + 1] - o.lvl_off[l];
        k_down<T><<<blocks_for(nc * q2 * ncol, tb), tb, tsh, s>>>(yh + o.lvl_off[l] * q2 * ncol,
                                                                   yh + o.lvl_off[l - 1] * q2 * ncol, Tm, nc, q2,
                                                                   ncol);
        launched("k_down");
      }
      set_smem_limit(k_leaf_down<T>, sizeof(T) * o.nld * q2);
      k_leaf_down<T><<<blocks_for(o.nleaf * o.nld * ncol, tb), tb, sizeof(T) * o.nld * q2, s>>>(
          yh + leaf_off * q2 * ncol, V, yl, o.nleaf, o.nld, q2, ncol);
      launched("k_leaf_down");
    }
  } else {
    cuda_check(cudaMemsetAsync(yl, 0, sizeof(T) * o.nlocal * ncol, s), "yl clear");
  }
  if (rows_kernel_fits(o.nld, nrhs, C, sizeof(T))) {
    // many right-hand sides: one CTA per target leaf row
    if (o.cplx)
      launch_bsr_rows<T, true>(o.d_near_ptr, o.d_near_col, o.nleaf, N, xl, yl, o.nld, nrhs, s);
    else
      launch_bsr_rows<T, false>(o.d_near_ptr, o.d_near_col, o.nleaf, N, xl, yl, o.nld, nrhs, s);
  } else if (o.cplx) {
    launch_bsr<T, true, false>(o.d_near_tgt, o.d_near_col, o.nnear, N, nullptr, 0.f, 0.f, xl, yl, o.nld, nrhs, s, o.bsr_chunk);
  } else {
    launch_bsr<T, false, false>(o.d_near_tgt, o.d_near_col, o.nnear, N, nullptr, 0.f, 0.f, xl, yl, o.nld, nrhs, s, o.bsr_chunk);
  }
  scatter_l<T>(o, yl, y, ncol, C, s);
}

}  // namespace

void cluster_moments(const Op& o, const double* x, double* xl, double* xh, int nrhs, cudaStream_t s) {
  if (o.q2 == 0 || o.efie) fail(BEMBEL_EUNSUPPORTED, "cluster moments: compressed S^2 operators only");
  const int C = o.cplx ? 2 : 1;
  const int ncol = nrhs * C;
  const int q2 = o.q2, tb = 256;
  gather_l<double>(o, x, xl, ncol, C, s);
  const int64_t leaf_off = o.lvl_off[o.leaf];
  set_smem_limit(k_leaf_up<double>, sizeof(double) * o.nld * q2);
  k_leaf_up<double><<<blocks_for(o.nleaf * q2 * ncol, tb), tb, sizeof(double) * o.nld * q2, s>>>(
      xl, xh + leaf_off * q2 * ncol, o.d_V, o.nleaf, o.nld, q2, ncol);
  launched("k_leaf_up");
  const size_t tsh = sizeof(double) * 4 * q2 * q2;
  set_smem_limit(k_up<double>, tsh);
  for (int l = o.leaf - 1; l >= 0; --l) {
    const int64_t np = o.lvl_off[l + 1] - o.lvl_off[l];
    k_up<double><<<blocks_for(np * q2 * ncol, tb), tb, tsh, s>>>(xh + o.lvl_off[l] * q2 * ncol,
                                                                  xh + o.lvl_off[l + 1] * q2 * ncol, o.d_T, np, q2,
                                                                  ncol);
    launched("k_up");
  }
}

void gather_to_local(const Op& o, const double* x, double* xl, int nrhs, cudaStream_t s) {
  const int C = o.cplx ? 2 : 1;
  const int ncol = nrhs * C;
  gather_l<double>(o, x, xl, ncol, C, s);
}

void scatter_to_global(const Op& o, const double* yl, double* y, int nrhs, cudaStream_t s) {
  const int C = o.cplx ? 2 : 1;
  const int ncol = nrhs * C;
  scatter_l<double>(o, yl, y, ncol, C, s);
}

size_t matvec_scratch_bytes(const Op& o, int nrhs, bool fp32) {
  const int C = o.cplx ? 2 : 1;
  const size_t el = fp32 ? sizeof(float) : sizeof(double);
  const size_t channels = o.efie ? 3 : 1;  // compressed EFIE: three moment channels
  return el * (size_t)nrhs * C * (2 * (size_t)o.nlocal + 2 * channels * (size_t)o.nclusters * o.q2);
}

void matvec_device(const Op& o, const void* x, void* y, int nrhs, bool fp32, cudaStream_t s) {
  ensure_scratch(const_cast<Op&>(o), matvec_scratch_bytes(o, nrhs, fp32));
  if (fp32) tc_prepare(const_cast<Op&>(o), nrhs);
  if (fp32) coupling_f32_prepare(const_cast<Op&>(o), nrhs);
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

// Looking the address up loads this file's module (and so the fixed array) on
// the current device when lazy module loading deferred it; assembly calls this
// so that a later matvec_noalloc on the device has nothing left to load.
void noalloc_prepare() { (void)noalloc_scratch_address(); }

void matvec_noalloc(const Op& o, const void* x, void* y, int nrhs, bool fp32, cudaStream_t s) {
  const size_t need = matvec_scratch_bytes(o, nrhs, fp32);
  if (need > kNoAllocScratchBytes)
    fail(BEMBEL_EINVAL, "matvec_noalloc: this operator and nrhs need " + std::to_string(need) +
                            " bytes of scratch; the fixed buffer holds " + std::to_string(kNoAllocScratchBytes) +
                            " bytes (use bembel_matvec)");
  if (fp32 && !o.d_N32) fail(BEMBEL_EINVAL, "FP32 matvec needs an operator assembled with precision MIXED");
  // every scratch element is written before it is read, so nothing is cleared
  void* scratch = noalloc_scratch_address();
  struct NoAlloc {
    NoAlloc() { t_no_alloc = true; }
    ~NoAlloc() { t_no_alloc = false; }
  } no_alloc_scope;
  if (fp32)
    matvec_impl<float>(o, static_cast<const float*>(x), static_cast<float*>(y), nrhs, s, o.d_K32, o.d_N32, o.d_V32,
                       o.d_T32, scratch);
  else
    matvec_impl<double>(o, static_cast<const double*>(x), static_cast<double*>(y), nrhs, s, o.d_K, o.d_N, o.d_V,
                        o.d_T, scratch);
}

namespace {
template <typename T>
void precond_impl(const Op& o, const T* x, T* y, int nrhs, cudaStream_t s, const T* Dinv) {
  const int C = o.cplx ? 2 : 1;
  const int ncol = nrhs * C;
  T* xl = static_cast<T*>(o.d_scratch);
  T* yl = xl + o.nlocal * ncol;
  gather_l<T>(o, x, xl, ncol, C, s);
  const bool learned = o.active_precond == BEMBEL_PRECOND_LEARNED && o.d_lw;
  if (learned) learned_scale_local(o, xl, nrhs, sizeof(T) == 4, s);
  cuda_check(cudaMemsetAsync(yl, 0, sizeof(T) * o.nlocal * ncol, s), "yl clear");
  if (o.cplx)
    launch_bsr<T, true, false>(o.d_leaf_ids, o.d_leaf_ids, o.nleaf, Dinv, nullptr, 0.f, 0.f, xl, yl, o.nld, nrhs, s, o.bsr_chunk);
  else
    launch_bsr<T, false, false>(o.d_leaf_ids, o.d_leaf_ids, o.nleaf, Dinv, nullptr, 0.f, 0.f, xl, yl, o.nld, nrhs, s, o.bsr_chunk);
  if (learned) learned_scale_local(o, yl, nrhs, sizeof(T) == 4, s);
  scatter_l<T>(o, yl, y, ncol, C, s);
  if (o.active_precond == BEMBEL_PRECOND_TWO_LEVEL || o.active_precond == BEMBEL_PRECOND_LEARNED)
    coarse_apply_add(o, x, y, nrhs, sizeof(T) == 4, s);
}
}  // namespace

void local_gather(const Op& o, const void* x, void* xl, int nrhs, bool fp32, cudaStream_t s) {
  const int C = o.cplx ? 2 : 1;
  const int ncol = nrhs * C;
  if (fp32)
    gather_l<float>(o, static_cast<const float*>(x), static_cast<float*>(xl), ncol, C, s);
  else
    gather_l<double>(o, static_cast<const double*>(x), static_cast<double*>(xl), ncol, C, s);
}

void local_scatter(const Op& o, const void* yl, void* y, int nrhs, bool fp32, cudaStream_t s) {
  const int C = o.cplx ? 2 : 1;
  const int ncol = nrhs * C;
  if (fp32)
    scatter_l<float>(o, static_cast<const float*>(yl), static_cast<float*>(y), ncol, C, s);
  else
    scatter_l<double>(o, static_cast<const double*>(yl), static_cast<double*>(y), ncol, C, s);
}

void blockdiag_apply(const Op& o, const void* Dinv, const void* xl, void* yl, int nrhs, bool fp32, cudaStream_t s) {
  const int C = o.cplx ? 2 : 1;
  const size_t el = fp32 ? sizeof(float) : sizeof(double);
  cuda_check(cudaMemsetAsync(yl, 0, el * o.nlocal * nrhs * C, s), "yl clear");
  if (fp32) {
    if (o.cplx)
      launch_bsr<float, true, false>(o.d_leaf_ids, o.d_leaf_ids, o.nleaf, static_cast<const float*>(Dinv), nullptr,
                                     0.f, 0.f, static_cast<const float*>(xl), static_cast<float*>(yl), o.nld, nrhs, s,
                                     o.bsr_chunk);
    else
      launch_bsr<float, false, false>(o.d_leaf_ids, o.d_leaf_ids, o.nleaf, static_cast<const float*>(Dinv), nullptr,
                                      0.f, 0.f, static_cast<const float*>(xl), static_cast<float*>(yl), o.nld, nrhs,
                                      s, o.bsr_chunk);
  } else {
    if (o.cplx)
      launch_bsr<double, true, false>(o.d_leaf_ids, o.d_leaf_ids, o.nleaf, static_cast<const double*>(Dinv),
                                      nullptr, 0.f, 0.f, static_cast<const double*>(xl), static_cast<double*>(yl),
                                      o.nld, nrhs, s, o.bsr_chunk);
    else
      launch_bsr<double, false, false>(o.d_leaf_ids, o.d_leaf_ids, o.nleaf, static_cast<const double*>(Dinv),
                                       nullptr, 0.f, 0.f, static_cast<const double*>(xl), static_cast<double*>(yl),
                                       o.nld, nrhs, s, o.bsr_chunk);
  }
}

void precond_apply(const Op& o, const void* x, void* y, int nrhs, bool fp32, cudaStream_t s) {
  if (!o.d_bj) fail(BEMBEL_EINVAL, "block-Jacobi preconditioner not set up");
  ensure_scratch(const_cast<Op&>(o), matvec_scratch_bytes(o, nrhs, fp32));
  if (fp32)
    precond_impl<float>(o, static_cast<const float*>(x), static_cast<float*>(y), nrhs, s, o.d_bj32);
  else
    precond_impl<double>(o, static_cast<const double*>(x), static_cast<double*>(y), nrhs, s, o.d_bj);
}

void ensure_dofmajor(Op& o, size_t bytes) {
  if (bytes <= o.dofmajor_bytes) return;
  if (capturing()) fail(BEMBEL_ECUDA, "dof-major buffer must be reserved before graph capture");
  if (o.d_dofmajor) {
    cuda_check(cudaStreamSynchronize(o.stream), "dof-major sync");
    dev_free(o.d_dofmajor);
  }
  o.d_dofmajor = dev_alloc(bytes);
  o.dofmajor_bytes = bytes;
}

void ensure_scratch(Op& o, size_t bytes) {
  if (bytes <= o.scratch_bytes) return;
  // a captured graph keeps the scratch address: growing it under capture
  // would leave earlier graphs pointing at freed memory
  if (capturing()) fail(BEMBEL_ECUDA, "matvec scratch must be reserved before graph capture");
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
