// coarse.cu - coarse-space correction of the two-level preconditioner.
//
// Not in the paper (which solves without a preconditioner); it extends the solver's
// block-Jacobi fallback.  The S^2 spaces of one degree on the dyadic levels are nested
// (App. E: the fine knot vector contains the coarse one, and the Piola lift is the same
// on every level), so coarse coefficients c give the same function as the fine
// coefficients P c.  Per patch P = R (x) R, with R (n1 x n1c) the 1-D refinement matrix
// from level Lc to level L.  The coarse Galerkin matrix A_c (= P^T A P up to quadrature)
// is assembled directly on level Lc by the dense assembly kernels, inverted once by
// Gauss-Jordan elimination on the device, and the preconditioners add
//     z += P A_c^-1 P^T r
// to their block-Jacobi part: restriction (one block per coarse dof and column), a dense
// product with A_c^-1 (one warp per coarse dof and column) and prolongation (one thread
// per fine dof and column).  The correction removes the smooth error components that a
// block-diagonal preconditioner cannot reach; for Helmholtz these include the modes
// near the interior resonances.
#include <cmath>
#include <vector>

#include "op.h"

namespace bembel {

namespace {

inline int nblk(int64_t n, int t) { return int(std::max<int64_t>(1, (n + t - 1) / t)); }

// 1-D refinement matrix R (n1f x n1c) of the open-knot B-splines of degree d from 2^Lc
// to 2^L uniform elements, by collocation at the fine Greville abscissae: the coarse
// spline b^c_a equals sum_i R[i][a] b^f_i exactly, and the fine collocation matrix at
// the Greville points is nonsingular (Schoenberg-Whitney).  Dense Gaussian elimination
// with partial pivoting (n1f <= 1 + 2^10 + 3).
std::vector<double> refinement_matrix(int d, int Lc, int L) {
  const int nelc = 1 << Lc, nelf = 1 << L;
  const int n1c = d + nelc, n1f = d + nelf;
  auto knots = [d](int nel) {
    std::vector<double> k;
    for (int i = 0; i <= d; ++i) k.push_back(0.0);
    for (int i = 1; i < nel; ++i) k.push_back(double(i) / nel);
    for (int i = 0; i <= d; ++i) k.push_back(1.0);
    return k;
  };
  const std::vector<double> kf = knots(nelf), kc = knots(nelc);
  // all B-splines of one knot vector at x (Cox-de Boor, right end point in the last interval)
  auto basis = [d](const std::vector<double>& kn, double x) {
    const int nk = int(kn.size());
    std::vector<double> b(nk - 1, 0.0);
    int last = 0;
    for (int i = 0; i < nk - 1; ++i)
      if (kn[i] < kn[i + 1]) last = i;
    for (int i = 0; i < nk - 1; ++i) b[i] = (kn[i] < kn[i + 1] && x >= kn[i] && x < kn[i + 1]) ? 1.0 : 0.0;
    if (x >= 1.0) {
      std::fill(b.begin(), b.end(), 0.0);
      b[last] = 1.0;
    }
    for (int p = 1; p <= d; ++p)
      for (int i = 0; i < nk - 1 - p; ++i) {
        const double d1 = kn[i + p] - kn[i], d2 = kn[i + p + 1] - kn[i + 1];
        const double t1 = d1 > 0 ? (x - kn[i]) / d1 * b[i] : 0.0;
        const double t2 = d2 > 0 ? (kn[i + p + 1] - x) / d2 * b[i + 1] : 0.0;
        b[i] = t1 + t2;
      }
    b.resize(nk - 1 - d);
    return b;
  };
  // Greville abscissae of the fine space (degree 0: element midpoints)
  std::vector<double> xg(n1f);
  for (int i = 0; i < n1f; ++i) {
    if (d == 0) {
      xg[i] = (i + 0.5) / nelf;
    } else {
      double s = 0.0;
      for (int j = 1; j <= d; ++j) s += kf[i + j];
      xg[i] = s / d;
    }
  }
  // solve Bf R = Bc, Bf (n1f x n1f) at the abscissae, n1c right-hand sides
  const int w = n1f + n1c;
  std::vector<double> M((size_t)n1f * w);
  for (int r = 0; r < n1f; ++r) {
    const std::vector<double> bf = basis(kf, xg[r]), bc = basis(kc, xg[r]);
    for (int j = 0; j < n1f; ++j) M[(size_t)r * w + j] = bf[j];
    for (int a = 0; a < n1c; ++a) M[(size_t)r * w + n1f + a] = bc[a];
  }
  for (int c = 0; c < n1f; ++c) {
    int piv = c;
    for (int r = c + 1; r < n1f; ++r)
      if (std::fabs(M[(size_t)r * w + c]) > std::fabs(M[(size_t)piv * w + c])) piv = r;
    if (M[(size_t)piv * w + c] == 0.0) fail(BEMBEL_EINVAL, "coarse space: singular collocation matrix");
    if (piv != c)
      for (int k = 0; k < w; ++k) std::swap(M[(size_t)c * w + k], M[(size_t)piv * w + k]);
    const double inv = 1.0 / M[(size_t)c * w + c];
    for (int k = c; k < w; ++k) M[(size_t)c * w + k] *= inv;
    for (int r = 0; r < n1f; ++r) {
      if (r == c) continue;
      const double f = M[(size_t)r * w + c];
      if (f == 0.0) continue;
      for (int k = c; k < w; ++k) M[(size_t)r * w + k] -= f * M[(size_t)c * w + k];
    }
  }
  std::vector<double> R((size_t)n1f * n1c);
  for (int i = 0; i < n1f; ++i)
    for (int a = 0; a < n1c; ++a) {
      const double v = M[(size_t)i * w + n1f + a];
      R[(size_t)i * n1c + a] = std::fabs(v) < 1e-14 ? 0.0 : v;  // exact zeros outside the band
    }
  return R;
}

// ---- Gauss-Jordan inversion of W = [A_c | I] (m x 2m, row-major, C components) ----

// Step k, part 1: pivot row (largest modulus in column k at or below k), swap, scale
// row k by the inverse pivot, and keep column k (the elimination factors) in f.
template <bool CPLX>
__global__ void k_gj_pivot(double* __restrict__ W, int m, int k, double* __restrict__ f, int* __restrict__ info) {
  constexpr int C = CPLX ? 2 : 1;
  const int w = 2 * m;
  __shared__ double best[256];
  __shared__ int bidx[256];
  double bm = -1.0;
  int bi = k;
  for (int r = k + threadIdx.x; r < m; r += blockDim.x) {
    const double re = W[((int64_t)r * w + k) * C], im = CPLX ? W[((int64_t)r * w + k) * C + 1] : 0.0;
    const double mag = re * re + im * im;
    if (mag > bm) {
      bm = mag;
      bi = r;
    }
  }
  best[threadIdx.x] = bm;
  bidx[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double o = best[threadIdx.x + s];
      const int oi = bidx[threadIdx.x + s];
      if (o > best[threadIdx.x] || (o == best[threadIdx.x] && oi < bidx[threadIdx.x])) {
        best[threadIdx.x] = o;
        bidx[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const int p = bidx[0];
  const bool singular = !(best[0] > 0.0);
  if (singular && threadIdx.x == 0) *info = 1;
  if (p != k)
    for (int c = k + threadIdx.x; c < w; c += blockDim.x)
      for (int t = 0; t < C; ++t) {
        const double a = W[((int64_t)k * w + c) * C + t];
        W[((int64_t)k * w + c) * C + t] = W[((int64_t)p * w + c) * C + t];
        W[((int64_t)p * w + c) * C + t] = a;
      }
  __syncthreads();
  // inverse pivot (1 for a singular column: the info flag reports it)
  double pr = singular ? 1.0 : W[((int64_t)k * w + k) * C], pi = (CPLX && !singular) ? W[((int64_t)k * w + k) * C + 1] : 0.0;
  const double den = pr * pr + pi * pi;
  const double ir = pr / den, ii = -pi / den;
  __syncthreads();
  for (int c = k + threadIdx.x; c < w; c += blockDim.x) {
    double* v = W + ((int64_t)k * w + c) * C;
    if (CPLX) {
      const double vr = v[0], vi = v[1];
      v[0] = vr * ir - vi * ii;
      v[1] = vr * ii + vi * ir;
    } else {
      v[0] *= ir;
    }
  }
  for (int r = threadIdx.x; r < m; r += blockDim.x)
    for (int t = 0; t < C; ++t) f[(int64_t)r * C + t] = r == k ? 0.0 : W[((int64_t)r * w + k) * C + t];
}

// Step k, part 2: W[r][c] -= f[r] W[k][c] for every row r != k and column c >= k.
template <bool CPLX>
__global__ void k_gj_eliminate(double* __restrict__ W, int m, int k, const double* __restrict__ f) {
  constexpr int C = CPLX ? 2 : 1;
  const int w = 2 * m, nc = w - k;
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= (int64_t)m * nc) return;
  const int r = int(id / nc), c = k + int(id % nc);
  if (r == k) return;
  const double* pk = W + ((int64_t)k * w + c) * C;
  double* v = W + ((int64_t)r * w + c) * C;
  const double fr = f[(int64_t)r * C];
  if (CPLX) {
    const double fi = f[(int64_t)r * C + 1];
    v[0] -= fr * pk[0] - fi * pk[1];
    v[1] -= fr * pk[1] + fi * pk[0];
  } else {
    v[0] -= fr * pk[0];
  }
}

// right half of W into A_c^-1 (FP64 and FP32 copies)
__global__ void k_gj_extract(const double* __restrict__ W, int m, int C, double* __restrict__ inv,
                             float* __restrict__ inv32) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= (int64_t)m * m * C) return;
  const int t = int(id % C);
  const int64_t rc = id / C;
  const int r = int(rc / m), c = int(rc % m);
  const double v = W[((int64_t)r * 2 * m + m + c) * C + t];
  inv[id] = v;
  inv32[id] = float(v);
}

// columns of the dense coarse matrix from A_c e_j: Y[j][i] = (A_c)_ij, into W = [A_c | I]
__global__ void k_gj_load(const double* __restrict__ Y, int m, int j0, int nj, int C, double* __restrict__ W) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= (int64_t)nj * m * C) return;
  const int t = int(id % C);
  const int64_t q = id / C;
  const int j = j0 + int(q / m), i = int(q % m);
  W[((int64_t)i * 2 * m + j) * C + t] = Y[id];
  W[((int64_t)i * 2 * m + m + j) * C + t] = (i == j && t == 0) ? 1.0 : 0.0;
}

// ---- the correction z += P A_c^-1 P^T r ----

// rc[col][pc] = sum_{j, i} R[j][b] R[i][a] x[col][patch, j, i]; one block per (coarse dof, rhs)
template <typename T, int C>
__global__ void k_restrict(const T* __restrict__ x, T* __restrict__ rc, const double* __restrict__ R,
                           const int* __restrict__ rrow, int n1, int n1c, int64_t ndofs, int64_t ncoarse) {
  const int64_t pc = blockIdx.x;
  const int r = blockIdx.y;
  const int per = n1c * n1c;
  const int patch = int(pc / per), a = int(pc % per) % n1c, b = int(pc % per) / n1c;
  const int i0 = rrow[2 * a], i1 = rrow[2 * a + 1], j0 = rrow[2 * b], j1 = rrow[2 * b + 1];
  const int ni = i1 - i0, cnt = ni * (j1 - j0);
  const T* xr = x + ((int64_t)r * ndofs + (int64_t)patch * n1 * n1) * C;
  double acc[C];
  for (int t = 0; t < C; ++t) acc[t] = 0.0;
  for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
    const int i = i0 + q % ni, j = j0 + q / ni;
    const double wgt = R[(int64_t)i * n1c + a] * R[(int64_t)j * n1c + b];
    for (int t = 0; t < C; ++t) acc[t] += wgt * double(xr[((int64_t)j * n1 + i) * C + t]);
  }
  __shared__ double red[C][128];
  for (int t = 0; t < C; ++t) red[t][threadIdx.x] = acc[t];
  __syncthreads();
  for (int s = 64; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int t = 0; t < C; ++t) red[t][threadIdx.x] += red[t][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < C) rc[((int64_t)r * ncoarse + pc) * C + threadIdx.x] = T(red[threadIdx.x][0]);
}

// zc[col][i] = sum_j Ainv[i][j] rc[col][j]; one warp per (coarse dof, rhs)
template <typename T, bool CPLX>
__global__ void k_coarse_mv(const T* __restrict__ Ainv, const T* __restrict__ rc, T* __restrict__ zc, int64_t m,
                            int nrhs) {
  constexpr int C = CPLX ? 2 : 1;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= m * nrhs) return;
  const int64_t i = wid % m;
  const int r = int(wid / m);
  const T* a = Ainv + i * m * C;
  const T* v = rc + (int64_t)r * m * C;
  T sr = 0, si = 0;
  for (int64_t j = lane; j < m; j += 32) {
    if (CPLX) {
      const T ar = a[2 * j], ai = a[2 * j + 1], vr = v[2 * j], vi = v[2 * j + 1];
      sr += ar * vr - ai * vi;
      si += ar * vi + ai * vr;
    } else {
      sr += a[j] * v[j];
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    if (CPLX) si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  if (lane == 0) {
    zc[((int64_t)r * m + i) * C] = sr;
    if (CPLX) zc[((int64_t)r * m + i) * C + 1] = si;
  }
}

// y[col][patch, j, i] += sum_{b, a} R[j][b] R[i][a] zc[col][patch, b, a]; one thread per fine dof and rhs
template <typename T, int C>
__global__ void k_prolong_add(const T* __restrict__ zc, T* __restrict__ y, const double* __restrict__ R,
                              const int* __restrict__ rcol, int n1, int n1c, int64_t ndofs, int64_t ncoarse,
                              int nrhs) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= ndofs * nrhs) return;
  const int64_t g = id % ndofs;
  const int r = int(id / ndofs);
  const int per = n1 * n1;
  const int patch = int(g / per), i = int(g % per) % n1, j = int(g % per) / n1;
  const T* zr = zc + ((int64_t)r * ncoarse + (int64_t)patch * n1c * n1c) * C;
  double acc[C];
  for (int t = 0; t < C; ++t) acc[t] = 0.0;
  for (int b = rcol[2 * j]; b < rcol[2 * j + 1]; ++b) {
    const double wb = R[(int64_t)j * n1c + b];
    for (int a = rcol[2 * i]; a < rcol[2 * i + 1]; ++a) {
      const double wgt = wb * R[(int64_t)i * n1c + a];
      for (int t = 0; t < C; ++t) acc[t] += wgt * double(zr[((int64_t)b * n1c + a) * C + t]);
    }
  }
  T* yr = y + ((int64_t)r * ndofs + g) * C;
  for (int t = 0; t < C; ++t) yr[t] += T(acc[t]);
}

template <typename T>
void apply_impl(const Op& o, const T* x, T* y, int nrhs, cudaStream_t s, const T* Ainv) {
  const int64_t m = o.ncoarse;
  T* rc = static_cast<T*>(o.d_cbuf);
  T* zc = rc + m * nrhs * (o.cplx ? 2 : 1);
  const dim3 grid{unsigned(m), unsigned(nrhs), 1u};
  if (o.cplx)
    k_restrict<T, 2><<<grid, 128, 0, s>>>(x, rc, o.d_R, o.d_rrow, o.n1, o.n1c, o.ndofs, m);
  else
    k_restrict<T, 1><<<grid, 128, 0, s>>>(x, rc, o.d_R, o.d_rrow, o.n1, o.n1c, o.ndofs, m);
  launched("k_restrict");
  const int64_t warps = m * nrhs;
  if (o.cplx)
    k_coarse_mv<T, true><<<nblk(warps * 32, 256), 256, 0, s>>>(Ainv, rc, zc, m, nrhs);
  else
    k_coarse_mv<T, false><<<nblk(warps * 32, 256), 256, 0, s>>>(Ainv, rc, zc, m, nrhs);
  launched("k_coarse_mv");
  if (o.cplx)
    k_prolong_add<T, 2><<<nblk(o.ndofs * nrhs, 256), 256, 0, s>>>(zc, y, o.d_R, o.d_rcol, o.n1, o.n1c, o.ndofs, m,
                                                                   nrhs);
  else
    k_prolong_add<T, 1><<<nblk(o.ndofs * nrhs, 256), 256, 0, s>>>(zc, y, o.d_R, o.d_rcol, o.n1, o.n1c, o.ndofs, m,
                                                                   nrhs);
  launched("k_prolong_add");
}

}  // namespace

// Level of the coarse space: the operator's coarse_level option, or L - 3 (at least 0).
static int coarse_level_of(const Op& o) {
  const int c = o.opts.coarse_level > 0 ? o.opts.coarse_level : std::max(0, o.L - 3);
  return std::min(c, o.L);
}

void coarse_setup(Op& o, int nrhs) {
  if (o.efie) fail(BEMBEL_EUNSUPPORTED, "two-level preconditioner: S^2 operators only");
  if (o.rep != 1) fail(BEMBEL_EUNSUPPORTED, "two-level preconditioner: knot_repetition 1 only");
  const int C = o.cplx ? 2 : 1;
  if (!o.d_cinv) {
    const int Lc = coarse_level_of(o);
    const int n1c = o.d + (1 << Lc);
    const int64_t m = int64_t(6) * n1c * n1c;
    if (m > 8192) fail(BEMBEL_EINVAL, "two-level preconditioner: coarse space above 8192 dofs");
    // refinement matrix and its band (first and end nonzero per row and per column)
    const std::vector<double> R = refinement_matrix(o.d, Lc, o.L);
    std::vector<int> rcol(2 * o.n1), rrow(2 * n1c);
    for (int i = 0; i < o.n1; ++i) {
      int lo = n1c, hi = 0;
      for (int a = 0; a < n1c; ++a)
        if (R[(size_t)i * n1c + a] != 0.0) {
          lo = std::min(lo, a);
          hi = a + 1;
        }
      rcol[2 * i] = std::min(lo, hi);
      rcol[2 * i + 1] = hi;
    }
    for (int a = 0; a < n1c; ++a) {
      int lo = o.n1, hi = 0;
      for (int i = 0; i < o.n1; ++i)
        if (R[(size_t)i * n1c + a] != 0.0) {
          lo = std::min(lo, i);
          hi = i + 1;
        }
      rrow[2 * a] = std::min(lo, hi);
      rrow[2 * a + 1] = hi;
    }
    // the dense coarse Galerkin matrix, column by column from A_c e_j
    Op* c = assemble_level(o, Lc);
    double* W = nullptr;
    double* f = nullptr;
    int* info = nullptr;
    double *X = nullptr, *Y = nullptr;
    try {
      if (c->ndofs != m) fail(BEMBEL_EINVAL, "two-level preconditioner: coarse dof count");
      const int nb = int(std::min<int64_t>(m, 64));
      W = static_cast<double*>(dev_alloc(sizeof(double) * m * 2 * m * C));
      f = static_cast<double*>(dev_alloc(sizeof(double) * m * C));
      info = static_cast<int*>(dev_alloc(sizeof(int)));
      X = static_cast<double*>(dev_alloc(sizeof(double) * m * nb * C));
      Y = static_cast<double*>(dev_alloc(sizeof(double) * m * nb * C));
      cuda_check(cudaMemsetAsync(info, 0, sizeof(int), o.stream), "gj info");
      for (int64_t j0 = 0; j0 < m; j0 += nb) {
        const int nj = int(std::min<int64_t>(nb, m - j0));
        std::vector<double> eye((size_t)m * nj * C, 0.0);
        for (int j = 0; j < nj; ++j) eye[((size_t)j * m + j0 + j) * C] = 1.0;
        cuda_check(cudaMemcpyAsync(X, eye.data(), sizeof(double) * eye.size(), cudaMemcpyHostToDevice, o.stream),
                   "coarse identity");
        matvec_device(*c, X, Y, nj, false, o.stream);
        k_gj_load<<<nblk(int64_t(nj) * m * C, 256), 256, 0, o.stream>>>(Y, int(m), int(j0), nj, C, W);
        launched("k_gj_load");
        cuda_check(cudaStreamSynchronize(o.stream), "coarse columns");  // eye is reused
      }
      for (int k = 0; k < int(m); ++k) {
        if (o.cplx) {
          k_gj_pivot<true><<<1, 256, 0, o.stream>>>(W, int(m), k, f, info);
          k_gj_eliminate<true><<<nblk(m * (2 * m - k), 256), 256, 0, o.stream>>>(W, int(m), k, f);
        } else {
          k_gj_pivot<false><<<1, 256, 0, o.stream>>>(W, int(m), k, f, info);
          k_gj_eliminate<false><<<nblk(m * (2 * m - k), 256), 256, 0, o.stream>>>(W, int(m), k, f);
        }
      }
      launched("k_gj_pivot");
      launched("k_gj_eliminate");
      o.d_cinv = static_cast<double*>(dev_alloc(sizeof(double) * m * m * C));
      o.d_cinv32 = static_cast<float*>(dev_alloc(sizeof(float) * m * m * C));
      k_gj_extract<<<nblk(m * m * C, 256), 256, 0, o.stream>>>(W, int(m), C, o.d_cinv, o.d_cinv32);
      launched("k_gj_extract");
      int h = 0;
      cuda_check(cudaMemcpyAsync(&h, info, sizeof(int), cudaMemcpyDeviceToHost, o.stream), "gj info");
      cuda_check(cudaStreamSynchronize(o.stream), "coarse inverse");
      if (h) fail(BEMBEL_EINVAL, "two-level preconditioner: the coarse matrix is singular");
    } catch (...) {
      for (void* p : {(void*)W, (void*)f, (void*)info, (void*)X, (void*)Y}) dev_free(p);
      destroy_op(c);
      throw;
    }
    for (void* p : {(void*)W, (void*)f, (void*)info, (void*)X, (void*)Y}) dev_free(p);
    destroy_op(c);
    o.d_R = static_cast<double*>(dev_alloc(sizeof(double) * R.size()));
    o.d_rcol = static_cast<int*>(dev_alloc(sizeof(int) * rcol.size()));
    o.d_rrow = static_cast<int*>(dev_alloc(sizeof(int) * rrow.size()));
    cuda_check(cudaMemcpy(o.d_R, R.data(), sizeof(double) * R.size(), cudaMemcpyHostToDevice), "R");
    cuda_check(cudaMemcpy(o.d_rcol, rcol.data(), sizeof(int) * rcol.size(), cudaMemcpyHostToDevice), "R cols");
    cuda_check(cudaMemcpy(o.d_rrow, rrow.data(), sizeof(int) * rrow.size(), cudaMemcpyHostToDevice), "R rows");
    o.coarse_level = Lc;
    o.n1c = n1c;
    o.ncoarse = m;
  }
  const size_t need = sizeof(double) * 2 * o.ncoarse * nrhs * C;
  if (need > o.cbuf_bytes) {
    if (capturing()) fail(BEMBEL_ECUDA, "coarse buffers must be reserved before graph capture");
    if (o.d_cbuf) {
      cuda_check(cudaStreamSynchronize(o.stream), "coarse buffer sync");
      dev_free(o.d_cbuf);
    }
    o.d_cbuf = dev_alloc(need);
    o.cbuf_bytes = need;
  }
}

void coarse_apply_add(const Op& o, const void* x, void* y, int nrhs, bool fp32, cudaStream_t s) {
  if (!o.d_cinv) fail(BEMBEL_EINVAL, "two-level preconditioner not set up");
  const size_t el = fp32 ? sizeof(float) : sizeof(double);
  if (el * 2 * o.ncoarse * nrhs * (o.cplx ? 2 : 1) > o.cbuf_bytes)
    fail(BEMBEL_EINVAL, "two-level preconditioner: coarse buffers set up for fewer columns");
  if (fp32)
    apply_impl<float>(o, static_cast<const float*>(x), static_cast<float*>(y), nrhs, s, o.d_cinv32);
  else
    apply_impl<double>(o, static_cast<const double*>(x), static_cast<double*>(y), nrhs, s, o.d_cinv);
}

}  // namespace bembel
