// solve.cu - restarted GMRES (Sec. 4.6) on the device.
//
// GMRES(m) runs nrhs independent systems side by side: one (preconditioned)
// matvec per Arnoldi step for all columns, classical Gram-Schmidt applied
// twice (CGS2), and the Givens update of the (m+1) x m Hessenberg
// least-squares problem, all on the device.  One Arnoldi step is captured once
// in a CUDA graph and replayed; the kernels read the step index from device
// memory, so the same graph serves every step.  The host only reads the
// residual estimates, one step behind (two graph copies write to alternate
// pinned buffers), so it never waits for the step it just launched.
// FP64 operators solve in FP64.  MIXED operators run FP32 Krylov vectors and
// FP32 matvecs inside FP64 iterative refinement (r = b - A x with the FP64
// matvec, x += correction), which restores FP64 residual accuracy.
// Preconditioning (block-Jacobi) is applied from the right: A M^-1 u = b,
// x = M^-1 u.
#include <chrono>
#include <cmath>
#include <vector>

#include "op.h"

namespace bembel {

namespace {

// max that treats a NaN residual as the worst possible (std::max would drop it)
inline double worse(double a, double b) { return std::isnan(b) ? HUGE_VAL : (b > a ? b : a); }

inline int nblk(int64_t n, int t) { return int(std::max<int64_t>(1, std::min<int64_t>((n + t - 1) / t, 65535 * 16))); }

struct cd_t {
  double r, i;
};
__device__ __forceinline__ cd_t cmul(cd_t a, cd_t b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ __forceinline__ cd_t cconj(cd_t a) { return {a.r, -a.i}; }
__device__ __forceinline__ cd_t cadd(cd_t a, cd_t b) { return {a.r + b.r, a.i + b.i}; }
__device__ __forceinline__ cd_t csub(cd_t a, cd_t b) { return {a.r - b.r, a.i - b.i}; }
__device__ __forceinline__ double cabs2(cd_t a) { return a.r * a.r + a.i * a.i; }
__device__ __forceinline__ cd_t cdiv(cd_t a, cd_t b) {
  const double d = cabs2(b);
  return {(a.r * b.r + a.i * b.i) / d, (a.i * b.r - a.r * b.i) / d};
}

// Device state of one GMRES cycle (all complex values as {re, im} pairs).
struct Gm {
  int m, nrhs;
  cd_t* H;       // [nrhs][m+1][m]
  cd_t* cs;      // [nrhs][m]
  cd_t* sn;      // [nrhs][m]
  cd_t* g;       // [nrhs][m+1]
  cd_t* h1;      // [m+1][nrhs] first Gram-Schmidt coefficients of the step
  cd_t* h2;      // [m+1][nrhs] second pass
  cd_t* hn;      // [nrhs] squared norm (real part) of the orthogonalised vector
  cd_t* y;       // [m+1][nrhs] least-squares solution
  double* bn;    // [nrhs] reference norm of the column
  double* alpha; // [nrhs] scale of the next basis vector
  double* stat;  // [2][nrhs]: residual estimate, active flag
  int* jend;     // [nrhs]
  int* j;        // current step
  int* ctr;      // completion counter of k_givens
};

// h[i][r] = sum_n conj(V_i[n, r]) w[n, r] for i < nv, nv = *dj + 1 (or nv_fixed)
template <typename T, bool CPLX>
__global__ void k_dots(const T* __restrict__ V, int64_t vstride, const int* __restrict__ dj, int nv_fixed,
                       const T* __restrict__ w, int64_t n, int nrhs, cd_t* __restrict__ h) {
  const int pair = blockIdx.x;
  const int i = pair / nrhs, r = pair % nrhs;
  const int nv = dj ? *dj + 1 : nv_fixed;
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
    h[pair] = {a, b};
  }
}

// h[i][r] += sum_n conj(V_i[n, r]) w[n, r] for i < *dj + 1.  Grid (blocks
// along n, nrhs, groups of 8 basis vectors): every group runs at once; each
// thread reads w once per group, sums are reduced per block and added
// atomically (h cleared before the launch).  Groups at or beyond *dj + 1 exit.
template <typename T, bool CPLX>
__global__ void __launch_bounds__(256) k_mdots(const T* __restrict__ V, int64_t vstride, const int* __restrict__ dj,
                                               const T* __restrict__ w, int64_t n, int nrhs, cd_t* __restrict__ h) {
  constexpr int G = 8;
  const int r = blockIdx.y;
  const int nv = *dj + 1;
  const int i0 = blockIdx.z * G;
  if (i0 >= nv) return;
  const int C = CPLX ? 2 : 1;
  __shared__ double red[G][2][8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double sr[G], si[G];
#pragma unroll
  for (int g = 0; g < G; ++g) sr[g] = si[g] = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const T* wk = w + ((int64_t)r * n + k) * C;
    const double wr = wk[0], wi = CPLX ? (double)wk[1] : 0.0;
#pragma unroll
    for (int g = 0; g < G; ++g) {
      if (i0 + g < nv) {
        const T* v = V + (int64_t)(i0 + g) * vstride + ((int64_t)r * n + k) * C;
        const double vr = v[0], vi = CPLX ? (double)v[1] : 0.0;
        sr[g] += vr * wr + vi * wi;
        if (CPLX) si[g] += vr * wi - vi * wr;
      }
    }
  }
#pragma unroll
  for (int g = 0; g < G; ++g) {
    for (int o = 16; o > 0; o >>= 1) {
      sr[g] += __shfl_xor_sync(0xffffffffu, sr[g], o);
      if (CPLX) si[g] += __shfl_xor_sync(0xffffffffu, si[g], o);
    }
    if (lane == 0) {
      red[g][0][warp] = sr[g];
      red[g][1][warp] = si[g];
    }
  }
  __syncthreads();
  if (threadIdx.x < G && i0 + (int)threadIdx.x < nv) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a += red[threadIdx.x][0][k];
      b += red[threadIdx.x][1][k];
    }
    cd_t* hp = h + (i0 + threadIdx.x) * nrhs + r;
    atomicAdd(&hp->r, a);
    if (CPLX) atomicAdd(&hp->i, b);
  }
}

// hn[r].r += sum_n |w[n, r]|^2: grid (blocks along n, nrhs), block sums added
// atomically (hn cleared before the launch).
template <typename T, bool CPLX>
__global__ void __launch_bounds__(256) k_norm2(const T* __restrict__ w, int64_t n, cd_t* __restrict__ hn) {
  const int r = blockIdx.y;
  const int C = CPLX ? 2 : 1;
  double s = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n * C; k += (int64_t)gridDim.x * blockDim.x) {
    const double v = w[(int64_t)r * n * C + k];
    s += v * v;
  }
  __shared__ double red[8];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) a += red[k];
    atomicAdd(&hn[r].r, a);
  }
}

// w[n, r] -= sum_{i <= *dj} V_i[n, r] h[i][r]
template <typename T, bool CPLX>
__global__ void k_orth(const T* __restrict__ V, int64_t vstride, const int* __restrict__ dj, T* __restrict__ w,
                       int64_t n, int nrhs, const cd_t* __restrict__ h) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= n * nrhs) return;
  const int r = int(id / n);
  const int64_t k = id % n;
  const int C = CPLX ? 2 : 1;
  const int nv = *dj + 1;
  double ar = CPLX ? (double)w[(r * n + k) * 2] : (double)w[r * n + k];
  double ai = CPLX ? (double)w[(r * n + k) * 2 + 1] : 0.0;
  for (int i = 0; i < nv; ++i) {
    const T* v = V + (int64_t)i * vstride + ((int64_t)r * n + k) * C;
    const cd_t c = h[i * nrhs + r];
    if (CPLX) {
      ar -= c.r * (double)v[0] - c.i * (double)v[1];
      ai -= c.r * (double)v[1] + c.i * (double)v[0];
    } else {
      ar -= c.r * (double)v[0];
    }
  }
  if (CPLX) {
    w[(r * n + k) * 2] = T(ar);
    w[(r * n + k) * 2 + 1] = T(ai);
  } else {
    w[r * n + k] = T(ar);
  }
}

// Givens update of step j = *dj, one block (one warp) per column: the new
// Hessenberg column and the previous rotations are staged in shared memory by
// all lanes, lane 0 applies the rotations, lanes write the column back.  The
// last block to finish advances *dj (grid-wide completion counter).
__global__ void k_givens(Gm st, double tol, int* __restrict__ done_ctr) {
  extern __shared__ cd_t gsh[];
  const int r = blockIdx.x;
  const int lane = threadIdx.x;
  const int j = *st.j;
  const int m = st.m, nrhs = st.nrhs;
  cd_t* col = gsh;           // m + 1
  cd_t* csv = gsh + m + 1;   // m
  cd_t* snv = csv + m;       // m
  const double hn = sqrt(fmax(0.0, st.hn[r].r));
  if (lane == 0) st.alpha[r] = hn > 0.0 ? 1.0 / hn : 0.0;
  const bool active = st.stat[nrhs + r] != 0.0 && j < m;
  if (active) {
    cd_t* H = st.H + (size_t)r * (m + 1) * m;
    const cd_t* cs = st.cs + (size_t)r * m;
    const cd_t* sn = st.sn + (size_t)r * m;
    for (int i = lane; i <= j; i += blockDim.x) {
      col[i] = cadd(st.h1[i * nrhs + r], st.h2[i * nrhs + r]);
      if (i < j) {
        csv[i] = cs[i];
        snv[i] = sn[i];
      }
    }
    __syncwarp();
    if (lane == 0) {
      col[j + 1] = {hn, 0.0};
      for (int i = 0; i < j; ++i) {
        const cd_t a = col[i], b = col[i + 1];
        col[i] = cadd(cmul(csv[i], a), cmul(snv[i], b));
        col[i + 1] = csub(cmul(csv[i], b), cmul(cconj(snv[i]), a));
      }
      const cd_t a = col[j], b = col[j + 1];
      const double den = sqrt(cabs2(a) + cabs2(b));
      cd_t c, sg;
      if (den == 0.0) {
        c = {1.0, 0.0};
        sg = {0.0, 0.0};
      } else if (cabs2(a) == 0.0) {
        c = {0.0, 0.0};
        const double bb = sqrt(cabs2(b));
        sg = {b.r / bb, -b.i / bb};
      } else {
        const double aa = sqrt(cabs2(a));
        c = {aa / den, 0.0};
        const cd_t ph = {a.r / aa, a.i / aa};
        sg = cmul(ph, {b.r / den, -b.i / den});
      }
      st.cs[(size_t)r * m + j] = c;
      st.sn[(size_t)r * m + j] = sg;
      col[j] = cadd(cmul(c, a), cmul(sg, b));
      col[j + 1] = {0.0, 0.0};
      cd_t* g = st.g + (size_t)r * (m + 1);
      const cd_t gj = g[j];
      g[j + 1] = {-(sg.r * gj.r + sg.i * gj.i), -(sg.r * gj.i - sg.i * gj.r)};  // -conj(s) g_j
      g[j] = cmul(c, gj);
      st.jend[r] = j + 1;
      const double res = sqrt(cabs2(g[j + 1])) / st.bn[r];
      st.stat[r] = res;
      if (res <= tol || hn == 0.0) st.stat[nrhs + r] = 0.0;
    }
    __syncwarp();
    for (int i = lane; i <= j + 1; i += blockDim.x) H[i * m + j] = col[i];
  }
  __syncwarp();
  if (lane == 0) {
    __threadfence();
    const int prev = atomicAdd(done_ctr, 1);
    if (prev == (int)gridDim.x - 1) {
      *st.j = j + 1;
      *done_ctr = 0;
      __threadfence();
    }
  }
}

// V_{*dj}[n, r] = alpha_r * w[n, r]   (after k_givens advanced *dj)
template <typename T>
__global__ void k_scale_next(const T* __restrict__ w, T* __restrict__ V, int64_t vstride, const int* __restrict__ dj,
                             int64_t nper, int nrhs, const double* __restrict__ alpha, int m) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= nper * nrhs) return;
  const int j = min(*dj, m);
  V[(int64_t)j * vstride + id] = T(alpha[id / nper] * (double)w[id]);
}

template <typename T>
__global__ void k_copy_vj(const T* __restrict__ V, int64_t vstride, const int* __restrict__ dj, T* __restrict__ out,
                          int64_t n, int m) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= n) return;
  out[id] = V[(int64_t)min(*dj, m) * vstride + id];
}

// y = R^{-1} g per column (R: upper triangle of the rotated H, size jend).
__global__ void k_backsolve(Gm st) {
  const int r = threadIdx.x;
  if (r >= st.nrhs) return;
  const int m = st.m, nrhs = st.nrhs, k = st.jend[r];
  const cd_t* H = st.H + (size_t)r * (m + 1) * m;
  const cd_t* g = st.g + (size_t)r * (m + 1);
  for (int i = m; i >= 0; --i) {
    if (i >= k) {
      st.y[i * nrhs + r] = {0.0, 0.0};
      continue;
    }
    cd_t acc = g[i];
    for (int l = i + 1; l < k; ++l) acc = csub(acc, cmul(H[i * m + l], st.y[l * nrhs + r]));
    st.y[i * nrhs + r] = cdiv(acc, H[i * m + i]);
  }
}

// z[n, r] = sum_{i < jend[r]} V_i[n, r] y[i][r]   (FP64 output).  Only the
// basis vectors built in this cycle enter: later columns hold stale memory
// (y is zero there, but 0 * NaN is not).
template <typename T, bool CPLX>
__global__ void k_combine(const T* __restrict__ V, int64_t vstride, int nv, double* __restrict__ z, int64_t n,
                          int nrhs, const cd_t* __restrict__ y, const int* __restrict__ jend) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= n * nrhs) return;
  const int r = int(id / n);
  const int64_t k = id % n;
  const int C = CPLX ? 2 : 1;
  double ar = 0.0, ai = 0.0;
  const int nvr = min(nv, jend[r]);
  for (int i = 0; i < nvr; ++i) {
    const T* v = V + (int64_t)i * vstride + ((int64_t)r * n + k) * C;
    const cd_t c = y[i * nrhs + r];
    if (CPLX) {
      ar += c.r * (double)v[0] - c.i * (double)v[1];
      ai += c.r * (double)v[1] + c.i * (double)v[0];
    } else {
      ar += c.r * (double)v[0];
    }
  }
  if (CPLX) {
    z[(r * n + k) * 2] = ar;
    z[(r * n + k) * 2 + 1] = ai;
  } else {
    z[r * n + k] = ar;
  }
}

// V_0 = r / ||r|| (column scale), converting to the basis type
template <typename T>
__global__ void k_scale_first(const double* __restrict__ r, T* __restrict__ V, int64_t nper, int nrhs,
                              const double* __restrict__ alpha) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= nper * nrhs) return;
  V[id] = T(alpha[id / nper] * r[id]);
}

__global__ void k_axpy(double* __restrict__ x, const double* __restrict__ d, int64_t n) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id < n) x[id] += d[id];
}

__global__ void k_sub(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ c, int64_t n) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id < n) c[id] = a[id] - b[id];
}

struct HostBuf {
  void* p = nullptr;
  explicit HostBuf(size_t bytes) { cuda_check(cudaMallocHost(&p, bytes), "cudaMallocHost"); }
  ~HostBuf() {
    if (p) cudaFreeHost(p);
  }
};

struct StreamGuard {
  cudaStream_t s = nullptr;
  StreamGuard() { cuda_check(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream create"); }
  ~StreamGuard() {
    if (s) cudaStreamDestroy(s);
  }
};

// Column norms ||x_r|| (FP64 result on the host, synchronises the stream).
template <bool CPLX>
void col_norms(const double* x, int64_t n, int nrhs, cd_t* d_h, std::vector<double>& out, cudaStream_t s) {
  k_dots<double, CPLX><<<nrhs, 256, 0, s>>>(x, 0, nullptr, 1, x, n, nrhs, d_h);
  launched("k_dots");
  std::vector<cd_t> h(nrhs);
  cuda_check(cudaMemcpyAsync(h.data(), d_h, sizeof(cd_t) * nrhs, cudaMemcpyDeviceToHost, s), "norm copy");
  cuda_check(cudaStreamSynchronize(s), "norm sync");
  out.resize(nrhs);
  // a NaN stays NaN (std::max(0, NaN) would return 0 and hide it)
  for (int r = 0; r < nrhs; ++r) out[r] = std::isnan(h[r].r) ? h[r].r : std::sqrt(std::max(0.0, h[r].r));
}

// One GMRES(m) solve of A x = b from x0 = 0 on stream s.  b, x: FP64 blocks
// (n x nrhs).  T = type of the Krylov basis and of the matvec (float for the
// inner solves of the mixed-precision form).  Returns Arnoldi steps taken.
template <typename T, bool CPLX>
int gmres_run(const Op& o, const double* b, double* x, int nrhs, double tol, int restart, int max_iter, bool prec,
              std::vector<double>& relres, cudaStream_t s) {
  const bool fp32 = sizeof(T) == 4;
  const int C = CPLX ? 2 : 1;
  const int64_t n = o.ndofs;
  const int64_t vstride = n * nrhs * C;
  const int m = restart;
  const int tb = 256;
  // FP64 bytes cover the FP32 products too; reserved before the graphs capture the address
  ensure_scratch(const_cast<Op&>(o), matvec_scratch_bytes(o, nrhs, false));
  if (fp32) tc_prepare(const_cast<Op&>(o), nrhs);  // tensor-core groups, if used, before capture
  if (fp32) coupling_f32_prepare(const_cast<Op&>(o), nrhs);
  // dof-major staging for wide products (the FP64 restart residuals need the larger size)
  if (!o.d_e_ptr && nrhs * C >= 32) ensure_dofmajor(const_cast<Op&>(o), sizeof(double) * (size_t)n * nrhs * C);
  DevBuf Vbuf(sizeof(T) * vstride * (m + 1)), wbuf(sizeof(T) * vstride), zbuf(sizeof(T) * vstride),
      rbuf(sizeof(double) * vstride), ubuf(sizeof(double) * vstride);
  T* V = static_cast<T*>(Vbuf.p);
  T* w = static_cast<T*>(wbuf.p);
  T* z = static_cast<T*>(zbuf.p);
  double* r = static_cast<double*>(rbuf.p);
  double* u = static_cast<double*>(ubuf.p);
  // device state
  const size_t ncd = (size_t)nrhs * ((m + 1) * m + 2 * m + 4 * (m + 1) + 1);
  DevBuf sbuf(sizeof(cd_t) * ncd + sizeof(double) * 4 * nrhs + sizeof(int) * (nrhs + 8));
  Gm st;
  st.m = m;
  st.nrhs = nrhs;
  cd_t* pc = static_cast<cd_t*>(sbuf.p);
  st.H = pc;
  pc += (size_t)nrhs * (m + 1) * m;
  st.cs = pc;
  pc += (size_t)nrhs * m;
  st.sn = pc;
  pc += (size_t)nrhs * m;
  st.g = pc;
  pc += (size_t)nrhs * (m + 1);
  st.h1 = pc;
  pc += (size_t)nrhs * (m + 1);
  st.h2 = pc;
  pc += (size_t)nrhs * (m + 1);
  st.y = pc;
  pc += (size_t)nrhs * (m + 1);
  st.hn = pc;
  pc += nrhs;
  double* pd = reinterpret_cast<double*>(pc);
  st.bn = pd;
  st.alpha = pd + nrhs;
  st.stat = pd + 2 * nrhs;
  int* pi = reinterpret_cast<int*>(pd + 4 * nrhs);
  st.jend = pi;
  st.j = pi + nrhs;
  st.ctr = pi + nrhs + 1;
  HostBuf hstat(sizeof(double) * 4 * nrhs);  // two pinned copies of stat
  double* hs[2] = {static_cast<double*>(hstat.p), static_cast<double*>(hstat.p) + 2 * nrhs};

  // ---- capture one Arnoldi step (two copies, each writing its own pinned buffer) ----
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  struct ExecGuard {
    cudaGraphExec_t* e;
    ~ExecGuard() {
      for (int c = 0; c < 2; ++c)
        if (e[c]) cudaGraphExecDestroy(e[c]);
    }
  } eg{exec};
  long long kernels_per_step = 0;
  // blocks along n for the reductions: about two elements per thread
  const int dots_blocks = int(std::max<int64_t>(1, std::min<int64_t>(256, (n * C + 511) / 512)));
  const int groups = (m + 1 + 7) / 8;
  for (int c = 0; c < 2; ++c) {
    cudaGraph_t graph;
    capture_begin(s);
    k_copy_vj<T><<<nblk(vstride, tb), tb, 0, s>>>(V, vstride, st.j, w, vstride, m);
    launched("k_copy_vj");
    if (prec) precond_apply(o, w, z, nrhs, fp32, s);
    matvec_device(o, prec ? static_cast<const void*>(z) : static_cast<const void*>(w), prec ? w : z, nrhs, fp32, s);
    T* av = prec ? w : z;  // A v_j (or A M^-1 v_j)
    cuda_check(cudaMemsetAsync(st.h1, 0, sizeof(cd_t) * 2 * (m + 1) * nrhs, s), "h clear");  // h1 and h2
    k_mdots<T, CPLX><<<dim3(dots_blocks, nrhs, groups), 256, 0, s>>>(V, vstride, st.j, av, n, nrhs, st.h1);
    launched("k_mdots");
    k_orth<T, CPLX><<<nblk(n * nrhs, tb), tb, 0, s>>>(V, vstride, st.j, av, n, nrhs, st.h1);
    launched("k_orth");
    k_mdots<T, CPLX><<<dim3(dots_blocks, nrhs, groups), 256, 0, s>>>(V, vstride, st.j, av, n, nrhs, st.h2);
    launched("k_mdots");
    k_orth<T, CPLX><<<nblk(n * nrhs, tb), tb, 0, s>>>(V, vstride, st.j, av, n, nrhs, st.h2);
    launched("k_orth");
    cuda_check(cudaMemsetAsync(st.hn, 0, sizeof(cd_t) * nrhs, s), "hn clear");
    k_norm2<T, CPLX><<<dim3(dots_blocks, nrhs), 256, 0, s>>>(av, n, st.hn);
    launched("k_norm2");
    k_givens<<<nrhs, 32, sizeof(cd_t) * (3 * m + 1), s>>>(st, tol, st.ctr);
    launched("k_givens");
    k_scale_next<T><<<nblk(vstride, tb), tb, 0, s>>>(av, V, vstride, st.j, n * C, nrhs, st.alpha, m);
    launched("k_scale_next");
    cuda_check(cudaMemcpyAsync(hs[c], st.stat, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, s), "stat copy");
    kernels_per_step = capture_end(s, &graph);
    cuda_check(cudaGraphInstantiate(&exec[c], graph, 0), "graph instantiate");
    cudaGraphDestroy(graph);
  }
  cudaEvent_t ev[2];
  cuda_check(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming), "event");
  cuda_check(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming), "event");

  cd_t* d_tmp = st.h1;  // scratch for column norms outside the graph
  cuda_check(cudaMemsetAsync(x, 0, sizeof(double) * vstride, s), "x0");
  std::vector<double> bnorm;
  col_norms<CPLX>(b, n, nrhs, d_tmp, bnorm, s);
  relres.assign(nrhs, 0.0);
  std::vector<char> done(nrhs, 0);
  for (int rr = 0; rr < nrhs; ++rr)
    if (bnorm[rr] == 0.0) done[rr] = 1;
  cuda_check(cudaMemcpyAsync(st.bn, bnorm.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s), "bn");
  int iters = 0;
  bool first = true;
  while (iters < max_iter) {
    // true residual r = b - A x
    if (first) {
      cuda_check(cudaMemcpyAsync(r, b, sizeof(double) * vstride, cudaMemcpyDeviceToDevice, s), "r0");
    } else {
      matvec_device(o, x, r, nrhs, false, s);
      k_sub<<<nblk(vstride, tb), tb, 0, s>>>(b, r, r, vstride);
      launched("k_sub");
    }
    first = false;
    std::vector<double> rn;
    col_norms<CPLX>(r, n, nrhs, d_tmp, rn, s);
    bool all = true;
    for (int rr = 0; rr < nrhs; ++rr) {
      relres[rr] = bnorm[rr] > 0 ? rn[rr] / bnorm[rr] : 0.0;
      if (relres[rr] <= tol) done[rr] = 1;
      all = all && done[rr];
    }
    if (all) break;
    // cycle set-up: V_0 = r/||r||, g = (||r||, 0, ...), active flags, step 0
    std::vector<double> alpha(nrhs), stat0(2 * nrhs);
    std::vector<cd_t> g0((size_t)nrhs * (m + 1), cd_t{0.0, 0.0});
    for (int rr = 0; rr < nrhs; ++rr) {
      alpha[rr] = rn[rr] > 0 ? 1.0 / rn[rr] : 0.0;
      g0[(size_t)rr * (m + 1)] = {rn[rr], 0.0};
      stat0[rr] = relres[rr];
      stat0[nrhs + rr] = done[rr] ? 0.0 : 1.0;
    }
    cuda_check(cudaMemcpyAsync(st.alpha, alpha.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s), "alpha");
    cuda_check(cudaMemcpyAsync(st.g, g0.data(), sizeof(cd_t) * g0.size(), cudaMemcpyHostToDevice, s), "g0");
    cuda_check(cudaMemcpyAsync(st.stat, stat0.data(), sizeof(double) * 2 * nrhs, cudaMemcpyHostToDevice, s), "stat");
    cuda_check(cudaMemsetAsync(st.jend, 0, sizeof(int) * (nrhs + 2), s), "jend/j/ctr");
    k_scale_first<T><<<nblk(vstride, tb), tb, 0, s>>>(r, V, n * C, nrhs, st.alpha);
    launched("k_scale_first");
    int steps = 0;
    for (int j = 0; j < m && iters + j < max_iter; ++j) {
      cuda_check(cudaGraphLaunch(exec[j & 1], s), "graph launch");
      note_graph_kernels(kernels_per_step);
      cuda_check(cudaEventRecord(ev[j & 1], s), "event");
      ++steps;
      if (j >= 1) {
        // look at step j-1 while step j runs
        cuda_check(cudaEventSynchronize(ev[(j - 1) & 1]), "step sync");
        const double* hsj = hs[(j - 1) & 1];
        bool any = false;
        for (int rr = 0; rr < nrhs; ++rr) any = any || hsj[nrhs + rr] != 0.0;
        if (!any) break;
      }
    }
    cuda_check(cudaStreamSynchronize(s), "cycle sync");
    iters += steps;
    // x += M^-1 V y
    k_backsolve<<<1, std::max(32, ((nrhs + 31) / 32) * 32), 0, s>>>(st);
    launched("k_backsolve");
    k_combine<T, CPLX><<<nblk(n * nrhs, tb), tb, 0, s>>>(V, vstride, m + 1, u, n, nrhs, st.y, st.jend);
    launched("k_combine");
    if (prec) {
      precond_apply(o, u, r, nrhs, false, s);
      k_axpy<<<nblk(vstride, tb), tb, 0, s>>>(x, r, vstride);
    } else {
      k_axpy<<<nblk(vstride, tb), tb, 0, s>>>(x, u, vstride);
    }
    launched("k_axpy");
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  return iters;
}

}  // namespace

int solve_gmres(const Op& o, const void* bv, void* xv, int nrhs, const bembel_solve_opts& so,
                bembel_solve_info* info) {
  const auto t0 = std::chrono::steady_clock::now();
  StreamGuard sg;  // graphs are captured on a private stream ordered after the operator's
  const cudaStream_t s = sg.s;
  {
    cudaEvent_t e;
    cuda_check(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    cuda_check(cudaEventRecord(e, o.stream), "event");
    cuda_check(cudaStreamWaitEvent(s, e, 0), "wait");
    cudaEventDestroy(e);
  }
  const bool prec = so.precond == BEMBEL_PRECOND_BLOCK_JACOBI || so.precond == BEMBEL_PRECOND_LEARNED ||
                    so.precond == BEMBEL_PRECOND_TWO_LEVEL;
  if (prec) precond_setup(const_cast<Op&>(o));
  if (so.precond == BEMBEL_PRECOND_TWO_LEVEL || so.precond == BEMBEL_PRECOND_LEARNED)
    coarse_setup(const_cast<Op&>(o), nrhs);
  if (so.precond == BEMBEL_PRECOND_LEARNED && !o.d_lw)
    fail(BEMBEL_EINVAL, "solve: the learned preconditioner needs bembel_learned_attach first");
  const_cast<Op&>(o).active_precond = so.precond;
  const double* b = static_cast<const double*>(bv);
  double* x = static_cast<double*>(xv);
  const int C = o.cplx ? 2 : 1;
  const int64_t vn = o.ndofs * nrhs * C;
  std::vector<double> relres;
  int iters = 0, refinements = 0;
  const bool mixed = o.opts.precision == BEMBEL_PREC_MIXED && so.refine;
  if (!mixed) {
    iters = o.cplx ? gmres_run<double, true>(o, b, x, nrhs, so.tol, so.restart, so.max_iter, prec, relres, s)
                   : gmres_run<double, false>(o, b, x, nrhs, so.tol, so.restart, so.max_iter, prec, relres, s);
  } else {
    DevBuf rbuf(sizeof(double) * vn), dbuf(sizeof(double) * vn), hbuf(sizeof(cd_t) * nrhs);
    double* r = static_cast<double*>(rbuf.p);
    double* dx = static_cast<double*>(dbuf.p);
    cd_t* dh = static_cast<cd_t*>(hbuf.p);
    cuda_check(cudaMemsetAsync(x, 0, sizeof(double) * vn, s), "x0");
    std::vector<double> bn, rn;
    if (o.cplx)
      col_norms<true>(b, o.ndofs, nrhs, dh, bn, s);
    else
      col_norms<false>(b, o.ndofs, nrhs, dh, bn, s);
    relres.assign(nrhs, 1.0);
    for (int outer = 0; outer < 30 && iters < so.max_iter; ++outer) {
      if (outer == 0) {
        cuda_check(cudaMemcpyAsync(r, b, sizeof(double) * vn, cudaMemcpyDeviceToDevice, s), "r");
      } else {
        matvec_device(o, x, r, nrhs, false, s);
        k_sub<<<nblk(vn, 256), 256, 0, s>>>(b, r, r, vn);
        launched("k_sub");
      }
      if (o.cplx)
        col_norms<true>(r, o.ndofs, nrhs, dh, rn, s);
      else
        col_norms<false>(r, o.ndofs, nrhs, dh, rn, s);
      double worst = 0.0;
      for (int rr = 0; rr < nrhs; ++rr) {
        relres[rr] = bn[rr] > 0 ? rn[rr] / bn[rr] : 0.0;
        worst = worse(worst, relres[rr]);
      }
      if (worst <= so.tol) break;
      ++refinements;
      // inner tolerance relative to the current residual: what is still
      // missing to reach tol, but not below what FP32 Krylov vectors and FP32
      // operator products resolve on ill-conditioned systems (each refinement
      // step then gains up to four digits)
      const double inner = std::min(0.5, std::max(1e-4, 0.3 * so.tol / worst));
      std::vector<double> rel_inner;
      iters += o.cplx ? gmres_run<float, true>(o, r, dx, nrhs, inner, so.restart, so.max_iter - iters, prec,
                                               rel_inner, s)
                      : gmres_run<float, false>(o, r, dx, nrhs, inner, so.restart, so.max_iter - iters, prec,
                                                rel_inner, s);
      k_axpy<<<nblk(vn, 256), 256, 0, s>>>(x, dx, vn);
      launched("k_axpy");
    }
  }
  cuda_check(cudaStreamSynchronize(s), "solve sync");
  double worst = 0.0;
  for (double v : relres) worst = worse(worst, v);
  if (info) {
    info->iterations = iters;
    info->refinements = refinements;
    info->rel_residual = worst;
    info->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return worst <= so.tol ? BEMBEL_OK : BEMBEL_ENOTCONV;
}

}  // namespace bembel
