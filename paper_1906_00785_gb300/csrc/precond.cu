// precond.cu - block-Jacobi preconditioner set-up.
//
// D = blockdiag(N_tau,tau): the near-field diagonal blocks of the leaf clusters
// in element-local (Bernstein) coordinates.  Each block is inverted once by
// Gauss-Jordan elimination with partial pivoting (one thread block per leaf,
// one thread per row, in shared memory).  The preconditioner applied to global
// vectors is M^-1 = E^T D^-1 E with E the Bezier extraction (gather); E is
// injective, so for the SPD Laplace blocks M^-1 is SPD.  Not part of the paper
// (which solves without a preconditioner); it is the fallback preconditioner
// of the solver.
#include <string>
#include <vector>

#include "op.h"

namespace bembel {

namespace {

struct cplx_t {
  double r, i;
};
__device__ __forceinline__ cplx_t cmul(cplx_t a, cplx_t b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ __forceinline__ cplx_t cdiv(cplx_t a, cplx_t b) {
  const double d = b.r * b.r + b.i * b.i;
  return {(a.r * b.r + a.i * b.i) / d, (a.i * b.r - a.r * b.i) / d};
}

// One block per leaf: invert the nld x nld diagonal block (row-major in N)
// into out (row-major, leaf order).  info[leaf] = 1 when a pivot vanished.
template <bool CPLX>
__global__ void k_invert_blocks(const double* __restrict__ N, const int* __restrict__ diag_blk, int nld,
                                int64_t nleaf, double* __restrict__ out, int* __restrict__ info) {
  extern __shared__ double sm[];
  const int C = CPLX ? 2 : 1;
  const int w = 2 * nld;  // augmented row width [A | I]
  double* A = sm;         // nld rows x w columns, complex pairs when CPLX
  __shared__ int piv;
  const int64_t leaf = blockIdx.x;
  if (leaf >= nleaf) return;
  const double* B = N + (int64_t)diag_blk[leaf] * nld * nld * C;
  const int i = threadIdx.x;
  if (i < nld) {
    for (int j = 0; j < nld; ++j) {
      A[(i * w + j) * C] = B[((int64_t)i * nld + j) * C];
      if (CPLX) A[(i * w + j) * C + 1] = B[((int64_t)i * nld + j) * C + 1];
      A[(i * w + nld + j) * C] = (i == j) ? 1.0 : 0.0;
      if (CPLX) A[(i * w + nld + j) * C + 1] = 0.0;
    }
  }
  __syncthreads();
  for (int k = 0; k < nld; ++k) {
    if (i == 0) {
      int p = k;
      double best = -1.0;
      for (int r = k; r < nld; ++r) {
        const double re = A[(r * w + k) * C], im = CPLX ? A[(r * w + k) * C + 1] : 0.0;
        const double mag = re * re + im * im;
        if (mag > best) {
          best = mag;
          p = r;
        }
      }
      piv = p;
      if (best == 0.0) info[leaf] = 1;
    }
    __syncthreads();
    const int p = piv;
    if (p != k && i < w) {  // swap rows k and p, one column per thread
      for (int c = i; c < w; c += blockDim.x)
        for (int q = 0; q < C; ++q) {
          const double t = A[(k * w + c) * C + q];
          A[(k * w + c) * C + q] = A[(p * w + c) * C + q];
          A[(p * w + c) * C + q] = t;
        }
    }
    __syncthreads();
    // normalise the pivot row
    cplx_t pv = {A[(k * w + k) * C], CPLX ? A[(k * w + k) * C + 1] : 0.0};
    __syncthreads();
    for (int c = i; c < w; c += blockDim.x) {
      cplx_t v = {A[(k * w + c) * C], CPLX ? A[(k * w + c) * C + 1] : 0.0};
      const cplx_t q = CPLX ? cdiv(v, pv) : cplx_t{v.r / pv.r, 0.0};
      A[(k * w + c) * C] = q.r;
      if (CPLX) A[(k * w + c) * C + 1] = q.i;
    }
    __syncthreads();
    // eliminate column k from the other rows, one row per thread
    if (i < nld && i != k) {
      const cplx_t f = {A[(i * w + k) * C], CPLX ? A[(i * w + k) * C + 1] : 0.0};
      for (int c = 0; c < w; ++c) {
        const cplx_t pr = {A[(k * w + c) * C], CPLX ? A[(k * w + c) * C + 1] : 0.0};
        const cplx_t t = CPLX ? cmul(f, pr) : cplx_t{f.r * pr.r, 0.0};
        A[(i * w + c) * C] -= t.r;
        if (CPLX) A[(i * w + c) * C + 1] -= t.i;
      }
    }
    __syncthreads();
  }
  double* O = out + leaf * nld * nld * C;
  if (i < nld)
    for (int j = 0; j < nld; ++j) {
      O[((int64_t)i * nld + j) * C] = A[(i * w + nld + j) * C];
      if (CPLX) O[((int64_t)i * nld + j) * C + 1] = A[(i * w + nld + j) * C + 1];
    }
}

__global__ void k_f64_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = float(a[i]);
}

}  // namespace

void precond_setup(Op& o) {
  if (o.d_bj) return;
  const int C = o.cplx ? 2 : 1;
  const size_t shm = sizeof(double) * o.nld * 2 * o.nld * C;
  // one CTA holds [D | I] of a leaf in shared memory (at most 227 KiB)
  if (shm > 227 * 1024)
    fail(BEMBEL_EUNSUPPORTED, "block-Jacobi: leaf blocks of " + std::to_string(o.nld) +
                                  " local dofs exceed one CTA's shared memory (use a finer leaf level)");
  const int64_t n = o.nleaf * (int64_t)o.nld * o.nld * C;
  o.d_bj = static_cast<double*>(dev_alloc(sizeof(double) * n));
  int* info = static_cast<int*>(dev_alloc(sizeof(int) * o.nleaf));
  cuda_check(cudaMemsetAsync(info, 0, sizeof(int) * o.nleaf, o.stream), "bj info");
  const int threads = std::max(32, ((o.nld + 31) / 32) * 32);
  if (o.cplx) {
    if (shm > 48 * 1024)
      cuda_check(cudaFuncSetAttribute(k_invert_blocks<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(shm)),
                 "smem attr");
    k_invert_blocks<true><<<int(o.nleaf), threads, shm, o.stream>>>(o.d_N, o.d_diag_blk, o.nld, o.nleaf, o.d_bj,
                                                                     info);
  } else {
    if (shm > 48 * 1024)
      cuda_check(cudaFuncSetAttribute(k_invert_blocks<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(shm)),
                 "smem attr");
    k_invert_blocks<false><<<int(o.nleaf), threads, shm, o.stream>>>(o.d_N, o.d_diag_blk, o.nld, o.nleaf, o.d_bj,
                                                                      info);
  }
  launched("k_invert_blocks");
  o.d_bj32 = static_cast<float*>(dev_alloc(sizeof(float) * n));
  k_f64_to_f32<<<1024, 256, 0, o.stream>>>(o.d_bj, o.d_bj32, n);
  launched("k_f64_to_f32");
  std::vector<int> h(o.nleaf);
  cuda_check(cudaMemcpyAsync(h.data(), info, sizeof(int) * o.nleaf, cudaMemcpyDeviceToHost, o.stream), "bj info");
  cuda_check(cudaStreamSynchronize(o.stream), "bj sync");
  dev_free(info);
  for (int v : h)
    if (v) fail(BEMBEL_EINVAL, "block-Jacobi: a near-field diagonal block is singular");
}

}  // namespace bembel
