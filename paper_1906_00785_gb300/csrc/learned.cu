// learned.cu - learned weighting of the block-Jacobi preconditioner.
//
// The block-Jacobi preconditioner M^-1 = E^T D^-1 E (precond.cu) sums, for a
// global dof shared by several elements or leaves, the contributions of every
// element-local copy.  The learned form
//   M_W^-1 = E^T W D^-1 W E + P A_c^-1 P^T,   W = diag(w_i),  w_i = exp(MLP(f_i)) > 0,
// weights every element-local dof by a small network of local features f_i
// (position of the basis function in its element and of the element in its
// leaf, patch and leaf boundary flags, element distortion, |kappa| h).  W = I
// (zero output layer) is exactly the two-level preconditioner (block-Jacobi plus the
// coarse-space correction P A_c^-1 P^T of coarse.cu, which does not depend on W).  The
// network is trained on systems the solver generates, with the unsupervised loss
//   L = sum_s |M_W^-1 A z_s - z_s|^2 / |z_s|^2,
// whose gradient in W is (y = A z, t = z - P A_c^-1 P^T y, u = E y, p = D^-1 W u,
// r = E^T W p - t,
// g = E r, D^-1 complex symmetric)
//   dL/dw_i = 2 Re[ conj(g_i) p_i + (D^-1 W conj(g))_i u_i ],
// and back-propagated through the network by this file's own kernels.  Not in
// the paper (which uses no preconditioner).
#include <chrono>
#include <random>
#include <vector>

#include "op.h"

namespace bembel {

constexpr int kNin = 8, kNh = 16;
constexpr int kNparam = kNh * kNin + kNh + kNh * kNh + kNh + kNh + 1;  // 433

namespace {

inline int nb(int64_t n, int t) { return int(std::max<int64_t>(1, (n + t - 1) / t)); }

// Features of element-local dof ld = e*nloc + k1 + (d+1) k2.
__global__ void k_features(Geom g, int L, int d, int leaf, int64_t nlocal, double kabs, float* __restrict__ F) {
  const int64_t ld = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (ld >= nlocal) return;
  const int D1 = d + 1, nloc = D1 * D1;
  const int64_t e = ld / nloc;
  const int k = int(ld % nloc), k1 = k % D1, k2 = k / D1;
  const int64_t per = int64_t(1) << (2 * L);
  const int patch = int(e / per);
  uint32_t i1, i2;
  morton_decode(uint32_t(e % per), i1, i2);
  const int nel = 1 << L, m = 1 << (L - leaf);
  const double h = ldexp(1.0, -L);
  double x00[3], x10[3], x01[3];
  gamma_eval(g, patch, i1 * h, i2 * h, x00);
  gamma_eval(g, patch, (i1 + 1) * h, i2 * h, x10);
  gamma_eval(g, patch, i1 * h, (i2 + 1) * h, x01);
  const double a0 = x10[0] - x00[0], a1 = x10[1] - x00[1], a2 = x10[2] - x00[2];
  const double b0 = x01[0] - x00[0], b1 = x01[1] - x00[1], b2 = x01[2] - x00[2];
  const double c0 = a1 * b2 - a2 * b1, c1 = a2 * b0 - a0 * b2, c2 = a0 * b1 - a1 * b0;
  const double area = sqrt(c0 * c0 + c1 * c1 + c2 * c2);
  float* f = F + ld * kNin;
  f[0] = d > 0 ? float(k1) / d : 0.5f;
  f[1] = d > 0 ? float(k2) / d : 0.5f;
  f[2] = m > 1 ? float(i1 % m) / (m - 1) : 0.5f;
  f[3] = m > 1 ? float(i2 % m) / (m - 1) : 0.5f;
  f[4] = (i1 == 0 || i2 == 0 || int(i1) == nel - 1 || int(i2) == nel - 1) ? 1.f : 0.f;
  f[5] = (i1 / m == 0 || i2 / m == 0 || int(i1 / m) == nel / m - 1 || int(i2 / m) == nel / m - 1) ? 1.f : 0.f;
  f[6] = float(log(area / (h * h)));
  f[7] = float(kabs * sqrt(area));
}

struct Net {
  const float *W1, *b1, *W2, *b2, *w3;
  float b3;
};
__device__ __forceinline__ Net net_view(const float* P) {
  Net n;
  n.W1 = P;
  n.b1 = P + kNh * kNin;
  n.W2 = n.b1 + kNh;
  n.b2 = n.W2 + kNh * kNh;
  n.w3 = n.b2 + kNh;
  n.b3 = n.w3[kNh];
  return n;
}

__device__ __forceinline__ float net_forward(const Net& n, const float* x, float* h1, float* h2) {
  for (int j = 0; j < kNh; ++j) {
    float z = n.b1[j];
    for (int c = 0; c < kNin; ++c) z = fmaf(n.W1[j * kNin + c], x[c], z);
    h1[j] = tanhf(z);
  }
  float o = n.b3;
  for (int j = 0; j < kNh; ++j) {
    float z = n.b2[j];
    for (int c = 0; c < kNh; ++c) z = fmaf(n.W2[j * kNh + c], h1[c], z);
    h2[j] = tanhf(z);
    o = fmaf(n.w3[j], h2[j], o);
  }
  return expf(o);
}

__global__ void k_mlp_fwd(const float* __restrict__ P, const float* __restrict__ F, int64_t n, float* __restrict__ W) {
  __shared__ float sp[kNparam];
  for (int i = threadIdx.x; i < kNparam; i += blockDim.x) sp[i] = P[i];
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Net net = net_view(sp);
  float x[kNin], h1[kNh], h2[kNh];
  for (int c = 0; c < kNin; ++c) x[c] = F[i * kNin + c];
  W[i] = net_forward(net, x, h1, h2);
}

// grad += d/dP sum_i gw_i * w_i; per-dof terms staged in shared memory and
// reduced per parameter by the block, then added atomically.
constexpr int kBwdThreads = 128;
__global__ void __launch_bounds__(kBwdThreads) k_mlp_bwd(const float* __restrict__ P, const float* __restrict__ F,
                                                          const float* __restrict__ gw, int64_t n,
                                                          float* __restrict__ grad) {
  __shared__ float sp[kNparam];
  __shared__ float sx[kBwdThreads][kNin], sh1[kBwdThreads][kNh], sh2[kBwdThreads][kNh];
  __shared__ float sg1[kBwdThreads][kNh], sg2[kBwdThreads][kNh], sgo[kBwdThreads];
  for (int i = threadIdx.x; i < kNparam; i += blockDim.x) sp[i] = P[i];
  __syncthreads();
  const int t = threadIdx.x;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + t;
  const Net net = net_view(sp);
  if (i < n) {
    float x[kNin], h1[kNh], h2[kNh];
    for (int c = 0; c < kNin; ++c) x[c] = F[i * kNin + c];
    const float w = net_forward(net, x, h1, h2);
    const float go = gw[i] * w;
    float gz2[kNh];
    for (int j = 0; j < kNh; ++j) gz2[j] = go * net.w3[j] * (1.f - h2[j] * h2[j]);
    for (int c = 0; c < kNh; ++c) {
      float acc = 0.f;
      for (int j = 0; j < kNh; ++j) acc = fmaf(gz2[j], net.W2[j * kNh + c], acc);
      sg1[t][c] = acc * (1.f - h1[c] * h1[c]);
    }
    for (int c = 0; c < kNin; ++c) sx[t][c] = x[c];
    for (int j = 0; j < kNh; ++j) {
      sh1[t][j] = h1[j];
      sh2[t][j] = h2[j];
      sg2[t][j] = gz2[j];
    }
    sgo[t] = go;
  } else {
    for (int c = 0; c < kNin; ++c) sx[t][c] = 0.f;
    for (int j = 0; j < kNh; ++j) sh1[t][j] = sh2[t][j] = sg1[t][j] = sg2[t][j] = 0.f;
    sgo[t] = 0.f;
  }
  __syncthreads();
  for (int pi = t; pi < kNparam; pi += blockDim.x) {
    float acc = 0.f;
    if (pi < kNh * kNin) {  // W1[j][c]
      const int j = pi / kNin, c = pi % kNin;
      for (int r = 0; r < kBwdThreads; ++r) acc = fmaf(sg1[r][j], sx[r][c], acc);
    } else if (pi < kNh * kNin + kNh) {  // b1[j]
      const int j = pi - kNh * kNin;
      for (int r = 0; r < kBwdThreads; ++r) acc += sg1[r][j];
    } else if (pi < kNh * kNin + kNh + kNh * kNh) {  // W2[j][c]
      const int q = pi - kNh * kNin - kNh, j = q / kNh, c = q % kNh;
      for (int r = 0; r < kBwdThreads; ++r) acc = fmaf(sg2[r][j], sh1[r][c], acc);
    } else if (pi < kNh * kNin + 2 * kNh + kNh * kNh) {  // b2[j]
      const int j = pi - kNh * kNin - kNh - kNh * kNh;
      for (int r = 0; r < kBwdThreads; ++r) acc += sg2[r][j];
    } else if (pi < kNparam - 1) {  // w3[j]
      const int j = pi - kNh * kNin - 2 * kNh - kNh * kNh;
      for (int r = 0; r < kBwdThreads; ++r) acc = fmaf(sgo[r], sh2[r][j], acc);
    } else {  // b3
      for (int r = 0; r < kBwdThreads; ++r) acc += sgo[r];
    }
    atomicAdd(&grad[pi], acc);
  }
}

// v = w .* u (conj of u when conj_in), per element-local dof, C components
__global__ void k_wmul(const float* __restrict__ u, const float* __restrict__ w, float* __restrict__ v, int64_t n,
                       int C, int conj_in) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float wi = w[i];
  v[i * C] = wi * u[i * C];
  if (C == 2) v[i * C + 1] = (conj_in ? -wi : wi) * u[i * C + 1];
}

template <typename T>
__global__ void k_wmul_t(const T* __restrict__ u, const float* __restrict__ w, T* __restrict__ v, int64_t n, int C) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n * C) return;
  v[i] = T(w[i / C]) * u[i];
}

// r = out - z, loss += |r|^2 * scale
__global__ void k_resid(const float* __restrict__ out, const float* __restrict__ z, float* __restrict__ r, int64_t n,
                        double scale, double* __restrict__ loss) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double v = 0.0;
  if (i < n) {
    const float d = out[i] - z[i];
    r[i] = d;
    v = double(d) * d * scale;
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, v);
}

// gw_i += scale * 2 Re[conj(g_i) p_i + s_i u_i]
__global__ void k_wgrad(const float* __restrict__ g, const float* __restrict__ p, const float* __restrict__ s,
                        const float* __restrict__ u, int64_t n, int C, float scale, float* __restrict__ gw) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float acc;
  if (C == 2) {
    acc = g[2 * i] * p[2 * i] + g[2 * i + 1] * p[2 * i + 1] + s[2 * i] * u[2 * i] - s[2 * i + 1] * u[2 * i + 1];
  } else {
    acc = g[i] * p[i] + s[i] * u[i];
  }
  gw[i] += 2.f * scale * acc;
}

__global__ void k_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M,
                       float* __restrict__ V, int n, float lr, float b1, float b2, float eps, int step) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = G[i];
  M[i] = b1 * M[i] + (1.f - b1) * g;
  V[i] = b2 * V[i] + (1.f - b2) * g * g;
  const float mh = M[i] / (1.f - powf(b1, float(step))), vh = V[i] / (1.f - powf(b2, float(step)));
  P[i] -= lr * mh / (sqrtf(vh) + eps);
}

}  // namespace

// Training data of one operator: a stripped operator description (mesh sizes,
// extraction, leaf lists, FP32 D^-1), the dof features and samples (z, A z).
struct LearnedSet {
  Op o;
  float* F = nullptr;
  float* Z = nullptr;
  float* Y = nullptr;
  int ns = 0;
  std::vector<double> zscale;
  ~LearnedSet() {
    void* ps[] = {o.d_ex, o.d_bj32, o.d_leaf_ids, o.d_scratch, F, Z, Y};
    for (void* p : ps) dev_free(p);
  }
};

void learned_features(const Op& o, float* F) {
  k_features<<<nb(o.nlocal, 256), 256, 0, o.stream>>>(o.geom, o.L, o.d, o.leaf, o.nlocal,
                                                      std::sqrt(o.kre * o.kre + o.kim * o.kim), F);
  launched("k_features");
}

void mlp_forward(const float* P_dev, const float* F, int64_t n, float* W, cudaStream_t s) {
  k_mlp_fwd<<<nb(n, 256), 256, 0, s>>>(P_dev, F, n, W);
  launched("k_mlp_fwd");
}

void mlp_backward(const float* P_dev, const float* F, const float* gw, int64_t n, float* grad, cudaStream_t s) {
  k_mlp_bwd<<<nb(n, kBwdThreads), kBwdThreads, 0, s>>>(P_dev, F, gw, n, grad);
  launched("k_mlp_bwd");
}

LearnedSet* learned_collect(Op& src, int ns, unsigned long long seed) {
  if (src.rep != 1) fail(BEMBEL_EUNSUPPORTED, "learned preconditioner: knot_repetition 1 only");
  precond_setup(src);
  auto* S = new LearnedSet();
  Op& o = S->o;
  o.geom = src.geom;
  o.cplx = src.cplx;
  o.kre = src.kre;
  o.kim = src.kim;
  o.L = src.L;
  o.d = src.d;
  o.leaf = src.leaf;
  o.nloc = src.nloc;
  o.n1 = src.n1;
  o.nel1 = src.nel1;
  o.m = src.m;
  o.nld = src.nld;
  o.nelem = src.nelem;
  o.ndofs = src.ndofs;
  o.nlocal = src.nlocal;
  o.nleaf = src.nleaf;
  o.h = src.h;
  o.bsr_chunk = src.bsr_chunk;
  o.stream = src.stream;
  const int C = o.cplx ? 2 : 1;
  const size_t nex = (size_t)o.nel1 * (o.d + 1) * (o.d + 1);
  const size_t nbj = (size_t)o.nleaf * o.nld * o.nld * C;
  o.d_ex = static_cast<double*>(dev_alloc(sizeof(double) * nex));
  o.d_bj32 = static_cast<float*>(dev_alloc(sizeof(float) * nbj));
  o.d_leaf_ids = static_cast<int*>(dev_alloc(sizeof(int) * o.nleaf));
  cuda_check(cudaMemcpyAsync(o.d_ex, src.d_ex, sizeof(double) * nex, cudaMemcpyDeviceToDevice, o.stream), "copy");
  cuda_check(cudaMemcpyAsync(o.d_bj32, src.d_bj32, sizeof(float) * nbj, cudaMemcpyDeviceToDevice, o.stream), "copy");
  cuda_check(cudaMemcpyAsync(o.d_leaf_ids, src.d_leaf_ids, sizeof(int) * o.nleaf, cudaMemcpyDeviceToDevice, o.stream),
             "copy");
  S->F = static_cast<float*>(dev_alloc(sizeof(float) * o.nlocal * kNin));
  learned_features(o, S->F);
  // samples z ~ N(0,1) (real and imaginary parts), y = A z with the FP64 product
  S->ns = ns;
  const int64_t nv = o.ndofs * C;
  std::vector<double> zh((size_t)nv * ns);
  std::mt19937_64 rng(seed);
  std::normal_distribution<double> nd(0.0, 1.0);
  for (auto& v : zh) v = nd(rng);
  double* zd = static_cast<double*>(dev_alloc(sizeof(double) * nv * ns));
  double* yd = static_cast<double*>(dev_alloc(sizeof(double) * nv * ns));
  cuda_check(cudaMemcpy(zd, zh.data(), sizeof(double) * nv * ns, cudaMemcpyHostToDevice), "z");
  matvec_device(src, zd, yd, ns, false, src.stream);
  // the coarse correction C y is fixed (independent of W): the weighted block-Jacobi term
  // is trained to reproduce t = z - C y, so that the loss is |M_W^-1 A z - z|^2 with
  // M_W^-1 = E^T W D^-1 W E + C
  coarse_setup(src, ns);
  double* cd = static_cast<double*>(dev_alloc(sizeof(double) * nv * ns));
  cuda_check(cudaMemsetAsync(cd, 0, sizeof(double) * nv * ns, src.stream), "cy clear");
  const int saved = src.active_precond;
  src.active_precond = BEMBEL_PRECOND_TWO_LEVEL;
  coarse_apply_add(src, yd, cd, ns, false, src.stream);
  src.active_precond = saved;
  std::vector<double> yh((size_t)nv * ns), ch((size_t)nv * ns);
  cuda_check(cudaMemcpyAsync(yh.data(), yd, sizeof(double) * nv * ns, cudaMemcpyDeviceToHost, src.stream), "y");
  cuda_check(cudaMemcpyAsync(ch.data(), cd, sizeof(double) * nv * ns, cudaMemcpyDeviceToHost, src.stream), "cy");
  cuda_check(cudaStreamSynchronize(src.stream), "collect sync");
  dev_free(zd);
  dev_free(yd);
  dev_free(cd);
  std::vector<float> zf(zh.size()), yf(yh.begin(), yh.end());
  for (size_t i = 0; i < zh.size(); ++i) zf[i] = float(zh[i] - ch[i]);
  S->Z = static_cast<float*>(dev_alloc(sizeof(float) * nv * ns));
  S->Y = static_cast<float*>(dev_alloc(sizeof(float) * nv * ns));
  cuda_check(cudaMemcpy(S->Z, zf.data(), sizeof(float) * nv * ns, cudaMemcpyHostToDevice), "z32");
  cuda_check(cudaMemcpy(S->Y, yf.data(), sizeof(float) * nv * ns, cudaMemcpyHostToDevice), "y32");
  S->zscale.resize(ns);
  for (int r = 0; r < ns; ++r) {
    double a = 0.0;
    for (int64_t k = 0; k < nv; ++k) a += zh[(size_t)r * nv + k] * zh[(size_t)r * nv + k];
    S->zscale[r] = a > 0 ? 1.0 / (a * ns) : 0.0;
  }
  // scratch: u, v, p, g, t, s_, local (C each) + out, r global
  o.scratch_bytes = sizeof(float) * (6 * (size_t)o.nlocal * C + 2 * (size_t)nv) + 64;
  o.d_scratch = dev_alloc(o.scratch_bytes);
  return S;
}

// One pass over a set: loss (returned) and gw accumulated for weights W.
double learned_loss_grad(LearnedSet& S, const float* W, float* gw, double* d_loss) {
  Op& o = S.o;
  const cudaStream_t s = o.stream;
  const int C = o.cplx ? 2 : 1;
  const int64_t nl = o.nlocal, nv = o.ndofs * C;
  float* u = static_cast<float*>(o.d_scratch);
  float* v = u + nl * C;
  float* p = v + nl * C;
  float* g = p + nl * C;
  float* t = g + nl * C;
  float* sv = t + nl * C;
  float* out = sv + nl * C;
  float* r = out + nv;
  cuda_check(cudaMemsetAsync(d_loss, 0, sizeof(double), s), "loss clear");
  for (int smp = 0; smp < S.ns; ++smp) {
    const float* y = S.Y + (int64_t)smp * nv;
    const float* z = S.Z + (int64_t)smp * nv;
    local_gather(o, y, u, 1, true, s);
    k_wmul<<<nb(nl, 256), 256, 0, s>>>(u, W, v, nl, C, 0);
    launched("k_wmul");
    blockdiag_apply(o, o.d_bj32, v, p, 1, true, s);
    k_wmul<<<nb(nl, 256), 256, 0, s>>>(p, W, v, nl, C, 0);
    launched("k_wmul");
    local_scatter(o, v, out, 1, true, s);
    k_resid<<<nb(nv, 256), 256, 0, s>>>(out, z, r, nv, S.zscale[smp], d_loss);
    launched("k_resid");
    local_gather(o, r, g, 1, true, s);
    k_wmul<<<nb(nl, 256), 256, 0, s>>>(g, W, t, nl, C, 1);
    launched("k_wmul");
    blockdiag_apply(o, o.d_bj32, t, sv, 1, true, s);
    k_wgrad<<<nb(nl, 256), 256, 0, s>>>(g, p, sv, u, nl, C, float(S.zscale[smp]), gw);
    launched("k_wgrad");
  }
  double loss = 0.0;
  cuda_check(cudaMemcpyAsync(&loss, d_loss, sizeof(double), cudaMemcpyDeviceToHost, s), "loss");
  cuda_check(cudaStreamSynchronize(s), "loss sync");
  return loss;
}

void learned_train(LearnedSet* const* sets, int nsets, int epochs, double lr, float* params, double* hist) {
  float *P, *G, *M, *V;
  P = static_cast<float*>(dev_alloc(sizeof(float) * kNparam * 4));
  G = P + kNparam;
  M = G + kNparam;
  V = M + kNparam;
  cuda_check(cudaMemcpy(P, params, sizeof(float) * kNparam, cudaMemcpyHostToDevice), "params");
  cuda_check(cudaMemset(M, 0, sizeof(float) * kNparam * 2), "adam state");
  double* d_loss = static_cast<double*>(dev_alloc(sizeof(double)));
  int64_t nmax = 0;
  for (int i = 0; i < nsets; ++i) nmax = std::max<int64_t>(nmax, sets[i]->o.nlocal);
  float* W = static_cast<float*>(dev_alloc(sizeof(float) * nmax));
  float* gw = static_cast<float*>(dev_alloc(sizeof(float) * nmax));
  for (int ep = 0; ep < epochs; ++ep) {
    cuda_check(cudaMemset(G, 0, sizeof(float) * kNparam), "grad clear");
    double loss = 0.0;
    for (int i = 0; i < nsets; ++i) {
      LearnedSet& S = *sets[i];
      const cudaStream_t s = S.o.stream;
      mlp_forward(P, S.F, S.o.nlocal, W, s);
      cuda_check(cudaMemsetAsync(gw, 0, sizeof(float) * S.o.nlocal, s), "gw clear");
      loss += learned_loss_grad(S, W, gw, d_loss);
      mlp_backward(P, S.F, gw, S.o.nlocal, G, s);
      cuda_check(cudaStreamSynchronize(s), "set sync");
    }
    const float scale = 1.0f / float(nsets);
    std::vector<float> gh(kNparam);
    cuda_check(cudaMemcpy(gh.data(), G, sizeof(float) * kNparam, cudaMemcpyDeviceToHost), "grad");
    for (auto& v : gh) v *= scale;
    cuda_check(cudaMemcpy(G, gh.data(), sizeof(float) * kNparam, cudaMemcpyHostToDevice), "grad");
    k_adam<<<nb(kNparam, 256), 256>>>(P, G, M, V, kNparam, float(lr), 0.9f, 0.999f, 1e-8f, ep + 1);
    launched("k_adam");
    if (hist) hist[ep] = loss / nsets;
  }
  cuda_check(cudaMemcpy(params, P, sizeof(float) * kNparam, cudaMemcpyDeviceToHost), "params out");
  dev_free(P);
  dev_free(d_loss);
  dev_free(W);
  dev_free(gw);
}

// Attach trained weights to an operator: w_i = exp(MLP(f_i)) per element-local dof.
void learned_attach(Op& o, const float* params) {
  precond_setup(o);
  float* P = static_cast<float*>(dev_alloc(sizeof(float) * kNparam));
  float* F = static_cast<float*>(dev_alloc(sizeof(float) * o.nlocal * kNin));
  cuda_check(cudaMemcpy(P, params, sizeof(float) * kNparam, cudaMemcpyHostToDevice), "params");
  if (!o.d_lw) o.d_lw = static_cast<float*>(dev_alloc(sizeof(float) * o.nlocal));
  learned_features(o, F);
  mlp_forward(P, F, o.nlocal, o.d_lw, o.stream);
  cuda_check(cudaStreamSynchronize(o.stream), "attach sync");
  dev_free(P);
  dev_free(F);
}

// y_loc <- w .* y_loc for the learned preconditioner (T = float or double)
void learned_scale_local(const Op& o, void* yl, int nrhs, bool fp32, cudaStream_t s) {
  const int C = o.cplx ? 2 : 1;
  // weights are per local dof; with nrhs columns the local layout is dof-major
  // with nrhs*C contiguous reals, so each dof's weight covers ncol reals
  const int ncol = nrhs * C;
  if (fp32)
    k_wmul_t<float><<<nb(o.nlocal * ncol, 256), 256, 0, s>>>(static_cast<float*>(yl), o.d_lw, static_cast<float*>(yl),
                                                            o.nlocal, ncol);
  else
    k_wmul_t<double><<<nb(o.nlocal * ncol, 256), 256, 0, s>>>(static_cast<double*>(yl), o.d_lw,
                                                              static_cast<double*>(yl), o.nlocal, ncol);
  launched("k_wmul_t");
}

void learned_set_free(LearnedSet* s) { delete s; }

void mlp_eval_dev(const float* params_host, const float* F, int64_t n, const float* gw, float* W, float* grad_host) {
  float* P = static_cast<float*>(dev_alloc(sizeof(float) * kNparam * 2));
  float* G = P + kNparam;
  cuda_check(cudaMemcpy(P, params_host, sizeof(float) * kNparam, cudaMemcpyHostToDevice), "params");
  cuda_check(cudaMemset(G, 0, sizeof(float) * kNparam), "grad clear");
  mlp_forward(P, F, n, W, nullptr);
  if (gw) mlp_backward(P, F, gw, n, G, nullptr);
  cuda_check(cudaDeviceSynchronize(), "mlp sync");
  if (grad_host) cuda_check(cudaMemcpy(grad_host, G, sizeof(float) * kNparam, cudaMemcpyDeviceToHost), "grad");
  dev_free(P);
}

}  // namespace bembel
