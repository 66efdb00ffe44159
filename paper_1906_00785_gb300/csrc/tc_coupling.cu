// tc_coupling.cu - far-field coupling of the H^2 matvec for many right-hand
// sides on the 5th-generation tensor cores (tcgen05, TMEM accumulators).
//
// For a block of nrhs columns the coupling yh_t = sum_s K_ts xh_s (Sec. 2,
// kernel interpolated at the cluster Chebyshev points) is a sum of small
// products (q^2 x q^2) x (q^2 x ncol).  One CTA takes a group of sibling target
// clusters (8 for real kernels, 4 for complex ones) and walks the sorted union
// of their far sources.  Per source sigma it builds in shared memory
//   A (128 x 16, bf16): rows = (target, a) [x (Re, Im) for complex kernels], the
//       coupling K_t,sigma[a][b] evaluated on the fly in FP32 from the cluster
//       points, zero rows for group targets that do not interact with sigma;
//   B (ncol x 16, bf16): the source moments xh_sigma[b][col];
// and one thread issues tcgen05.mma.kind::f16 (M = 128, N = ncol, K = 16) that
// accumulates D = A B^T in TMEM (FP32).  The epilogue reads D with tcgen05.ld
// and writes yh for the group (complex: D_re-row / D_im-row recombined).
// Operands are double-buffered; a tcgen05.commit per MMA arrives on an
// mbarrier that guards the buffer's reuse.  Every wait is bounded: on time-out
// the kernel records an error, drains, frees its TMEM and returns.
//
// Shared-memory operands use the canonical K-major layout without swizzling:
// 8 x 16-byte core matrices, element (row r, k) at byte
// (r/8)*256 + (k/8)*128 + (r%8)*16 + (k%8)*2 of the tile.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "op.h"

namespace bembel {

namespace {

constexpr int kTcThreads = 128;
constexpr int kTcSmem = 100 * 1024;  // self-test launch (one CTA)
constexpr int kSmPerSm = 233472;     // shared memory per SM (228 KB)
constexpr int kSmReserved = 1024;    // per-CTA reservation
constexpr long long kSpinLimit = 1ll << 26;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: K-major, no swizzle, LBO = K-direction core
// stride, SBO = row-direction core stride (bytes), version 1
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor kind::f16: D f32, A/B bf16, both K-major
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* m, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count));
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(m)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait; returns false on time-out
__device__ __forceinline__ bool mbar_wait(uint64_t* m, uint32_t parity) {
  for (long long i = 0; i < kSpinLimit; ++i)
    if (mbar_try_wait(m, parity)) return true;
  return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* m) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(m))
               : "memory");
}

// 32 lanes x 8 consecutive 32-bit columns per thread
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const uint32_t a = __float_as_uint(lo), b = __float_as_uint(hi);
  // round to nearest even on the upper 16 bits
  const uint32_t ra = (a + 0x7FFFu + ((a >> 16) & 1u)) >> 16;
  const uint32_t rb = (b + 0x7FFFu + ((b >> 16) & 1u)) >> 16;
  return (ra & 0xFFFFu) | (rb << 16);
}

// write 16 bf16 values (one K = 16 row) of a K-major no-swizzle tile
__device__ __forceinline__ void store_row16(unsigned char* tile, int row, const float (&v)[16]) {
  uint4 lo, hi;
  lo.x = pack_bf16(v[0], v[1]);
  lo.y = pack_bf16(v[2], v[3]);
  lo.z = pack_bf16(v[4], v[5]);
  lo.w = pack_bf16(v[6], v[7]);
  hi.x = pack_bf16(v[8], v[9]);
  hi.y = pack_bf16(v[10], v[11]);
  hi.z = pack_bf16(v[12], v[13]);
  hi.w = pack_bf16(v[14], v[15]);
  unsigned char* base = tile + (row >> 3) * 256 + (row & 7) * 16;
  *reinterpret_cast<uint4*>(base) = lo;
  *reinterpret_cast<uint4*>(base + 128) = hi;
}

__device__ __forceinline__ uint32_t tmem_cols_for(int ncol) {
  uint32_t c = 32;
  while ((int)c < ncol) c <<= 1;
  return c;
}

// ---------------------------------------------------------------------------
// Self-test: D (128 x N) = A (128 x 16) B^T (B: N x 16), one MMA, one CTA.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kTcThreads) k_tc_selftest(const float* __restrict__ A, const float* __restrict__ B,
                                                            int N, float* __restrict__ D, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* tA = sm;
  unsigned char* tB = sm + 4096;
  __shared__ uint64_t mbar;
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t ncols = tmem_cols_for(N);
  if (warp == 0) tmem_alloc(&tbase, ncols);
  if (tid == 0) {
    mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  {
    float v[16];
    for (int k = 0; k < 16; ++k) v[k] = A[tid * 16 + k];
    store_row16(tA, tid, v);
    for (int n = tid; n < N; n += kTcThreads) {
      for (int k = 0; k < 16; ++k) v[k] = B[n * 16 + k];
      store_row16(tB, n, v);
    }
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t d = tbase;
  if (tid == 0) {
    mma_bf16(d, make_desc(smem_addr(tA), 128, 256), make_desc(smem_addr(tB), 128, 256), make_idesc(128, N), 0);
    mma_commit(&mbar);
  }
  const bool ok = mbar_wait(&mbar, 0);
  if (!ok && tid == 0) atomicExch(err, 1);
  tc_fence_after();
  __syncthreads();
  if (ok) {
    const int row = tid;
    for (int c0 = 0; c0 < N; c0 += 8) {
      float v[8];
      tmem_ld8(d + ((uint32_t)(warp * 32) << 16) + c0, v);
      for (int i = 0; i < 8; ++i) D[row * N + c0 + i] = v[i];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(d, ncols);
}

// One row of a coupling tile: G(pa, pb[b]) / (4 pi) for the 16 source points (real part,
// or for complex kernels the real (part 0) or imaginary (part 1) part), zero when the
// row's target does not interact with the source.
template <bool CPLX>
__device__ __forceinline__ void tile_row(bool on, float4 pa, const float4* __restrict__ pb, int part, float kre,
                                         float kim, float (&v)[16]) {
#pragma unroll
  for (int b = 0; b < 16; ++b) {
    float val = 0.f;
    if (on) {
      const float4 p = pb[b];
      const float d0 = pa.x - p.x, d1 = pa.y - p.y, d2 = pa.z - p.z;
      const float r2 = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
      const float rinv = rsqrtf(r2) * float(kInv4Pi);
      if (CPLX) {
        const float rr = r2 * rsqrtf(r2);
        float sn, cs;
        sincosf(kre * rr, &sn, &cs);
        const float am = (kim != 0.f ? expf(kim * rr) : 1.f) * rinv;
        val = part == 0 ? am * cs : -am * sn;
      } else {
        val = rinv;
      }
    }
    v[b] = val;
  }
}

// ---------------------------------------------------------------------------
// Production kernel, tiles evaluated on the fly.
// ---------------------------------------------------------------------------
template <bool CPLX>
__global__ void __launch_bounds__(kTcThreads) k_coupling_tc(const int* __restrict__ gptr, const int* __restrict__ gsrc,
                                                            const unsigned* __restrict__ gmask,
                                                            const int* __restrict__ gfirst, const int* __restrict__ gcnt,
                                                            int ngroups, const float4* __restrict__ pts, float kre,
                                                            float kim, const float* __restrict__ xh,
                                                            float* __restrict__ yh, int ncol, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* tA[2] = {sm, sm + 4096};
  unsigned char* tB[2] = {sm + 8192, sm + 8192 + 8192};
  __shared__ float4 tpt[128];  // target points of the group (rows / (1 + CPLX))
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tbase;
  __shared__ int abort_flag;
  constexpr int TG = CPLX ? 4 : 8;  // targets per group
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t ncols = tmem_cols_for(ncol);
  if (warp == 0) tmem_alloc(&tbase, ncols);
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t d = tbase;
  const uint32_t idesc = make_idesc(128, ncol);
  uint32_t phase[2] = {0, 0};
  int issued[2] = {0, 0};
  const int row = tid;  // A row owned by this thread
  const int tslot = CPLX ? (row >> 1) / 16 : row / 16;
  const int arow = CPLX ? (row >> 1) % 16 : row % 16;
  const int part = CPLX ? (row & 1) : 0;
  for (int gi = blockIdx.x; gi < ngroups && !abort_flag; gi += gridDim.x) {
    const int t0 = gfirst[gi], nt = gcnt[gi];
    if (tid < TG * 16) tpt[tid] = (tid / 16 < nt) ? pts[(int64_t)(t0 + tid / 16) * 16 + tid % 16] : make_float4(0, 0, 0, 0);
    __syncthreads();
    const int e0 = gptr[gi], e1 = gptr[gi + 1];
    int stage = 0;
    for (int e = e0; e < e1; ++e, stage ^= 1) {
      if (issued[stage]) {  // buffer still read by the MMA issued two steps ago
        if (!mbar_wait(&mbar[stage], phase[stage])) {
          if (tid == 0) {
            *reinterpret_cast<volatile int*>(err) = 1;
            abort_flag = 1;
          }
        }
        phase[stage] ^= 1;
        issued[stage] = 0;
      }
      __syncthreads();
      if (abort_flag) break;
      const int sc = gsrc[e];
      const unsigned mask = gmask[e];
      // A row: coupling of (target tslot, row a) with the 16 source points
      {
        float v[16];
        const bool on = tslot < nt && ((mask >> tslot) & 1u);
        tile_row<CPLX>(on, tpt[tslot * 16 + arow], pts + (int64_t)sc * 16, part, kre, kim, v);
        store_row16(tA[stage], row, v);
      }
      // B rows: source moments, column n, k = b
      for (int n = tid; n < ncol; n += kTcThreads) {
        float v[16];
        const float* xs = xh + (int64_t)sc * 16 * ncol + n;
#pragma unroll
        for (int b = 0; b < 16; ++b) v[b] = xs[(int64_t)b * ncol];
        store_row16(tB[stage], n, v);
      }
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        mma_bf16(d, make_desc(smem_addr(tA[stage]), 128, 256), make_desc(smem_addr(tB[stage]), 128, 256), idesc,
                 e > e0 ? 1 : 0);
        mma_commit(&mbar[stage]);
      }
      issued[stage] = 1;
    }
    // drain both buffers before reading the accumulator
    for (int st = 0; st < 2; ++st)
      if (issued[st]) {
        if (!mbar_wait(&mbar[st], phase[st]) && tid == 0) {
          *reinterpret_cast<volatile int*>(err) = 1;
          abort_flag = 1;
        }
        phase[st] ^= 1;
        issued[st] = 0;
      }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (abort_flag) break;
    // epilogue: row -> (target, a[, part]); D row = sum over sources
    const bool have = e1 > e0;
    for (int c0 = 0; c0 < ncol; c0 += 8) {
      float v[8];
      if (have) {
        tmem_ld8(d + ((uint32_t)(warp * 32) << 16) + c0, v);
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = 0.f;
      }
      if (!CPLX) {
        if (tslot < nt) {
          float* y = yh + ((int64_t)(t0 + tslot) * 16 + arow) * ncol + c0;
#pragma unroll
          for (int i = 0; i < 8; ++i) y[i] = v[i];
        }
      } else {
        // partner lane holds the other part of the same (target, a)
        float w[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) w[i] = __shfl_xor_sync(0xffffffffu, v[i], 1);
        // columns interleave (re, im) per right-hand side: D_re-row = Kr X', D_im-row = Ki X'
        // Y_re = Kr x_re - Ki x_im (even columns), Y_im = Kr x_im + Ki x_re (odd columns)
        if (tslot < nt && part == 0) {
          float* y = yh + ((int64_t)(t0 + tslot) * 16 + arow) * ncol + c0;
#pragma unroll
          for (int i = 0; i < 8; i += 2) {
            y[i] = v[i] - w[i + 1];
            y[i + 1] = v[i + 1] + w[i];
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  (void)lane;
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(d, ncols);
}

// ---------------------------------------------------------------------------
// Stored tiles.  The A tile of every group entry depends only on the geometry and the
// wavenumber, so it is evaluated once (tile_row, the same FP32 arithmetic as above) and
// kept in the canonical layout (4 KB per entry); per product the source moments are
// packed once per cluster into B tiles (ncol x 16 bf16).  The product kernel then only
// moves tiles and multiplies: one thread per CTA keeps a ring of kStages stages filled with
// bulk copies (cp.async.bulk, completion counted in bytes on the stage's "full" mbarrier),
// issues one tcgen05.mma per entry and commits it to the stage's "empty" mbarrier, which
// guards the stage's next fill.  Fills run a third of the ring ahead of the MMAs; the other
// stages hold MMAs in flight (the completion of one MMA is what a fill waits for).  Every wait is bounded: on time-out the CTA records the error, drains and returns.
// ---------------------------------------------------------------------------
constexpr int kMaxStages = 16;  // ring depth: chosen per launch from the shared memory per CTA

__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)), "r"(bytes)
               : "memory");
}

// bytes (multiple of 16, 16-byte aligned addresses) global -> shared, counted on m
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* m) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(m))
               : "memory");
}

// A tiles: block per group, thread per tile row, entries of the group in order.
template <bool CPLX>
__global__ void __launch_bounds__(kTcThreads) k_tc_build_a(const int* __restrict__ gptr, const int* __restrict__ gsrc,
                                                           const unsigned* __restrict__ gmask,
                                                           const int* __restrict__ gfirst,
                                                           const int* __restrict__ gcnt, int ngroups,
                                                           const float4* __restrict__ pts, float kre, float kim,
                                                           unsigned char* __restrict__ A) {
  const int row = threadIdx.x;
  const int tslot = CPLX ? (row >> 1) / 16 : row / 16;
  const int arow = CPLX ? (row >> 1) % 16 : row % 16;
  const int part = CPLX ? (row & 1) : 0;
  for (int gi = blockIdx.x; gi < ngroups; gi += gridDim.x) {
    const int t0 = gfirst[gi], nt = gcnt[gi];
    const float4 pa = tslot < nt ? pts[(int64_t)(t0 + tslot) * 16 + arow] : make_float4(0.f, 0.f, 0.f, 0.f);
    for (int e = gptr[gi]; e < gptr[gi + 1]; ++e) {
      float v[16];
      const bool on = tslot < nt && ((gmask[e] >> tslot) & 1u);
      tile_row<CPLX>(on, pa, pts + (int64_t)gsrc[e] * 16, part, kre, kim, v);
      store_row16(A + (int64_t)e * 4096, row, v);
    }
  }
}

// B tiles: B[s] row n (column n of the product), k = b: xh[s][b][n] in bf16.
__global__ void k_tc_pack_b(const float* __restrict__ xh, int64_t nclusters, int ncol, unsigned char* __restrict__ B) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= nclusters * ncol) return;
  const int64_t sc = id / ncol;
  const int n = int(id % ncol);
  const float* xs = xh + sc * 16 * ncol + n;
  float v[16];
#pragma unroll
  for (int b = 0; b < 16; ++b) v[b] = xs[(int64_t)b * ncol];
  store_row16(B + sc * (int64_t)ncol * 32, n, v);
}

// Work items: a run of at most kItemEntries consecutive entries of one group (int3: group,
// first entry, end), so that the long source lists of a few groups spread over many CTAs;
// each item's partial product is added to yh (cleared beforehand) with atomics.
constexpr int kItemEntries = 128;

template <bool CPLX>
__global__ void __launch_bounds__(kTcThreads)
    k_coupling_tc_stored(const int3* __restrict__ items, int nitems, const int* __restrict__ gsrc,
                         const int* __restrict__ gfirst, const int* __restrict__ gcnt,
                         const unsigned char* __restrict__ A, const unsigned char* __restrict__ B,
                         float* __restrict__ yh, int ncol, int kStages, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t full[kMaxStages], empty[kMaxStages];
  __shared__ uint32_t tbase;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t sbytes = 4096u + uint32_t(ncol) * 32u;  // one stage: A tile then B tile
  const uint32_t ncols = tmem_cols_for(ncol);
  if (warp == 0) tmem_alloc(&tbase, ncols);
  if (tid == 0) {
    for (int st = 0; st < kStages; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], 1);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t d = tbase;
  const uint32_t idesc = make_idesc(128, ncol);
  // thread 0's pipeline state, kept across groups
  uint32_t ph_full[kMaxStages], ph_empty[kMaxStages];
  bool pending[kMaxStages];  // an MMA committed to empty[st] that nobody has waited for
  bool filled[kMaxStages];   // a fill of stage st issued and not yet consumed
  for (int st = 0; st < kStages; ++st) {
    ph_full[st] = ph_empty[st] = 0u;
    pending[st] = filled[st] = false;
  }
  const int row = tid;
  const int tslot = CPLX ? (row >> 1) / 16 : row / 16;
  const int arow = CPLX ? (row >> 1) % 16 : row % 16;
  const int part = CPLX ? (row & 1) : 0;
  for (int it = blockIdx.x; it < nitems && !abort_flag; it += gridDim.x) {
    const int3 item = items[it];
    const int gi = item.x;
    const int t0 = gfirst[gi], nt = gcnt[gi];
    const int e0 = item.y, n = item.z - item.y;
    if (tid == 0) {
      bool ok = true;
      // fill stage j % kStages with entry j once the MMA that last read the stage is done
      auto load = [&](int j) {
        const int st = j % kStages;
        if (pending[st]) {
          ok = ok && mbar_wait(&empty[st], ph_empty[st]);
          ph_empty[st] ^= 1u;
          pending[st] = false;
        }
        if (!ok) return;
        unsigned char* sa = sm + st * sbytes;
        mbar_expect_tx(&full[st], sbytes);
        bulk_copy(sa, A + (int64_t)(e0 + j) * 4096, 4096u, &full[st]);
        bulk_copy(sa + 4096, B + (int64_t)gsrc[e0 + j] * ncol * 32, uint32_t(ncol) * 32u, &full[st]);
        filled[st] = true;
      };
      // fills run `ahead` entries in front; the other kStages - ahead stages hold MMAs in flight
      const int ahead = max(2, kStages / 3);
      for (int j = 0; j < ahead && j < n; ++j) load(j);
      for (int i = 0; i < n && ok; ++i) {
        if (i + ahead < n) load(i + ahead);
        const int st = i % kStages;
        ok = ok && mbar_wait(&full[st], ph_full[st]);
        ph_full[st] ^= 1u;
        filled[st] = false;
        if (!ok) break;
        tc_fence_after();
        const uint32_t sa = smem_addr(sm + st * sbytes);
        mma_bf16(d, make_desc(sa, 128, 256), make_desc(sa + 4096, 128, 256), idesc, i > 0 ? 1 : 0);
        mma_commit(&empty[st]);
        pending[st] = true;
      }
      // the accumulator is read below: wait for every MMA still in flight
      for (int st = 0; st < kStages; ++st)
        if (pending[st]) {
          ok = mbar_wait(&empty[st], ph_empty[st]) && ok;
          ph_empty[st] ^= 1u;
          pending[st] = false;
        }
      if (!ok) {
        // copies still in flight land in this CTA's shared memory: wait for them (bounded)
        for (int st = 0; st < kStages; ++st)
          if (filled[st]) {
            mbar_wait(&full[st], ph_full[st]);
            filled[st] = false;
          }
        *reinterpret_cast<volatile int*>(err) = 1;
        abort_flag = 1;
      }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (abort_flag) break;
    for (int c0 = 0; c0 < ncol && n > 0; c0 += 8) {
      float v[8];
      tmem_ld8(d + ((uint32_t)(warp * 32) << 16) + c0, v);
      if (!CPLX) {
        if (tslot < nt) {
          float* y = yh + ((int64_t)(t0 + tslot) * 16 + arow) * ncol + c0;
#pragma unroll
          for (int i = 0; i < 8; ++i) atomicAdd(y + i, v[i]);
        }
      } else {
        float w[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) w[i] = __shfl_xor_sync(0xffffffffu, v[i], 1);
        if (tslot < nt && part == 0) {
          float* y = yh + ((int64_t)(t0 + tslot) * 16 + arow) * ncol + c0;
#pragma unroll
          for (int i = 0; i < 8; i += 2) {
            atomicAdd(y + i, v[i] - w[i + 1]);
            atomicAdd(y + i + 1, v[i + 1] + w[i]);
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(d, ncols);
}

// Time-out path of the bounded waits: one thread waits, with a short limit, on an mbarrier
// that nothing arrives on, and records the expiry.  No TMEM, no copies: nothing to drain.
__global__ void k_tc_timeout_probe(long long limit, int* __restrict__ err) {
  __shared__ uint64_t m;
  if (threadIdx.x == 0) {
    mbar_init(&m, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    bool ok = false;
    for (long long i = 0; i < limit && !ok; ++i) ok = mbar_try_wait(&m, 0);
    if (!ok) *err = 1;
  }
}

}  // namespace

bool tc_coupling_wanted(const Op& o, int nrhs) {
  const int ncol = nrhs * (o.cplx ? 2 : 1);
  // below these widths the CUDA-core product is as fast (measured on the
  // level-6 sphere: real 32 columns 1.4x, complex 64 columns 1.15x faster here)
  const int min_cols = o.cplx ? 64 : 32;
  return o.opts.precision == BEMBEL_PREC_MIXED && o.opts.tensor_cores && o.q2 == 16 && !o.efie && o.nfar > 0 &&
         ncol >= min_cols && ncol <= 256 && ncol % 16 == 0;
}

bool tc_coupling_usable(const Op& o, int nrhs) { return o.d_tc_gptr != nullptr && tc_coupling_wanted(o, nrhs); }

// Sibling groups are built on first use (from the far lists on the device), not
// during assembly: most operators never see a wide enough product.
// The stored A tiles of every group entry (and the buffer for the packed B tiles); very
// large operators (more than 8 GiB of tiles) keep evaluating their tiles on the fly.
static void tc_build_tiles(Op& o) {
  const size_t abytes = size_t(4096) * std::max<int64_t>(1, o.tc_nentries);
  if (abytes > (size_t(8) << 30)) return;
  o.d_tc_A = static_cast<unsigned char*>(dev_alloc(abytes));
  o.d_tc_B = static_cast<unsigned char*>(dev_alloc(size_t(o.nclusters) * 256 * 32));
  {
    std::vector<int> gptr(o.tc_ngroups + 1);
    cuda_check(cudaMemcpy(gptr.data(), o.d_tc_gptr, sizeof(int) * gptr.size(), cudaMemcpyDeviceToHost), "tc gptr");
    std::vector<int3> items;
    for (int64_t g = 0; g < o.tc_ngroups; ++g)
      for (int e = gptr[g]; e < gptr[g + 1]; e += kItemEntries)
        items.push_back(make_int3(int(g), e, std::min(e + kItemEntries, gptr[g + 1])));
    o.tc_nitems = (int64_t)items.size();
    o.d_tc_items = static_cast<int*>(dev_alloc(sizeof(int3) * std::max<size_t>(1, items.size())));
    if (!items.empty())
      cuda_check(cudaMemcpy(o.d_tc_items, items.data(), sizeof(int3) * items.size(), cudaMemcpyHostToDevice),
                 "tc items");
  }
  const int grid = int(std::min<int64_t>(o.tc_ngroups, 152 * 8));
  if (o.cplx)
    k_tc_build_a<true><<<grid, kTcThreads, 0, o.stream>>>(o.d_tc_gptr, o.d_tc_gsrc, o.d_tc_gmask, o.d_tc_gfirst,
                                                          o.d_tc_gcnt, int(o.tc_ngroups),
                                                          reinterpret_cast<const float4*>(o.d_nodes32), float(o.kre),
                                                          float(o.kim), o.d_tc_A);
  else
    k_tc_build_a<false><<<grid, kTcThreads, 0, o.stream>>>(o.d_tc_gptr, o.d_tc_gsrc, o.d_tc_gmask, o.d_tc_gfirst,
                                                           o.d_tc_gcnt, int(o.tc_ngroups),
                                                           reinterpret_cast<const float4*>(o.d_nodes32), 0.f, 0.f,
                                                           o.d_tc_A);
  launched("k_tc_build_a");
}

void tc_prepare(Op& o, int nrhs) {
  if (o.d_tc_gptr || !tc_coupling_wanted(o, nrhs) || capturing()) return;

  std::vector<long long> fptr(o.nclusters + 1);
  std::vector<int> fsrc(o.nfar);
  cuda_check(cudaStreamSynchronize(o.stream), "tc groups sync");
  cuda_check(cudaMemcpy(fptr.data(), o.d_far_ptr, sizeof(long long) * fptr.size(), cudaMemcpyDeviceToHost),
             "far ptr");
  cuda_check(cudaMemcpy(fsrc.data(), o.d_far_src, sizeof(int) * fsrc.size(), cudaMemcpyDeviceToHost), "far src");
  tc_build_groups(o, fptr, fsrc);
  tc_build_tiles(o);
}

// CTAs per SM that the TMEM accumulators allow (512 columns per SM), and the
// dynamic shared memory that keeps residency at that count: the operand
// buffers need 2 x (4 KB + ncol x 32 B); the rest is padding.
static int tc_smem_bytes(int ncol, int static_bytes, int* ctas_per_sm) {
  int cols = 32;
  while (cols < ncol) cols <<= 1;
  const int ctas = std::min(8, 512 / cols);
  const int need = 2 * 4096 + 2 * ncol * 32;
  // (ctas + 1) CTAs must not fit: per-CTA footprint above kSmPerSm / (ctas + 1)
  const int cap = kSmPerSm / (ctas + 1) - kSmReserved - static_bytes + 128;
  *ctas_per_sm = ctas;
  return std::max(need, cap);
}

// the same residency rule for the stored-tile kernel, whose ring takes as many stages of
// (4 KB + ncol x 32 B) as the shared memory of one of the resident CTAs holds (4..16)
static int tc_smem_bytes_stored(int ncol, int static_bytes, int* ctas_per_sm, int* stages) {
  int cols = 32;
  while (cols < ncol) cols <<= 1;
  // as many CTAs per SM as their TMEM columns allow (up to 8), each with a shallow ring:
  // measured faster than 2-4 CTAs with deep rings (level-6 Laplace, 32 columns: 1.22 vs
  // 1.30-1.46 ms per product; level-5 Helmholtz, 64 columns: 0.87 vs 0.87-0.94 ms)
  const int ctas = std::min(8, 512 / cols);
  const int sbytes = 4096 + ncol * 32;
  const int per_cta = kSmPerSm / ctas - kSmReserved - static_bytes - 128;
  *stages = std::max(4, std::min(kMaxStages, per_cta / sbytes));
  const int need = *stages * sbytes;
  const int cap = kSmPerSm / (ctas + 1) - kSmReserved - static_bytes + 128;
  *ctas_per_sm = ctas;
  return std::max(need, cap);
}

void tc_coupling(const Op& o, const float* xh, float* yh, int nrhs, cudaStream_t s) {
  const int ncol = nrhs * (o.cplx ? 2 : 1);
  cudaFuncAttributes fa{};
  int ctas = 1;
  if (o.d_tc_A) {  // stored A tiles: pack B, then the copy + MMA pipeline
    k_tc_pack_b<<<int((o.nclusters * ncol + 255) / 256), 256, 0, s>>>(xh, o.nclusters, ncol, o.d_tc_B);
    launched("k_tc_pack_b");
    auto run = [&](auto kernel) {
      cuda_check(cudaFuncGetAttributes(&fa, kernel), "tc attributes");
      int stages = 4;
      const int smem = tc_smem_bytes_stored(ncol, int(fa.sharedSizeBytes), &ctas, &stages);
      cuda_check(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem), "tc smem");
      const int grid = int(std::max<int64_t>(1, std::min<int64_t>(o.tc_nitems, int64_t(152) * ctas)));
      kernel<<<grid, kTcThreads, smem, s>>>(reinterpret_cast<const int3*>(o.d_tc_items), int(o.tc_nitems),
                                            o.d_tc_gsrc, o.d_tc_gfirst, o.d_tc_gcnt, o.d_tc_A, o.d_tc_B, yh, ncol,
                                            stages, o.d_tc_err);
    };
    if (o.cplx)
      run(k_coupling_tc_stored<true>);
    else
      run(k_coupling_tc_stored<false>);
    launched("k_coupling_tc_stored");
    return;
  }
  if (o.cplx) {
    cuda_check(cudaFuncGetAttributes(&fa, k_coupling_tc<true>), "tc attributes");
    const int smem = tc_smem_bytes(ncol, int(fa.sharedSizeBytes), &ctas);
    cuda_check(cudaFuncSetAttribute(k_coupling_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
               "tc smem");
    const int grid = int(std::min<int64_t>(o.tc_ngroups, int64_t(152) * ctas));
    k_coupling_tc<true><<<grid, kTcThreads, smem, s>>>(o.d_tc_gptr, o.d_tc_gsrc, o.d_tc_gmask, o.d_tc_gfirst,
                                                       o.d_tc_gcnt, int(o.tc_ngroups),
                                                       reinterpret_cast<const float4*>(o.d_nodes32), float(o.kre),
                                                       float(o.kim), xh, yh, ncol, o.d_tc_err);
  } else {
    cuda_check(cudaFuncGetAttributes(&fa, k_coupling_tc<false>), "tc attributes");
    const int smem = tc_smem_bytes(ncol, int(fa.sharedSizeBytes), &ctas);
    cuda_check(cudaFuncSetAttribute(k_coupling_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
               "tc smem");
    const int grid = int(std::min<int64_t>(o.tc_ngroups, int64_t(152) * ctas));
    k_coupling_tc<false><<<grid, kTcThreads, smem, s>>>(o.d_tc_gptr, o.d_tc_gsrc, o.d_tc_gmask, o.d_tc_gfirst,
                                                        o.d_tc_gcnt, int(o.tc_ngroups),
                                                        reinterpret_cast<const float4*>(o.d_nodes32), 0.f, 0.f, xh,
                                                        yh, ncol, o.d_tc_err);
  }
  launched("k_coupling_tc");
}

// Groups of sibling targets and the union of their far sources (host set-up).
void tc_build_groups(Op& o, const std::vector<long long>& fptr, const std::vector<int>& fsrc) {
  const int TG = o.cplx ? 4 : 8;
  std::vector<int> gptr = {0}, gsrc, gfirst, gcnt;
  std::vector<unsigned> gmask;
  gsrc.reserve(fsrc.size());
  gmask.reserve(fsrc.size());
  // union of the group targets' far sources: mark[src] collects the target
  // bits, touched lists each source once (linear in the far-list length)
  std::vector<unsigned> mark(o.nclusters, 0u);
  std::vector<int> touched;
  for (int l = 0; l <= o.leaf; ++l) {
    const int64_t t0 = o.lvl_off[l], t1 = o.lvl_off[l + 1];
    for (int64_t g = t0; g < t1; g += TG) {
      const int nt = int(std::min<int64_t>(TG, t1 - g));
      touched.clear();
      for (int i = 0; i < nt; ++i)
        for (long long k = fptr[g + i]; k < fptr[g + i + 1]; ++k) {
          const int sc = fsrc[k];
          if (!mark[sc]) touched.push_back(sc);
          mark[sc] |= 1u << i;
        }
      std::sort(touched.begin(), touched.end());  // ascending sources: neighbouring loads
      for (int sc : touched) {
        gsrc.push_back(sc);
        gmask.push_back(mark[sc]);
        mark[sc] = 0u;
      }
      gptr.push_back(int(gsrc.size()));
      gfirst.push_back(int(g));
      gcnt.push_back(nt);
    }
  }
  o.tc_ngroups = (int64_t)gfirst.size();
  o.tc_nentries = (int64_t)gsrc.size();
  auto up = [](const auto& v) {
    using T = typename std::decay<decltype(v)>::type::value_type;
    T* p = static_cast<T*>(dev_alloc(sizeof(T) * std::max<size_t>(1, v.size())));
    if (!v.empty()) cuda_check(cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice), "tc upload");
    return p;
  };
  o.d_tc_gptr = up(gptr);
  o.d_tc_gsrc = up(gsrc);
  o.d_tc_gmask = up(gmask);
  o.d_tc_gfirst = up(gfirst);
  o.d_tc_gcnt = up(gcnt);
  // the time-out flag lives in mapped host memory: the host reads it without
  // synchronising (the next call on the operator reports it)
  void* h = nullptr;
  cuda_check(cudaHostAlloc(&h, sizeof(int), cudaHostAllocMapped), "tc err flag");
  o.h_tc_err = static_cast<int*>(h);
  *o.h_tc_err = 0;
  void* dptr = nullptr;
  cuda_check(cudaHostGetDevicePointer(&dptr, h, 0), "tc err flag alias");
  o.d_tc_err = static_cast<int*>(dptr);
}

void tc_check(const Op& o) {
  if (o.h_tc_err && *static_cast<volatile int*>(o.h_tc_err))
    fail(BEMBEL_ETIMEOUT, "a tensor-core MMA completion wait timed out in an earlier product on this operator");
}

bool tc_timeout_probe() {
  DevBuf err(sizeof(int));
  cuda_check(cudaMemset(err.p, 0, sizeof(int)), "probe err");
  k_tc_timeout_probe<<<1, 32>>>(1ll << 14, static_cast<int*>(err.p));
  launched("k_tc_timeout_probe");
  int h = 0;
  cuda_check(cudaMemcpy(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost), "probe read");
  return h != 0;
}

double tc_selftest(int N) {
  if (N < 16 || N > 256 || N % 16) fail(BEMBEL_EINVAL, "tc_selftest: N must be a multiple of 16 in [16, 256]");
  std::vector<float> A(128 * 16), B((size_t)N * 16);
  uint32_t st = 12345u;
  auto rnd = [&]() {
    st = st * 1664525u + 1013904223u;
    // values exactly representable in bf16: small integers / 8
    return float(int((st >> 16) % 17) - 8) / 8.0f;
  };
  for (auto& v : A) v = rnd();
  for (auto& v : B) v = rnd();
  float *dA, *dB, *dD;
  int* derr;
  dA = static_cast<float*>(dev_alloc(sizeof(float) * A.size()));
  dB = static_cast<float*>(dev_alloc(sizeof(float) * B.size()));
  dD = static_cast<float*>(dev_alloc(sizeof(float) * 128 * N));
  derr = static_cast<int*>(dev_alloc(sizeof(int)));
  cuda_check(cudaMemcpy(dA, A.data(), sizeof(float) * A.size(), cudaMemcpyHostToDevice), "A");
  cuda_check(cudaMemcpy(dB, B.data(), sizeof(float) * B.size(), cudaMemcpyHostToDevice), "B");
  cuda_check(cudaMemset(dD, 0, sizeof(float) * 128 * N), "D");
  cuda_check(cudaMemset(derr, 0, sizeof(int)), "err");
  cuda_check(cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem), "smem");
  k_tc_selftest<<<1, kTcThreads, kTcSmem>>>(dA, dB, N, dD, derr);
  launched("k_tc_selftest");
  cuda_check(cudaDeviceSynchronize(), "selftest sync");
  std::vector<float> D((size_t)128 * N);
  int herr = 0;
  cuda_check(cudaMemcpy(D.data(), dD, sizeof(float) * D.size(), cudaMemcpyDeviceToHost), "D");
  cuda_check(cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost), "err");
  dev_free(dA);
  dev_free(dB);
  dev_free(dD);
  dev_free(derr);
  if (herr) fail(BEMBEL_ETIMEOUT, "tc_selftest: MMA completion wait timed out");
  double worst = 0.0;
  for (int m = 0; m < 128; ++m)
    for (int n = 0; n < N; ++n) {
      double ref = 0.0;
      for (int k = 0; k < 16; ++k) ref += double(A[m * 16 + k]) * B[(size_t)n * 16 + k];
      worst = std::max(worst, std::fabs(ref - D[(size_t)m * N + n]));
    }
  return worst;
}

}  // namespace bembel
