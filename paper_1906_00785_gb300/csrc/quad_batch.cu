// quad_batch.cu - assembly of several meshes in one persistent launch (FP64; for MIXED
// operators the separated pairs beyond the ring in FP32, as in quad.cu).
#include <algorithm>
#include <vector>

#include "op.h"
#include "pairkernels.cuh"

namespace bembel {

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
  const float4* Xqf32;  // MIXED: FP32 far-order points (regular_pair_f32), else null
  const double* cen;
  const float* BWf32;
  int f32k;             // MIXED: coupling entries evaluated in FP32 (coupling_entry_f32)
  const double* ccen;   // MIXED: cluster centres and FP32 point offsets
  const float4* rel;
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
                                                                int G2, int G2f, int scratch,
                                                                const double* __restrict__ gauss, int4 gi, int4 ge,
                                                                int4 gv, int3 goff, int q2) {
  extern __shared__ double sh[];
  double* ubuf = sh + (threadIdx.x >> 5) * scratch;  // regular pairs' sums or staged Duffy points
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
          if (m.pairs[kRegular][w].pad && m.Xqf32)
            regular_pair_f32<D, CPLX>(m.pairs[kRegular][w], m.Xqf32, m.cen, m.BWf32, m.BWf, ubuf, G2f, float(m.kre),
                                      float(m.kim), m.N, m.nld, lane);
          else if (m.pairs[kRegular][w].pad)
            regular_pair<D, CPLX>(m.pairs[kRegular][w], m.Xqf, m.BWf, ubuf, G2f, m.kre, m.kim, m.N, m.nld, lane);
          else
            regular_pair<D, CPLX>(m.pairs[kRegular][w], m.Xq, m.BW, ubuf, G2, m.kre, m.kim, m.N, m.nld, lane);
        break;
      case kIdentical:
        for (long long w = first; w < last; ++w)
          singular_pair<D, CPLX, kIdentical>(m.pairs[kIdentical][w], m.geom, m.L, gi, gx[0], gw[0], m.kre, m.kim,
                                             m.N, m.nld, lane, ubuf);
        break;
      case kEdge:
        for (long long w = first; w < last; ++w)
          singular_pair<D, CPLX, kEdge>(m.pairs[kEdge][w], m.geom, m.L, ge, gx[1], gw[1], m.kre, m.kim, m.N,
                                        m.nld, lane, ubuf);
        break;
      case kVertex:
        for (long long w = first; w < last; ++w)
          singular_pair<D, CPLX, kVertex>(m.pairs[kVertex][w], m.geom, m.L, gv, gx[2], gw[2], m.kre, m.kim, m.N,
                                          m.nld, lane, ubuf);
        break;
      default: {
        const int per = q2 * q2;
        for (long long blk = first; blk < last; ++blk) {
          if (m.f32k && m.rel) {
            const int t = m.far_tgt[blk], sc = m.far_src[blk];
            const float3 dc = centre_difference(m.ccen, t, sc);
            for (int r = lane; r < per; r += 32)
              coupling_entry_f32<CPLX>(blk, r, t, sc, dc, m.rel, q2, float(m.kre), float(m.kim), m.K);
          } else {
            for (int r = lane; r < per; r += 32)
              coupling_entry<CPLX>(blk, r, m.far_tgt, m.far_src, m.nodes, q2, m.kre, m.kim, m.K, m.f32k != 0);
          }
        }
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
  const int scratch = std::max(std::max(G2, G2f) * NL * (CPLX ? 2 : 1), stage_doubles(kVertex, NL));
  const size_t shm = sizeof(double) * kWarps * scratch;
  // opt in always: the static tables and segments come on top of shm
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
  k_assemble_multi<D, CPLX><<<grid, 32 * kWarps, shm, s>>>(d_ms, d_seg, nseg, nitems, d_next, G2, G2f, scratch,
                                                           o.d_gauss,
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
    w.Xqf32 = reinterpret_cast<const float4*>(o.d_Xq_far32);
    w.f32k = o.opts.precision == BEMBEL_PREC_MIXED ? 1 : 0;
    w.ccen = o.d_ccen;
    w.rel = reinterpret_cast<const float4*>(o.d_nodes_rel32);
    w.cen = o.d_cen;
    w.BWf32 = o.d_BW_far32;
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
  for (Op* o : ops) points_f32(*o, s);
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
  for (Op* o : ops) coupling_f32(*o, s);
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

}  // namespace bembel
