// Coreness of every vertex (§4 "k-core"; Alg. 16, the bucketing peeling of
// Julienne) as one persistent cooperative kernel.  D starts at the degrees.
// For each k in increasing order:
//   - NextBucket: k = the smallest D over unfinished vertices.  It is
//     gathered while the previous bucket runs, with no pass of its own:
//     its vertex pass sees every untouched unfinished D, and a decrement
//     that leaves a vertex above the previous k offers its new D.  An
//     offered value may belong to a vertex finished later in the same
//     bucket, so k can fall below the true minimum; the bucket is then
//     empty and only costs its pass.  Empty buckets are otherwise skipped;
//   - the bucket: every unfinished vertex with D <= k is finished with
//     coreness k and put on a frontier queue (CTA-staged compaction);
//   - peeling rounds: the blocked sparse edgeMap over the frontier lowers
//     D of each unfinished neighbour by the number of its arcs from the
//     frontier (Histogram + DecrementCoreness: the arcs of a warp window
//     to the same neighbour are combined into one fetch-and-add); the
//     neighbour whose D crosses from above k to k or below in that add is
//     finished with coreness k and joins the next frontier (UpdateBuckets
//     into the current bucket), until the frontier is empty.
// Neighbours already at or below k are not decremented further (their
// coreness is k already), so D never has to be clamped.
#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "gbf_impl.h"

namespace gbf {
using namespace dev;

struct KcParams {
  DevGraph g;
  int32_t *core;   // output
  int32_t *D;      // remaining degree
  uint32_t *fin;   // finished vertices
  int32_t *q[2];
  uint32_t *qoff[2];
  uint32_t *qadj[2];
  uint32_t *cs[2];
  uint32_t cs_cap;
  Ctl *ctl;
  TraceRec *trace;
  int trace_cap;
  int bmax;
  int cap;
  int inject_wait;
  long long cap_ns;
};

namespace {

// DecrementCoreness over kU windows of arcs out of the frontier.
struct PeelFn {
  static constexpr int kWin = kU;
  template <class Sink>
  __device__ __forceinline__ void drain(Sink &, PushSmem &) {}
  const uint32_t *off;
  const int32_t *tgt;
  int32_t *D;
  int32_t *core;
  uint32_t *fin;
  int32_t k;
  unsigned long long peeled;
  int32_t nmin;  // smallest D left above k by this thread's decrements
  // Applies one decrement of c to v; true if v crossed into bucket k.
  __device__ __forceinline__ bool decrement(int32_t v, int32_t c) {
    const int32_t old = atomicSub(D + v, c);
    if (old - c > k) nmin = min(nmin, old - c);
    if (old > k && old - c <= k) {  // crossed into bucket k: finished now
      core[v] = k;
      atomicOr(fin + (v >> 5), 1u << (v & 31));
      peeled++;
      return true;
    }
    return false;
  }
  template <class Sink>
  __device__ __forceinline__ void batch(const bool *ok, const int32_t *, const uint32_t *idx,
                                        Sink &sink, PushSmem &S) {
    const int lane = threadIdx.x & 31;
    int32_t v[kU], dv[kU];
    bool live[kU];
#pragma unroll
    for (int r = 0; r < kU; r++) v[r] = ok[r] ? __ldg(tgt + idx[r]) : 0;
#pragma unroll
    for (int r = 0; r < kU; r++) dv[r] = ok[r] ? __ldcg(D + v[r]) : 0;
#pragma unroll
    for (int r = 0; r < kU; r++) live[r] = ok[r] && dv[r] > k;
    bool win[kU];
#pragma unroll
    for (int r = 0; r < kU; r++) {
      win[r] = false;
      // one fetch-and-add per distinct neighbour of the window
      const uint32_t key = live[r] ? (uint32_t)v[r] : (0x80000000u | (uint32_t)lane);
      const unsigned grp = __match_any_sync(kFull, key);
      if (live[r] && lane == __ffs(grp) - 1) win[r] = decrement(v[r], __popc(grp));
    }
    uint32_t a[kU], z[kU];
#pragma unroll
    for (int r = 0; r < kU; r++) {
      a[r] = z[r] = 0;
      if (win[r]) {
        a[r] = __ldg(off + v[r]);
        z[r] = __ldg(off + v[r] + 1);
      }
      z[r] -= a[r];
    }
    sink.template append_n<kU>(S, win, v, z, a);
  }
};


}  // namespace

__global__ void __launch_bounds__(1024) kcore_kernel(KcParams P) {
  extern __shared__ unsigned long long smem_raw[];
  __shared__ int s_flag;
  __shared__ int s_min[40];
  PushSmem S = carve_push_smem(smem_raw, SmemShape{P.bmax, P.cap, 0, 0, 1});
  if (threadIdx.x == 0) S.misc[0] = 0;
  Ctl *ctl = P.ctl;
  Barrier bar{0u, P.cap_ns};
  const DevGraph g = P.g;
  const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  const uint32_t n = (uint32_t)g.n;
  const uint32_t nwords = (n + 31) >> 5;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned long long scanned = 0, peeled = 0;
  const unsigned long long t_start = globaltimer();

  // D = degrees.  The first bucket is k = 0 (isolated vertices; empty if
  // there are none), whose pass gathers the smallest degree above 0.
  for (uint32_t i = gt; i < n; i += gs) P.D[i] = (int32_t)(__ldg(g.off + i + 1) - __ldg(g.off + i));
  for (uint32_t i = gt; i < nwords; i += gs) P.fin[i] = 0u;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st_vol(ctl->gmin[0], 0);
    st_vol(ctl->gmin[1], kInf);
  }
  if (P.inject_wait && blockIdx.x == 0 && threadIdx.x == 0) injected_wait(ctl, P.cap_ns);
  __syncthreads();
  bool ok = grid_sync(ctl, bar, &s_flag);

  // CTA-contiguous word ranges for the vertex passes
  const uint32_t per = (nwords + gridDim.x - 1) / gridDim.x;
  const uint32_t wlo = min(nwords, blockIdx.x * per), whi = min(nwords, wlo + per);
  // Counter slots.  fr[sub % 3] is zero at the top of each bucket; every
  // phase zeroes the slot after its own, read by nobody since two barriers.
  // gmin[it % 3] holds bucket it's k at its top; bucket it gathers the next
  // k in gmin[(it + 1) % 3] and zeroes gmin[(it + 2) % 3] for the one after.
  int bem = 0, sub = 0, tr = 0;  // tr: trace records (bucket passes and peeling rounds)
  for (int it = 0; ok; it++) {
    // ---------------- NextBucket: the smallest D over unfinished vertices,
    // gathered during the previous bucket (its pass and its decrements)
    const int32_t k = ld_vol(ctl->gmin[it % 3]);
    if (k >= kInf) break;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st_vol(ctl->gmin[(it + 2) % 3], kInf);
      st_vol(ctl->fr[(sub + 1) % 3], 0ull);
    }
    // ---------------- the bucket: unfinished vertices with D <= k; the
    // others give the next bucket's candidate minimum
    int lm = kInf;
    {
      QueueOut out{P.q[0], P.qoff[0], P.qadj[0], P.cs[0], &ctl->fr[sub % 3], n, P.cs_cap};
      constexpr int R = 2 * kU;
      for (uint32_t base = wlo; base < whi; base += R * nw) {
        uint32_t fw[R];
        int32_t dv[R];
#pragma unroll
        for (int r = 0; r < R; r++) {  // all loads first
          const uint32_t wi = base + warp + r * nw;
          const uint32_t v = wi * 32 + lane;
          fw[r] = wi < whi ? __ldcg(P.fin + wi) : ~0u;
          dv[r] = (wi < whi && v < n) ? __ldcg(P.D + v) : kInf;
        }
        uint32_t a[R], z[R];
        bool take[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
          const uint32_t wi = base + warp + r * nw;
          const uint32_t v = wi * 32 + lane;
          const bool un = v < n && !((fw[r] >> lane) & 1u);
          take[r] = un && dv[r] <= k;
          if (un && dv[r] > k) lm = min(lm, dv[r]);
          const unsigned tb = __ballot_sync(kFull, take[r]);
          if (lane == 0 && tb) P.fin[wi] = fw[r] | tb;  // the CTA owns these words here
          a[r] = z[r] = 0;
          if (take[r]) {
            P.core[v] = k;
            a[r] = __ldg(g.off + v);
            z[r] = __ldg(g.off + v + 1);
          }
        }
#pragma unroll
        for (int r = 0; r < R; r++) {
          const uint32_t d = z[r] - a[r];
          if (take[r]) peeled++;
          stage_append(S, take[r] && d > 0, (int32_t)((base + warp + r * nw) * 32 + lane), d, a[r]);
        }
        __syncthreads();
        stage_make_room(S, out, ctl, R * blockDim.x);
      }
      stage_flush(S, out, ctl);
    }
    {
      const int bm = block_min_i32(lm, s_min);
      if (threadIdx.x == 0 && bm < ld_vol(ctl->gmin[(it + 1) % 3])) atomicMin(&ctl->gmin[(it + 1) % 3], bm);
    }
    if (!grid_sync(ctl, bar, &s_flag)) break;
    // ---------------- peeling rounds within bucket k
    int qb = 0;
    unsigned long long fr = ld_vol(ctl->fr[sub % 3]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      atomicAdd(&ctl->rounds, 1);
      if (P.trace && tr < P.trace_cap)
        P.trace[tr] = TraceRec{tr + 1, 5, (uint32_t)(fr >> 32), (uint32_t)fr,
                               (long long)(globaltimer() - t_start), 0};
    }
    tr++;
    while (ok) {
      const uint32_t cnt = (uint32_t)(fr >> 32), Dsum = (uint32_t)fr;
      if (cnt == 0) break;
      sub++;
      unsigned long long *outc = &ctl->fr[sub % 3];
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        st_vol(ctl->fr[(sub + 1) % 3], 0ull);
        atomicAdd(&ctl->rounds, 1);
        atomicAdd(&ctl->push_rounds, 1);
        scanned += Dsum;
      }
      QueueIn in{P.q[qb], P.qoff[qb], P.qadj[qb], P.cs[qb], cnt, Dsum};
      PeelFn fn{g.off, g.tgt, P.D, P.core, P.fin, k, 0, kInf};
      StagedSink sink{QueueOut{P.q[qb ^ 1], P.qoff[qb ^ 1], P.qadj[qb ^ 1], P.cs[qb ^ 1], outc, n,
                               P.cs_cap},
                      ctl, nullptr};
      blocked_edge_map(g, in, chunk_shift(Dsum, 4u, chunk_shift_cap(PeelFn::kWin * blockDim.x)),
                       (uint32_t)P.bmax, S, fn, sink, ctl, bem++);
      sink.finish(S);
      peeled += fn.peeled;
      {
        const int bm = block_min_i32(fn.nmin, s_min);
        if (threadIdx.x == 0 && bm < ld_vol(ctl->gmin[(it + 1) % 3]))
          atomicMin(&ctl->gmin[(it + 1) % 3], bm);
      }
      qb ^= 1;
      if (!grid_sync(ctl, bar, &s_flag)) {
        ok = false;
        break;
      }
      fr = ld_vol(*outc);
      if (P.trace && blockIdx.x == 0 && threadIdx.x == 0 && tr < P.trace_cap)
        P.trace[tr] = TraceRec{tr + 1, 1, cnt, Dsum, (long long)(globaltimer() - t_start), 0};
      tr++;
    }
    sub++;  // the next bucket's pass uses the slot zeroed by the last phase
  }
  unsigned long long t;
  t = block_sum64(scanned, S.misc64);
  if (threadIdx.x == 0 && t) atomicAdd(&ctl->edges_scanned, t);
  t = block_sum64(peeled, S.misc64);
  if (threadIdx.x == 0 && t) atomicAdd(&ctl->reached, t);
}

gbf_status launch_kcore(Graph &g, Workspace &ws, int32_t *core, const Opts &o, cudaStream_t st) {
  KcParams P;
  P.g = g.dev();
  P.core = core;
  P.D = ws.dist_tmp == core ? ws.parent_tmp : ws.dist_tmp;
  P.fin = ws.visited;
  for (int i = 0; i < 2; i++) {
    P.q[i] = ws.q[i];
    P.qoff[i] = ws.qoff[i];
    P.qadj[i] = ws.qadj[i];
    P.cs[i] = ws.cs[i];
  }
  P.cs_cap = (uint32_t)(((uint64_t)g.m + kFine - 1) / kFine + 2);
  P.ctl = ws.ctl;
  P.trace = ws.trace;
  P.trace_cap = ws.trace_cap;
  P.bmax = o.heavy_cutoff;
  P.cap = stage_capacity(o.block);
  P.inject_wait = o.inject_wait;
  P.cap_ns = o.spin_cap_ns;
  const size_t smem = push_smem_bytes(SmemShape{P.bmax, P.cap, 0, 0, 1});
  {
    const gbf_status sm = check_smem(smem, "kcore_kernel");
    if (sm != GBF_OK) return sm;
  }
  GBF_CUDA(cudaFuncSetAttribute(kcore_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  int per_sm = 0;
  GBF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kcore_kernel, o.block, smem));
  if (per_sm < 1) {
    set_error("kcore kernel does not fit on an SM with this block size");
    return GBF_ERR_INVALID;
  }
  int grid = per_sm * g.num_sms;
  if (o.ctas > 0 && o.ctas < grid) grid = o.ctas;
  GBF_CUDA(cudaMemsetAsync(ws.ctl, 0, sizeof(Ctl), st));
  if (ws.trace) GBF_CUDA(cudaMemsetAsync(ws.trace, 0, sizeof(TraceRec) * (size_t)ws.trace_cap, st));
  void *args[] = {&P};
  GBF_CUDA(cudaLaunchCooperativeKernel((const void *)kcore_kernel, dim3(grid), dim3(o.block), args,
                                       smem, st));
  ws.last_kind = 6;
  ws.last_grid = grid;
  ws.last_block = o.block;
  return GBF_OK;
}

}  // namespace gbf

using namespace gbf;

extern "C" gbf_status gbf_kcore(gbf_graph *h, int32_t *core, int mem, const gbf_options *opt,
                                void *cuda_stream) {
  if (!h || !core) return set_error("graph or core is NULL"), GBF_ERR_INVALID;
  Graph &g = h->g;
  if (mem != GBF_HOST && mem != GBF_DEVICE) return set_error("bad mem"), GBF_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  std::lock_guard<std::mutex> lk(g.mu);
  const Opts o = resolve(opt, g, GBF_TUNE_BFS);
  {
    const gbf_status s = ws_ensure_base(g, g.ws);
    if (s != GBF_OK) return s;
  }
  int32_t *dd = mem == GBF_HOST ? g.ws.parent_tmp : core;
  {
    const gbf_status s = launch_kcore(g, g.ws, dd, o, st);
    if (s != GBF_OK) return s;
  }
  if (mem == GBF_DEVICE) return GBF_OK;
  GBF_CUDA(cudaMemcpyAsync(core, dd, sizeof(int32_t) * (size_t)g.n, cudaMemcpyDeviceToHost, st));
  return ws_collect(g.ws, st, nullptr);
}
