// Frontier Bellman-Ford (Alg. 4, general-weight SSSP) and single-source
// widest path (the same rounds over the (max, min) semiring, §5 "Widest
// Path") as one persistent cooperative kernel: one bounded grid barrier per
// round.  Each round is the blocked sparse edgeMap of §6.2 over the
// frontier queue with the Update of Alg. 4: the candidate value
// (D[s] + w, or min(W[s], w)) is compared with the target's, written with
// writeMin (writeMax), and a target whose value improved joins the next
// frontier once through a test-and-set on a per-round flag bitmap.  The
// flags of a frontier are reset one round later (ResetFlags), while the
// other bitmap serves the round in between.
//
// Values: Bellman-Ford D = INT32_MAX until reached, D[src] = 0; widest path
// W = 0 ("no path yet"; weights are >= 1) and W[src] = INT32_MAX (the empty
// path), then unreached vertices get INT32_MAX at the end, the paper's
// output convention.  Graphs are symmetric with weights >= 1, so there are
// no negative cycles and a round limit of n is never reached.
#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "gbf_impl.h"

namespace gbf {
using namespace dev;

struct BfParams {
  DevGraph g;
  int32_t src;
  int32_t *val;
  uint32_t *flags[2];
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
  int widest;  // 0: (min, +) Bellman-Ford; 1: (max, min) widest path
  int inject_wait;
  long long cap_ns;
};

namespace {

// Update of Alg. 4 for kU windows of arcs out of the frontier: target,
// weight and source-value loads, then the target values, then writeMin /
// writeMax, then the flag test-and-set of the improved targets, whose
// degrees and first arcs are then read for the next frontier.
struct SemiringFn {
  static constexpr int kWin = kU;  // windows per walk step
  template <class Sink>
  __device__ __forceinline__ void drain(Sink &, PushSmem &) {}  // nothing deferred
  const uint32_t *off;
  const int32_t *tgt;
  const uint32_t *w;
  int32_t *val;
  uint32_t *flags;
  int widest;
  unsigned long long relax;
  template <class Sink>
  __device__ __forceinline__ void batch(const bool *ok, const int32_t *u, const uint32_t *idx,
                                        Sink &sink, PushSmem &S) {
    int32_t v[kU], c[kU];
#pragma unroll
    for (int r = 0; r < kU; r++) {
      v[r] = 0;
      c[r] = widest ? 0 : kInf;  // never better than any value
      if (ok[r]) {
        v[r] = __ldg(tgt + idx[r]);
        const int32_t wt = (int32_t)__ldg(w + idx[r]);
        // the source's value now (it may have improved earlier this round)
        const int32_t su = __ldcg(val + u[r]);
        c[r] = widest ? min(su, wt) : su + wt;  // su < kInf: u is on the frontier
      }
    }
    int32_t cur[kU];
#pragma unroll
    for (int r = 0; r < kU; r++) cur[r] = ok[r] ? __ldcg(val + v[r]) : 0;
    bool win[kU];
#pragma unroll
    for (int r = 0; r < kU; r++) {
      win[r] = false;
      const bool better = ok[r] && (widest ? c[r] > cur[r] : c[r] < cur[r]);
      if (better) {
        const int32_t old = widest ? atomicMax(val + v[r], c[r]) : atomicMin(val + v[r], c[r]);
        if (widest ? old < c[r] : old > c[r]) {
          relax++;
          const uint32_t bit = 1u << (v[r] & 31);
          if (!(__ldcg(flags + (v[r] >> 5)) & bit))
            win[r] = !(atomicOr(flags + (v[r] >> 5), bit) & bit);
        }
      }
    }
    uint32_t a[kU], z[kU];
    bool emit[kU];
#pragma unroll
    for (int r = 0; r < kU; r++) {
      a[r] = z[r] = 0;
      if (win[r]) {
        a[r] = __ldg(off + v[r]);
        z[r] = __ldg(off + v[r] + 1);
      }
      z[r] -= a[r];  // degree
      // a degree-1 vertex improved through its only neighbour cannot improve it back
      emit[r] = win[r] && z[r] >= 2;
    }
    sink.template append_n<kU>(S, emit, v, z, a);
  }
};

}  // namespace

__global__ void __launch_bounds__(1024) bf_kernel(BfParams P) {
  extern __shared__ unsigned long long smem_raw[];
  __shared__ int s_flag;
  PushSmem S = carve_push_smem(smem_raw, SmemShape{P.bmax, P.cap, 0, 0, 1});
  if (threadIdx.x == 0) S.misc[0] = 0;
  Ctl *ctl = P.ctl;
  Barrier bar{0u, P.cap_ns};
  const DevGraph g = P.g;
  const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  const uint32_t nwords = ((uint32_t)g.n + 31) >> 5;
  const int32_t src = P.src;
  const int32_t unset = P.widest ? 0 : kInf;
  unsigned long long scanned = 0, expanded = 0, relax = 0;
  const unsigned long long t_start = globaltimer();

  for (uint32_t i = gt; i < (uint32_t)g.n; i += gs)
    P.val[i] = (i == (uint32_t)src) ? (P.widest ? kInf : 0) : unset;
  for (uint32_t i = gt; i < nwords; i += gs) {
    P.flags[0][i] = 0u;
    P.flags[1][i] = 0u;
  }
  if (blockIdx.x == 0) {
    const uint32_t a0 = __ldg(g.off + src), d0 = __ldg(g.off + src + 1) - a0;
    if (threadIdx.x == 0 && d0 > 0) {
      P.q[0][0] = src;
      P.qoff[0][0] = 0;
      P.qadj[0][0] = a0;
      st_vol(ctl->fr[0], (1ull << 32) | d0);
    }
    for (uint32_t c = threadIdx.x; c < (d0 + kFine - 1) / kFine; c += blockDim.x)
      if (c < P.cs_cap) P.cs[0][c] = 0;
  }
  if (P.inject_wait && blockIdx.x == 0 && threadIdx.x == 0) injected_wait(ctl, P.cap_ns);
  __syncthreads();
  bool ok = grid_sync(ctl, bar, &s_flag);

  int qb = 0, bem = 0;
  unsigned long long fr = ok ? ld_vol(ctl->fr[0]) : 0ull;
  for (int32_t round = 1; ok && round <= g.n; round++) {
    const uint32_t cnt = (uint32_t)(fr >> 32), D = (uint32_t)fr;
    if (cnt == 0) break;
    unsigned long long *outc = &ctl->fr[round % 3];
    uint32_t *fl = P.flags[round & 1];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st_vol(ctl->fr[(round + 1) % 3], 0ull);
      atomicAdd(&ctl->rounds, 1);
      atomicAdd(&ctl->push_rounds, 1);
      scanned += D;
      expanded += cnt;
    }
    // ResetFlags of this frontier (set in the other bitmap last round)
    for (uint32_t i = gt; i < cnt; i += gs) {
      const int32_t v = P.q[qb][i];
      atomicAnd(P.flags[(round + 1) & 1] + (v >> 5), ~(1u << (v & 31)));
    }
    QueueIn in{P.q[qb], P.qoff[qb], P.qadj[qb], P.cs[qb], cnt, D};
    SemiringFn fn{g.off, g.tgt, g.w, P.val, fl, P.widest, 0};
    StagedSink sink{QueueOut{P.q[qb ^ 1], P.qoff[qb ^ 1], P.qadj[qb ^ 1], P.cs[qb ^ 1], outc,
                             (uint32_t)g.n, P.cs_cap},
                    ctl, nullptr};
    blocked_edge_map(g, in, chunk_shift(D, 4u, chunk_shift_cap(SemiringFn::kWin * blockDim.x)),
                     (uint32_t)P.bmax, S, fn, sink, ctl, bem++);
    sink.finish(S);
    relax += fn.relax;
    qb ^= 1;
    if (!grid_sync(ctl, bar, &s_flag)) break;
    fr = ld_vol(*outc);
    if (P.trace && blockIdx.x == 0 && threadIdx.x == 0 && round <= P.trace_cap)
      P.trace[round - 1] = TraceRec{round, 1, cnt, D, (long long)(globaltimer() - t_start), 0};
  }
  if (ok && P.widest)
    for (uint32_t i = gt; i < (uint32_t)g.n; i += gs)
      if (P.val[i] == 0) P.val[i] = kInf;
  unsigned long long t;
  t = block_sum64(scanned, S.misc64);
  if (threadIdx.x == 0 && t) atomicAdd(&ctl->edges_scanned, t);
  t = block_sum64(expanded, S.misc64);
  if (threadIdx.x == 0 && t) atomicAdd(&ctl->expanded, t);
  t = block_sum64(relax, S.misc64);
  if (threadIdx.x == 0 && t) atomicAdd(&ctl->relax, t);
}

gbf_status launch_bf(Graph &g, Workspace &ws, int32_t src, int32_t *val, int widest,
                     const Opts &o, cudaStream_t st) {
  BfParams P;
  P.g = g.dev();
  P.src = src;
  P.val = val;
  P.flags[0] = ws.visited;
  P.flags[1] = ws.fbm[0];
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
  P.widest = widest;
  P.inject_wait = o.inject_wait;
  P.cap_ns = o.spin_cap_ns;
  const size_t smem = push_smem_bytes(SmemShape{P.bmax, P.cap, 0, 0, 1});
  {
    const gbf_status sm = check_smem(smem, "bf_kernel");
    if (sm != GBF_OK) return sm;
  }
  GBF_CUDA(cudaFuncSetAttribute(bf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  GBF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bf_kernel, o.block, smem));
  if (per_sm < 1) {
    set_error("bf kernel does not fit on an SM with this block size");
    return GBF_ERR_INVALID;
  }
  int grid = per_sm * g.num_sms;
  if (o.ctas > 0 && o.ctas < grid) grid = o.ctas;
  GBF_CUDA(cudaMemsetAsync(ws.ctl, 0, sizeof(Ctl), st));
  if (ws.trace) GBF_CUDA(cudaMemsetAsync(ws.trace, 0, sizeof(TraceRec) * (size_t)ws.trace_cap, st));
  void *args[] = {&P};
  GBF_CUDA(cudaLaunchCooperativeKernel((const void *)bf_kernel, dim3(grid), dim3(o.block), args,
                                       smem, st));
  ws.last_kind = 4;
  ws.last_grid = grid;
  ws.last_block = o.block;
  return GBF_OK;
}

}  // namespace gbf

using namespace gbf;

namespace {
gbf_status run_bf(gbf_graph *h, int32_t src, int32_t *out, int mem, const gbf_options *opt,
                  void *cuda_stream, int widest) {
  if (!h || !out) return set_error("graph or output is NULL"), GBF_ERR_INVALID;
  Graph &g = h->g;
  if (!g.w) return set_error("graph has no weights"), GBF_ERR_INVALID;
  if (src < 0 || src >= g.n) return set_error("src out of range"), GBF_ERR_INVALID;
  if (mem != GBF_HOST && mem != GBF_DEVICE) return set_error("bad mem"), GBF_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  std::lock_guard<std::mutex> lk(g.mu);
  const Opts o = resolve(opt, g, GBF_TUNE_BFS);
  {
    const gbf_status ws = ws_ensure_base(g, g.ws);
    if (ws != GBF_OK) return ws;
  }
  int32_t *dd = mem == GBF_HOST ? g.ws.dist_tmp : out;
  {
    const gbf_status ls = launch_bf(g, g.ws, src, dd, widest, o, st);
    if (ls != GBF_OK) return ls;
  }
  if (mem == GBF_DEVICE) return GBF_OK;
  GBF_CUDA(cudaMemcpyAsync(out, dd, sizeof(int32_t) * (size_t)g.n, cudaMemcpyDeviceToHost, st));
  return ws_collect(g.ws, st, nullptr);
}
}  // namespace

extern "C" gbf_status gbf_bellman_ford(gbf_graph *g, int32_t src, int32_t *dist, int mem,
                                       const gbf_options *opt, void *cuda_stream) {
  return run_bf(g, src, dist, mem, opt, cuda_stream, 0);
}

extern "C" gbf_status gbf_widest_path(gbf_graph *g, int32_t src, int32_t *width, int mem,
                                      const gbf_options *opt, void *cuda_stream) {
  return run_bf(g, src, width, mem, opt, cuda_stream, 1);
}
