// Connectivity (§4 "Connectivity") as one persistent cooperative kernel:
// label[v] = the smallest vertex id in v's connected component.
//
// The paper reaches the partition by decomposing (Alg. 6), contracting the
// clusters and recursing (Alg. 7).  Here every round sweeps all arcs once
// with the blocked edgeMap over every vertex that has arcs (one queue, built
// once by CTA-staged compaction with its degree prefix and chunk starts),
// then shortcuts the labels:
//   - hooking: for an arc (u, v) with L[u] < L[v], writeMin L[u] into L[v]
//     and into L[L[v]] (the label v points at), so whole label trees move;
//   - shortcutting: L[v] = L[L[v]].
// Labels only decrease and always name a vertex of the same component, so
// the smallest vertex of a component keeps its own id; a round that changes
// nothing leaves L[u] == L[v] across every arc and L[L[v]] == L[v], i.e.
// every vertex labelled with its component's smallest id.  Changes are
// counted per round in triple-buffered slots, so every CTA reads the same
// count after the barrier and all stop in the same round.
#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "gbf_impl.h"

namespace gbf {
using namespace dev;

struct CcParams {
  DevGraph g;
  int32_t *L;  // labels (output)
  int32_t *q;  // the vertices with arcs, their degree prefix, first arcs, chunk starts
  uint32_t *qoff;
  uint32_t *qadj;
  uint32_t *cs;
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

constexpr int kMaxRounds = 1 << 12;

// Hooking over kU windows of arcs.
struct HookFn {
  static constexpr int kWin = kU;
  template <class Sink>
  __device__ __forceinline__ void drain(Sink &, PushSmem &) {}
  const int32_t *tgt;
  int32_t *L;
  unsigned long long changed;
  template <class Sink>
  __device__ __forceinline__ void batch(const bool *ok, const int32_t *uu, const uint32_t *idx,
                                        Sink &, PushSmem &) {
    int32_t lu[kU], lv[kU];
#pragma unroll
    for (int r = 0; r < kU; r++) {
      const int32_t v = ok[r] ? __ldg(tgt + idx[r]) : 0;
      lu[r] = ok[r] ? __ldcg(L + uu[r]) : 0;
      lv[r] = ok[r] ? __ldcg(L + v) : 0;
      if (ok[r] && lu[r] < lv[r]) {
        if (atomicMin(L + lv[r], lu[r]) > lu[r]) changed++;
        if (atomicMin(L + v, lu[r]) > lu[r]) changed++;
      }
    }
  }
};

struct NoOutput {
  template <int U>
  __device__ __forceinline__ void append_n(PushSmem &, const bool *, const int32_t *,
                                           const uint32_t *, const uint32_t *) {}
  __device__ __forceinline__ void chunk_end(PushSmem &) { __syncthreads(); }
};

}  // namespace

__global__ void __launch_bounds__(1024) cc_kernel(CcParams P) {
  extern __shared__ unsigned long long smem_raw[];
  __shared__ int s_flag;
  PushSmem S = carve_push_smem(smem_raw, SmemShape{P.bmax, P.cap, 0, 0, 1});
  if (threadIdx.x == 0) S.misc[0] = 0;
  Ctl *ctl = P.ctl;
  Barrier bar{0u, P.cap_ns};
  const DevGraph g = P.g;
  const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  const uint32_t n = (uint32_t)g.n;
  unsigned long long scanned = 0;
  const unsigned long long t_start = globaltimer();

  // labels, and one queue of every vertex with arcs (CTA-contiguous ranges,
  // staged compaction: the walk needs entries of positive degree)
  {
    const uint32_t per = (n + gridDim.x - 1) / gridDim.x;
    const uint32_t vlo = min(n, blockIdx.x * per), vhi = min(n, vlo + per);
    QueueOut out{P.q, P.qoff, P.qadj, P.cs, &ctl->fr[0], n, P.cs_cap};
    for (uint32_t base = vlo; base < vhi; base += blockDim.x) {
      const uint32_t v = base + threadIdx.x;
      uint32_t a = 0, d = 0;
      if (v < vhi) {
        P.L[v] = (int32_t)v;
        a = __ldg(g.off + v);
        d = __ldg(g.off + v + 1) - a;
      }
      stage_append(S, v < vhi && d > 0, (int32_t)v, d, a);
      __syncthreads();
      stage_make_room(S, out, ctl, blockDim.x);
    }
    stage_flush(S, out, ctl);
  }
  if (P.inject_wait && blockIdx.x == 0 && threadIdx.x == 0) injected_wait(ctl, P.cap_ns);
  __syncthreads();
  bool ok = grid_sync(ctl, bar, &s_flag);
  const unsigned long long qf = ld_vol(ctl->fr[0]);  // written before the barrier, never after
  const uint32_t qcnt = (uint32_t)(qf >> 32), qD = (uint32_t)qf;

  int bem = 0;
  for (int32_t r = 0; ok; r++) {
    if (r >= kMaxRounds) {
      if (blockIdx.x == 0 && threadIdx.x == 0) raise_error(ctl, GBF_ERR_OVERFLOW, 40);
      break;
    }
    // slot (r + 1) % 3 was last read two barriers ago
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st_vol(ctl->scnt[(r + 1) % 3], 0u);
      atomicAdd(&ctl->rounds, 1);
      scanned += qD;
    }
    unsigned long long changed = 0;
    if (qcnt > 0) {
      QueueIn in{P.q, P.qoff, P.qadj, P.cs, qcnt, qD};
      HookFn fn{g.tgt, P.L, 0};
      NoOutput sink;
      blocked_edge_map(g, in, chunk_shift(qD, 4u, chunk_shift_cap(HookFn::kWin * blockDim.x)),
                       (uint32_t)P.bmax, S, fn, sink, ctl, bem++);
      changed = fn.changed;
    }
    if (!grid_sync(ctl, bar, &s_flag)) break;
    // shortcutting
    for (uint32_t v = gt; v < n; v += gs) {
      const int32_t l = __ldcg(P.L + v);
      const int32_t ll = __ldcg(P.L + l);
      if (ll < l) {
        atomicMin(P.L + v, ll);
        changed++;
      }
    }
    {
      const unsigned long long t = block_sum64(changed, S.misc64);
      if (threadIdx.x == 0 && t) atomicAdd(&ctl->scnt[r % 3], t > 0xffffffffull ? 0xffffffffu : (unsigned)t);
    }
    if (!grid_sync(ctl, bar, &s_flag)) break;
    if (P.trace && blockIdx.x == 0 && threadIdx.x == 0 && r < P.trace_cap)
      P.trace[r] = TraceRec{r + 1, 1, qcnt, qD, (long long)(globaltimer() - t_start), 0};
    if (ld_vol(ctl->scnt[r % 3]) == 0u) break;  // nothing changed: every label is final
  }
  {
    const unsigned long long t = block_sum64(scanned, S.misc64);
    if (threadIdx.x == 0 && t) atomicAdd(&ctl->edges_scanned, t);
  }
}

gbf_status launch_cc(Graph &g, Workspace &ws, int32_t *label, const Opts &o, cudaStream_t st) {
  CcParams P;
  P.g = g.dev();
  P.L = label;
  P.q = ws.q[0];
  P.qoff = ws.qoff[0];
  P.qadj = ws.qadj[0];
  P.cs = ws.cs[0];
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
    const gbf_status sm = check_smem(smem, "cc_kernel");
    if (sm != GBF_OK) return sm;
  }
  GBF_CUDA(cudaFuncSetAttribute(cc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  GBF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cc_kernel, o.block, smem));
  if (per_sm < 1) {
    set_error("cc kernel does not fit on an SM with this block size");
    return GBF_ERR_INVALID;
  }
  int grid = per_sm * g.num_sms;
  if (o.ctas > 0 && o.ctas < grid) grid = o.ctas;
  GBF_CUDA(cudaMemsetAsync(ws.ctl, 0, sizeof(Ctl), st));
  if (ws.trace) GBF_CUDA(cudaMemsetAsync(ws.trace, 0, sizeof(TraceRec) * (size_t)ws.trace_cap, st));
  void *args[] = {&P};
  GBF_CUDA(cudaLaunchCooperativeKernel((const void *)cc_kernel, dim3(grid), dim3(o.block), args,
                                       smem, st));
  ws.last_kind = 8;
  ws.last_grid = grid;
  ws.last_block = o.block;
  return GBF_OK;
}

}  // namespace gbf

using namespace gbf;

extern "C" gbf_status gbf_connectivity(gbf_graph *h, int32_t *label, int mem, const gbf_options *opt,
                                       void *cuda_stream) {
  if (!h || !label) return set_error("graph or label is NULL"), GBF_ERR_INVALID;
  Graph &g = h->g;
  if (mem != GBF_HOST && mem != GBF_DEVICE) return set_error("bad mem"), GBF_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  std::lock_guard<std::mutex> lk(g.mu);
  const Opts o = resolve(opt, g, GBF_TUNE_BFS);
  {
    const gbf_status s = ws_ensure_base(g, g.ws);
    if (s != GBF_OK) return s;
  }
  int32_t *dd = mem == GBF_HOST ? g.ws.dist_tmp : label;
  {
    const gbf_status s = launch_cc(g, g.ws, dd, o, st);
    if (s != GBF_OK) return s;
  }
  if (mem == GBF_DEVICE) return GBF_OK;
  GBF_CUDA(cudaMemcpyAsync(label, dd, sizeof(int32_t) * (size_t)g.n, cudaMemcpyDeviceToHost, st));
  return ws_collect(g.ws, st, nullptr);
}
