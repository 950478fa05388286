// Multi-source BFS: k <= 64 independent BFSs (§4 "Breadth-First Search",
// Alg. 1) advanced together, source i in bit lane i of a uint64 per vertex.
// The paper's nearest precedent is the SCC algorithm's simultaneous
// searches from many centres (§5, "Strongly Connected Components"); here the
// lanes share every edge scan and every level barrier.
//
// Per vertex: seen (lanes that reached it), visit[2] (lanes for which it is
// on the current / next frontier), next (lanes pushed into it this level).
// One persistent cooperative kernel runs every level; each level is one
// edgeMap in one direction (§3), chosen from the frontier's out-degree sum
// against m / pull_divisor:
//   - push: the blocked edgeMap (§6.2) over the frontier queue; for an arc
//     (u, v) the lanes visit[u] & ~seen[v] are OR-ed into next[v] (64-bit
//     atomicOr); the first OR into v records v in a touched list, and a
//     second phase turns next[v] & ~seen[v] into v's new lanes;
//   - pull: every vertex with unreached lanes ORs visit[u] over its
//     neighbours, stopping once every missing lane is covered.
// Vertices reached by lane i at level L get dist[i][L] written once, in
// warp-wide bit loops so a warp of consecutive vertices writes each row
// coalesced; lanes that never reach a vertex get GBF_INF at the end.
//
// The graph, sources, k and the output rows are read from a device parameter
// block (MsCall), so one captured CUDA graph replays any call on any graph
// the workspace is sized for.
//
// Lane words come in two widths: 64-bit lanes for batches of more than 8
// sources, and 8-bit lanes (one byte per vertex, four vertices per 32-bit
// word for the atomic ORs) for batches of 2..8, whose per-vertex arrays are
// an eighth of the size and stay in L2 at the serving graphs' sizes.
#include <cuda_runtime.h>

#include <algorithm>

#include "dev_common.cuh"
#include "gbf_impl.h"

namespace gbf {
using namespace dev;

struct MsCall {
  DevGraph g;         // the graph of this call
  int32_t srcs[64];
  int32_t *rows[64];  // rows[i][v] = distance of v from srcs[i]
  int32_t k;
  int32_t pad;
};

struct MsParams {
  const MsCall *call;
  void *seen;       // lane words (LaneT of the kernel instance), n each
  void *visit[2];
  void *next;
  int32_t *q[3];
  uint32_t *qoff[3];
  uint32_t *qadj[3];
  uint32_t *cs[3];
  uint32_t cs_cap;
  int32_t *touched;
  Ctl *ctl;
  TraceRec *trace;
  int trace_cap;
  int pull_divisor;
  int pull_serial;
  int bmax;
  int cap;
  int inject_wait;
  long long cap_ns;
};

namespace {

typedef unsigned long long u64;

// Access to the per-vertex lane words of one width; values travel as u64.
template <class T>
struct Lanes;
template <>
struct Lanes<u64> {
  static __device__ __forceinline__ u64 ld(const void *a, uint32_t v) { return ((const u64 *)a)[v]; }
  static __device__ __forceinline__ void st(void *a, uint32_t v, u64 x) { ((u64 *)a)[v] = x; }
  // atomic OR of m into vertex v's word; returns the word before
  static __device__ __forceinline__ u64 bor(void *a, uint32_t v, u64 m) {
    return atomicOr((u64 *)a + v, m);
  }
};
template <>
struct Lanes<uint8_t> {
  static __device__ __forceinline__ u64 ld(const void *a, uint32_t v) {
    return (u64)((const uint8_t *)a)[v];
  }
  static __device__ __forceinline__ void st(void *a, uint32_t v, u64 x) {
    ((uint8_t *)a)[v] = (uint8_t)x;
  }
  // the byte of v inside its aligned 32-bit word (the array is 4-byte aligned)
  static __device__ __forceinline__ u64 bor(void *a, uint32_t v, u64 m) {
    unsigned *w = (unsigned *)((uint8_t *)a + (v & ~3u));
    const unsigned sh = 8u * (v & 3u);
    return (u64)((atomicOr(w, (unsigned)m << sh) >> sh) & 0xffu);
  }
};

// Warp-collective: write level L into dist[i][v] for every lane bit i of
// `bits`, iterating lanes so that a warp of consecutive v writes each row
// with one coalesced store.
__device__ __forceinline__ void write_rows(int32_t *const *rows, int k, int32_t v, u64 bits,
                                           int32_t L) {
  u64 any = 0;
  // OR of bits across the warp, to skip lanes nobody has
  const unsigned lo32 = __reduce_or_sync(kFull, (unsigned)bits);
  const unsigned hi32 = __reduce_or_sync(kFull, (unsigned)(bits >> 32));
  any = ((u64)hi32 << 32) | lo32;
  while (any) {
    const int i = __ffsll((long long)any) - 1;
    any &= any - 1;
    if (i >= k) break;
    if ((bits >> i) & 1ull) rows[i][v] = L;
  }
}

struct TouchSink {
  int32_t *list;
  unsigned int *count;
  uint32_t cap;
  Ctl *ctl;
  // Warp-collective: the U appends of one walk step with one atomic.
  template <int U>
  __device__ __forceinline__ void append_n(PushSmem &, const bool *emit, const int32_t *v,
                                           const uint32_t *, const uint32_t *) {
    unsigned bal[U];
    uint32_t tot = 0;
#pragma unroll
    for (int r = 0; r < U; r++) {
      bal[r] = __ballot_sync(kFull, emit[r]);
      tot += __popc(bal[r]);
    }
    if (tot == 0) return;
    const int lane = threadIdx.x & 31;
    uint32_t pos = 0;
    if (lane == 0) pos = atomicAdd(count, tot);
    pos = __shfl_sync(kFull, pos, 0);
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int r = 0; r < U; r++) {
      if (emit[r]) {
        const uint32_t i = pos + __popc(bal[r] & lt);
        if (i < cap) list[i] = v[r];
        else raise_error(ctl, GBF_ERR_OVERFLOW, 10);
      }
      pos += __popc(bal[r]);
    }
  }
  __device__ __forceinline__ void chunk_end(PushSmem &) { __syncthreads(); }
};

// Push Update for kU windows: lanes visit[u] & ~seen[v] are OR-ed into next[v].
template <class T>
struct MsPushFn {
  static constexpr int kWin = kU;  // windows per walk step
  template <class Sink>
  __device__ __forceinline__ void drain(Sink &, PushSmem &) {}  // nothing deferred
  const int32_t *tgt;
  const void *cur;
  const void *seen;
  void *next;
  unsigned long long scanned;
  template <class Sink>
  __device__ __forceinline__ void batch(const bool *val, const int32_t *u, const uint32_t *idx,
                                        Sink &sink, PushSmem &S) {
    int32_t v[kU];
    u64 w[kU], sv[kU];
#pragma unroll
    for (int r = 0; r < kU; r++) {
      v[r] = val[r] ? __ldg(tgt + idx[r]) : 0;
      w[r] = val[r] ? Lanes<T>::ld(cur, (uint32_t)u[r]) : 0ull;
    }
#pragma unroll
    for (int r = 0; r < kU; r++) sv[r] = val[r] ? Lanes<T>::ld(seen, (uint32_t)v[r]) : ~0ull;
    bool first[kU];
#pragma unroll
    for (int r = 0; r < kU; r++) {
      const u64 m = w[r] & ~sv[r];
      first[r] = false;
      if (m) first[r] = Lanes<T>::bor(next, (uint32_t)v[r], m) == 0ull;
    }
    sink.template append_n<kU>(S, first, v, nullptr, nullptr);
  }
};

}  // namespace

template <class T>
__global__ void __launch_bounds__(1024) msbfs_kernel(MsParams P) {
  typedef Lanes<T> LN;
  extern __shared__ unsigned long long smem_raw[];
  __shared__ int s_flag;
  PushSmem S = carve_push_smem(smem_raw, SmemShape{P.bmax, P.cap, 0, 0, 1});
  if (threadIdx.x == 0) S.misc[0] = 0;
  Ctl *ctl = P.ctl;
  Barrier bar{0u, P.cap_ns};
  const DevGraph g = P.call->g;
  const uint32_t n = (uint32_t)g.n;
  const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int k = P.call->k;
  int32_t *const *rows = P.call->rows;
  const u64 ALL = (k >= 64) ? ~0ull : ((1ull << k) - 1ull);
  unsigned long long scanned = 0, expanded = 0, reached = 0, pulled = 0;
  const unsigned long long t_start = globaltimer();

  for (uint32_t i = gt; i < n; i += gs) {
    LN::st(P.seen, i, 0ull);
    LN::st(P.visit[0], i, 0ull);
    LN::st(P.visit[1], i, 0ull);
    LN::st(P.next, i, 0ull);
  }
  if (P.inject_wait && blockIdx.x == 0 && threadIdx.x == 0) injected_wait(ctl, P.cap_ns);
  bool ok = grid_sync(ctl, bar, &s_flag);
  // sources: lane i starts at srcs[i] (level 0); the level-0 queue holds each
  // distinct source with at least one edge
  if (ok && blockIdx.x == 0) {
    bool emit = false;
    int32_t s = 0;
    uint32_t d = 0, a = 0;
    if ((int)threadIdx.x < k) {
      s = P.call->srcs[threadIdx.x];
      LN::bor(P.seen, (uint32_t)s, 1ull << threadIdx.x);
      LN::bor(P.visit[0], (uint32_t)s, 1ull << threadIdx.x);
      rows[threadIdx.x][s] = 0;
      bool dup = false;
      for (int j = 0; j < (int)threadIdx.x; j++) dup |= P.call->srcs[j] == s;
      a = __ldg(g.off + s);
      d = __ldg(g.off + s + 1) - a;
      emit = !dup && d > 0;
    }
    stage_append(S, emit, s, d, a);  // whole CTA: warp-collective
    stage_flush(S, QueueOut{P.q[0], P.qoff[0], P.qadj[0], P.cs[0], &ctl->fr[0], n, P.cs_cap}, ctl);
    if (threadIdx.x == 0) reached = (unsigned long long)k;
  }
  ok = ok && grid_sync(ctl, bar, &s_flag);

  unsigned long long fr = ok ? ld_vol(ctl->fr[0]) : 0ull;
  int bem = 0;  // blocked edgeMap invocations so far
  for (int32_t L = 1; ok; L++) {
    const uint32_t cnt = (uint32_t)(fr >> 32), D = (uint32_t)fr;
    if (cnt == 0) break;
    const int qc = (L - 1) % 3, qn = L % 3, qo = (L + 1) % 3;  // queues of levels L-1, L, L-2
    const void *cur = P.visit[(L - 1) & 1];
    void *nxt = P.visit[L & 1];
    const bool dense =
        P.pull_divisor > 0 && (unsigned long long)D * (unsigned)P.pull_divisor > g.m;
    unsigned long long *outc = &ctl->fr[qn];
    unsigned int *tcount = &ctl->mcnt[L & 1];
    // counters of level L+1 were last read at level L-1
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st_vol(ctl->mcnt[(L + 1) & 1], 0u);
      atomicAdd(&ctl->rounds, 1);
      atomicAdd(dense ? &ctl->pull_rounds : &ctl->push_rounds, 1);
    }
    QueueOut fout{P.q[qn], P.qoff[qn], P.qadj[qn], P.cs[qn], outc, n, P.cs_cap};
    if (!dense) {
      // nxt still holds the frontier of level L-2 (queue qo, plus every
      // source when L == 2): clear it while the push reads cur
      if (L >= 2) {
        const uint32_t c2 = (uint32_t)(ld_vol(ctl->fr[qo]) >> 32);
        for (uint32_t i = gt; i < c2; i += gs) LN::st(nxt, (uint32_t)P.q[qo][i], 0ull);
        if (L == 2 && blockIdx.x == 0 && (int)threadIdx.x < k)
          LN::st(nxt, (uint32_t)P.call->srcs[threadIdx.x], 0ull);
      }
      QueueIn in{P.q[qc], P.qoff[qc], P.qadj[qc], P.cs[qc], cnt, D};
      MsPushFn<T> fn{g.tgt, cur, P.seen, P.next, 0};
      TouchSink sink{P.touched, tcount, n, ctl};
      blocked_edge_map(g, in, chunk_shift(D, 4u, 8), (uint32_t)P.bmax, S, fn, sink,
                       ctl, bem++);
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        scanned += D;
        expanded += cnt;
      }
      if (!grid_sync(ctl, bar, &s_flag)) break;
      // update over the touched vertices
      if (blockIdx.x == 0 && threadIdx.x == 0) st_vol(ctl->fr[qo], 0ull);  // queue qo is consumed
      const uint32_t tc = min(ld_vol(*tcount), n);
      for (uint32_t it = blockIdx.x * blockDim.x; it < tc; it += gs) {
        const uint32_t i = it + threadIdx.x;
        int32_t v = 0;
        u64 nwb = 0;
        uint32_t d = 0, a = 0;
        if (i < tc) {
          v = P.touched[i];
          const u64 x = LN::ld(P.next, (uint32_t)v);
          LN::st(P.next, (uint32_t)v, 0ull);
          const u64 sv = LN::ld(P.seen, (uint32_t)v);
          nwb = x & ~sv;
          if (nwb) {
            LN::st(P.seen, (uint32_t)v, sv | nwb);
            LN::st(nxt, (uint32_t)v, nwb);
            a = __ldg(g.off + v);
            d = __ldg(g.off + v + 1) - a;
            reached += __popcll(nwb);
          }
        }
        // scattered vertices: each lane writes its own rows
        u64 bits = nwb;
        while (bits) {
          const int bi = __ffsll((long long)bits) - 1;
          bits &= bits - 1;
          if (bi < k) rows[bi][v] = L;
        }
        stage_append(S, nwb != 0ull && d > 0, v, d, a);
        __syncthreads();
        stage_make_room(S, fout, ctl, blockDim.x);
      }
      stage_flush(S, fout, ctl);
    } else {
      // pull: owner-computes over CTA-contiguous word ranges; every entry of
      // nxt is written, so it needs no clearing
      if (blockIdx.x == 0 && threadIdx.x == 0) st_vol(ctl->fr[qo], 0ull);
      const uint32_t nwords = (n + 31) >> 5;
      const uint32_t per = (nwords + gridDim.x - 1) / gridDim.x;
      const uint32_t wlo = min(nwords, blockIdx.x * per), whi = min(nwords, wlo + per);
      for (uint32_t base = wlo; base < whi; base += nw) {
        const uint32_t wi = base + warp;
        const int32_t v = (int32_t)(wi * 32 + lane);
        const bool inr = wi < whi && (uint32_t)v < n;
        const u64 sv = inr ? LN::ld(P.seen, (uint32_t)v) : ALL;
        uint32_t s = 0, e = 0;
        bool cand = inr && sv != ALL;
        if (cand) {
          s = __ldg(g.off + v);
          e = __ldg(g.off + v + 1);
          cand = e > s;
        }
        u64 acc = 0;
        uint32_t kk = s;
        if (cand) {
          const uint32_t lim = min(e, s + (uint32_t)P.pull_serial);
          for (; kk < lim && ((acc | sv) != ALL); kk++) acc |= LN::ld(cur, (uint32_t)__ldg(g.tgt + kk));
          scanned += kk - s;
        }
        unsigned rm = __ballot_sync(kFull, cand && ((acc | sv) != ALL) && kk < e);
        while (rm) {
          const int l = __ffs(rm) - 1;
          rm &= rm - 1;
          const uint32_t ks = __shfl_sync(kFull, kk, l), ke = __shfl_sync(kFull, e, l);
          const u64 need = ALL & ~__shfl_sync(kFull, sv, l);
          u64 wacc = __shfl_sync(kFull, acc, l);
          uint32_t looked = 0;
          for (uint32_t c0 = ks; c0 < ke && ((wacc & need) != need); c0 += 32) {
            const uint32_t c = c0 + lane;
            const u64 x = (c < ke) ? LN::ld(cur, (uint32_t)__ldg(g.tgt + c)) : 0ull;
            const unsigned xl = __reduce_or_sync(kFull, (unsigned)x);
            const unsigned xh = __reduce_or_sync(kFull, (unsigned)(x >> 32));
            wacc |= ((u64)xh << 32) | xl;
            looked += min(32u, ke - c0);
          }
          if (lane == l) {
            acc = wacc;
            scanned += looked;
          }
        }
        const u64 nwb = acc & ~sv & ALL;
        if (inr) {
          LN::st(nxt, (uint32_t)v, nwb);
          if (nwb) {
            LN::st(P.seen, (uint32_t)v, sv | nwb);
            reached += __popcll(nwb);
          }
        }
        if (cand) pulled++;
        write_rows(rows, k, v, inr ? nwb : 0ull, L);
        stage_append(S, nwb != 0ull && e > s, v, e - s, s);
        __syncthreads();
        stage_make_room(S, fout, ctl, blockDim.x);
      }
      stage_flush(S, fout, ctl);
    }
    if (!grid_sync(ctl, bar, &s_flag)) break;
    fr = ld_vol(*outc);
    if (P.trace && blockIdx.x == 0 && threadIdx.x == 0 && L <= P.trace_cap)
      P.trace[L - 1] = TraceRec{L, dense ? 2 : 1, cnt, D, (long long)(globaltimer() - t_start), 0};
  }
  // lanes that never reached a vertex: GBF_INF
  if (ok) {
    const uint32_t nwords = (n + 31) >> 5;
    const uint32_t gw = gt >> 5, tw = gs >> 5;
    for (uint32_t wi = gw; wi < nwords; wi += tw) {
      const uint32_t v = wi * 32 + lane;
      const u64 miss = (v < n) ? (ALL & ~LN::ld(P.seen, v)) : 0ull;
      write_rows(rows, k, (int32_t)v, miss, kInf);
    }
  }
  unsigned long long tt;
  tt = block_sum64(scanned, S.misc64);
  if (threadIdx.x == 0 && tt) atomicAdd(&ctl->edges_scanned, tt);
  tt = block_sum64(expanded, S.misc64);
  if (threadIdx.x == 0 && tt) atomicAdd(&ctl->expanded, tt);
  tt = block_sum64(pulled, S.misc64);
  if (threadIdx.x == 0 && tt) atomicAdd(&ctl->pulled, tt);
  tt = block_sum64(reached, S.misc64);
  if (threadIdx.x == 0 && tt) atomicAdd(&ctl->reached, tt);
}

// Host side: a CUDA graph per workspace holding [parameter copy, control
// reset, cooperative kernel], replayed for every call with the same knobs.
gbf_status launch_msbfs_rows(Graph &g, Workspace &ws, const int32_t *srcs_host, int32_t k,
                             int32_t *const *rows, const Opts &o, cudaStream_t user_st) {
  static_assert(sizeof(MsCall) <= 1024, "parameter block size");
  // the previous replay must be done with the pinned parameter block
  if (ws.ms_done) GBF_CUDA(cudaEventSynchronize(ws.ms_done));
  MsCall *hc = (MsCall *)ws.ms_call_host;
  hc->g = g.dev();
  for (int i = 0; i < 64; i++) {
    hc->srcs[i] = i < k ? srcs_host[i] : 0;
    hc->rows[i] = i < k ? rows[i] : nullptr;
  }
  hc->k = k;
  hc->pad = 0;
  const bool narrow = k <= 8;  // 8-bit lanes
  const long long key[7] = {o.block, o.pull_divisor, o.heavy_cutoff, o.pull_serial, o.ctas,
                            o.spin_cap_ns, narrow ? 1 : 0};
  bool same = ws.ms_exec != nullptr;
  for (int i = 0; i < 7 && same; i++) same = ws.ms_key[i] == key[i];
  same = same && o.inject_wait == 0;
  if (!same) {
    if (ws.ms_exec) {
      cudaGraphExecDestroy(ws.ms_exec);
      ws.ms_exec = nullptr;
    }
    MsParams P;
    P.call = (const MsCall *)ws.ms_call;
    P.seen = ws.ms_seen;
    P.visit[0] = ws.ms_visit;
    P.visit[1] = ws.ms_visit + (size_t)ws.n;  // the workspace's size, not this graph's
    const void *kern = narrow ? (const void *)msbfs_kernel<uint8_t> : (const void *)msbfs_kernel<u64>;
    P.next = ws.ms_next;
    for (int i = 0; i < 3; i++) {
      P.q[i] = ws.ms_q[i];
      P.qoff[i] = ws.ms_qoff[i];
      P.qadj[i] = ws.ms_qadj[i];
      P.cs[i] = ws.ms_cs[i];
    }
    P.cs_cap = (uint32_t)(((uint64_t)ws.m + kFine - 1) / kFine + 2);
    P.touched = ws.ms_touched;
    P.ctl = ws.ctl;
    P.trace = ws.trace;
    P.trace_cap = ws.trace_cap;
    P.pull_divisor = o.pull_divisor;
    P.pull_serial = o.pull_serial;
    P.bmax = o.heavy_cutoff;
    P.cap = stage_capacity(o.block);
    P.inject_wait = o.inject_wait;
    P.cap_ns = o.spin_cap_ns;
    const size_t smem = push_smem_bytes(SmemShape{P.bmax, P.cap, 0, 0, 1});
    {
    const gbf_status sm = check_smem(smem, "msbfs_kernel");
    if (sm != GBF_OK) return sm;
  }
    GBF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GBF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, o.block, smem));
    if (per_sm < 1) {
      set_error("msbfs kernel does not fit on an SM with this block size");
      return GBF_ERR_INVALID;
    }
    int grid = per_sm * g.num_sms;
    if (o.ctas > 0 && o.ctas < grid) grid = o.ctas;
    ws.ms_grid = grid;
    cudaStream_t cs = ws.ms_stream;
    GBF_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaMemcpyAsync(ws.ms_call, ws.ms_call_host, sizeof(MsCall), cudaMemcpyHostToDevice, cs);
    cudaMemsetAsync(ws.ctl, 0, sizeof(Ctl), cs);
    cudaMemsetAsync(ws.trace, 0, sizeof(TraceRec) * (size_t)ws.trace_cap, cs);
    void *args[] = {&P};
    cudaError_t le = cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(o.block), args, smem, cs);
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (le != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail(le, "capture cooperative msbfs launch");
    }
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
    cudaError_t ie = cudaGraphInstantiate(&ws.ms_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      ws.ms_exec = nullptr;
      return cuda_fail(ie, "cudaGraphInstantiate");
    }
    for (int i = 0; i < 7; i++) ws.ms_key[i] = o.inject_wait ? -1 : key[i];
  }
  // order: user stream -> graph replay on the workspace stream -> user stream
  GBF_CUDA(cudaEventRecord(ws.ms_ready, user_st));
  GBF_CUDA(cudaStreamWaitEvent(ws.ms_stream, ws.ms_ready, 0));
  GBF_CUDA(cudaGraphLaunch(ws.ms_exec, ws.ms_stream));
  GBF_CUDA(cudaEventRecord(ws.ms_done, ws.ms_stream));
  GBF_CUDA(cudaStreamWaitEvent(user_st, ws.ms_done, 0));
  ws.last_kind = 3;
  ws.last_grid = ws.ms_grid;
  ws.last_block = o.block;
  return GBF_OK;
}

gbf_status launch_msbfs(Graph &g, Workspace &ws, const int32_t *srcs_host, int32_t k,
                        int32_t *dist, const Opts &o, cudaStream_t st) {
  int32_t *rows[64];
  for (int i = 0; i < 64; i++) rows[i] = i < k ? dist + (size_t)i * (size_t)g.n : nullptr;
  return launch_msbfs_rows(g, ws, srcs_host, k, rows, o, st);
}

int resident_ctas_per_sm_msbfs(const Opts &o) {
  const size_t smem = push_smem_bytes(SmemShape{o.heavy_cutoff, stage_capacity(o.block), 0, 0, 1});
  int best = 0;
  for (int w = 0; w < 2; w++) {  // the fewer of the two widths
    const void *kern = w ? (const void *)msbfs_kernel<uint8_t> : (const void *)msbfs_kernel<u64>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, o.block, smem) != cudaSuccess)
      return 0;
    best = w == 0 ? per_sm : std::min(best, per_sm);
  }
  return best;
}

}  // namespace gbf
