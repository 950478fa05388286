// Multi-source integral-weight SSSP: up to 8 single-source shortest-path
// problems (§4 "Integral-Weight SSSP") on one graph advanced together as the
// frontier rounds of Bellman-Ford (Alg. 4), one int32 distance lane per
// source.  The lanes of a vertex sit next to each other (32 bytes, one
// sector), so one read of an arc and of its target's lanes serves every
// source at once, and all sources share each round's barrier: the rounds
// number about the largest hop count of a shortest path (a dozen on the
// RMAT graphs) instead of one bucket round per distance value per source.
//
// Round r: the frontier queue holds every vertex some lane improved in round
// r-1, and imp[(r-1) % 3][v] says which lanes.  For an arc (u, v, w) of the
// frontier, each such lane i proposes D_i[u] + w (u's lane read now: it may
// have improved since) and writes it into D_i[v] with writeMin when smaller;
// the lanes that improved are OR-ed into imp[r % 3][v] (a byte per vertex,
// four vertices per 32-bit word), and the OR that finds v's byte empty puts
// v on the next frontier (the test-and-set of Alg. 4).  imp[(r + 1) % 3],
// last read in round r-1, is cleared during round r (ResetFlags).  A vertex
// of degree 1 improved through its only neighbour cannot improve it back and
// is not expanded.  Weights are >= 1 on a symmetric graph, so there is no
// negative cycle and the rounds end when no lane improves.
//
// Results are the unique shortest-path distances of each source, the same
// as the single-source weighted BFS; unreachable vertices get GBF_INF.
#include <cuda_runtime.h>

#include <algorithm>

#include "dev_common.cuh"
#include "gbf_impl.h"

namespace gbf {
using namespace dev;

constexpr int kMsspLanes = 8;

struct MsspParams {
  DevGraph g;
  int32_t srcs[kMsspLanes];
  int32_t *rows[kMsspLanes];  // rows[i][v] = distance of v from srcs[i]
  int32_t k;
  int32_t *dd;       // n x kMsspLanes distances, vertex-major (32-byte rows)
  unsigned *imp[3];  // lanes improved in round r % 3: byte v & 3 of word v >> 2
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

__device__ __forceinline__ unsigned lane_byte(const unsigned *words, uint32_t v) {
  return (__ldcg(words + (v >> 2)) >> (8u * (v & 3u))) & 0xffu;
}

// The 8 lanes of vertex v (two 16-byte loads at L2: other SMs lower them).
__device__ __forceinline__ void load_lanes(const int32_t *dd, uint32_t v, int32_t (&x)[kMsspLanes]) {
  const int4 *p = reinterpret_cast<const int4 *>(dd + (size_t)v * kMsspLanes);
  const int4 a = __ldcg(p), b = __ldcg(p + 1);
  x[0] = a.x;
  x[1] = a.y;
  x[2] = a.z;
  x[3] = a.w;
  x[4] = b.x;
  x[5] = b.y;
  x[6] = b.z;
  x[7] = b.w;
}

// Update of Alg. 4 for the lanes of kWin windows of frontier arcs.
struct MsspFn {
  static constexpr int kWin = 2;  // windows per walk step (each carries 16 lane values)
  template <class Sink>
  __device__ __forceinline__ void drain(Sink &, PushSmem &) {}  // nothing deferred
  const uint32_t *off;
  const int32_t *tgt;
  const uint32_t *w;
  int32_t *dd;
  const unsigned *lanes_in;
  unsigned *imp_out;
  unsigned long long relax;
  template <class Sink>
  __device__ __forceinline__ void batch(const bool *ok, const int32_t *u, const uint32_t *idx,
                                        Sink &sink, PushSmem &S) {
    int32_t v[kWin], wt[kWin];
    unsigned lm[kWin];
#pragma unroll
    for (int r = 0; r < kWin; r++) {
      v[r] = 0;
      wt[r] = 0;
      lm[r] = 0;
      if (ok[r]) {
        v[r] = __ldg(tgt + idx[r]);
        wt[r] = (int32_t)__ldg(w + idx[r]);
        lm[r] = lane_byte(lanes_in, (uint32_t)u[r]);
      }
    }
    bool win[kWin];
    uint32_t a[kWin], z[kWin];
#pragma unroll
    for (int r = 0; r < kWin; r++) {
      win[r] = false;
      a[r] = z[r] = 0;
      if (lm[r]) {
        int32_t du[kMsspLanes], dv[kMsspLanes];
        load_lanes(dd, (uint32_t)u[r], du);
        load_lanes(dd, (uint32_t)v[r], dv);
        unsigned better = 0;
#pragma unroll
        for (int i = 0; i < kMsspLanes; i++) {
          if ((lm[r] >> i) & 1u) {
            const int32_t c = du[i] + wt[r];  // du[i] < INF: u improved in lane i
            if (c < dv[i] && atomicMin(dd + (size_t)v[r] * kMsspLanes + i, c) > c) better |= 1u << i;
          }
        }
        if (better) {
          relax += __popc(better);
          const unsigned sh = 8u * ((uint32_t)v[r] & 3u);
          const unsigned old = atomicOr(imp_out + ((uint32_t)v[r] >> 2), better << sh);
          win[r] = ((old >> sh) & 0xffu) == 0u;  // v's first improvement this round
        }
      }
      if (win[r]) {
        a[r] = __ldg(off + v[r]);
        z[r] = __ldg(off + v[r] + 1);
      }
    }
    bool emit[kWin];
#pragma unroll
    for (int r = 0; r < kWin; r++) {
      z[r] -= a[r];  // degree
      emit[r] = win[r] && z[r] >= 2;
    }
    sink.template append_n<kWin>(S, emit, v, z, a);
  }
};

}  // namespace

__global__ void __launch_bounds__(1024) mssp_kernel(MsspParams P) {
  extern __shared__ unsigned long long smem_raw[];
  __shared__ int s_flag;
  PushSmem S = carve_push_smem(smem_raw, SmemShape{P.bmax, P.cap, 0, 0, 1});
  if (threadIdx.x == 0) S.misc[0] = 0;
  Ctl *ctl = P.ctl;
  Barrier bar{0u, P.cap_ns};
  const DevGraph g = P.g;
  const uint32_t n = (uint32_t)g.n;
  const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  const uint32_t nw4 = (n + 3) >> 2;
  const int k = P.k;
  unsigned long long scanned = 0, expanded = 0, relax = 0;
  const unsigned long long t_start = globaltimer();

  // every lane unreached, no lane improved anywhere
  for (uint32_t i = gt; i < n * 2u; i += gs)
    reinterpret_cast<int4 *>(P.dd)[i] = make_int4(kInf, kInf, kInf, kInf);
  for (uint32_t i = gt; i < nw4; i += gs) {
    P.imp[0][i] = 0u;
    P.imp[1][i] = 0u;
    P.imp[2][i] = 0u;
  }
  if (P.inject_wait && blockIdx.x == 0 && threadIdx.x == 0) injected_wait(ctl, P.cap_ns);
  bool ok = grid_sync(ctl, bar, &s_flag);
  // sources: D_i[srcs[i]] = 0, lane i improved at its source in round 0; the
  // first frontier holds each distinct source with at least one arc
  if (ok && blockIdx.x == 0) {
    bool emit = false;
    int32_t s = 0;
    uint32_t d = 0, a = 0;
    if ((int)threadIdx.x < k) {
      s = P.srcs[threadIdx.x];
      P.dd[(size_t)s * kMsspLanes + threadIdx.x] = 0;
      atomicOr(P.imp[0] + ((uint32_t)s >> 2), (1u << threadIdx.x) << (8u * ((uint32_t)s & 3u)));
      bool dup = false;
      for (int j = 0; j < (int)threadIdx.x; j++) dup |= P.srcs[j] == s;
      a = __ldg(g.off + s);
      d = __ldg(g.off + s + 1) - a;
      emit = !dup && d > 0;
    }
    stage_append(S, emit, s, d, a);  // whole CTA: warp-collective
    stage_flush(S, QueueOut{P.q[0], P.qoff[0], P.qadj[0], P.cs[0], &ctl->fr[0], n, P.cs_cap}, ctl);
  }
  ok = ok && grid_sync(ctl, bar, &s_flag);

  int qb = 0, bem = 0;
  unsigned long long fr = ok ? ld_vol(ctl->fr[0]) : 0ull;
  for (int32_t round = 1; ok && round <= g.n; round++) {
    const uint32_t cnt = (uint32_t)(fr >> 32), D = (uint32_t)fr;
    if (cnt == 0) break;
    unsigned long long *outc = &ctl->fr[round % 3];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st_vol(ctl->fr[(round + 1) % 3], 0ull);
      atomicAdd(&ctl->rounds, 1);
      atomicAdd(&ctl->push_rounds, 1);
      scanned += D;
      expanded += cnt;
    }
    // ResetFlags: the lane masks of round r-2, last read in round r-1
    unsigned *stale = P.imp[(round + 1) % 3];
    for (uint32_t i = gt; i < nw4; i += gs) stale[i] = 0u;
    QueueIn in{P.q[qb], P.qoff[qb], P.qadj[qb], P.cs[qb], cnt, D};
    MsspFn fn{g.off, g.tgt, g.w, P.dd, P.imp[(round - 1) % 3], P.imp[round % 3], 0};
    StagedSink sink{QueueOut{P.q[qb ^ 1], P.qoff[qb ^ 1], P.qadj[qb ^ 1], P.cs[qb ^ 1], outc, n,
                             P.cs_cap},
                    ctl, nullptr};
    blocked_edge_map(g, in, chunk_shift(D, 4u, chunk_shift_cap(MsspFn::kWin * blockDim.x)),
                     (uint32_t)P.bmax, S, fn, sink, ctl, bem++);
    sink.finish(S);
    relax += fn.relax;
    qb ^= 1;
    if (!grid_sync(ctl, bar, &s_flag)) break;
    fr = ld_vol(*outc);
    if (P.trace && blockIdx.x == 0 && threadIdx.x == 0 && round <= P.trace_cap)
      P.trace[round - 1] = TraceRec{round, 1, cnt, D, (long long)(globaltimer() - t_start), 0};
  }
  // each lane's row of the output (consecutive vertices: coalesced per row)
  if (ok && ld_vol(ctl->err) == 0) {
    for (uint32_t v = gt; v < n; v += gs) {
      int32_t x[kMsspLanes];
      load_lanes(P.dd, v, x);
#pragma unroll
      for (int i = 0; i < kMsspLanes; i++)
        if (i < k) P.rows[i][v] = x[i];
    }
  }
  unsigned long long t;
  t = block_sum64(scanned, S.misc64);
  if (threadIdx.x == 0 && t) atomicAdd(&ctl->edges_scanned, t);
  t = block_sum64(expanded, S.misc64);
  if (threadIdx.x == 0 && t) atomicAdd(&ctl->expanded, t);
  t = block_sum64(relax, S.misc64);
  if (threadIdx.x == 0 && t) atomicAdd(&ctl->relax, t);
}

gbf_status ws_ensure_mssp(Graph &g, Workspace &ws, bool host_out) {
  gbf_status s = ws_ensure_base(g, ws);
  if (s != GBF_OK) return s;
  const size_t n = (size_t)g.n;
  size_t acc = 0;
  if (!ws.mssp_dd) {
    cudaError_t e = cudaMalloc((void **)&ws.mssp_dd, sizeof(int32_t) * kMsspLanes * std::max<size_t>(n, 1));
    if (e != cudaSuccess) {
      ws.mssp_dd = nullptr;
      return cuda_fail(e, "cudaMalloc");
    }
    acc += sizeof(int32_t) * kMsspLanes * n;
    const size_t w4 = (n + 3) / 4;
    e = cudaMalloc((void **)&ws.mssp_imp, sizeof(unsigned) * 3 * std::max<size_t>(w4, 1));
    if (e != cudaSuccess) {
      ws.mssp_imp = nullptr;
      return cuda_fail(e, "cudaMalloc");
    }
    acc += sizeof(unsigned) * 3 * w4;
  }
  if (host_out && !ws.mssp_out_tmp) {
    cudaError_t e = cudaMalloc((void **)&ws.mssp_out_tmp, sizeof(int32_t) * kMsspLanes * std::max<size_t>(n, 1));
    if (e != cudaSuccess) {
      ws.mssp_out_tmp = nullptr;
      return cuda_fail(e, "cudaMalloc");
    }
    acc += sizeof(int32_t) * kMsspLanes * n;
  }
  ws.bytes += acc;
  return GBF_OK;
}

gbf_status launch_mssp_rows(Graph &g, Workspace &ws, const int32_t *srcs_host, int32_t k,
                            int32_t *const *rows, const Opts &o, cudaStream_t st) {
  if (k < 1 || k > kMsspLanes) return set_error("k must be in [1, 8]"), GBF_ERR_INVALID;
  if (!ws.mssp_dd || !ws.mssp_imp) return set_error("no multi-source SSSP workspace"), GBF_ERR_INVALID;
  MsspParams P;
  P.g = g.dev();
  for (int i = 0; i < kMsspLanes; i++) {
    P.srcs[i] = i < k ? srcs_host[i] : 0;
    P.rows[i] = i < k ? rows[i] : nullptr;
  }
  P.k = k;
  P.dd = ws.mssp_dd;
  const size_t w4 = ((size_t)ws.n + 3) / 4;  // the workspace's size, not this graph's
  for (int i = 0; i < 3; i++) P.imp[i] = ws.mssp_imp + (size_t)i * w4;
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
    const gbf_status sm = check_smem(smem, "mssp_kernel");
    if (sm != GBF_OK) return sm;
  }
  GBF_CUDA(cudaFuncSetAttribute(mssp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  GBF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mssp_kernel, o.block, smem));
  if (per_sm < 1) {
    set_error("mssp kernel does not fit on an SM with this block size");
    return GBF_ERR_INVALID;
  }
  int grid = per_sm * g.num_sms;
  if (o.ctas > 0 && o.ctas < grid) grid = o.ctas;
  GBF_CUDA(cudaMemsetAsync(ws.ctl, 0, sizeof(Ctl), st));
  if (ws.trace) GBF_CUDA(cudaMemsetAsync(ws.trace, 0, sizeof(TraceRec) * (size_t)ws.trace_cap, st));
  void *args[] = {&P};
  GBF_CUDA(cudaLaunchCooperativeKernel((const void *)mssp_kernel, dim3(grid), dim3(o.block), args,
                                       smem, st));
  ws.last_kind = 5;
  ws.last_grid = grid;
  ws.last_block = o.block;
  return GBF_OK;
}

int resident_ctas_per_sm_mssp(const Opts &o) {
  const size_t smem = push_smem_bytes(SmemShape{o.heavy_cutoff, stage_capacity(o.block), 0, 0, 1});
  if (cudaFuncSetAttribute(mssp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mssp_kernel, o.block, smem) != cudaSuccess)
    return 0;
  return per_sm;
}

}  // namespace gbf

using namespace gbf;

extern "C" gbf_status gbf_mssp(gbf_graph *h, const int32_t *srcs, int32_t k, int32_t *dist,
                               int mem, const gbf_options *opt, void *cuda_stream) {
  if (!h || !srcs || !dist) return set_error("graph, srcs or dist is NULL"), GBF_ERR_INVALID;
  Graph &g = h->g;
  if (!g.w) return set_error("graph has no weights"), GBF_ERR_INVALID;
  if (k < 1 || k > kMsspLanes) return set_error("k must be in [1, 8]"), GBF_ERR_INVALID;
  for (int i = 0; i < k; i++)
    if (srcs[i] < 0 || srcs[i] >= g.n) return set_error("source out of range"), GBF_ERR_INVALID;
  if (mem != GBF_HOST && mem != GBF_DEVICE) return set_error("bad mem"), GBF_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  std::lock_guard<std::mutex> lk(g.mu);
  {
    const gbf_status s = ws_ensure_mssp(g, g.ws, mem == GBF_HOST);
    if (s != GBF_OK) return s;
  }
  const Opts o = resolve(opt, g, GBF_TUNE_BFS);
  int32_t *base = mem == GBF_HOST ? g.ws.mssp_out_tmp : dist;
  int32_t *rows[kMsspLanes];
  for (int i = 0; i < kMsspLanes; i++) rows[i] = i < k ? base + (size_t)i * (size_t)g.n : nullptr;
  {
    const gbf_status s = launch_mssp_rows(g, g.ws, srcs, k, rows, o, st);
    if (s != GBF_OK) return s;
  }
  if (mem == GBF_DEVICE) return GBF_OK;
  GBF_CUDA(cudaMemcpyAsync(dist, base, sizeof(int32_t) * (size_t)k * (size_t)g.n,
                           cudaMemcpyDeviceToHost, st));
  return ws_collect(g.ws, st, nullptr);
}
