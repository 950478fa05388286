// Single-source betweenness centrality (§4 "Single-Source Betweenness
// Centrality"; Alg. 2) as one persistent cooperative kernel.
//   Forward: frontier rounds of the blocked sparse edgeMap (§6.2); each arc
//   (s, d) with d not visited before the round adds NumPaths[s] to
//   NumPaths[d] (fp64 fetch-and-add); d joins the next frontier at its
//   first contribution (the add that found 0).  Every frontier is kept, in
//   order, as a level of one array (vertices, degree prefix, first arcs,
//   chunk starts), so the backward pass can walk them again.
//   Backward: the levels in reverse.  For level L the coefficient
//   (1 + D[s]) / NumPaths[s] of each of its vertices is computed once
//   (stored over NumPaths[s], which no later step reads), then each arc
//   (s, d) with d one level up adds NumPaths[d] * coefficient to D[d]
//   (fp64 fetch-and-add).  "Not visited" in the backward edgeMap of Alg. 2
//   is exactly "one level up": the other neighbours of a level-L vertex
//   are on levels L and L+1, already marked.
// Readings: the source starts with one path and is visited before the first
// round; path counts and dependencies are fp64.
#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "gbf_impl.h"

namespace gbf {
using namespace dev;

struct LevelInfo {
  uint32_t lo, cnt, D, cs_lo;  // first entry, entries, degree sum, first chunk start
};

struct BcParams {
  DevGraph g;
  int32_t src;
  double *dep;       // output D
  double *paths;     // NumPaths, then the backward coefficients
  int32_t *lvl;      // hop level, -1 if not reached
  int32_t *order;    // all levels, one after another
  uint32_t *offs;    // degree prefix within the level
  uint32_t *adj;     // first arc
  uint32_t *cs;      // chunk starts of all levels
  uint32_t cs_total;
  LevelInfo *info;
  int max_levels;
  Ctl *ctl;
  TraceRec *trace;
  int trace_cap;
  int bmax;
  int cap;
  int inject_wait;
  long long cap_ns;
};

namespace {

// PathUpdate of Alg. 2 for kU windows: targets, their levels, then the
// fetch-and-adds of the source's path count into the targets not visited
// before this round; a target whose add found 0 is new this round.
struct PathFn {
  static constexpr int kWin = kU;
  template <class Sink>
  __device__ __forceinline__ void drain(Sink &, PushSmem &) {}
  const uint32_t *off;
  const int32_t *tgt;
  double *paths;
  int32_t *lvl;
  int32_t round;
  unsigned long long reached;
  template <class Sink>
  __device__ __forceinline__ void batch(const bool *ok, const int32_t *u, const uint32_t *idx,
                                        Sink &sink, PushSmem &S) {
    int32_t v[kU], lv[kU];
#pragma unroll
    for (int r = 0; r < kU; r++) v[r] = ok[r] ? __ldg(tgt + idx[r]) : 0;
#pragma unroll
    for (int r = 0; r < kU; r++) lv[r] = ok[r] ? __ldcg(lvl + v[r]) : 0;
    bool win[kU];
#pragma unroll
    for (int r = 0; r < kU; r++) {
      win[r] = false;
      if (ok[r] && (lv[r] < 0 || lv[r] == round)) {
        const double prev = atomicAdd(paths + v[r], __ldcg(paths + u[r]));
        if (prev == 0.0) {
          win[r] = true;
          lvl[v[r]] = round;
          reached++;
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
      z[r] -= a[r];
      emit[r] = win[r];  // every level vertex is walked again backwards
    }
    sink.template append_n<kU>(S, emit, v, z, a);
  }
};

// DependencyUpdate of Alg. 2 for kU windows of arcs out of level L: each
// target one level up gets NumPaths[d] * (1 + D[s]) / NumPaths[s].
struct DepFn {
  static constexpr int kWin = kU;
  template <class Sink>
  __device__ __forceinline__ void drain(Sink &, PushSmem &) {}
  const int32_t *tgt;
  const double *coef;  // per level-L vertex: (1 + D[s]) / NumPaths[s]
  const double *paths;
  const int32_t *lvl;
  double *dep;
  int32_t up;  // L - 1
  template <class Sink>
  __device__ __forceinline__ void batch(const bool *ok, const int32_t *u, const uint32_t *idx,
                                        Sink &, PushSmem &) {
    int32_t d[kU];
    bool hit[kU];
#pragma unroll
    for (int r = 0; r < kU; r++) d[r] = ok[r] ? __ldg(tgt + idx[r]) : 0;
    // levels, path counts and coefficients were written earlier in this
    // launch: read them at L2 (.cg), not through the read-only path
#pragma unroll
    for (int r = 0; r < kU; r++) hit[r] = ok[r] && __ldcg(lvl + d[r]) == up;
#pragma unroll
    for (int r = 0; r < kU; r++)
      if (hit[r]) atomicAdd(dep + d[r], __ldcg(paths + d[r]) * __ldcg(coef + u[r]));
  }
};

// Sink of the backward edgeMap: nothing is emitted.
struct NoSink {
  template <int U>
  __device__ __forceinline__ void append_n(PushSmem &, const bool *, const int32_t *,
                                           const uint32_t *, const uint32_t *) {}
  __device__ __forceinline__ void chunk_end(PushSmem &) { __syncthreads(); }
};

}  // namespace

__global__ void __launch_bounds__(1024) bc_kernel(BcParams P) {
  extern __shared__ unsigned long long smem_raw[];
  __shared__ int s_flag;
  PushSmem S = carve_push_smem(smem_raw, SmemShape{P.bmax, P.cap, 0, 0, 1});
  if (threadIdx.x == 0) S.misc[0] = 0;
  Ctl *ctl = P.ctl;
  Barrier bar{0u, P.cap_ns};
  const DevGraph g = P.g;
  const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  const int32_t src = P.src;
  unsigned long long scanned = 0, reached = 0;
  const unsigned long long t_start = globaltimer();

  for (uint32_t i = gt; i < (uint32_t)g.n; i += gs) {
    const bool s = i == (uint32_t)src;
    P.dep[i] = 0.0;
    P.paths[i] = s ? 1.0 : 0.0;
    P.lvl[i] = s ? 0 : -1;
  }
  // level 0: the source (if it has arcs)
  const uint32_t a0 = __ldg(g.off + src), d0 = __ldg(g.off + src + 1) - a0;
  if (blockIdx.x == 0) {
    if (threadIdx.x == 0) {
      P.order[0] = src;
      P.offs[0] = 0;
      P.adj[0] = a0;
      reached = 1;
    }
    for (uint32_t c = threadIdx.x; c < (d0 + kFine - 1) / kFine; c += blockDim.x)
      if (c < P.cs_total) P.cs[c] = 0;
  }
  if (P.inject_wait && blockIdx.x == 0 && threadIdx.x == 0) injected_wait(ctl, P.cap_ns);
  __syncthreads();
  bool ok = grid_sync(ctl, bar, &s_flag);

  // ---------------- forward
  LevelInfo cur{0u, d0 > 0 ? 1u : 0u, d0, 0u};
  int levels = 0;  // levels 0 .. levels-1 are recorded (nonempty)
  int bem = 0;
  for (int32_t r = 1; ok && cur.cnt > 0; r++) {
    if (levels >= P.max_levels) {
      if (threadIdx.x == 0) raise_error(ctl, GBF_ERR_OVERFLOW, 20);
      ok = false;
      break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      P.info[levels] = cur;
      st_vol(ctl->fr[(r + 1) % 3], 0ull);
      atomicAdd(&ctl->rounds, 1);
      atomicAdd(&ctl->push_rounds, 1);
      scanned += cur.D;
    }
    levels++;
    const LevelInfo nxt{cur.lo + cur.cnt, 0u, 0u, cur.cs_lo + (cur.D + kFine - 1) / kFine + 1};
    unsigned long long *outc = &ctl->fr[r % 3];
    QueueIn in{P.order + cur.lo, P.offs + cur.lo, P.adj + cur.lo, P.cs + cur.cs_lo, cur.cnt, cur.D};
    PathFn fn{g.off, g.tgt, P.paths, P.lvl, r, 0};
    StagedSink sink{QueueOut{P.order + nxt.lo, P.offs + nxt.lo, P.adj + nxt.lo, P.cs + nxt.cs_lo,
                             outc, (uint32_t)g.n - nxt.lo,
                             nxt.cs_lo < P.cs_total ? P.cs_total - nxt.cs_lo : 0u},
                    ctl, nullptr};
    blocked_edge_map(g, in, chunk_shift(cur.D, 4u, chunk_shift_cap(PathFn::kWin * blockDim.x)),
                     (uint32_t)P.bmax, S, fn, sink, ctl, bem++);
    sink.finish(S);
    reached += fn.reached;
    if (!grid_sync(ctl, bar, &s_flag)) {
      ok = false;
      break;
    }
    const unsigned long long fr = ld_vol(*outc);
    if (P.trace && blockIdx.x == 0 && threadIdx.x == 0 && r <= P.trace_cap)
      P.trace[r - 1] = TraceRec{r, 1, cur.cnt, cur.D, (long long)(globaltimer() - t_start), 0};
    cur = LevelInfo{nxt.lo, (uint32_t)(fr >> 32), (uint32_t)fr, nxt.cs_lo};
  }

  // ---------------- backward over levels levels-1 .. 1
  for (int L = levels - 1; ok && L >= 1; L--) {
    const LevelInfo li = P.info[L];
    for (uint32_t i = gt; i < li.cnt; i += gs) {
      const int32_t s = P.order[li.lo + i];
      P.paths[s] = (1.0 + P.dep[s]) / P.paths[s];
    }
    if (!grid_sync(ctl, bar, &s_flag)) break;
    QueueIn in{P.order + li.lo, P.offs + li.lo, P.adj + li.lo, P.cs + li.cs_lo, li.cnt, li.D};
    DepFn fn{g.tgt, P.paths, P.paths, P.lvl, P.dep, L - 1};
    NoSink sink;
    blocked_edge_map(g, in, chunk_shift(li.D, 4u, 8), (uint32_t)P.bmax, S, fn, sink, ctl, bem++);
    if (blockIdx.x == 0 && threadIdx.x == 0) scanned += li.D;
    if (!grid_sync(ctl, bar, &s_flag)) break;
  }
  unsigned long long t;
  t = block_sum64(scanned, S.misc64);
  if (threadIdx.x == 0 && t) atomicAdd(&ctl->edges_scanned, t);
  t = block_sum64(reached, S.misc64);
  if (threadIdx.x == 0 && t) atomicAdd(&ctl->reached, t);
}

gbf_status launch_bc(Graph &g, Workspace &ws, int32_t src, double *dep, const Opts &o,
                     cudaStream_t st) {
  BcParams P;
  P.g = g.dev();
  P.src = src;
  P.dep = dep;
  P.paths = ws.bc_paths;
  P.lvl = ws.bc_lvl;
  P.order = ws.q[0];
  P.offs = ws.qoff[0];
  P.adj = ws.qadj[0];
  P.cs = ws.bc_cs;
  P.cs_total = ws.bc_cs_total;
  P.info = (LevelInfo *)ws.bc_info;
  P.max_levels = ws.bc_max_levels;
  P.ctl = ws.ctl;
  P.trace = ws.trace;
  P.trace_cap = ws.trace_cap;
  P.bmax = o.heavy_cutoff;
  P.cap = stage_capacity(o.block);
  P.inject_wait = o.inject_wait;
  P.cap_ns = o.spin_cap_ns;
  const size_t smem = push_smem_bytes(SmemShape{P.bmax, P.cap, 0, 0, 1});
  {
    const gbf_status sm = check_smem(smem, "bc_kernel");
    if (sm != GBF_OK) return sm;
  }
  GBF_CUDA(cudaFuncSetAttribute(bc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  GBF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bc_kernel, o.block, smem));
  if (per_sm < 1) {
    set_error("bc kernel does not fit on an SM with this block size");
    return GBF_ERR_INVALID;
  }
  int grid = per_sm * g.num_sms;
  if (o.ctas > 0 && o.ctas < grid) grid = o.ctas;
  GBF_CUDA(cudaMemsetAsync(ws.ctl, 0, sizeof(Ctl), st));
  if (ws.trace) GBF_CUDA(cudaMemsetAsync(ws.trace, 0, sizeof(TraceRec) * (size_t)ws.trace_cap, st));
  void *args[] = {&P};
  GBF_CUDA(cudaLaunchCooperativeKernel((const void *)bc_kernel, dim3(grid), dim3(o.block), args,
                                       smem, st));
  ws.last_kind = 5;
  ws.last_grid = grid;
  ws.last_block = o.block;
  return GBF_OK;
}

}  // namespace gbf

using namespace gbf;

extern "C" gbf_status gbf_betweenness(gbf_graph *h, int32_t src, double *dep, int mem,
                                      const gbf_options *opt, void *cuda_stream) {
  if (!h || !dep) return set_error("graph or dep is NULL"), GBF_ERR_INVALID;
  Graph &g = h->g;
  if (src < 0 || src >= g.n) return set_error("src out of range"), GBF_ERR_INVALID;
  if (mem != GBF_HOST && mem != GBF_DEVICE) return set_error("bad mem"), GBF_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  std::lock_guard<std::mutex> lk(g.mu);
  const Opts o = resolve(opt, g, GBF_TUNE_BFS);
  {
    const gbf_status s = ws_ensure_bc(g, g.ws);
    if (s != GBF_OK) return s;
  }
  double *dd = mem == GBF_HOST ? g.ws.bc_out_tmp : dep;
  {
    const gbf_status s = launch_bc(g, g.ws, src, dd, o, st);
    if (s != GBF_OK) return s;
  }
  if (mem == GBF_DEVICE) return GBF_OK;
  GBF_CUDA(cudaMemcpyAsync(dep, dd, sizeof(double) * (size_t)g.n, cudaMemcpyDeviceToHost, st));
  return ws_collect(g.ws, st, nullptr);
}
