// Low-diameter decomposition (§4 "Low-Diameter Decomposition"; Alg. 6, the
// Miller-Peng-Xu clustering) as one persistent cooperative kernel.
//
// The shifts delta[v] ~ Exp(beta) are an input.  Vertex v may start its own
// cluster in round s(v) = floor(max delta - delta[v]) unless a search has
// reached it by then; in every round each frontier vertex hands its cluster
// to its unclaimed neighbours (compare-and-swap on C, the Update of Alg. 6),
// and the claimed neighbours form the next frontier.  Per round:
//   - a vertex pass: unclaimed vertices whose start round has come become
//     centres (C[v] = v, T[v] = round) and join the frontier queue that the
//     previous round's edgeMap filled (CTA-staged compaction);
//   - the blocked sparse edgeMap over that queue: an unclaimed neighbour d
//     of u takes C[u] by atomicCAS; the winner records T[d] = round + 1 and
//     joins the next queue.
// Until v is claimed, T[v] holds -(s(v)) - 1, so no array beyond the outputs
// is needed.  The loop ends when every vertex is claimed: each CTA adds up
// the per-round claim counts (triple-buffered, so the count it reads after a
// barrier is not being written), and all reach n in the same round.  T is
// unique; where searches reach a vertex in the same round, which cluster
// wins is not.
#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "gbf_impl.h"

namespace gbf {
using namespace dev;

struct LddParams {
  DevGraph g;
  const double *delta;
  int32_t *C;  // cluster centre of each vertex (-1: unclaimed)
  int32_t *T;  // round in which the vertex joined a frontier (-(start) - 1 before)
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

constexpr int32_t kMaxStart = 1 << 22;  // start rounds beyond this are rejected

// Block-wide maximum of a 64-bit value (result valid in thread 0).
__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long x,
                                                            unsigned long long *s_tmp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) x = max(x, __shfl_down_sync(kFull, x, d));
  if (lane == 0) s_tmp[warp] = x;
  __syncthreads();
  unsigned long long r = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < nw; i++) r = max(r, s_tmp[i]);
  __syncthreads();
  return r;
}

// Update of Alg. 6 over kU windows of arcs out of the frontier.
struct ClaimFn {
  static constexpr int kWin = kU;
  template <class Sink>
  __device__ __forceinline__ void drain(Sink &, PushSmem &) {}
  const uint32_t *off;
  const int32_t *tgt;
  int32_t *C;
  int32_t *T;
  int32_t next_round;
  unsigned long long claimed;
  template <class Sink>
  __device__ __forceinline__ void batch(const bool *ok, const int32_t *uu, const uint32_t *idx,
                                        Sink &sink, PushSmem &S) {
    int32_t v[kU], cu[kU];
#pragma unroll
    for (int r = 0; r < kU; r++) {
      v[r] = ok[r] ? __ldg(tgt + idx[r]) : 0;
      cu[r] = ok[r] ? __ldcg(C + uu[r]) : -1;  // the frontier vertex's cluster (set)
    }
    bool win[kU];
#pragma unroll
    for (int r = 0; r < kU; r++)
      win[r] = ok[r] && cu[r] >= 0 && __ldcg(C + v[r]) < 0 && atomicCAS(C + v[r], -1, cu[r]) == -1;
    uint32_t a[kU], z[kU];
#pragma unroll
    for (int r = 0; r < kU; r++) {
      a[r] = z[r] = 0;
      if (win[r]) {
        T[v[r]] = next_round;
        claimed++;
        a[r] = __ldg(off + v[r]);
        z[r] = __ldg(off + v[r] + 1);
      }
      z[r] -= a[r];
    }
    sink.template append_n<kU>(S, win, v, z, a);
  }
};

}  // namespace

__global__ void __launch_bounds__(1024) ldd_kernel(LddParams P) {
  extern __shared__ unsigned long long smem_raw[];
  __shared__ int s_flag, s_err;
  PushSmem S = carve_push_smem(smem_raw, SmemShape{P.bmax, P.cap, 0, 0, 1});
  if (threadIdx.x == 0) S.misc[0] = 0;
  Ctl *ctl = P.ctl;
  Barrier bar{0u, P.cap_ns};
  const DevGraph g = P.g;
  const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  const uint32_t n = (uint32_t)g.n;
  unsigned long long scanned = 0, claimed = 0;
  const unsigned long long t_start = globaltimer();

  // max delta: shifts are finite and >= 0, so their IEEE bit patterns order
  // like their values and a 64-bit atomicMax finds the maximum
  {
    unsigned long long mx = 0;
    bool bad = false;
    for (uint32_t v = gt; v < n; v += gs) {
      const double d = P.delta[v];
      if (!(d >= 0.0) || !(d <= 1.0e300)) bad = true;  // negative, NaN or infinite
      else mx = max(mx, (unsigned long long)__double_as_longlong(d));
    }
    if (bad) raise_error(ctl, GBF_ERR_INVALID, 30);
    mx = block_max_u64(mx, S.misc64);
    if (threadIdx.x == 0 && mx) atomicMax(&ctl->conv, mx);
  }
  if (P.inject_wait && blockIdx.x == 0 && threadIdx.x == 0) injected_wait(ctl, P.cap_ns);
  __syncthreads();
  bool ok = grid_sync(ctl, bar, &s_flag);
  if (ok) {
    const double dmax = __longlong_as_double((long long)ld_vol(ctl->conv));
    for (uint32_t v = gt; v < n; v += gs) {
      const double s = floor(dmax - P.delta[v]);
      if (s > (double)kMaxStart) raise_error(ctl, GBF_ERR_INVALID, 31);
      const int32_t si = s <= 0.0 ? 0 : (s > (double)kMaxStart ? kMaxStart : (int32_t)s);
      P.C[v] = -1;
      P.T[v] = -si - 1;
    }
    __syncthreads();
    ok = grid_sync(ctl, bar, &s_flag);
    // invalid shifts: stop before any round (one read per CTA, so its threads agree)
    if (threadIdx.x == 0) s_err = ld_vol(ctl->err);
    __syncthreads();
    if (ok && s_err != 0) ok = false;
  }

  // CTA-contiguous vertex ranges for the centre passes
  const uint32_t per = (n + gridDim.x - 1) / gridDim.x;
  const uint32_t vlo = min(n, blockIdx.x * per), vhi = min(n, vlo + per);
  // Counter slots.  fr[sub % 3] counts the queue being filled for the
  // current round; scnt[r % 3] counts the claims of round r's centre pass and
  // of round r - 1's edgeMap.  Each round zeroes the slots the next round's
  // edgeMap fills, last read two barriers earlier.
  int bem = 0, sub = 0, qb = 0;
  unsigned long long total = 0;  // vertices claimed so far (identical in every CTA)
  for (int32_t r = 0; ok; r++) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st_vol(ctl->fr[(sub + 1) % 3], 0ull);
      st_vol(ctl->scnt[(r + 1) % 3], 0u);
    }
    // ---------------- centres whose start round has come
    {
      QueueOut out{P.q[qb], P.qoff[qb], P.qadj[qb], P.cs[qb], &ctl->fr[sub % 3], n, P.cs_cap};
      unsigned int mine = 0;
      for (uint32_t base = vlo; base < vhi; base += blockDim.x) {
        const uint32_t v = base + threadIdx.x;
        bool start = false;
        uint32_t a = 0, d = 0;
        if (v < vhi && __ldcg(P.C + v) < 0 && -__ldcg(P.T + v) - 1 <= r) {
          start = true;
          P.C[v] = (int32_t)v;  // unclaimed: nobody else writes it during this pass
          P.T[v] = r;
          mine++;
          a = __ldg(g.off + v);
          d = __ldg(g.off + v + 1) - a;
        }
        stage_append(S, start && d > 0, (int32_t)v, d, a);
        __syncthreads();
        stage_make_room(S, out, ctl, blockDim.x);
      }
      stage_flush(S, out, ctl);
      claimed += mine;
      const unsigned long long t = block_sum64(mine, S.misc64);
      if (threadIdx.x == 0 && t) atomicAdd(&ctl->scnt[r % 3], (unsigned int)t);
    }
    if (!grid_sync(ctl, bar, &s_flag)) break;
    total += ld_vol(ctl->scnt[r % 3]);
    if (total >= (unsigned long long)n) break;  // every vertex claimed
    const unsigned long long fr = ld_vol(ctl->fr[sub % 3]);
    const uint32_t cnt = (uint32_t)(fr >> 32), Dsum = (uint32_t)fr;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      atomicAdd(&ctl->rounds, 1);
      if (cnt) atomicAdd(&ctl->push_rounds, 1);
      scanned += Dsum;
    }
    // ---------------- edgeMap: the frontier claims its unclaimed neighbours
    if (cnt > 0) {
      unsigned long long *outc = &ctl->fr[(sub + 1) % 3];
      QueueIn in{P.q[qb], P.qoff[qb], P.qadj[qb], P.cs[qb], cnt, Dsum};
      ClaimFn fn{g.off, g.tgt, P.C, P.T, r + 1, 0};
      StagedSink sink{QueueOut{P.q[qb ^ 1], P.qoff[qb ^ 1], P.qadj[qb ^ 1], P.cs[qb ^ 1], outc, n,
                               P.cs_cap},
                      ctl, nullptr};
      blocked_edge_map(g, in, chunk_shift(Dsum, 4u, chunk_shift_cap(ClaimFn::kWin * blockDim.x)),
                       (uint32_t)P.bmax, S, fn, sink, ctl, bem++);
      sink.finish(S);
      claimed += fn.claimed;
      const unsigned long long t = block_sum64(fn.claimed, S.misc64);
      if (threadIdx.x == 0 && t) atomicAdd(&ctl->scnt[(r + 1) % 3], (unsigned int)t);
    }
    if (!grid_sync(ctl, bar, &s_flag)) break;
    if (P.trace && blockIdx.x == 0 && threadIdx.x == 0 && r < P.trace_cap)
      P.trace[r] = TraceRec{r + 1, 1, cnt, Dsum, (long long)(globaltimer() - t_start), 0};
    // the next round's queue is the one this edgeMap filled, counted in fr[(sub + 1) % 3]
    qb ^= 1;
    sub++;
  }
  {
    const unsigned long long t = block_sum64(claimed, S.misc64);
    if (threadIdx.x == 0 && t) atomicAdd(&ctl->reached, t);
  }
  const unsigned long long t = block_sum64(scanned, S.misc64);
  if (threadIdx.x == 0 && t) atomicAdd(&ctl->edges_scanned, t);
}

gbf_status launch_ldd(Graph &g, Workspace &ws, const double *delta, int32_t *C, int32_t *T,
                      const Opts &o, cudaStream_t st) {
  LddParams P;
  P.g = g.dev();
  P.delta = delta;
  P.C = C;
  P.T = T;
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
    const gbf_status sm = check_smem(smem, "ldd_kernel");
    if (sm != GBF_OK) return sm;
  }
  GBF_CUDA(cudaFuncSetAttribute(ldd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  GBF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ldd_kernel, o.block, smem));
  if (per_sm < 1) {
    set_error("ldd kernel does not fit on an SM with this block size");
    return GBF_ERR_INVALID;
  }
  int grid = per_sm * g.num_sms;
  if (o.ctas > 0 && o.ctas < grid) grid = o.ctas;
  GBF_CUDA(cudaMemsetAsync(ws.ctl, 0, sizeof(Ctl), st));
  if (ws.trace) GBF_CUDA(cudaMemsetAsync(ws.trace, 0, sizeof(TraceRec) * (size_t)ws.trace_cap, st));
  void *args[] = {&P};
  GBF_CUDA(cudaLaunchCooperativeKernel((const void *)ldd_kernel, dim3(grid), dim3(o.block), args,
                                       smem, st));
  ws.last_kind = 7;
  ws.last_grid = grid;
  ws.last_block = o.block;
  return GBF_OK;
}

}  // namespace gbf

using namespace gbf;

extern "C" gbf_status gbf_ldd(gbf_graph *h, const double *delta, int32_t *cluster, int32_t *round,
                              int mem, const gbf_options *opt, void *cuda_stream) {
  if (!h || !delta || !cluster || !round)
    return set_error("graph, delta, cluster or round is NULL"), GBF_ERR_INVALID;
  Graph &g = h->g;
  if (mem != GBF_HOST && mem != GBF_DEVICE) return set_error("bad mem"), GBF_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  std::lock_guard<std::mutex> lk(g.mu);
  const Opts o = resolve(opt, g, GBF_TUNE_BFS);
  {
    const gbf_status s = ws_ensure_base(g, g.ws);
    if (s != GBF_OK) return s;
  }
  if (mem == GBF_DEVICE) return launch_ldd(g, g.ws, delta, cluster, round, o, st);
  // host buffers: the shifts are staged in a stream-ordered allocation, the
  // outputs in the workspace's host-output arrays
  double *dd = nullptr;
  GBF_CUDA(cudaMallocAsync((void **)&dd, sizeof(double) * (size_t)g.n, st));
  cudaError_t e = cudaMemcpyAsync(dd, delta, sizeof(double) * (size_t)g.n, cudaMemcpyHostToDevice, st);
  gbf_status s = e == cudaSuccess ? launch_ldd(g, g.ws, dd, g.ws.dist_tmp, g.ws.parent_tmp, o, st)
                                  : cuda_fail(e, "upload delta");
  cudaFreeAsync(dd, st);
  if (s != GBF_OK) return s;
  GBF_CUDA(cudaMemcpyAsync(cluster, g.ws.dist_tmp, sizeof(int32_t) * (size_t)g.n,
                           cudaMemcpyDeviceToHost, st));
  GBF_CUDA(cudaMemcpyAsync(round, g.ws.parent_tmp, sizeof(int32_t) * (size_t)g.n,
                           cudaMemcpyDeviceToHost, st));
  return ws_collect(g.ws, st, nullptr);
}
