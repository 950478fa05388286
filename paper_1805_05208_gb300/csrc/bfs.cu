// BFS (§4 "Breadth-First Search"; Alg. 1) as one persistent cooperative
// kernel: the whole level loop stays on the device, one bounded grid barrier
// per level.  Each level runs Ligra's edgeMap (§3) in one of two directions:
//   - sparse (push): the blocked edgeMap of §6.2 over a frontier queue;
//     Update is a test-and-set on the visited bitmap (atomicOr) and the winner
//     writes D[v] = level and parent[v] = u (Alg. 1 Update);
//   - dense (pull): every unvisited vertex scans its neighbours in CSR order
//     and stops at the first one in the frontier bitmap (the early-exit dense
//     method of §3), writing its bit of the next frontier.
// The direction is chosen per level from the frontier's out-degree sum:
// dense when it exceeds m / pull_divisor (§3 "based on the number of edges
// incident to the current frontier").
//
// Readings of Alg. 1 used here: the source is marked visited with D = 0 and
// vertices first reached while expanding level k-1 get D = k.  A vertex of
// degree 1 reached from its only neighbour is never expanded: in a symmetric
// graph all its neighbours are already visited.
#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "gbf_impl.h"

namespace gbf {
using namespace dev;

struct BfsParams {
  DevGraph g;
  int32_t src;
  int32_t *dist;
  int32_t *parent;
  uint32_t *visited;
  uint32_t *fbm[2];
  int32_t *q[2];
  uint32_t *qoff[2];
  uint32_t *cs[2];
  uint32_t cs_cap;
  Ctl *ctl;
  TraceRec *trace;
  int trace_cap;
  int pull_divisor;
  int log2_bmax_fine;  // log2(Bmax / 256)
  int bmax;
  int cap;             // staging capacity
  int pull_serial;
  int inject_wait;
  long long cap_ns;
};

namespace {

// Sparse-direction Update of Alg. 1: test-and-set on the visited bit; the
// winner writes D and the parent.  kU windows at a time: all target loads,
// then all bitmap loads, then the test-and-sets, then the winners' degrees.
struct BfsPushFn {
  const uint32_t *off;
  const int32_t *tgt;
  uint32_t *visited;
  int32_t *dist, *parent;
  int32_t level;
  unsigned long long reached;
  template <class Sink>
  __device__ __forceinline__ void batch(const bool *val, const int32_t *u, const uint32_t *idx,
                                        Sink &sink, PushSmem &S) {
    int32_t v[kU];
    uint32_t wd[kU];
#pragma unroll
    for (int r = 0; r < kU; r++) v[r] = val[r] ? __ldg(tgt + idx[r]) : 0;
#pragma unroll
    for (int r = 0; r < kU; r++) wd[r] = val[r] ? visited[v[r] >> 5] : ~0u;
    bool win[kU];
#pragma unroll
    for (int r = 0; r < kU; r++) {
      const uint32_t bit = 1u << (v[r] & 31);
      win[r] = false;
      if (!(wd[r] & bit)) win[r] = !(atomicOr(visited + (v[r] >> 5), bit) & bit);
    }
    uint32_t a[kU], z[kU];
#pragma unroll
    for (int r = 0; r < kU; r++) {
      a[r] = z[r] = 0;
      if (win[r]) {
        dist[v[r]] = level;
        if (parent) parent[v[r]] = u[r];
        a[r] = __ldg(off + v[r]);
        z[r] = __ldg(off + v[r] + 1);
        reached++;
      }
    }
#pragma unroll
    for (int r = 0; r < kU; r++) {
      const uint32_t d = z[r] - a[r];
      sink.append(S, win[r] && d >= 2, v[r], d);
    }
  }
};

// Dense direction: one warp per 32-vertex word of the bitmaps.  Each
// unvisited vertex checks its first arcs (4 at a time, loads batched); the
// warp then walks the remaining arcs of every still-unresolved vertex of the
// word together, 32 consecutive arcs per window and kU windows per step,
// dropping a vertex as soon as one of its arcs hits the frontier.  Arcs are
// taken in CSR order and the first hit becomes the parent, as in a
// sequential early-exit scan.
__device__ void pull_level(const BfsParams &P, const uint32_t *fin, uint32_t *fout, int32_t level,
                           unsigned long long *counter, unsigned long long &scanned,
                           unsigned long long &reached, unsigned long long &cand_cnt,
                           unsigned long long *s64) {
  const DevGraph &g = P.g;
  const int lane = threadIdx.x & 31;
  const uint32_t nwords = ((uint32_t)g.n + 31) >> 5;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t tw = (gridDim.x * blockDim.x) >> 5;
  const uint32_t first = (uint32_t)P.pull_serial;
  uint32_t my_cnt = 0, my_deg = 0;
  for (uint32_t wi = gw; wi < nwords; wi += tw) {
    const uint32_t vis = P.visited[wi];
    const int32_t v = (int32_t)(wi * 32 + lane);
    bool cand = v < g.n && !((vis >> lane) & 1u);
    uint32_t s = 0, e = 0;
    if (cand) {
      s = __ldg(g.off + v);
      e = __ldg(g.off + v + 1);
      cand = e > s;
      cand_cnt++;
    }
    int32_t par = -1;
    // pass 1: the first arcs of each candidate, four loads in flight per lane
    uint32_t k = s;
    for (uint32_t c = 0; c < first; c += 4) {
      int32_t u[4];
      bool h[4];
#pragma unroll
      for (int r = 0; r < 4; r++) {
        const uint32_t kk = k + r;
        u[r] = (cand && par < 0 && kk < e) ? __ldg(g.tgt + kk) : -1;
      }
#pragma unroll
      for (int r = 0; r < 4; r++) h[r] = u[r] >= 0 && ((fin[u[r] >> 5] >> (u[r] & 31)) & 1u);
      if (cand && par < 0) {
        uint32_t used = min(4u, e - min(k, e));
#pragma unroll
        for (int r = 3; r >= 0; r--)
          if (h[r]) {
            par = u[r];
            used = (uint32_t)r + 1;
          }
        scanned += used;
        k += used;
      }
    }
    // pass 2: the remaining arcs of the unresolved candidates, warp windows
    const uint32_t rem = (cand && par < 0 && k < e) ? e - k : 0u;
    uint32_t incl = rem;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    const uint32_t excl = incl - rem;
    unsigned pending = __ballot_sync(kFull, rem > 0);
    for (uint32_t w0 = 0; w0 < total && pending; w0 += 32 * kU) {
      int32_t uu[kU];
      int own[kU];
      bool hit[kU];
#pragma unroll
      for (int r = 0; r < kU; r++) {
        const uint32_t ee = w0 + 32 * r + lane;
        int o = 0;
#pragma unroll
        for (int st = 16; st > 0; st >>= 1) {
          const uint32_t cv = __shfl_sync(kFull, incl, o + st - 1);
          if (cv <= ee) o += st;
        }
        o = min(o, 31);
        const uint32_t eo = __shfl_sync(kFull, excl, o);
        const uint32_t ko = __shfl_sync(kFull, k, o);
        const bool val = ee < total && ((pending >> o) & 1u);
        own[r] = o;
        uu[r] = val ? __ldg(g.tgt + ko + (ee - eo)) : -1;
      }
#pragma unroll
      for (int r = 0; r < kU; r++) hit[r] = uu[r] >= 0 && ((fin[uu[r] >> 5] >> (uu[r] & 31)) & 1u);
#pragma unroll
      for (int r = 0; r < kU; r++) {
        const unsigned lb = __ballot_sync(kFull, uu[r] >= 0);
        if (lane == 0) scanned += __popc(lb);
        unsigned hb = __ballot_sync(kFull, hit[r]);
        while (hb) {
          const int f = __ffs(hb) - 1;
          const int o = __shfl_sync(kFull, own[r], f);
          const int32_t uf = __shfl_sync(kFull, uu[r], f);
          if (lane == o && par < 0) par = uf;
          hb &= ~__ballot_sync(kFull, hit[r] && own[r] == o);
          pending &= ~(1u << o);
        }
      }
    }
    const bool got = par >= 0;
    const unsigned nb = __ballot_sync(kFull, got);
    if (got) {
      P.dist[v] = level;
      if (P.parent) P.parent[v] = par;
      reached++;
      const uint32_t d = e - s;
      if (d >= 2) {
        my_cnt++;
        my_deg += d;
      }
    }
    if (lane == 0) {
      fout[wi] = nb;
      if (nb) P.visited[wi] = vis | nb;
    }
  }
  unsigned long long packed = ((unsigned long long)my_cnt << 32) | my_deg;
  unsigned long long tot = block_sum64(packed, s64);
  if (threadIdx.x == 0 && tot) atomicAdd(counter, tot);
}

// Sparse queue -> bitmap (cleared first; two barriers).
__device__ bool queue_to_bitmap(const BfsParams &P, const int32_t *q, uint32_t cnt, uint32_t *fb,
                                Barrier &bar, int *s_flag) {
  const uint32_t nwords = ((uint32_t)P.g.n + 31) >> 5;
  const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (uint32_t i = gt; i < nwords; i += gs) fb[i] = 0u;
  if (!grid_sync(P.ctl, bar, s_flag)) return false;
  for (uint32_t i = gt; i < cnt; i += gs) {
    const int32_t v = q[i];
    atomicOr(fb + (v >> 5), 1u << (v & 31));
  }
  return grid_sync(P.ctl, bar, s_flag);
}

// Bitmap -> sparse queue with degree prefix (CTA-contiguous word ranges).
__device__ void bitmap_to_queue(const BfsParams &P, const uint32_t *fb, PushSmem &S,
                                const QueueOut &out) {
  const uint32_t nwords = ((uint32_t)P.g.n + 31) >> 5;
  const uint32_t per = (nwords + gridDim.x - 1) / gridDim.x;
  const uint32_t wlo = min(nwords, blockIdx.x * per), whi = min(nwords, wlo + per);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (uint32_t base = wlo; base < whi; base += nw) {
    const uint32_t wi = base + warp;
    const uint32_t bits = (wi < whi) ? fb[wi] : 0u;
    bool emit = false;
    int32_t v = (int32_t)(wi * 32 + lane);
    uint32_t d = 0;
    if ((bits >> lane) & 1u) {
      d = __ldg(P.g.off + v + 1) - __ldg(P.g.off + v);
      emit = d >= 2;
    }
    stage_append(S, emit, v, d);
    __syncthreads();
    if (S.misc[0] + blockDim.x > S.cap_out) stage_flush(S, out, P.ctl);
  }
  stage_flush(S, out, P.ctl);
}

}  // namespace

__global__ void __launch_bounds__(1024) bfs_kernel(BfsParams P) {
  extern __shared__ unsigned long long smem_raw[];
  __shared__ int s_flag;
  PushSmem S = carve_push_smem(smem_raw, SmemShape{P.bmax, P.cap, 0, 0});
  if (threadIdx.x == 0) S.misc[0] = 0;
  Ctl *ctl = P.ctl;
  Barrier bar{0u, P.cap_ns};
  const DevGraph g = P.g;
  const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  const uint32_t nwords = ((uint32_t)g.n + 31) >> 5;
  const int32_t src = P.src;
  unsigned long long scanned = 0, reached = 0, expanded = 0;
  const unsigned long long t_start = globaltimer();

  // Initialisation (Alg. 1 line 1 and BFS line 1): D = inf, Fl = 0, then the source.
  for (uint32_t i = gt; i < (uint32_t)g.n; i += gs) {
    P.dist[i] = (i == (uint32_t)src) ? 0 : kInf;
    if (P.parent) P.parent[i] = (i == (uint32_t)src) ? src : -1;
  }
  for (uint32_t i = gt; i < nwords; i += gs)
    P.visited[i] = (i == ((uint32_t)src >> 5)) ? (1u << (src & 31)) : 0u;
  if (blockIdx.x == 0) {
    const uint32_t d0 = __ldg(g.off + src + 1) - __ldg(g.off + src);
    if (threadIdx.x == 0 && d0 > 0) {
      P.q[0][0] = src;
      P.qoff[0][0] = 0;
      st_vol(ctl->fr[0], (1ull << 32) | d0);
    }
    for (uint32_t c = threadIdx.x; c < (d0 + kFine - 1) / kFine; c += blockDim.x)
      if (c < P.cs_cap) P.cs[0][c] = 0;
    if (threadIdx.x == 0) reached = 1;
  }
  if (P.inject_wait && blockIdx.x == 0 && threadIdx.x == 0) injected_wait(ctl, P.cap_ns);
  __syncthreads();
  bool ok = grid_sync(ctl, bar, &s_flag);

  int fmt_bitmap = 0, qb = 0, fb = 0;
  int bem = 0;  // blocked edgeMap invocations so far
  int level = 1;
  unsigned long long fr = ok ? ld_vol(ctl->fr[0]) : 0ull;
  while (ok) {
    const uint32_t cnt = (uint32_t)(fr >> 32), D = (uint32_t)fr;
    if (cnt == 0) break;
    const bool dense =
        P.pull_divisor > 0 && (unsigned long long)D * (unsigned)P.pull_divisor > g.m;
    if (dense && !fmt_bitmap) {
      if (!queue_to_bitmap(P, P.q[qb], cnt, P.fbm[0], bar, &s_flag)) break;
      fmt_bitmap = 1;
      fb = 0;
    } else if (!dense && fmt_bitmap) {
      QueueOut out{P.q[0], P.qoff[0], P.cs[0], &ctl->conv, (uint32_t)g.n, P.cs_cap};
      bitmap_to_queue(P, P.fbm[fb], S, out);
      if (!grid_sync(ctl, bar, &s_flag)) break;
      fmt_bitmap = 0;
      qb = 0;
    }
    unsigned long long *outc = &ctl->fr[level % 3];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st_vol(ctl->fr[(level + 1) % 3], 0ull);
      st_vol(ctl->conv, 0ull);
      if (dense) atomicAdd(&ctl->pull_rounds, 1);
      else {
        atomicAdd(&ctl->push_rounds, 1);
        scanned += D;
        expanded += cnt;
      }
      atomicAdd(&ctl->rounds, 1);
    }
    if (!fmt_bitmap) {
      QueueIn in{P.q[qb], P.qoff[qb], P.cs[qb], cnt, D};
      BfsPushFn fn{g.off, g.tgt, P.visited, P.dist, P.parent, level, 0};
      StagedSink sink{QueueOut{P.q[qb ^ 1], P.qoff[qb ^ 1], P.cs[qb ^ 1], outc, (uint32_t)g.n,
                               P.cs_cap},
                      ctl};
      // every queued vertex has degree >= 2
      const int s = chunk_shift(D, (uint32_t)P.bmax, 2u);
      blocked_edge_map(g, in, s, (uint32_t)P.bmax, S, fn, sink, ctl, bem++);
      sink.finish(S);
      reached += fn.reached;
      qb ^= 1;
    } else {
      pull_level(P, P.fbm[fb], P.fbm[fb ^ 1], level, outc, scanned, reached, expanded,
                 S.misc64);
      fb ^= 1;
    }
    if (!grid_sync(ctl, bar, &s_flag)) break;
    fr = ld_vol(*outc);
    if (P.trace && blockIdx.x == 0 && threadIdx.x == 0 && level <= P.trace_cap)
      P.trace[level - 1] = TraceRec{level, fmt_bitmap ? 2 : 1, cnt, D,
                                    (long long)(globaltimer() - t_start), 0};
    level++;
  }
  // statistics
  unsigned long long t;
  t = block_sum64(scanned, S.misc64);
  if (threadIdx.x == 0 && t) atomicAdd(&ctl->edges_scanned, t);
  t = block_sum64(reached, S.misc64);
  if (threadIdx.x == 0 && t) atomicAdd(&ctl->reached, t);
  t = block_sum64(expanded, S.misc64);
  if (threadIdx.x == 0 && t) atomicAdd(&ctl->expanded, t);
}

gbf_status launch_bfs(Graph &g, Workspace &ws, int32_t src, int32_t *dist, int32_t *parent,
                      const Opts &o, cudaStream_t st) {
  BfsParams P;
  P.g = g.dev();
  P.src = src;
  P.dist = dist;
  P.parent = parent;
  P.visited = ws.visited;
  for (int i = 0; i < 2; i++) {
    P.fbm[i] = ws.fbm[i];
    P.q[i] = ws.q[i];
    P.qoff[i] = ws.qoff[i];
    P.cs[i] = ws.cs[i];
  }
  P.cs_cap = (uint32_t)(((uint64_t)g.m + kFine - 1) / kFine + 2);
  P.ctl = ws.ctl;
  P.trace = ws.trace;
  P.trace_cap = ws.trace_cap;
  P.pull_divisor = o.pull_divisor;
  P.bmax = o.heavy_cutoff;
  P.cap = stage_capacity(o.block);
  int l = 0;
  while ((kFine << l) < (uint32_t)o.heavy_cutoff) l++;
  P.log2_bmax_fine = l;
  P.pull_serial = o.pull_serial;
  P.inject_wait = o.inject_wait;
  P.cap_ns = o.spin_cap_ns;
  const size_t smem = push_smem_bytes(SmemShape{P.bmax, P.cap, 0, 0});
  {
    const gbf_status sm = check_smem(smem, "bfs_kernel");
    if (sm != GBF_OK) return sm;
  }
  GBF_CUDA(cudaFuncSetAttribute(bfs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  int per_sm = 0;
  GBF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bfs_kernel, o.block, smem));
  if (per_sm < 1) {
    set_error("bfs kernel does not fit on an SM with this block size");
    return GBF_ERR_INVALID;
  }
  int grid = per_sm * g.num_sms;
  if (o.ctas > 0 && o.ctas < grid) grid = o.ctas;
  GBF_CUDA(cudaMemsetAsync(ws.ctl, 0, sizeof(Ctl), st));
  if (ws.trace) GBF_CUDA(cudaMemsetAsync(ws.trace, 0, sizeof(TraceRec) * (size_t)ws.trace_cap, st));
  void *args[] = {&P};
  GBF_CUDA(cudaLaunchCooperativeKernel((const void *)bfs_kernel, dim3(grid), dim3(o.block), args,
                                       smem, st));
  ws.last_kind = 1;
  ws.last_grid = grid;
  ws.last_block = o.block;
  return GBF_OK;
}

int resident_ctas_per_sm_bfs(const Opts &o) {
  const size_t smem = push_smem_bytes(SmemShape{o.heavy_cutoff, stage_capacity(o.block), 0, 0});
  if (cudaFuncSetAttribute(bfs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bfs_kernel, o.block, smem) != cudaSuccess)
    return 0;
  return per_sm;
}

}  // namespace gbf
