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

#include <algorithm>

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
  uint32_t *fbm[3];  // frontier bitmaps: input, output, cleared for the next level
  int32_t *q[2];
  uint32_t *qoff[2];
  uint32_t *qadj[2];
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
  static constexpr int kWin = kU;  // windows per walk step
  template <class Sink>
  __device__ __forceinline__ void drain(Sink &, PushSmem &) {}  // nothing deferred
  const uint32_t *off;
  const int32_t *tgt;
  uint32_t *visited;
  int32_t *dist, *parent;
  int32_t level;
  unsigned long long reached;
  template <class Sink>
  __device__ __forceinline__ void batch(const bool *val, const int32_t *u, const uint32_t *idx,
                                        Sink &sink, PushSmem &S) {
    int32_t v[kWin];
    uint32_t wd[kWin];
#pragma unroll
    for (int r = 0; r < kWin; r++) v[r] = val[r] ? __ldg(tgt + idx[r]) : 0;
#pragma unroll
    for (int r = 0; r < kWin; r++) wd[r] = val[r] ? visited[v[r] >> 5] : ~0u;
    bool win[kWin];
#pragma unroll
    for (int r = 0; r < kWin; r++) {
      const uint32_t bit = 1u << (v[r] & 31);
      win[r] = false;
      if (!(wd[r] & bit)) win[r] = !(atomicOr(visited + (v[r] >> 5), bit) & bit);
    }
    uint32_t a[kWin], z[kWin];
#pragma unroll
    for (int r = 0; r < kWin; r++) {
      a[r] = z[r] = 0;
      if (win[r]) {
        dist[v[r]] = level;
        if (parent) parent[v[r]] = u[r];
        a[r] = __ldg(off + v[r]);
        z[r] = __ldg(off + v[r] + 1);
        reached++;
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

// Dense direction (the early-exit pull of §3) as one stream of candidates per
// warp.  Warps take chunks of kChunkWords bitmap words from a global counter;
// a word group (kGroupWords words: visited word and the offsets of every
// vertex) is loaded one step before it is needed and its candidates
// (unvisited, degree > 0) are appended to the warp's ring in shared memory.
// Every step each lane checks the next 4 arcs of its candidate in CSR order
// and takes a new candidate from the ring as soon as its own resolves, so no
// lane waits for another except at the end of the level.  A candidate still
// unresolved after `pull_serial` arcs is parked in the lane (a lane whose
// slot is taken keeps scanning its candidate itself); once kWalkLanes lanes
// hold one, the warp walks the remaining arcs of all parked candidates
// together (pull_walk_parked), 128 arcs per step.  Words are owned by one warp, whose
// found vertices set their next-frontier and visited bits with one atomicOr
// per word and step.  The first frontier neighbour in CSR order becomes the
// parent, as in a sequential early-exit scan.
constexpr uint32_t kChunkWords = 32;
constexpr uint32_t kGroupWords = 4;
constexpr uint32_t kRing = 256;  // ring entries per warp: 8 per thread of the staging area
constexpr int kWalkLanes = 16;   // parked candidates that start a warp walk

// Per-thread counters of a pull level (32-bit: a thread's share of one level
// fits), and the write of a found vertex's distance and parent.
struct PullCtx {
  int32_t level;
  uint32_t scanned, reached;
  uint32_t cnt, deg;  // found vertices of degree >= 2 and their degree sum

  __device__ __forceinline__ void record(const BfsParams &P, int32_t v, int32_t par, uint32_t d) {
    P.dist[v] = level;
    if (P.parent) P.parent[v] = par;
    reached++;
    if (d >= 2) {
      cnt++;
      deg += d;
    }
  }
};

// Warp-collective: walk the remaining arcs [k, e) of the lanes' parked
// entries (v >= 0) in 32-arc windows, kU windows per step, in CSR order; a
// vertex drops out at its first frontier neighbour.  Clears the parked slots.
__device__ __forceinline__ void pull_walk_parked(const BfsParams &P, const uint32_t *fin,
                                                 uint32_t *fout, PullCtx &C, int32_t &v,
                                                 uint32_t k, uint32_t e, uint32_t s0) {
  const int lane = threadIdx.x & 31;
  const uint32_t rem = v >= 0 ? e - k : 0u;
  uint32_t incl = rem;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  const uint32_t total = __shfl_sync(kFull, incl, 31);
  const uint32_t excl = incl - rem;
  unsigned pending = __ballot_sync(kFull, rem > 0);
  int32_t par = -1;
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
      uu[r] = val ? __ldg(P.g.tgt + ko + (ee - eo)) : -1;
    }
#pragma unroll
    for (int r = 0; r < kU; r++)
      hit[r] = uu[r] >= 0 && ((fin[uu[r] >> 5] >> (uu[r] & 31)) & 1u);
#pragma unroll
    for (int r = 0; r < kU; r++) {
      const unsigned lb = __ballot_sync(kFull, uu[r] >= 0);
      if (lane == 0) C.scanned += __popc(lb);
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
  if (par >= 0) {
    C.record(P, v, par, e - s0);
    const uint32_t w = (uint32_t)v >> 5, bit = 1u << (v & 31);
    atomicOr(fout + w, bit);
    atomicOr(P.visited + w, bit);
  }
  v = -1;
}

__device__ void pull_level(const BfsParams &P, PushSmem &S, const uint32_t *fin, uint32_t *fout,
                           uint32_t *fzero, int32_t level, unsigned long long *counter,
                           unsigned long long &scanned, unsigned long long &reached,
                           unsigned long long &cand_cnt, int inv) {
  const DevGraph &g = P.g;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t nwords = ((uint32_t)g.n + 31) >> 5;
  const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  // the bitmap the next dense level writes (nobody reads it in this level)
  for (uint32_t i = gt; i < nwords; i += gs) fzero[i] = 0u;
  const uint32_t nchunk = (nwords + kChunkWords - 1) / kChunkWords;
  const uint32_t F = (uint32_t)P.pull_serial;
  const unsigned lt = (1u << lane) - 1u;
  int32_t *rv = S.out_v + warp * kRing;
  uint32_t *rs = S.out_d + warp * kRing, *re = S.pref + warp * kRing;
  uint32_t *scr = S.base + warp * 32;  // per-word bit gathering of one step
  scr[lane] = 0u;
  __syncwarp();
  PullCtx C{level, 0u, 0u, 0u, 0u};
  unsigned int *work = &P.ctl->work[inv & 3];
  if (blockIdx.x == 0 && threadIdx.x == 0) st_vol(P.ctl->work[(inv + 2) & 3], 0u);
  const uint32_t twarps = gridDim.x * (uint32_t)nw;

  // word supply: chunk = first chunk of this warp, then from the counter (the
  // next one is requested by lane 0 one chunk ahead)
  uint32_t chunk = blockIdx.x * (uint32_t)nw + (uint32_t)warp;
  uint32_t next_chunk = 0;
  if (lane == 0) next_chunk = twarps + atomicAdd(work, 1u);
  uint32_t gw = chunk * kChunkWords;  // first word of the next group to load
  bool more = chunk < nchunk;
  bool have = false;
  uint32_t pw = 0;
  // the loaded group: offsets of its vertices (pa[r]: word r; the end offset of
  // a lane's vertex is the next lane's start, pnext after the last word) and
  // its visited words (lane r holds word r)
  uint32_t pa[kGroupWords], pnext = 0, pvis = ~0u;
  uint32_t head = 0, tail = 0;
  int32_t cv = -1, pv = -1;
  uint32_t ck = 0, ce = 0, cs0 = 0, pk = 0, pe = 0, ps0 = 0;

  // load the next word group (warp-uniform)
#define GBF_PULL_PREFETCH()                                                              \
  do {                                                                                   \
    _Pragma("unroll") for (uint32_t r = 0; r < kGroupWords; r++) {                       \
      const uint32_t v = (gw + r) * 32 + lane;                                           \
      pa[r] = v <= (uint32_t)g.n ? __ldg(g.off + v) : 0u;                                \
    }                                                                                    \
    {                                                                                    \
      const uint32_t vn = (gw + kGroupWords) * 32;                                       \
      pnext = (lane == 31 && vn <= (uint32_t)g.n) ? __ldg(g.off + vn) : 0u;              \
      pvis = ((uint32_t)lane < kGroupWords && gw + lane < nwords) ? P.visited[gw + lane]  \
                                                                  : ~0u;                 \
    }                                                                                    \
    pw = gw;                                                                             \
    have = true;                                                                         \
    gw += kGroupWords;                                                                   \
    if (gw >= min(chunk * kChunkWords + kChunkWords, nwords)) {                          \
      chunk = __shfl_sync(kFull, next_chunk, 0);                                         \
      more = chunk < nchunk;                                                             \
      if (more) {                                                                        \
        gw = chunk * kChunkWords;                                                        \
        if (lane == 0) next_chunk = twarps + atomicAdd(work, 1u);                        \
      }                                                                                  \
    }                                                                                    \
  } while (0)

  if (more) GBF_PULL_PREFETCH();
  while (true) {
    // append the loaded group's candidates, then start loading the next group
    if (have && tail - head < kRing - 32 * kGroupWords - 32) {
#pragma unroll
      for (uint32_t r = 0; r < kGroupWords; r++) {
        const uint32_t vis = __shfl_sync(kFull, pvis, r);
        const uint32_t a = pa[r];
        uint32_t z = __shfl_down_sync(kFull, a, 1);
        const uint32_t zn = (r + 1 < kGroupWords) ? __shfl_sync(kFull, pa[r + 1 < kGroupWords ? r + 1 : r], 0)
                                                  : pnext;
        if (lane == 31) z = zn;
        const uint32_t v = (pw + r) * 32 + lane;
        const bool c = v < (uint32_t)g.n && !((vis >> lane) & 1u) && z > a;
        const unsigned bal = __ballot_sync(kFull, c);
        if (c) {
          const uint32_t i = (tail + __popc(bal & lt)) & (kRing - 1);
          rv[i] = (int32_t)v;
          rs[i] = a;
          re[i] = z;
        }
        tail += __popc(bal);
      }
      have = false;
      __syncwarp();
      if (more) GBF_PULL_PREFETCH();
    }
    // lanes without a candidate take the next ones from the ring
    const unsigned need = __ballot_sync(kFull, cv < 0);
    const uint32_t avail = tail - head;
    if (cv < 0) {
      const uint32_t r = __popc(need & lt);
      if (r < avail) {
        const uint32_t i = (head + r) & (kRing - 1);
        cv = rv[i];
        ck = cs0 = rs[i];
        ce = re[i];
        cand_cnt++;
      }
    }
    head += min((uint32_t)__popc(need), avail);
    const bool act = cv >= 0;
    if (!__any_sync(kFull, act)) {
      if (!have) break;
      continue;
    }
    // one step: the next 4 arcs of each lane's candidate
    int32_t u[4];
#pragma unroll
    for (int r = 0; r < 4; r++) u[r] = (act && ck + r < ce) ? __ldg(g.tgt + ck + r) : -1;
    bool h[4];
#pragma unroll
    for (int r = 0; r < 4; r++) h[r] = u[r] >= 0 && ((fin[u[r] >> 5] >> (u[r] & 31)) & 1u);
    bool park = false, got = false;
    int32_t gv = 0;
    if (act) {
      uint32_t used = min(4u, ce - ck);
      int32_t par = -1;
#pragma unroll
      for (int r = 3; r >= 0; r--)
        if (h[r]) {
          par = u[r];
          used = (uint32_t)r + 1;
        }
      C.scanned += used;
      ck += used;
      if (par >= 0) {
        C.record(P, cv, par, ce - cs0);
        got = true;
        gv = cv;
        cv = -1;
      } else if (ck >= ce) {
        cv = -1;
      } else {
        park = pv < 0 && ck - cs0 >= F;
      }
    }
    // one atomicOr per distinct word of this step's found vertices
    if (__any_sync(kFull, got)) {
      const uint32_t key = got ? ((uint32_t)gv >> 5) : (0xF0000000u | (uint32_t)lane);
      const unsigned grp = __match_any_sync(kFull, key);
      const int leader = __ffs(grp) - 1;
      if (got) atomicOr(scr + leader, 1u << (gv & 31));
      __syncwarp();
      if (got && lane == leader) {
        const uint32_t bits = scr[lane];
        scr[lane] = 0u;
        atomicOr(fout + key, bits);
        atomicOr(P.visited + key, bits);
      }
      __syncwarp();
    }
    if (park) {
      pv = cv;
      pk = ck;
      pe = ce;
      ps0 = cs0;
      cv = -1;
    }
    if (__popc(__ballot_sync(kFull, pv >= 0)) >= kWalkLanes)
      pull_walk_parked(P, fin, fout, C, pv, pk, pe, ps0);
  }
#undef GBF_PULL_PREFETCH
  if (__any_sync(kFull, pv >= 0)) pull_walk_parked(P, fin, fout, C, pv, pk, pe, ps0);
  scanned += C.scanned;
  reached += C.reached;
  unsigned long long packed = ((unsigned long long)C.cnt << 32) | C.deg;
  unsigned long long tot = block_sum64(packed, S.misc64);
  if (threadIdx.x == 0 && tot) atomicAdd(counter, tot);
}

// Sparse queue -> bitmap fb (cleared first, with the bitmap fo the next
// dense level writes; two barriers).
__device__ bool queue_to_bitmap(const BfsParams &P, const int32_t *q, uint32_t cnt, uint32_t *fb,
                                uint32_t *fo, Barrier &bar, int *s_flag) {
  const uint32_t nwords = ((uint32_t)P.g.n + 31) >> 5;
  const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (uint32_t i = gt; i < nwords; i += gs) {
    fb[i] = 0u;
    fo[i] = 0u;
  }
  if (!grid_sync(P.ctl, bar, s_flag)) return false;
  for (uint32_t i = gt; i < cnt; i += gs) {
    const int32_t v = q[i];
    atomicOr(fb + (v >> 5), 1u << (v & 31));
  }
  return grid_sync(P.ctl, bar, s_flag);
}

// Bitmap -> sparse queue with degree prefix (CTA-contiguous word ranges).
// Each warp takes 2 kU words per step with all their loads in flight; the
// staging area holds one step of the whole CTA (2 kU entries per thread, the
// staging capacity), so it is flushed between steps whenever it is not empty.
__device__ void bitmap_to_queue(const BfsParams &P, const uint32_t *fb, PushSmem &S,
                                const QueueOut &out) {
  constexpr int R = 2 * kU;
  const uint32_t nwords = ((uint32_t)P.g.n + 31) >> 5;
  const uint32_t per = (nwords + gridDim.x - 1) / gridDim.x;
  const uint32_t wlo = min(nwords, blockIdx.x * per), whi = min(nwords, wlo + per);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (uint32_t base = wlo; base < whi; base += R * nw) {
    uint32_t a[R], z[R];
    bool set[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
      const uint32_t wi = base + warp + r * nw;
      const uint32_t bits = (wi < whi) ? fb[wi] : 0u;
      set[r] = (bits >> lane) & 1u;
      const int32_t v = (int32_t)(wi * 32 + lane);
      a[r] = set[r] ? __ldg(P.g.off + v) : 0u;
      z[r] = set[r] ? __ldg(P.g.off + v + 1) : 0u;
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
      const uint32_t wi = base + warp + r * nw;
      const uint32_t d = z[r] - a[r];
      stage_append(S, set[r] && d >= 2, (int32_t)(wi * 32 + lane), d, a[r]);
    }
    __syncthreads();
    stage_make_room(S, out, P.ctl, R * blockDim.x);
  }
  stage_flush(S, out, P.ctl);
}

}  // namespace

__global__ void __launch_bounds__(1024) bfs_kernel(BfsParams P) {
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
      P.qadj[0][0] = __ldg(g.off + src);
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
      if (!queue_to_bitmap(P, P.q[qb], cnt, P.fbm[0], P.fbm[1], bar, &s_flag)) break;
      fmt_bitmap = 1;
      fb = 0;
    } else if (!dense && fmt_bitmap) {
      QueueOut out{P.q[0], P.qoff[0], P.qadj[0], P.cs[0], &ctl->conv, (uint32_t)g.n, P.cs_cap};
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
      QueueIn in{P.q[qb], P.qoff[qb], P.qadj[qb], P.cs[qb], cnt, D};
      BfsPushFn fn{g.off, g.tgt, P.visited, P.dist, P.parent, level, 0};
      StagedSink sink{QueueOut{P.q[qb ^ 1], P.qoff[qb ^ 1], P.qadj[qb ^ 1], P.cs[qb ^ 1], outc,
                               (uint32_t)g.n, P.cs_cap},
                      ctl, nullptr};
      // chunks of one walk step of the whole CTA (kWin 32-edge windows per
      // warp): a step appends at most half the staging capacity, which
      // chunk_end keeps free
      const int s = chunk_shift(D, 4u, chunk_shift_cap(BfsPushFn::kWin * blockDim.x));
      blocked_edge_map(g, in, s, (uint32_t)P.bmax, S, fn, sink, ctl, bem++);
      sink.finish(S);
      reached += fn.reached;
      qb ^= 1;
    } else {
      pull_level(P, S, P.fbm[fb], P.fbm[(fb + 1) % 3], P.fbm[(fb + 2) % 3], level, outc, scanned,
                 reached, expanded, bem++);
      fb = (fb + 1) % 3;
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
  for (int i = 0; i < 3; i++) P.fbm[i] = ws.fbm[i];
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
  P.pull_divisor = o.pull_divisor;
  P.bmax = o.heavy_cutoff;
  P.cap = stage_capacity(o.block);
  int l = 0;
  while ((kFine << l) < (uint32_t)o.heavy_cutoff) l++;
  P.log2_bmax_fine = l;
  P.pull_serial = o.pull_serial;
  P.inject_wait = o.inject_wait;
  P.cap_ns = o.spin_cap_ns;
  const size_t smem = push_smem_bytes(SmemShape{P.bmax, P.cap, 0, 0, 1});
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
  const size_t smem = push_smem_bytes(SmemShape{o.heavy_cutoff, stage_capacity(o.block), 0, 0, 1});
  if (cudaFuncSetAttribute(bfs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bfs_kernel, o.block, smem) != cudaSuccess)
    return 0;
  return per_sm;
}

}  // namespace gbf
