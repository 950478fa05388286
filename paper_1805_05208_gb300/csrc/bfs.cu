// BFS (§4 "Breadth-First Search"; Alg. 1) as one persistent cooperative
// kernel: the whole level loop stays on the device, one bounded grid barrier
// per level.  Each level runs Ligra's edgeMap (§3) in one of two directions:
//   - sparse (push): the blocked edgeMap of §6.2 over a frontier queue;
//     Update is a test-and-set on the visited bitmap (atomicOr) and the winner
//     records its parent (Alg. 1 Update);
//   - dense (pull): every unvisited vertex scans its neighbours in CSR order
//     and stops at the first one in the frontier bitmap (the early-exit dense
//     method of §3), writing its bit of the next frontier.
// The direction is chosen per level from the frontier's out-degree sum:
// dense when it exceeds m / pull_divisor (§3 "based on the number of edges
// incident to the current frontier"); after a dense level the next one stays
// dense while the frontier holds more than n / pull_stay vertices.
//
// Layout of the per-level output.  A level whose frontier is large (every
// dense level, and a sparse level with at least bulk_min frontier edges)
// writes its new vertices as a bitmap, one of jmax kept for the whole query;
// their distances are not written during the traversal but by one coalesced
// pass at the end, which reads each vertex's level from those bitmaps, so the
// scattered 4-byte writes of D disappear.  Small sparse levels write D
// directly and hand the next level a compact queue with its degree prefix.
// The next level converts between the two forms when its direction needs the
// other one.
//
// Graph-side arrays used when the graph provides them: a bitmap of the
// vertices of degree 0 (they start out visited, so no dense level looks at
// them) and the target of every vertex's first arc (`f1`; graph creation puts
// the arc to the highest-degree neighbour first): when the frontier holds
// more than an eighth of all arcs, or is made of hubs, the dense step checks
// that arc from a coalesced stream before it touches the vertex's adjacency
// list, which is the sequential scan's first step read from a copy.
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

constexpr int kMaxDeferred = 8;  // bitmaps of levels whose D is written at the end

struct BfsParams {
  DevGraph g;
  const uint32_t *iso;  // bit v set iff deg(v) == 0 (nullable)
  const int32_t *f1;    // target of each vertex's first arc (nullable)
  int32_t src;
  int32_t *dist;
  int32_t *parent;
  uint32_t *visited;
  uint32_t *lb;       // jmax bitmaps of deferred levels, nwords each
  int jmax;
  uint32_t *rb[3];    // rotating bitmaps: converted queues, levels written directly
  int32_t *q[2];
  uint32_t *qoff[2];
  uint32_t *qadj[2];
  uint32_t *cs[2];
  uint32_t cs_cap;
  Ctl *ctl;
  TraceRec *trace;
  int trace_cap;
  int pull_divisor;
  int pull_stay;      // > 0: stay dense while |F| * pull_stay > n
  uint32_t bulk_min;  // frontier edges from which a sparse level writes a bitmap
  int bmax;
  int cap;            // staging capacity
  int pull_serial;
  int inject_wait;
  long long cap_ns;
};

namespace {

// Sparse-direction Update of Alg. 1 for small frontiers: test-and-set on the
// visited bit; the winner writes D and the parent and is appended to the next
// queue.  kU windows at a time: all target loads, then all bitmap loads, then
// the test-and-sets, then the winners' degrees.
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

// Sparse-direction Update for large frontiers: the winner records its parent
// and sets its bit of the output bitmap (a reduction, nothing waits for it);
// D is written directly only when the level has no deferred bitmap.  The
// next frontier's size and degree sum are counted afterwards from the
// bitmap (count_bitmap), so a winner costs no offset loads here and a walk
// step keeps kBulkWin windows of loads in flight.
constexpr int kBulkWin = 8;
struct BfsBulkPushFn {
  static constexpr int kWin = kBulkWin;
  const int32_t *tgt;
  uint32_t *visited;
  uint32_t *fout;
  int32_t *dist;  // NULL: the level's D is written by the final pass
  int32_t *parent;
  int32_t level;
  unsigned long long reached;

  template <class Sink>
  __device__ __forceinline__ void drain(Sink &, PushSmem &) {}
  template <class Sink>
  __device__ __forceinline__ void batch(const bool *val, const int32_t *u, const uint32_t *idx,
                                        Sink &, PushSmem &) {
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
#pragma unroll
    for (int r = 0; r < kWin; r++) {
      if (win[r]) {
        if (parent) parent[v[r]] = u[r];
        if (dist) dist[v[r]] = level;
        atomicOr(fout + (v[r] >> 5), 1u << (v[r] & 31));  // result unused: a reduction
        reached++;
      }
    }
  }
};

// Set bits a lane takes per step when it walks its word of a bitmap: their
// offset loads are in flight together.
constexpr int kBitBatch = 4;

// Size and degree sum of a frontier bitmap (vertices of degree >= 2), added
// into *counter with one atomicAdd per CTA: warps take blocks of 32 words,
// every lane walks the set bits of its word kBitBatch at a time.
__device__ void count_bitmap(const BfsParams &P, const uint32_t *fb, unsigned long long *counter,
                             PushSmem &S) {
  const DevGraph &g = P.g;
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const uint32_t nwords = ((uint32_t)g.n + 31) >> 5;
  const uint32_t nblk = (nwords + 31) >> 5;
  const uint32_t gwarp = blockIdx.x * (uint32_t)nw + (threadIdx.x >> 5);
  const uint32_t twarps = gridDim.x * (uint32_t)nw;
  uint32_t c = 0, dg = 0;
  for (uint32_t blk = gwarp; blk < nblk; blk += twarps) {
    const uint32_t wi = blk * 32 + lane;
    uint32_t b = wi < nwords ? fb[wi] : 0u;
    while (b) {  // kBitBatch set bits at a time, their loads in flight together
      uint32_t a[kBitBatch], z[kBitBatch];
#pragma unroll
      for (int k = 0; k < kBitBatch; k++) {
        a[k] = z[k] = 0u;
        if (b) {
          const uint32_t v = wi * 32 + (uint32_t)(__ffs(b) - 1);
          b &= b - 1;
          a[k] = __ldg(g.off + v);
          z[k] = __ldg(g.off + v + 1);
        }
      }
#pragma unroll
      for (int k = 0; k < kBitBatch; k++) {
        const uint32_t d = z[k] - a[k];
        if (d >= 2) {
          c++;
          dg += d;
        }
      }
    }
  }
  const unsigned long long tot = block_sum64(((unsigned long long)c << 32) | dg, S.misc64);
  if (threadIdx.x == 0 && tot) atomicAdd(counter, tot);
}

// Sink of the bulk push: nothing is staged; chunk_end keeps the barrier that
// protects the shared chunk arrays between pieces.
struct NullSink {
  __device__ __forceinline__ void chunk_end(PushSmem &) { __syncthreads(); }
};

// Dense direction (the early-exit pull of §3) as one stream of candidates per
// warp.  Warps take chunks of kChunkWords bitmap words from a global counter;
// a word group (kGroupWords words: visited words, the offsets of every vertex
// and, with f1, the target of every vertex's first arc) is loaded one step
// before it is needed.  A candidate (unvisited, degree > 0) whose first arc
// leads into the frontier is found at once; the others are appended to the
// warp's ring in shared memory with the rest of their list.  Every step each
// lane checks the next 4 arcs of its candidate in CSR order and takes a new
// candidate from the ring as soon as its own resolves, so no lane waits for
// another except at the end of the level.  A candidate still unresolved after
// `pull_serial` arcs is parked in the lane (a lane whose slot is taken keeps
// scanning its candidate itself); once kWalkLanes lanes hold one, the warp
// walks the remaining arcs of all parked candidates together
// (pull_walk_parked), 128 arcs per step.  Words are owned by one warp, whose
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
  bool direct;  // write D now (else the final pass writes it)
  uint32_t scanned, reached;
  uint32_t cnt, deg;  // found vertices of degree >= 2 and their degree sum

  __device__ __forceinline__ void record(const BfsParams &P, int32_t v, int32_t par, uint32_t d) {
    if (direct) P.dist[v] = level;
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
                           const int32_t *f1, bool direct, int32_t level,
                           unsigned long long *counter, unsigned long long &scanned,
                           unsigned long long &reached, unsigned long long &pulled, int inv) {
  const DevGraph &g = P.g;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t nwords = ((uint32_t)g.n + 31) >> 5;
  const uint32_t nchunk = (nwords + kChunkWords - 1) / kChunkWords;
  const uint32_t F = (uint32_t)P.pull_serial;
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t skip = f1 ? 1u : 0u;  // arcs already checked before a candidate enters the ring
  int32_t *rv = S.out_v + warp * kRing;
  uint32_t *rs = S.out_d + warp * kRing, *re = S.pref + warp * kRing;
  uint32_t *scr = S.base + warp * 32;  // per-word bit gathering of one step
  scr[lane] = 0u;
  __syncwarp();
  PullCtx C{level, direct, 0u, 0u, 0u, 0u};
  uint32_t cand_cnt = 0;
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
  // a lane's vertex is the next lane's start, pnext after the last word), the
  // first-arc targets (ph[r]) and its visited words (lane r holds word r)
  uint32_t pa[kGroupWords], pnext = 0, pvis = ~0u;
  int32_t ph[kGroupWords];
  uint32_t head = 0, tail = 0;
  int32_t cv = -1, pv = -1;
  uint32_t ck = 0, ce = 0, cs0 = 0, pk = 0, pe = 0, ps0 = 0;

  // load the next word group (warp-uniform)
#define GBF_PULL_PREFETCH()                                                              \
  do {                                                                                   \
    _Pragma("unroll") for (uint32_t r = 0; r < kGroupWords; r++) {                       \
      const uint32_t v = (gw + r) * 32 + lane;                                           \
      pa[r] = v <= (uint32_t)g.n ? __ldg(g.off + v) : 0u;                                \
      ph[r] = (f1 && v < (uint32_t)g.n) ? __ldg(f1 + v) : -1;                            \
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
    // check the loaded group's candidates' first arcs, append the rest to the
    // ring, then start loading the next group
    if (have && tail - head < kRing - 32 * kGroupWords - 32) {
      bool cd[kGroupWords];
      uint32_t za[kGroupWords];
      unsigned cb[kGroupWords];
      uint32_t ncand = 0;
#pragma unroll
      for (uint32_t r = 0; r < kGroupWords; r++) {
        const uint32_t vis = __shfl_sync(kFull, pvis, r);
        const uint32_t a = pa[r];
        uint32_t z = __shfl_down_sync(kFull, a, 1);
        const uint32_t zn = (r + 1 < kGroupWords) ? __shfl_sync(kFull, pa[r + 1 < kGroupWords ? r + 1 : r], 0)
                                                  : pnext;
        if (lane == 31) z = zn;
        const uint32_t v = (pw + r) * 32 + lane;
        cd[r] = v < (uint32_t)g.n && !((vis >> lane) & 1u) && z > a;
        za[r] = z;
        cb[r] = __ballot_sync(kFull, cd[r]);
        ncand += __popc(cb[r]);
      }
      if (f1 && ncand <= 32) {
        // a sparse group: its candidates side by side, one per lane (lane j
        // takes the j-th, found in its word's ballot), so the first-arc
        // checks, the records and the ring appends run once for all words
        const uint32_t c0 = __popc(cb[0]), c1 = c0 + __popc(cb[1]), c2 = c1 + __popc(cb[2]);
        const uint32_t j = (uint32_t)lane;
        const bool act = j < ncand;
        const uint32_t r = (j >= c0 ? 1u : 0u) + (j >= c1 ? 1u : 0u) + (j >= c2 ? 1u : 0u);
        const uint32_t nth = j - (r == 0 ? 0u : r == 1 ? c0 : r == 2 ? c1 : c2);
        const unsigned br = r == 0 ? cb[0] : r == 1 ? cb[1] : r == 2 ? cb[2] : cb[3];
        const int own = act ? (int)__fns(br, 0u, (int)nth + 1) : 0;  // the candidate's lane
        uint32_t a = 0, z = 0;
        int32_t h = -1;
#pragma unroll
        for (uint32_t q = 0; q < kGroupWords; q++) {
          const uint32_t xa = __shfl_sync(kFull, pa[q], own), xz = __shfl_sync(kFull, za[q], own);
          const int32_t xh = __shfl_sync(kFull, ph[q], own);
          if (q == r) {
            a = xa;
            z = xz;
            h = xh;
          }
        }
        const uint32_t v = (pw + r) * 32 + (uint32_t)own;
        const uint32_t fwv = act ? fin[(uint32_t)h >> 5] : 0u;
        const bool hit = act && ((fwv >> (h & 31)) & 1u);
        if (act) {
          cand_cnt++;
          C.scanned += skip;
        }
        if (hit) C.record(P, (int32_t)v, h, z - a);
#pragma unroll
        for (uint32_t q = 0; q < kGroupWords; q++) {
          const unsigned hb = __reduce_or_sync(kFull, (hit && r == q) ? 1u << own : 0u);
          if (hb && lane == (int)q) {
            atomicOr(fout + pw + q, hb);
            atomicOr(P.visited + pw + q, hb);
          }
        }
        const bool c = act && !hit && z - a > skip;
        const unsigned bal = __ballot_sync(kFull, c);
        if (c) {
          const uint32_t i = (tail + __popc(bal & lt)) & (kRing - 1);
          rv[i] = (int32_t)v;
          rs[i] = a;
          re[i] = z;
        }
        tail += __popc(bal);
      } else {
        uint32_t fw[kGroupWords];
#pragma unroll
        for (uint32_t r = 0; r < kGroupWords; r++)
          fw[r] = (f1 && cd[r]) ? fin[(uint32_t)ph[r] >> 5] : 0u;
#pragma unroll
        for (uint32_t r = 0; r < kGroupWords; r++) {
          const uint32_t a = pa[r], z = za[r];
          const uint32_t v = (pw + r) * 32 + lane;
          const bool hit = f1 && cd[r] && ((fw[r] >> (ph[r] & 31)) & 1u);
          if (cd[r]) {
            cand_cnt++;
            C.scanned += skip;
          }
          const unsigned hb = __ballot_sync(kFull, hit);
          if (hit) C.record(P, (int32_t)v, ph[r], z - a);
          if (hb && lane == 0) {
            atomicOr(fout + pw + r, hb);
            atomicOr(P.visited + pw + r, hb);
          }
          const bool c = cd[r] && !hit && z - a > skip;
          const unsigned bal = __ballot_sync(kFull, c);
          if (c) {
            const uint32_t i = (tail + __popc(bal & lt)) & (kRing - 1);
            rv[i] = (int32_t)v;
            rs[i] = a;
            re[i] = z;
          }
          tail += __popc(bal);
        }
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
        cs0 = rs[i];
        ck = cs0 + skip;
        ce = re[i];
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
  pulled += cand_cnt;
  unsigned long long packed = ((unsigned long long)C.cnt << 32) | C.deg;
  unsigned long long tot = block_sum64(packed, S.misc64);
  if (threadIdx.x == 0 && tot) atomicAdd(counter, tot);
}

// Grid-stride clear of one bitmap.
__device__ __forceinline__ void clear_bitmap(uint32_t *b, uint32_t nwords) {
  const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (uint32_t i = gt; i < nwords; i += gs) b[i] = 0u;
}

// Sparse queue -> bitmap fb (cleared first; two barriers).
__device__ bool queue_to_bitmap(const BfsParams &P, const int32_t *q, uint32_t cnt, uint32_t *fb,
                                Barrier &bar, int *s_flag) {
  const uint32_t nwords = ((uint32_t)P.g.n + 31) >> 5;
  const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  clear_bitmap(fb, nwords);
  if (!grid_sync(P.ctl, bar, s_flag)) return false;
  for (uint32_t i = gt; i < cnt; i += gs) {
    const int32_t v = q[i];
    atomicOr(fb + (v >> 5), 1u << (v & 31));
  }
  return grid_sync(P.ctl, bar, s_flag);
}

// Bitmap -> sparse queue with degree prefix, first-arc offsets and chunk
// starts, warp by warp over blocks of 32 words (1,024 vertices), lane l
// owning word l of the block: a block with no bit set costs one coalesced
// load; otherwise every lane walks the set bits of its word (all lanes'
// offset loads in flight together), the warp scans the lanes' entry counts
// (set bits of degree >= 2) and degree sums, reserves its queue and edge
// range with one 64-bit atomicAdd, and the lanes walk their bits again to
// write the entries (the offsets come back from L1/L2).  No CTA barrier:
// warps finish their blocks independently.
__device__ void bitmap_to_queue(const BfsParams &P, const uint32_t *fb, const QueueOut &out) {
  const DevGraph &g = P.g;
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const uint32_t nwords = ((uint32_t)g.n + 31) >> 5;
  const uint32_t nblk = (nwords + 31) >> 5;
  const uint32_t gwarp = blockIdx.x * (uint32_t)nw + (threadIdx.x >> 5);
  const uint32_t twarps = gridDim.x * (uint32_t)nw;
  for (uint32_t blk = gwarp; blk < nblk; blk += twarps) {
    const uint32_t wi = blk * 32 + lane;
    const uint32_t bits = wi < nwords ? fb[wi] : 0u;
    if (__ballot_sync(kFull, bits != 0u) == 0u) continue;
    // pass 1: this lane's entries and their degree sum
    uint32_t c = 0, dg = 0;
    for (uint32_t b = bits; b;) {
      uint32_t a[kBitBatch], z[kBitBatch];
#pragma unroll
      for (int k = 0; k < kBitBatch; k++) {
        a[k] = z[k] = 0u;
        if (b) {
          const uint32_t v = wi * 32 + (uint32_t)(__ffs(b) - 1);
          b &= b - 1;
          a[k] = __ldg(g.off + v);
          z[k] = __ldg(g.off + v + 1);
        }
      }
#pragma unroll
      for (int k = 0; k < kBitBatch; k++) {
        const uint32_t d = z[k] - a[k];
        if (d >= 2) {
          c++;
          dg += d;
        }
      }
    }
    uint32_t ic = c, id = dg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t yc = __shfl_up_sync(kFull, ic, o), yd = __shfl_up_sync(kFull, id, o);
      if (lane >= o) {
        ic += yc;
        id += yd;
      }
    }
    const uint32_t tc = __shfl_sync(kFull, ic, 31), td = __shfl_sync(kFull, id, 31);
    if (tc == 0u) continue;
    unsigned long long old = 0;
    if (lane == 0) old = atomicAdd(out.counter, ((unsigned long long)tc << 32) | td);
    old = __shfl_sync(kFull, old, 0);
    const uint32_t pos = (uint32_t)(old >> 32), dpos = (uint32_t)old;
    if ((unsigned long long)pos + tc > out.q_cap) {
      if (lane == 0) raise_error(P.ctl, GBF_ERR_OVERFLOW, 12);
      continue;
    }
    // pass 2: write this lane's entries at its exclusive prefix
    uint32_t qi = pos + ic - c, e0 = dpos + id - dg;
    for (uint32_t b = bits; b;) {
      uint32_t vv[kBitBatch], a[kBitBatch], z[kBitBatch];
#pragma unroll
      for (int k = 0; k < kBitBatch; k++) {
        vv[k] = a[k] = z[k] = 0u;
        if (b) {
          vv[k] = wi * 32 + (uint32_t)(__ffs(b) - 1);
          b &= b - 1;
          a[k] = __ldg(g.off + vv[k]);
          z[k] = __ldg(g.off + vv[k] + 1);
        }
      }
#pragma unroll
      for (int k = 0; k < kBitBatch; k++) {
        const uint32_t d = z[k] - a[k];
        if (d < 2) continue;
        out.q[qi] = (int32_t)vv[k];
        out.qoff[qi] = e0;
        out.adj[qi] = a[k];
        for (uint32_t ch = (e0 + kFine - 1) >> kFineLog; (ch << kFineLog) < e0 + d; ch++)
          if (ch < out.cs_cap) out.cs[ch] = qi;
        qi++;
        e0 += d;
      }
    }
  }
}

// Distances of the deferred levels, and INF for every vertex never reached,
// in one coalesced pass; vertices reached in levels that wrote D directly
// (and the source) keep their value.  A warp takes blocks of 32 words: lane
// l loads word l of every bitmap (all loads in flight together), then the
// warp writes the block's 1,024 distances 128 at a time, each lane 4
// consecutive vertices with one 16-byte store.
__device__ void final_dist(const BfsParams &P, int jused, const int32_t *s_lvl) {
  const DevGraph &g = P.g;
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const uint32_t n = (uint32_t)g.n;
  const uint32_t nwords = (n + 31) >> 5;
  const uint32_t nblk = (nwords + 31) >> 5;
  const uint32_t gwarp = blockIdx.x * (uint32_t)nw + (threadIdx.x >> 5);
  const uint32_t twarps = gridDim.x * (uint32_t)nw;
  const bool a16 = ((uintptr_t)P.dist & 15u) == 0;
  for (uint32_t blk = gwarp; blk < nblk; blk += twarps) {
    const uint32_t wi = blk * 32 + lane;
    const bool in = wi < nwords;
    // reached in a direct level (or the source): keep
    uint32_t keep = in ? P.visited[wi] & ~(P.iso ? P.iso[wi] : 0u) : 0u;
    if (in && wi == ((uint32_t)P.src >> 5)) keep |= 1u << (P.src & 31);
    uint32_t lw[kMaxDeferred];
#pragma unroll
    for (int j = 0; j < kMaxDeferred; j++)
      lw[j] = (j < jused && in) ? P.lb[(size_t)j * nwords + wi] : 0u;
#pragma unroll
    for (int j = 0; j < kMaxDeferred; j++) keep &= ~lw[j];
    // step q: vertices blk*1024 + 128 q + 4 lane .. + 3, in word 4 q + lane / 8
    for (int q = 0; q < 8; q++) {
      const int sl = 4 * q + (lane >> 3);
      const uint32_t sh = 4u * (uint32_t)(lane & 7);
      const uint32_t kp = __shfl_sync(kFull, keep, sl) >> sh;
      int32_t d[4] = {kInf, kInf, kInf, kInf};
#pragma unroll
      for (int j = 0; j < kMaxDeferred; j++) {
        if (j < jused) {
          const uint32_t b = __shfl_sync(kFull, lw[j], sl) >> sh;
          const int32_t lv = s_lvl[j];
#pragma unroll
          for (int k = 0; k < 4; k++)
            if ((b >> k) & 1u) d[k] = lv;
        }
      }
      const uint32_t v0 = blk * 1024u + 128u * (uint32_t)q + 4u * (uint32_t)lane;
      if (a16 && (kp & 15u) == 0 && v0 + 4 <= n) {
        *reinterpret_cast<int4 *>(P.dist + v0) = make_int4(d[0], d[1], d[2], d[3]);
      } else {
#pragma unroll
        for (int k = 0; k < 4; k++)
          if (v0 + k < n && !((kp >> k) & 1u)) P.dist[v0 + k] = d[k];
      }
    }
  }
}

}  // namespace

__global__ void __launch_bounds__(1024) bfs_kernel(BfsParams P) {
  extern __shared__ unsigned long long smem_raw[];
  __shared__ int s_flag;
  __shared__ int32_t s_lvl[kMaxDeferred];
  PushSmem S = carve_push_smem(smem_raw, SmemShape{P.bmax, P.cap, 0, 0, 1});
  if (threadIdx.x == 0) S.misc[0] = 0;
  Ctl *ctl = P.ctl;
  Barrier bar{0u, P.cap_ns};
  const DevGraph g = P.g;
  const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  const uint32_t nwords = ((uint32_t)g.n + 31) >> 5;
  const int32_t src = P.src;
  unsigned long long scanned = 0, reached = 0, expanded = 0, pulled = 0;
  const unsigned long long t_start = globaltimer();

  // Initialisation (Alg. 1): parents -1, the visited
  // bitmap holds the vertices of degree 0 (never candidates) and the source;
  // D is written by the final pass or by the level that reaches a vertex.
  if (P.parent) {
    const uint32_t n4 = ((uintptr_t)P.parent & 15u) == 0 ? (uint32_t)g.n >> 2 : 0u;
    for (uint32_t i = gt; i < n4; i += gs)
      *reinterpret_cast<int4 *>(P.parent + 4 * i) = make_int4(-1, -1, -1, -1);
    for (uint32_t i = 4 * n4 + gt; i < (uint32_t)g.n; i += gs) P.parent[i] = -1;
  }
  for (uint32_t i = gt; i < nwords; i += gs)
    P.visited[i] = (P.iso ? P.iso[i] : 0u) | ((i == ((uint32_t)src >> 5)) ? (1u << (src & 31)) : 0u);
  if (P.jmax > 0) clear_bitmap(P.lb, nwords);
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
    if (threadIdx.x == 0) {
      reached = 1;
      P.dist[src] = 0;
    }
  }
  if (P.inject_wait && blockIdx.x == 0 && threadIdx.x == 0) injected_wait(ctl, P.cap_ns);
  __syncthreads();
  // the source's parent after the parent initialisation of every CTA
  bool ok = grid_sync(ctl, bar, &s_flag);
  if (ok && P.parent && blockIdx.x == 0 && threadIdx.x == 0) P.parent[src] = src;

  int in_bm = 0;                  // input frontier: 0 = queue q[qb], 1 = bitmap fin
  const uint32_t *fin = nullptr;
  int fin_rb = -1;                // rotating bitmap holding fin, or -1
  int qb = 0, jn = 0, rr = 0, was_dense = 0;
  int cleared = P.jmax > 0 ? 1 : 0;  // deferred bitmaps cleared so far
  int bem = 0;  // blocked edgeMap / pull invocations so far
  int level = 1;
  unsigned long long fr = ok ? ld_vol(ctl->fr[0]) : 0ull;
  while (ok) {
    uint32_t cnt = (uint32_t)(fr >> 32), D = (uint32_t)fr;
    if (cnt == 0) break;
    bool dense = P.pull_divisor > 0 && (unsigned long long)D * (unsigned)P.pull_divisor > g.m;
    if (!dense && was_dense && P.pull_divisor > 0 && P.pull_stay > 0 &&
        (unsigned long long)cnt * (unsigned)P.pull_stay > (unsigned long long)g.n)
      dense = true;
    bool converted = false;
    long long t_mid = 0;  // end of the level's first phase (conversion, or push before its count)
    // the input frontier in the form this direction reads
    if (!dense && in_bm) {
      unsigned long long *cv = &ctl->cv[level % 3];
      QueueOut out{P.q[0], P.qoff[0], P.qadj[0], P.cs[0], cv, (uint32_t)g.n, P.cs_cap};
      bitmap_to_queue(P, fin, out);
      if (!grid_sync(ctl, bar, &s_flag)) break;
      t_mid = (long long)(globaltimer() - t_start);
      const unsigned long long c2 = ld_vol(*cv);
      cnt = (uint32_t)(c2 >> 32);
      D = (uint32_t)c2;
      in_bm = 0;
      qb = 0;
      fin_rb = -1;
      converted = true;
    } else if (dense && !in_bm) {
      const int x = rr;
      rr = (rr + 1) % 3;
      if (!queue_to_bitmap(P, P.q[qb], cnt, P.rb[x], bar, &s_flag)) break;
      fin = P.rb[x];
      fin_rb = x;
      in_bm = 1;
    }
    // the output: a deferred bitmap, a rotating bitmap (D written now), or a queue
    const bool bulk = dense || D >= P.bulk_min;
    uint32_t *fout = nullptr;
    bool direct = true;
    if (bulk) {
      if (jn < P.jmax) {
        fout = P.lb + (size_t)jn * nwords;
        if (threadIdx.x == 0) s_lvl[jn] = level;
        jn++;
        direct = false;
      } else {
        int x = rr;
        if (x == fin_rb) x = (x + 1) % 3;
        rr = (x + 1) % 3;
        fout = P.rb[x];
        clear_bitmap(fout, nwords);
        if (!grid_sync(ctl, bar, &s_flag)) break;
      }
    }
    // clear the deferred bitmap a later level will take
    if (cleared < P.jmax && cleared <= jn) {
      clear_bitmap(P.lb + (size_t)cleared * nwords, nwords);
      cleared++;
    }
    unsigned long long *outc = &ctl->fr[level % 3];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st_vol(ctl->fr[(level + 1) % 3], 0ull);
      st_vol(ctl->cv[(level + 1) % 3], 0ull);
      if (dense) atomicAdd(&ctl->pull_rounds, 1);
      else {
        atomicAdd(&ctl->push_rounds, 1);
        scanned += D;
        expanded += cnt;
      }
      atomicAdd(&ctl->rounds, 1);
    }
    if (!dense) {
      QueueIn in{P.q[qb], P.qoff[qb], P.qadj[qb], P.cs[qb], cnt, D};
      if (!bulk) {
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
        BfsBulkPushFn fn{g.tgt, P.visited, fout, direct ? P.dist : nullptr, P.parent, level, 0};
        NullSink sink;
        // nothing is staged, so a chunk may span many walk steps
        const int s = chunk_shift(D, 4u, 6);
        blocked_edge_map(g, in, s, (uint32_t)P.bmax, S, fn, sink, ctl, bem++);
        reached += fn.reached;
        if (!grid_sync(ctl, bar, &s_flag)) break;
        t_mid = (long long)(globaltimer() - t_start);
        count_bitmap(P, fout, outc, S);
      }
    } else {
      // the first-arc check pays when a candidate's first arc (the arc to its
      // highest-degree neighbour) leads into the frontier often: when the
      // frontier holds more than an eighth of all arcs, or when its vertices
      // average more than 8 times the graph's mean degree (a frontier of hubs)
      const bool hubs = (unsigned long long)D * (unsigned)g.n >
                        8ull * (unsigned long long)g.m * (unsigned long long)cnt;
      const int32_t *f1 = ((unsigned long long)D * 8ull > g.m || hubs) ? P.f1 : nullptr;
      pull_level(P, S, fin, fout, f1, direct, level, outc, scanned, reached, pulled, bem++);
    }
    if (!grid_sync(ctl, bar, &s_flag)) break;
    fr = ld_vol(*outc);
    if (bulk) {
      in_bm = 1;
      fin = fout;
      fin_rb = direct ? (fout == P.rb[0] ? 0 : fout == P.rb[1] ? 1 : 2) : -1;
    } else {
      in_bm = 0;
    }
    was_dense = dense;
    if (P.trace && blockIdx.x == 0 && threadIdx.x == 0 && level <= P.trace_cap) {
      // 1 sparse (queue out), 2 dense, 6 sparse with bitmap out; +1 (1 -> 4,
      // 6 -> 7) after a bitmap -> queue conversion
      int kind = dense ? 2 : bulk ? 6 : 1;
      if (converted) kind = kind == 1 ? 4 : 7;
      P.trace[level - 1] =
          TraceRec{level, kind, cnt, D, (long long)(globaltimer() - t_start), t_mid};
    }
    level++;
  }
  if (ok) {
    __syncthreads();
    if (ld_vol(ctl->err) == 0) final_dist(P, jn, s_lvl);
  }
  // the last CTA to get here records the kernel's end (for the trace)
  __syncthreads();
  if (threadIdx.x == 0 && atomicAdd(&ctl->done, 1u) == gridDim.x - 1)
    st_vol(ctl->t_end_ns, (long long)(globaltimer() - t_start));
  // statistics
  unsigned long long t;
  t = block_sum64(scanned, S.misc64);
  if (threadIdx.x == 0 && t) atomicAdd(&ctl->edges_scanned, t);
  t = block_sum64(reached, S.misc64);
  if (threadIdx.x == 0 && t) atomicAdd(&ctl->reached, t);
  t = block_sum64(expanded, S.misc64);
  if (threadIdx.x == 0 && t) atomicAdd(&ctl->expanded, t);
  t = block_sum64(pulled, S.misc64);
  if (threadIdx.x == 0 && t) atomicAdd(&ctl->pulled, t);
}

// Dynamic shared memory of bfs_kernel for a heavy cutoff and block size (the
// dense step's rings live inside the staging area).
static size_t bfs_smem_bytes(int heavy_cutoff, int block) {
  return push_smem_bytes(SmemShape{heavy_cutoff, stage_capacity(block), 0, 0, 1});
}

gbf_status launch_bfs(Graph &g, Workspace &ws, int32_t src, int32_t *dist, int32_t *parent,
                      const Opts &o, cudaStream_t st) {
  BfsParams P;
  P.g = g.dev();
  P.iso = g.iso;
  P.f1 = g.f1;
  P.src = src;
  P.dist = dist;
  P.parent = parent;
  P.visited = ws.visited;
  P.lb = ws.lb;
  P.jmax = ws.lb ? std::min(ws.lb_count, kMaxDeferred) : 0;
  for (int i = 0; i < 3; i++) P.rb[i] = ws.fbm[i];
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
  P.pull_stay = o.pull_stay;
  P.bulk_min = std::max<uint32_t>((uint32_t)g.n / 16u, 1u);
  P.bmax = o.heavy_cutoff;
  P.cap = stage_capacity(o.block);
  P.pull_serial = o.pull_serial;
  P.inject_wait = o.inject_wait;
  P.cap_ns = o.spin_cap_ns;
  const size_t smem = bfs_smem_bytes(o.heavy_cutoff, o.block);
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
  const size_t smem = bfs_smem_bytes(o.heavy_cutoff, o.block);
  if (cudaFuncSetAttribute(bfs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bfs_kernel, o.block, smem) != cudaSuccess)
    return 0;
  return per_sm;
}

}  // namespace gbf
