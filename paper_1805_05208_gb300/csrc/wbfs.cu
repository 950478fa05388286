// Weighted BFS (integral-weight SSSP, §4; Alg. 3) as one persistent
// cooperative kernel.  One bucket round:
//
//   nextBucket: every CTA computes, from the bucket counters, the smallest
//     bucket value b with unconsumed entries (identically in every CTA).
//   edgeMapData (Alg. 3 Update): the live entries of bucket b (D[v] == b;
//     entries whose distance dropped after they were filed are stale — lazy
//     deletion) relax their arcs: nDist = b + w; if nDist < D[d], priority-
//     write D[d] with atomicMin.  A successful write files d straight into
//     the bucket of its new distance (Reset + updateBuckets of Alg. 3, done
//     at the write instead of in a later vertexMap pass, so a round needs no
//     Moved list and no test-and-set: a vertex lowered twice in a round
//     leaves one stale entry behind).  A vertex of degree 1 is not filed:
//     lowered through its only neighbour, it has its final distance and
//     nothing to relax.
//       - vertices with at most heavy_cutoff / 8 arcs (32 at least) are
//         expanded by the CTA that extracted them: a CTA-local degree prefix
//         over the staged entries, then warps walk their arcs in 32-arc
//         windows (the blocked edgeMap's walk, on one CTA's entries);
//       - heavier vertices are compacted into a frontier queue with a global
//         degree prefix and expanded afterwards by the blocked edgeMap
//         (§6.2) over all CTAs, so one hub is spread over the whole GPU.
//   With dense_wbfs, a bucket with more than n / pull_divisor entries is
//   instead pulled: every vertex with D[v] > b + 1 takes the minimum of b + w
//   over neighbours with D[u] == b (the dense switch of the SSSP experiments).
//
// One bounded grid barrier per round, two when heavy vertices were found.
//
// Bucket structure (Julienne's makeBuckets / nextBucket / updateBuckets,
// INCREASING order): nB open buckets, value x in slot x mod nB; each slot is
// a ring buffer of n entries with a monotone append counter, and every CTA
// keeps the consumed position of each slot in shared memory (all CTAs consume
// identically).  A value has at most n entries (D only decreases), so a ring
// never overwrites unconsumed entries.  If nB > max weight the window slides
// to the current bucket and nothing overflows.  Otherwise the window is fixed
// and values beyond it go to an overflow bucket, which refills a window
// starting at its minimum once the open buckets run dry.
//
// Δ-stepping (the coarsening the SSSP discussion of §7 sets wBFS against;
// the kDelta instance, Δ = 2^dl): bucket q holds the distances [qΔ, (q+1)Δ)
// and "value" above reads "bucket index" (an entry is live iff D[v] / Δ is
// its bucket).  Each arc adds w to its source's current D.  A vertex lowered
// into the bucket being processed goes on the round's side list (a
// test-and-set on a per-round flag bitmap keeps it there once) and the next
// round expands the side list, again in bucket b, until a round leaves it
// empty; only then is the next bucket taken.  Distances are exact for any Δ:
// every vertex is expanded again after its last lowering.
#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "gbf_impl.h"

namespace gbf {
using namespace dev;

struct WbfsParams {
  DevGraph g;
  const uint32_t *leaf;  // bit v set iff deg(v) == 1
  int32_t src;
  int32_t *dist;
  int32_t *slots;
  uint32_t *slot_cnt;
  int32_t nB;
  int slide;
  int2 *ovf[2];
  uint32_t ovf_cap;
  int32_t *q;
  uint32_t *qoff;
  uint32_t *cs;
  uint32_t cs_cap;
  Ctl *ctl;
  TraceRec *trace;
  int trace_cap;
  int pull_divisor;
  int dense;
  int bmax;
  int cap;
  int log2_bmax_fine;
  int heavy;
  int local_arcs;  // CTA-local rounds: most live arcs of a bucket one CTA expands alone
  int inject_wait;
  long long cap_ns;
  // Δ-stepping (dl > 0): buckets hold distance ranges [qΔ, (q+1)Δ), Δ = 2^dl;
  // a vertex lowered into the bucket being processed joins that round's side
  // list (once per round: test-and-set on a flag bitmap) instead of a ring
  int dl;
  int32_t *side[2];   // side lists by round parity, n entries each
  uint32_t *sflag[2]; // their flag bitmaps, ceil(n/32) words each
  int32_t *xround;    // the last round each vertex was expanded in (n)
};

namespace {

constexpr int kMaskWords = 8;  // pending / filed slot masks: nB <= 256
constexpr int32_t kNoSlot = -1;  // a staged entry dropped at the flush (overflow slots are <= -2)

struct Counters {
  unsigned long long scanned, relax, inserts, expanded, heavy, pulled;
};

// Bucket filing, staged per CTA: lanes whose writeMin succeeded reserve a
// place in the shared-memory stage (one shared atomic per warp); the CTA then
// flushes the stage with one global atomicAdd per bucket slot touched, so
// the few slot counters are not hammered once per warp.
struct FileSink {
  const WbfsParams *P;
  int32_t lo;
  int cur;
  Counters *c;
  unsigned *imask;   // this round's filed-slot mask (global)
  unsigned *s_pub;   // slots this CTA already published this round
  int32_t bq;        // bucket being processed (Δ-stepping), -1 if none
  int32_t *sq;       // this round's side list, its flag bitmap and count
  uint32_t *sfl;
  unsigned *scnt;
  uint32_t *cnt_out;  // CTA-local rounds: the CTA's copy of the slot counters, kept current

  __device__ __forceinline__ void append(PushSmem &S, bool low, int32_t v, uint32_t ndu) {
    const unsigned bal = __ballot_sync(kFull, low);
    if (bal == 0) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(bal) - 1;
    uint32_t pos = 0;
    if (lane == leader) pos = atomicAdd(&S.misc[4], (uint32_t)__popc(bal));
    pos = __shfl_sync(kFull, pos, leader);
    if (!low) return;
    const int32_t sl = slot_of((int32_t)ndu);
    const uint32_t r = pos + __popc(bal & lanemask_lt());
    if (r < S.cap_out) {
      S.fv[r] = v;
      S.fs[r] = sl;
      return;
    }
    file_direct(v, (int32_t)ndu, sl);  // the stage is full
  }
  // Where distance nd is filed: ring slot q mod nB of its bucket q, the
  // overflow bucket (-q - 2) beyond a fixed window, or nB: the side list of
  // the bucket being processed (Δ-stepping only; in exact wBFS every filed
  // distance lies above the current bucket).
  __device__ __forceinline__ int32_t slot_of(int32_t nd) const {
    const int32_t q = nd >> P->dl;
    if (q == bq) return P->nB;
    return (P->slide || q < lo + P->nB) ? q % P->nB : -q - 2;
  }
  // An entry that found the stage full, filed directly.
  __device__ __forceinline__ void file_direct(int32_t v, int32_t nd, int32_t sl) {
    if (sl == P->nB) {
      const unsigned bit = 1u << (v & 31);
      if (atomicOr(sfl + (v >> 5), bit) & bit) return;  // already on this round's side list
      const uint32_t gp = atomicAdd(scnt, 1u);
      if (gp < (uint32_t)P->g.n) sq[gp] = v;
      else raise_error(P->ctl, GBF_ERR_OVERFLOW, 13);
    } else if (sl >= 0) {
      const uint32_t raw = atomicAdd(P->slot_cnt + sl, 1u);
      P->slots[(size_t)sl * (size_t)P->g.n + raw % (uint32_t)P->g.n] = v;
      atomicOr(imask + (sl >> 5), 1u << (sl & 31));
      if (cnt_out) {  // CTA-local round: the filed mask and counter of this CTA alone
        atomicOr(s_pub + (sl >> 5), 1u << (sl & 31));
        atomicMax(cnt_out + sl, raw + 1u);
      }
    } else {
      const uint32_t gp = atomicAdd(&P->ctl->ovf_cnt[cur], 1u);
      if (gp < P->ovf_cap) {
        P->ovf[cur][gp] = make_int2(v, -sl - 2);
        atomicMin(&P->ctl->ovf_min[cur], -sl - 2);
      } else {
        raise_error(P->ctl, GBF_ERR_OVERFLOW, 12);
      }
    }
    c->inserts++;
  }
  // Warp-collective: the U filings of one walk step with one shared-memory
  // atomic for the whole warp.
  template <int U>
  __device__ __forceinline__ void append_n(PushSmem &S, const bool *low, const int32_t *v,
                                           const uint32_t *ndu, const uint32_t *) {
    unsigned bal[U];
    uint32_t tot = 0;
#pragma unroll
    for (int r = 0; r < U; r++) {
      bal[r] = __ballot_sync(kFull, low[r]);
      tot += __popc(bal[r]);
    }
    if (tot == 0) return;
    const int lane = threadIdx.x & 31;
    uint32_t pos = 0;
    if (lane == 0) pos = atomicAdd(&S.misc[4], tot);
    pos = __shfl_sync(kFull, pos, 0);
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int r = 0; r < U; r++) {
      if (low[r]) {
        const int32_t nd = (int32_t)ndu[r];
        const int32_t sl = slot_of(nd);
        const uint32_t i = pos + __popc(bal[r] & lt);
        if (i < S.cap_out) {
          S.fv[i] = v[r];
          S.fs[i] = sl;
        } else {
          file_direct(v[r], nd, sl);
        }
      }
      pos += __popc(bal[r]);
    }
  }
  // CTA-collective, between chunks / loop iterations.
  __device__ __forceinline__ void chunk_end(PushSmem &S) {
    __syncthreads();
    if (S.misc[4] > (S.cap_out >> 1)) flush(S);
  }
  // CTA-collective.
  __device__ void flush(PushSmem &S) {
    __syncthreads();
    const uint32_t k = min(S.misc[4], S.cap_out);  // entries beyond cap were filed directly
    if (k == 0) return;
    const int nB = P->nB;
    const uint32_t n = (uint32_t)P->g.n;
    for (int i = threadIdx.x; i <= nB; i += blockDim.x) S.hist[i] = 0u;  // [nB]: side list
    if (threadIdx.x == 0) {
      S.misc[5] = 0u;
      S.misc[7] = (uint32_t)kInf;
    }
    __syncthreads();
    // A vertex of degree 1 lowered here was lowered through its only
    // neighbour, whose distance is final: its own distance is final too and
    // expanding it could not lower anything, so it is not filed (its entry
    // would only be extracted and skipped).  The source is never filed here.
    for (uint32_t i = threadIdx.x; i < k; i += blockDim.x) {
      const int32_t v = S.fv[i];
      if ((__ldg(P->leaf + (v >> 5)) >> (v & 31)) & 1u) {
        S.fs[i] = kNoSlot;
        continue;
      }
      const int32_t sl = S.fs[i];
      if (sl == nB) {  // side list: once per vertex and round
        const unsigned bit = 1u << (v & 31);
        if (atomicOr(sfl + (v >> 5), bit) & bit) {
          S.fs[i] = kNoSlot;
          continue;
        }
        S.pref[i] = atomicAdd(&S.hist[nB], 1u);
      } else if (sl >= 0) {
        S.pref[i] = atomicAdd(&S.hist[sl], 1u);
      } else {
        S.pref[i] = atomicAdd(&S.misc[5], 1u);
        atomicMin(&S.misc[7], (uint32_t)(-sl - 2));
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && S.hist[nB]) S.gbase[nB] = atomicAdd(scnt, S.hist[nB]);
    for (int i = threadIdx.x; i < nB; i += blockDim.x) {
      const uint32_t h = S.hist[i];
      if (h) {
        S.gbase[i] = atomicAdd(P->slot_cnt + i, h);
        if (cnt_out) cnt_out[i] = S.gbase[i] + h;
        const unsigned bit = 1u << (i & 31);
        if (!(s_pub[i >> 5] & bit)) {
          atomicOr(s_pub + (i >> 5), bit);
          atomicOr(imask + (i >> 5), bit);
        }
      }
    }
    if (threadIdx.x == 0 && S.misc[5]) {
      S.misc[6] = atomicAdd(&P->ctl->ovf_cnt[cur], S.misc[5]);
      atomicMin(&P->ctl->ovf_min[cur], (int)S.misc[7]);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < k; i += blockDim.x) {
      const int32_t sl = S.fs[i];
      const int32_t v = S.fv[i];
      if (sl == kNoSlot) continue;
      if (sl == nB) {
        const uint32_t pos = S.gbase[nB] + S.pref[i];
        if (pos < n) sq[pos] = v;
        else raise_error(P->ctl, GBF_ERR_OVERFLOW, 14);
        c->inserts++;
      } else if (sl >= 0) {
        const uint32_t pos = (S.gbase[sl] + S.pref[i]) % n;
        P->slots[(size_t)sl * n + pos] = v;
        c->inserts++;
      } else {
        const uint32_t pos = S.misc[6] + S.pref[i];
        if (pos < P->ovf_cap) P->ovf[cur][pos] = make_int2(v, -sl - 2);
        else raise_error(P->ctl, GBF_ERR_OVERFLOW, 6);
        c->inserts++;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) S.misc[4] = 0;
    __syncthreads();
  }
};

// Update of Alg. 3 for kU windows of arcs out of bucket b: all target and
// weight loads, then the distance loads, then the writeMins.  The writeMins
// of a step are consumed (successes filed) at the next step, after its
// target loads are issued, so their latency overlaps the next step's loads;
// drain() files the last step's.  In exact wBFS every live entry of bucket b
// has D == b, so nDist = b + w; under Δ-stepping (kDelta) the bucket holds a
// range of distances and each arc adds w to its source's current D.
template <bool kDelta>
struct RelaxFn {
  static constexpr int kWin = kU;  // windows per walk step
  const int32_t *tgt;
  const uint32_t *w;
  int32_t *dist;
  int32_t b;
  unsigned long long relax;
  // the previous step: targets, proposed distances, writeMin results (equal
  // to the proposal where no writeMin was issued)
  int32_t pv[kU], pnd[kU], pold[kU];
  uint64_t stream_pol, keep_pol;  // L2 policies: arcs leave first, D stays

  template <class Sink>
  __device__ __forceinline__ void drain(Sink &sink, PushSmem &S) {
    bool low[kU];
#pragma unroll
    for (int r = 0; r < kU; r++) {
      low[r] = pold[r] > pnd[r];
      if (low[r]) relax++;
    }
    sink.template append_n<kU>(S, low, pv, (const uint32_t *)pnd, nullptr);
#pragma unroll
    for (int r = 0; r < kU; r++) pold[r] = pnd[r];
  }
  template <class Sink>
  __device__ __forceinline__ void batch(const bool *val, const int32_t *uu, const uint32_t *idx,
                                        Sink &sink, PushSmem &S) {
    int32_t v[kU], nd[kU];
#pragma unroll
    for (int r = 0; r < kU; r++) {
      const int32_t base = kDelta ? (val[r] ? __ldcg(dist + uu[r]) : 0) : b;
      v[r] = val[r] ? (int32_t)ldg_pol(tgt + idx[r], stream_pol) : 0;
      nd[r] = val[r] ? base + (int32_t)ldg_pol(w + idx[r], stream_pol) : kInf;
    }
    drain(sink, S);
    // read D at L2 (.cg): L1 lines of D go stale as other SMs lower it, and a
    // stale (larger) value only costs a writeMin that cannot succeed
    int32_t dv[kU];
#pragma unroll
    for (int r = 0; r < kU; r++) dv[r] = val[r] ? (int32_t)ldcg_pol(dist + v[r], keep_pol) : kInf;
#pragma unroll
    for (int r = 0; r < kU; r++) {
      pold[r] = nd[r] < dv[r] ? atomicMin(dist + v[r], nd[r]) : nd[r];
      pv[r] = v[r];
      pnd[r] = nd[r];
    }
  }
};

// Dense edgeMap for one bucket: owner-computes pull of min(b + w) over
// neighbours with D[u] == b, into every vertex with D[v] > b + 1.  Word-
// contiguous CTA ranges keep the loop CTA-uniform for the filing stage.
__device__ void dense_round(const WbfsParams &P, int32_t b, PushSmem &S, FileSink &sink,
                            Counters &c) {
  const DevGraph &g = P.g;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t nwords = ((uint32_t)g.n + 31) >> 5;
  const uint32_t per = (nwords + gridDim.x - 1) / gridDim.x;
  const uint32_t wlo = min(nwords, blockIdx.x * per), whi = min(nwords, wlo + per);
  for (uint32_t base = wlo; base < whi; base += nw) {
    const uint32_t wi = base + warp;
    const int32_t v = (int32_t)(wi * 32 + lane);
    int32_t dv = kInf;
    uint32_t s = 0, e = 0;
    bool cand = false;
    if (wi < whi && v < g.n) {
      dv = P.dist[v];
      if (dv > b + 1) {
        s = __ldg(g.off + v);
        e = __ldg(g.off + v + 1);
        cand = e > s;
      }
    }
    int32_t best = kInf;
    if (cand) c.pulled++;
    unsigned rm = __ballot_sync(kFull, cand);
    // each candidate's list is scanned by the whole warp, 32 arcs at a time,
    // stopping once the lower bound b + 1 is reached
    while (rm) {
      const int l = __ffs(rm) - 1;
      rm &= rm - 1;
      const uint32_t ks = __shfl_sync(kFull, s, l), ke = __shfl_sync(kFull, e, l);
      int32_t wb = kInf;
      for (uint32_t k0 = ks; k0 < ke && wb != b + 1; k0 += 32) {
        const uint32_t kk = k0 + lane;
        int32_t cd = kInf;
        if (kk < ke) {
          const int32_t u = __ldg(g.tgt + kk);
          if (P.dist[u] == b) cd = b + (int32_t)__ldg(g.w + kk);
        }
        wb = min(wb, (int32_t)__reduce_min_sync(kFull, cd));
        if (lane == 0) c.scanned += min(32u, ke - k0);
      }
      if (lane == l) best = wb;
    }
    const bool low = cand && best < dv;
    if (low) {
      P.dist[v] = best;
      c.relax++;
    }
    sink.append(S, low, v, (uint32_t)best);
    sink.chunk_end(S);
  }
  sink.flush(S);
}

// nextBucket from the CTA's pending-slot set (identical in every CTA): the
// smallest value among slots marked pending, or kInf.  Values of the window
// [lo, lo + nB) map one-to-one to slots.
__device__ int32_t next_bucket(const unsigned *s_pend, int nB, int32_t lo, int *s_tmp) {
  int32_t best = kInf;
  for (int i = threadIdx.x; i < nB; i += blockDim.x) {
    if ((s_pend[i >> 5] >> (i & 31)) & 1u) {
      const int32_t rel = ((i - lo % nB) % nB + nB) % nB;
      best = min(best, lo + rel);
    }
  }
  best = block_min_i32(best, s_tmp);
  if (threadIdx.x == 0) s_tmp[32] = best;
  __syncthreads();
  best = s_tmp[32];
  __syncthreads();
  return best;
}

}  // namespace

// Shared-memory shape of the kernel: the filing histogram has nB ring slots
// and the side list.
__host__ __device__ inline SmemShape wbfs_smem_shape(int bmax, int cap, int nB) {
  return SmemShape{bmax, cap, 1, nB + 1};
}
// Dynamic shared memory: the edgeMap stage, then per ring slot the consumed
// position and the append counter as read after the last barrier.
__host__ __device__ inline size_t wbfs_smem_bytes(int bmax, int cap, int nB) {
  return push_smem_bytes(wbfs_smem_shape(bmax, cap, nB)) + 2 * sizeof(uint32_t) * (size_t)nB;
}

// What round t + 1 starts from, read in one batch after the barrier that
// completes round t's filings (with whatever else the caller loads there):
// the slots filed in round t (mask t % 3; this thread's word), the length of
// round t's side list (Δ-stepping) and every slot's append counter.  The
// counter of the slot that round t + 1 consumes is final here: no round
// files into its own bucket's slot.
struct RoundState {
  unsigned mask;
  uint32_t side;
};
__device__ __forceinline__ RoundState read_round_state(const WbfsParams &P, int t, uint32_t *s_cnt) {
  RoundState r{0u, 0u};
  if (threadIdx.x < kMaskWords) r.mask = ld_vol(P.ctl->imask[t % 3][threadIdx.x]);
  if (P.dl > 0) r.side = ld_vol(P.ctl->scnt[t % 3]);
  for (int i = threadIdx.x; i < P.nB; i += blockDim.x) s_cnt[i] = ld_vol(P.slot_cnt[i]);
  return r;
}

// kLocal: the instance with CTA-local rounds (local_arcs > 0): a bucket of
// at most blockDim entries whose live entries hold at most local_arcs arcs
// is expanded by CTA 0 alone, and so are the following buckets while they
// stay that small, with CTA barriers only; the other CTAs wait at one grid
// barrier and resume from the bucket state CTA 0 hands back.  A separate
// instance, so that the other one's registers are those of the rounds alone.
template <bool kDelta, bool kLocal>
__global__ void __launch_bounds__(1024) wbfs_kernel(WbfsParams P) {
  extern __shared__ unsigned long long smem_raw[];
  __shared__ int s_flag;
  __shared__ int s_int[40];
  __shared__ unsigned s_pend[kMaskWords];  // slots with unconsumed entries
  __shared__ unsigned s_pub[kMaskWords];   // slots this CTA already published this round
  const int nB = P.nB;
  const SmemShape sh = wbfs_smem_shape(P.bmax, P.cap, nB);
  PushSmem S = carve_push_smem(smem_raw, sh);
  uint32_t *s_base = (uint32_t *)((char *)smem_raw + push_smem_bytes(sh));
  uint32_t *s_cnt = s_base + nB;
  for (int i = threadIdx.x; i < nB; i += blockDim.x) s_base[i] = 0u;
  for (int i = threadIdx.x; i < kMaskWords; i += blockDim.x) {
    s_pend[i] = (i == 0) ? 1u : 0u;  // the source sits in slot 0
    s_pub[i] = 0u;
  }
  if (threadIdx.x == 0) {
    S.misc[0] = 0;
    S.misc[4] = 0;
  }
  Ctl *ctl = P.ctl;
  Barrier bar{0u, P.cap_ns};
  const DevGraph g = P.g;
  const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  const int32_t src = P.src;
  Counters c{0, 0, 0, 0, 0, 0};
  const unsigned long long t_start = globaltimer();

  // makeBuckets: D = inf except D[src] = 0; src filed in bucket 0.
  for (uint32_t i = gt; i < (uint32_t)g.n; i += gs) P.dist[i] = (i == (uint32_t)src) ? 0 : kInf;
  if (kDelta) {
    const uint32_t nwords = ((uint32_t)g.n + 31) >> 5;
    for (uint32_t i = gt; i < nwords; i += gs) {
      P.sflag[0][i] = 0u;
      P.sflag[1][i] = 0u;
    }
    for (uint32_t i = gt; i < (uint32_t)g.n; i += gs) P.xround[i] = 0;
  }
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < nB; i += blockDim.x) P.slot_cnt[i] = (i == 0) ? 1u : 0u;
    if (threadIdx.x == 0) {
      P.slots[0] = src;
      ctl->ovf_min[0] = kInf;
      ctl->ovf_min[1] = kInf;
    }
  }
  if (P.inject_wait && blockIdx.x == 0 && threadIdx.x == 0) injected_wait(ctl, P.cap_ns);
  __syncthreads();
  bool ok = grid_sync(ctl, bar, &s_flag);
  // the slot counters after makeBuckets; no round has filed yet
  RoundState rs = read_round_state(P, 0, s_cnt);
  rs.mask = 0u;
  rs.side = 0u;

  int32_t lo = 0;
  int bem = 0;         // blocked edgeMap invocations so far
  int cur = 0;         // active overflow buffer
  int32_t prev = -1;   // slot consumed by the previous round (-1: none)
  int32_t bcur = -1;   // Δ-stepping: the bucket being processed
  bool in_local = false;         // kLocal, CTA 0: inside a run of CTA-local rounds
  unsigned long long t_loc = 0;  // kLocal, thread 0 of CTA 0: when that run began
  for (int32_t t = 1; ok; t++) {
    // ---------------- nextBucket.  Pending slots: those of the last round
    // minus the one it consumed, plus every slot filed into during it (the
    // masks of round t-1 are complete: a grid barrier separates the rounds).
    // Fast CTAs already filing in round t write mask t % 3, read by nobody yet.
    unsigned *imask = ctl->imask[t % 3];
    if (threadIdx.x < kMaskWords) {
      unsigned pm = s_pend[threadIdx.x];
      if (prev >= 0 && (prev >> 5) == (int)threadIdx.x) pm &= ~(1u << (prev & 31));
      pm |= rs.mask;
      s_pend[threadIdx.x] = pm;
      s_pub[threadIdx.x] = 0u;
    }
    // a run of CTA-local rounds ends after an eighth of the barrier's time
    // limit, so the CTAs waiting for it never come near that limit
    if (kLocal && in_local && threadIdx.x == 0)
      s_int[34] = (long long)(globaltimer() - t_loc) > P.cap_ns / 8 ? 1 : 0;
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x < kMaskWords) st_vol(ctl->imask[(t + 1) % 3][threadIdx.x], 0u);
    if (blockIdx.x == 0 && threadIdx.x == 0) st_vol(ctl->fr[(t + 1) % 3], 0ull);
    // Δ-stepping: vertices lowered into the current bucket during round t-1
    // (its side list, complete at the barrier) are expanded again before the
    // bucket is left.  Counter slots by t % 3: this round files into t % 3,
    // round t - 1's count was read after its barrier, and (t + 1) % 3 was
    // last read before round t - 1 began.
    uint32_t side_cnt = 0;
    if (kDelta) {
      side_cnt = min(rs.side, (uint32_t)g.n);
      if (blockIdx.x == 0 && threadIdx.x == 0) st_vol(ctl->scnt[(t + 1) % 3], 0u);
    }
    const bool side_round = kDelta && side_cnt > 0;
    const int32_t b = side_round ? bcur : next_bucket(s_pend, nB, lo, s_int);
    // ---------------- CTA-local rounds (kLocal, exact wBFS).  Every CTA
    // loads the bucket's entries and sums their live degrees, so all take
    // the same decision without a barrier; CTA 0 keeps the loads for its
    // expansion, thread i's entry in S.u/S.adj/S.base[i] (degree, or ~0 if
    // not live; bmax >= blockDim).
    bool pre = false;
    if constexpr (kLocal && !kDelta) {
      bool loc = false;
      if (b != kInf) {
        const int sb0 = b % nB;
        const uint32_t rb0 = s_base[sb0], cnt0 = min(s_cnt[sb0] - rb0, (uint32_t)g.n);
        const bool dense0 = P.dense && P.pull_divisor > 0 &&
                            (unsigned long long)cnt0 * (unsigned)P.pull_divisor > (unsigned long long)g.n;
        if (!dense0 && cnt0 <= blockDim.x) {
          pre = true;
          uint32_t deg = 0;
          S.base[threadIdx.x] = ~0u;
          if (threadIdx.x < cnt0) {
            const int32_t v = P.slots[(size_t)sb0 * (size_t)g.n + (rb0 + threadIdx.x) % (uint32_t)g.n];
            const int32_t dv = P.dist[v];
            const uint32_t o0 = __ldg(g.off + v), o1 = __ldg(g.off + v + 1);
            deg = o1 - o0;
            if (dv == b && (deg >= 2u || (deg == 1u && v == src))) {
              S.u[threadIdx.x] = v;
              S.adj[threadIdx.x] = o0;
              S.base[threadIdx.x] = deg;
            } else {
              deg = 0;
            }
          }
          uint32_t tot;
          block_excl_scan(deg, S.misc + 8, &tot);
          loc = tot <= (uint32_t)P.local_arcs;
        }
      }
      bool wait_local = false;
      if (in_local && (!loc || s_int[34])) {
        // CTA 0 ends its run before round t: the state as of this point
        for (int i = threadIdx.x; i < nB; i += blockDim.x) ctl->loc_base[i] = s_base[i];
        if (threadIdx.x < kMaskWords) ctl->loc_pend[threadIdx.x] = s_pend[threadIdx.x];
        if (threadIdx.x == 0) {
          ctl->loc_t = t;
          ctl->loc_lo = lo;
        }
        in_local = false;
        wait_local = true;
      } else if (!in_local && loc) {
        if (blockIdx.x == 0) {
          in_local = true;
          if (threadIdx.x == 0) t_loc = globaltimer();
        } else {
          wait_local = true;
        }
      }
      if (wait_local) {
        if (!grid_sync(ctl, bar, &s_flag)) break;
        // every CTA resumes at round loc_t from the state CTA 0 handed back
        t = ld_vol(ctl->loc_t) - 1;
        lo = ld_vol(ctl->loc_lo);
        for (int i = threadIdx.x; i < nB; i += blockDim.x) s_base[i] = ld_vol(ctl->loc_base[i]);
        if (threadIdx.x < kMaskWords) s_pend[threadIdx.x] = ld_vol(ctl->loc_pend[threadIdx.x]);
        prev = -1;
        rs = read_round_state(P, t, s_cnt);
        rs.mask = 0u;
        rs.side = 0u;
        continue;
      }
    }
    if (b == kInf) {
      // open buckets are dry: refill from the overflow bucket, or finish
      const uint32_t oc = min(ld_vol(ctl->ovf_cnt[cur]), P.ovf_cap);
      if (P.slide || oc == 0) break;
      const int32_t nlo = ld_vol(ctl->ovf_min[cur]);
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&ctl->refills, 1);
      // into the new window [nlo, nlo + nB), the rest into the other buffer
      FileSink fs{&P, nlo, cur ^ 1, &c, imask, s_pub, -1, nullptr, nullptr, nullptr};
      for (uint32_t base = blockIdx.x * blockDim.x; base < oc; base += gs) {
        const uint32_t i = base + threadIdx.x;
        const bool valid = i < oc;
        const int2 e = valid ? P.ovf[cur][i] : make_int2(0, 0);  // (vertex, bucket)
        const bool live = valid && (P.dist[e.x] >> P.dl) == e.y;
        fs.append(S, live, e.x, (uint32_t)e.y << P.dl);
        fs.chunk_end(S);
      }
      fs.flush(S);
      lo = nlo;
      prev = -1;
      if (!grid_sync(ctl, bar, &s_flag)) break;
      // the scanned buffer is consumed; the other one holds the remainder
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        st_vol(ctl->ovf_cnt[cur], 0u);
        st_vol(ctl->ovf_min[cur], kInf);
      }
      cur ^= 1;
      if (!grid_sync(ctl, bar, &s_flag)) break;
      // the refill filed into mask t % 3
      rs = read_round_state(P, t, s_cnt);
      continue;
    }
    // The entries of this round: bucket b's ring slot, or (Δ-stepping) the
    // side list of round t-1.
    uint32_t rb = 0, cntb = side_cnt;
    const int32_t *elist;
    if (side_round) {
      prev = -1;
      elist = P.side[(t + 1) & 1];
    } else {
      if (P.slide) lo = b;
      const int sb = b % nB;
      prev = sb;
      bcur = b;
      // No CTA files into slot sb during this round (exact wBFS files values
      // above b, less than nB above; Δ-stepping files bucket b into the side
      // list), so its counter is stable here.
      rb = s_base[sb];
      const uint32_t avail = s_cnt[sb] - rb;
      if (avail > (uint32_t)g.n && blockIdx.x == 0 && threadIdx.x == 0)
        raise_error(ctl, GBF_ERR_OVERFLOW, 15);  // a ring wrapped over unconsumed entries
      cntb = min(avail, (uint32_t)g.n);
      __syncthreads();
      if (threadIdx.x == 0) s_base[sb] = rb + cntb;
      __syncthreads();
      elist = P.slots + (size_t)sb * (size_t)g.n;
    }
    unsigned long long *fctr = &ctl->fr[t % 3];
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&ctl->rounds, 1);
    FileSink fsink{&P, lo, cur, &c, imask, s_pub, kDelta ? b : -1, P.side[t & 1], P.sflag[t & 1],
                   &ctl->scnt[t % 3], kLocal && in_local ? s_cnt : nullptr};
    const bool dense = !kDelta && P.dense && P.pull_divisor > 0 &&
                       (unsigned long long)cntb * (unsigned)P.pull_divisor > (unsigned long long)g.n;
    if (dense) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&ctl->pull_rounds, 1);
      dense_round(P, b, S, fsink, c);
      if (!grid_sync(ctl, bar, &s_flag)) break;
      rs = read_round_state(P, t, s_cnt);
      if (P.trace && blockIdx.x == 0 && threadIdx.x == 0 && t <= P.trace_cap)
        P.trace[t - 1] = TraceRec{t, 2, cntb, 0u, (long long)(globaltimer() - t_start), 0};
      continue;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&ctl->push_rounds, 1);
    // ---------------- edgeMapData over the live entries of bucket b
    QueueOut fout{P.q, P.qoff, nullptr, P.cs, fctr, (uint32_t)g.n, P.cs_cap};
    RelaxFn<kDelta> fn{g.tgt, g.w, P.dist, b, 0};
    fn.stream_pol = l2_evict_first();
    fn.keep_pol = l2_evict_last();
    for (uint32_t it = blockIdx.x * blockDim.x; it < cntb; it += gs) {
      const uint32_t i = it + threadIdx.x;
      int32_t v = 0;
      bool live = false;
      uint32_t a0 = 0, deg = 0;
      if (kLocal && pre && it == 0) {  // CTA 0: the entries the test above loaded
        const uint32_t d = S.base[threadIdx.x];
        live = d != ~0u;
        if (live) {
          v = S.u[threadIdx.x];
          a0 = S.adj[threadIdx.x];
          deg = d;
        }
      } else if (i < cntb) {
        v = elist[side_round ? i : (rb + i) % (uint32_t)g.n];
        if (side_round) atomicAnd(P.sflag[(t + 1) & 1] + (v >> 5), ~(1u << (v & 31)));
        // the entry's distance and its CSR range, loaded together
        const int32_t dv = P.dist[v];
        const uint32_t o0 = __ldg(g.off + v), o1 = __ldg(g.off + v + 1);
        // Δ-stepping: a bucket may hold a vertex more than once (lowered
        // twice inside its range before the bucket came up); it is expanded
        // once per round, which also bounds a round's arcs by m
        if ((dv >> P.dl) == b && (!kDelta || atomicExch(P.xround + v, t) != t)) {
          a0 = o0;
          deg = o1 - o0;
          // a degree-1 vertex other than the source was reached from its only
          // neighbour, which it cannot improve
          live = deg >= 2u || (deg == 1u && v == src);
        }
      }
      // (a CTA-local round expands every entry itself: its arcs fit the
      // 20-bit degree field below)
      const bool heavy = !(kLocal && in_local) && live && deg > (uint32_t)P.heavy;
      stage_append(S, heavy, v, deg, a0);
      const bool light = live && !heavy;
      if (live) c.expanded++;
      if (heavy) c.heavy++;
      // CTA-local degree prefix of the light entries (count in the high bits)
      uint32_t tot;
      const uint32_t ex = block_excl_scan(light ? ((1u << 20) | deg) : 0u, S.misc + 8, &tot);
      if (light) {
        const uint32_t j = ex >> 20;
        S.base[j] = ex & 0xfffffu;
        S.u[j] = v;
        S.adj[j] = a0;
      }
      const uint32_t nv = tot >> 20, E = tot & 0xfffffu;
      if (threadIdx.x == 0) {
        S.base[nv] = E;
        c.scanned += E;
      }
      __syncthreads();
      walk_chunk(S, g.m, nv, 0u, E, fn, fsink);
      fsink.chunk_end(S);  // starts with __syncthreads; leaves misc[0] alone
      stage_make_room(S, fout, ctl, blockDim.x);
    }
    stage_flush(S, fout, ctl);
    fsink.flush(S);
    if (kLocal && in_local) {
      // the next round starts from this CTA's own filings (complete after
      // the flush's barriers) and its own slot counters
      if (threadIdx.x < kMaskWords) rs.mask = s_pub[threadIdx.x];
      rs.side = 0u;
      c.relax += fn.relax;
      if (threadIdx.x == 0) {
        atomicAdd(&ctl->local_rounds, 1);
        if (P.trace && t <= P.trace_cap)
          P.trace[t - 1] = TraceRec{t, 8, cntb, 0u, (long long)(globaltimer() - t_start), 0};
      }
      continue;
    }
    if (!grid_sync(ctl, bar, &s_flag)) break;
    // heavy-vertex counter of this round (triple-buffered: the slot zeroed by
    // CTA 0 in round t + 1 is (t + 2) % 3, never this one), loaded with the
    // state the next round starts from, which is final here unless a heavy
    // pass follows
    const unsigned long long fr = ld_vol(*fctr);
    rs = read_round_state(P, t, s_cnt);
    const uint32_t hcnt = (uint32_t)(fr >> 32), hD = (uint32_t)fr;
    const long long t_mid = (long long)(globaltimer() - t_start);
    if (hcnt > 0 && ((uint64_t)hD + kFine - 1) / kFine > P.cs_cap) {
      // more arcs than the chunk-start table covers (a round expands every
      // vertex at most once, so never expected)
      if (blockIdx.x == 0 && threadIdx.x == 0) raise_error(ctl, GBF_ERR_OVERFLOW, 16);
    } else if (hcnt > 0) {
      // heavy vertices of the bucket: blocked edgeMap over all CTAs
      QueueIn in{P.q, P.qoff, nullptr, P.cs, hcnt, hD};
      // every heavy vertex has more than P.heavy edges; chunks of at most
      // 256 << 6 arcs keep the last chunks of the round short
      blocked_edge_map(g, in, chunk_shift(hD, 4u, 6),
                       (uint32_t)P.bmax, S, fn, fsink, ctl, bem++);
      fsink.flush(S);
      if (blockIdx.x == 0 && threadIdx.x == 0) c.scanned += hD;
      if (!grid_sync(ctl, bar, &s_flag)) break;
      rs = read_round_state(P, t, s_cnt);
    }
    c.relax += fn.relax;
    if (P.trace && blockIdx.x == 0 && threadIdx.x == 0 && t <= P.trace_cap)
      P.trace[t - 1] = TraceRec{t, hcnt ? 3 : 1, cntb, hD, (long long)(globaltimer() - t_start),
                                hcnt ? t_mid : 0};
  }
  // statistics
  unsigned long long tt;
  tt = block_sum64(c.scanned, S.misc64);
  if (threadIdx.x == 0 && tt) atomicAdd(&ctl->edges_scanned, tt);
  tt = block_sum64(c.relax, S.misc64);
  if (threadIdx.x == 0 && tt) atomicAdd(&ctl->relax, tt);
  tt = block_sum64(c.inserts, S.misc64);
  if (threadIdx.x == 0 && tt) atomicAdd(&ctl->inserts, tt);
  tt = block_sum64(c.expanded, S.misc64);
  if (threadIdx.x == 0 && tt) atomicAdd(&ctl->expanded, tt);
  tt = block_sum64(c.heavy, S.misc64);
  if (threadIdx.x == 0 && tt) atomicAdd(&ctl->heavy, tt);
  tt = block_sum64(c.pulled, S.misc64);
  if (threadIdx.x == 0 && tt) atomicAdd(&ctl->pulled, tt);
}

gbf_status launch_wbfs(Graph &g, Workspace &ws, int32_t src, int32_t *dist, const Opts &o,
                       cudaStream_t st, int dl) {
  if (!g.leaf) return set_error("graph has no degree-1 bitmap"), GBF_ERR_INVALID;
  if (dl < 0 || dl > 20) return set_error("delta must be 2^0 .. 2^20"), GBF_ERR_INVALID;
  if (dl > 0 && (!ws.side[0] || !ws.side[1] || !ws.xround))
    return set_error("no side lists"), GBF_ERR_INVALID;
  WbfsParams P;
  P.g = g.dev();
  P.leaf = g.leaf;
  P.src = src;
  P.dist = dist;
  P.slots = ws.slots;
  P.slot_cnt = ws.slot_cnt;
  P.nB = ws.nB;
  // the largest bucket step of one relaxation is floor((Δ - 1 + w_max) / Δ)
  const uint32_t jump = (((1u << dl) - 1u) + g.w_max) >> dl;
  P.slide = (uint32_t)ws.nB > jump ? 1 : 0;
  P.ovf[0] = ws.ovf[0];
  P.ovf[1] = ws.ovf[1];
  P.ovf_cap = (uint32_t)ws.ovf_cap;
  P.q = ws.q[0];
  P.qoff = ws.qoff[0];
  P.cs = ws.cs[0];
  P.cs_cap = (uint32_t)(((uint64_t)g.m + kFine - 1) / kFine + 2);
  P.ctl = ws.ctl;
  P.trace = ws.trace;
  P.trace_cap = ws.trace_cap;
  P.pull_divisor = o.pull_divisor;
  P.dense = dl == 0 ? o.dense_wbfs : 0;
  P.bmax = o.heavy_cutoff;
  P.cap = stage_capacity(o.block);
  int l = 0;
  while ((kFine << l) < (uint32_t)o.heavy_cutoff) l++;
  P.log2_bmax_fine = l;
  // vertices with more arcs than this go through the blocked edgeMap pass
  P.heavy = o.heavy_cutoff / 8 > 32 ? o.heavy_cutoff / 8 : 32;
  P.local_arcs = dl == 0 ? o.local_arcs : 0;
  P.inject_wait = o.inject_wait;
  P.cap_ns = o.spin_cap_ns;
  P.dl = dl;
  P.side[0] = ws.side[0];
  P.side[1] = ws.side[1];
  P.sflag[0] = ws.fbm[0];
  P.sflag[1] = ws.fbm[1];
  P.xround = ws.xround;
  const void *kern = dl > 0 ? (const void *)wbfs_kernel<true, false>
                            : (P.local_arcs > 0 ? (const void *)wbfs_kernel<false, true>
                                                : (const void *)wbfs_kernel<false, false>);
  const size_t smem = wbfs_smem_bytes(P.bmax, P.cap, ws.nB);
  {
    const gbf_status sm = check_smem(smem, "wbfs_kernel");
    if (sm != GBF_OK) return sm;
  }
  GBF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  GBF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, o.block, smem));
  if (per_sm < 1) {
    set_error("wbfs kernel does not fit on an SM with this block size");
    return GBF_ERR_INVALID;
  }
  int grid = per_sm * g.num_sms;
  if (o.ctas > 0 && o.ctas < grid) grid = o.ctas;
  GBF_CUDA(cudaMemsetAsync(ws.ctl, 0, sizeof(Ctl), st));
  if (ws.trace) GBF_CUDA(cudaMemsetAsync(ws.trace, 0, sizeof(TraceRec) * (size_t)ws.trace_cap, st));
  void *args[] = {&P};
  GBF_CUDA(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(o.block), args, smem, st));
  ws.last_kind = 2;
  ws.last_grid = grid;
  ws.last_block = o.block;
  return GBF_OK;
}

int resident_ctas_per_sm_wbfs(const Opts &o, int nB) {
  const size_t smem = wbfs_smem_bytes(o.heavy_cutoff, stage_capacity(o.block), nB);
  if (cudaFuncSetAttribute(wbfs_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wbfs_kernel<false, false>, o.block, smem) !=
      cudaSuccess)
    return 0;
  return per_sm;
}

}  // namespace gbf
