// Weighted BFS (integral-weight SSSP, §4; Alg. 3) as one persistent
// cooperative kernel.  Each bucket round is two phases separated by bounded
// grid barriers:
//
//   R (edgeMapData, Alg. 3 Update): for every arc (s, d, w) out of the
//     current bucket F (all with D[s] = b): nDist = b + w; if nDist < D[d],
//     priority-write (atomicMin) D[d]; the first successful writer of the
//     round wins a test-and-set (a round stamp) and appends d to Moved.  The
//     sparse form is the blocked edgeMap of §6.2; with dense_wbfs the round
//     may instead pull: every vertex with D[v] > b + 1 takes the minimum of
//     b + w over neighbours with D[u] = b (the dense switch of the SSSP
//     experiments, "switch to a dense edgeMap once the frontiers are
//     sufficiently dense").
//   E (vertexMap(Moved, Reset) + updateBuckets + nextBucket): the next bucket
//     id is the smallest of (the minimum distance written in R, the lowest
//     non-empty open bucket, the overflow minimum); moved vertices are filed
//     under their final distance, and the live entries of the next bucket
//     (D[v] equal to the bucket id; stale ones are dropped) become the next
//     frontier, compacted with its degree prefix for the blocked edgeMap.
//
// The bucket structure (Julienne's makeBuckets / nextBucket / updateBuckets,
// INCREASING order) is a window of nB open buckets, bucket value x in slot
// x mod nB, plus an overflow bucket for values beyond the window; when the
// window runs dry the overflow is scanned and refilled into a window that
// starts at its minimum.  With nB > max weight nothing ever overflows.
#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "gbf_impl.h"

namespace gbf {
using namespace dev;

struct WbfsParams {
  DevGraph g;
  int32_t src;
  int32_t *dist;
  int32_t *stamp;
  int32_t *moved[2];
  int32_t *slots;
  uint32_t *slot_cnt;
  int32_t nB;
  int2 *ovf[2];
  uint32_t ovf_cap;
  int32_t *q;
  uint32_t *qoff;
  uint32_t *cs;
  uint32_t cs_cap;
  Ctl *ctl;
  int pull_divisor;
  int dense;
  int bmax;
  int log2_bmax_fine;
  int pull_serial;
  int inject_wait;
  long long cap_ns;
};

namespace {

// Update of Alg. 3 (sparse direction).
struct RelaxFn {
  const uint32_t *w;
  int32_t *dist;
  int32_t *stamp;
  int32_t b, t;
  int32_t gmin;
  unsigned long long relax;
  __device__ __forceinline__ void operator()(int32_t, int32_t v, uint32_t idx, bool &emit,
                                             int32_t &ov, uint32_t &) {
    const int32_t nd = b + (int32_t)__ldg(w + idx);
    if (nd >= dist[v]) return;
    const int32_t old = atomicMin(dist + v, nd);
    if (old <= nd) return;
    relax++;
    gmin = min(gmin, nd);
    if (atomicExch(stamp + v, t) != t) {
      emit = true;
      ov = v;
    }
  }
};

// Warp-aggregated append of (v) to bucket slot `slot` (lanes with slot < 0 skip).
__device__ __forceinline__ void slot_insert(const WbfsParams &P, int32_t slot, int32_t v,
                                            unsigned long long &inserts) {
  const unsigned grp = __match_any_sync(kFull, slot);
  if (slot < 0) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(grp) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(P.slot_cnt + slot, (unsigned)__popc(grp));
  base = __shfl_sync(grp, base, leader);
  const uint32_t pos = base + __popc(grp & lanemask_lt());
  if (pos < (uint32_t)P.g.n) P.slots[(size_t)slot * (size_t)P.g.n + pos] = v;
  else raise_error(P.ctl, GBF_ERR_OVERFLOW, 5);
  inserts++;
}

// Warp-aggregated append of (v, d) to overflow buffer `which`.
__device__ __forceinline__ void ovf_insert(const WbfsParams &P, int which, bool ins, int32_t v,
                                           int32_t d, unsigned long long &inserts) {
  const unsigned bal = __ballot_sync(kFull, ins);
  if (!bal) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(bal) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(&P.ctl->ovf_cnt[which], (unsigned)__popc(bal));
  base = __shfl_sync(kFull, base, leader);
  if (ins) {
    const uint32_t pos = base + __popc(bal & lanemask_lt());
    if (pos < P.ovf_cap) {
      P.ovf[which][pos] = make_int2(v, d);
      atomicMin(&P.ctl->ovf_min[which], d);
    } else {
      raise_error(P.ctl, GBF_ERR_OVERFLOW, 6);
    }
    inserts++;
  }
}

// Dense edgeMap for one bucket: pull the minimum of b + w over neighbours in
// the bucket (D[u] == b) into every vertex with D[v] > b + 1.
__device__ void dense_relax(const WbfsParams &P, int32_t b, int32_t t, int32_t &gmin,
                            unsigned long long &relax, unsigned long long &scanned) {
  const DevGraph &g = P.g;
  const int lane = threadIdx.x & 31;
  const uint32_t nwords = ((uint32_t)g.n + 31) >> 5;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t tw = (gridDim.x * blockDim.x) >> 5;
  int32_t *mlist = P.moved[t & 1];
  unsigned int *mcount = &P.ctl->mcnt[t & 1];
  for (uint32_t wi = gw; wi < nwords; wi += tw) {
    const int32_t v = (int32_t)(wi * 32 + lane);
    int32_t dv = kInf;
    uint32_t s = 0, e = 0;
    bool cand = false;
    if (v < g.n) {
      dv = P.dist[v];
      if (dv > b + 1) {
        s = __ldg(g.off + v);
        e = __ldg(g.off + v + 1);
        cand = e > s;
      }
    }
    int32_t best = kInf;
    uint32_t k = s;
    if (cand) {
      const uint32_t lim = min(e, s + (uint32_t)P.pull_serial);
      for (; k < lim && best != b + 1; k++) {
        const int32_t u = __ldg(g.tgt + k);
        if (P.dist[u] == b) best = min(best, b + (int32_t)__ldg(g.w + k));
      }
      scanned += k - s;
    }
    unsigned rm = __ballot_sync(kFull, cand && best != b + 1 && k < e);
    while (rm) {
      const int l = __ffs(rm) - 1;
      rm &= rm - 1;
      const uint32_t ks = __shfl_sync(kFull, k, l), ke = __shfl_sync(kFull, e, l);
      int32_t wb = __shfl_sync(kFull, best, l);
      uint32_t looked = 0;
      for (uint32_t c = ks; c < ke && wb != b + 1; c += 32) {
        const uint32_t kk = c + lane;
        int32_t cand_d = kInf;
        if (kk < ke) {
          const int32_t u = __ldg(g.tgt + kk);
          if (P.dist[u] == b) cand_d = b + (int32_t)__ldg(g.w + kk);
        }
        wb = min(wb, __reduce_min_sync(kFull, cand_d));
        looked += min(32u, ke - c);
      }
      if (lane == l) {
        best = wb;
        scanned += looked;
      }
    }
    const bool low = cand && best < dv;
    if (low) {
      P.dist[v] = best;
      relax++;
      gmin = min(gmin, best);
    }
    const unsigned bal = __ballot_sync(kFull, low);
    if (bal) {
      const int leader = __ffs(bal) - 1;
      uint32_t pos = 0;
      if (lane == leader) pos = atomicAdd(mcount, (unsigned)__popc(bal));
      pos = __shfl_sync(kFull, pos, leader);
      if (low) {
        const uint32_t r = pos + __popc(bal & lanemask_lt());
        if (r < (uint32_t)g.n) mlist[r] = v;
        else raise_error(P.ctl, GBF_ERR_OVERFLOW, 7);
      }
    }
  }
}

}  // namespace

__global__ void __launch_bounds__(1024) wbfs_kernel(WbfsParams P) {
  extern __shared__ unsigned long long smem_raw[];
  __shared__ int s_flag;
  __shared__ int s_int[40];
  PushSmem S = carve_push_smem(smem_raw, P.bmax);
  if (threadIdx.x == 0) S.misc[0] = 0;
  Ctl *ctl = P.ctl;
  Barrier bar{0u, P.cap_ns};
  const DevGraph g = P.g;
  const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  const int32_t src = P.src, nB = P.nB;
  unsigned long long scanned = 0, relax = 0, inserts = 0, expanded = 0;

  // makeBuckets: D = inf except D[src] = 0; only src in bucket 0.
  for (uint32_t i = gt; i < (uint32_t)g.n; i += gs) {
    P.dist[i] = (i == (uint32_t)src) ? 0 : kInf;
    P.stamp[i] = 0;
  }
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < nB; i += blockDim.x) P.slot_cnt[i] = 0u;
    const uint32_t d0 = __ldg(g.off + src + 1) - __ldg(g.off + src);
    if (threadIdx.x == 0) {
      ctl->gmin[0] = kInf;
      ctl->gmin[1] = kInf;
      ctl->ovf_min[0] = kInf;
      ctl->ovf_min[1] = kInf;
      if (d0 > 0) {
        P.q[0] = src;
        P.qoff[0] = 0;
        st_vol(ctl->fr[0], (1ull << 32) | d0);
      }
    }
    for (uint32_t c = threadIdx.x; c < (d0 + kFine - 1) / kFine; c += blockDim.x)
      if (c < P.cs_cap) P.cs[c] = 0;
  }
  if (P.inject_wait && blockIdx.x == 0 && threadIdx.x == 0) injected_wait(ctl, P.cap_ns);
  __syncthreads();
  bool ok = grid_sync(ctl, bar, &s_flag);

  int32_t b = 0, lo = 0;
  int cur = 0;  // active overflow buffer
  for (int32_t t = 1; ok; t++) {
    // ---------------- R phase: relax the frontier of bucket b
    const unsigned long long fr = ld_vol(ctl->fr[(t - 1) & 1]);
    const uint32_t cnt = (uint32_t)(fr >> 32), D = (uint32_t)fr;
    // Snapshot the bucket state for the next nextBucket decision now: the
    // open buckets and the overflow bucket only change in E phases, so every
    // CTA sees the same values here.  The slot of the bucket just extracted
    // (value b) is skipped: it is being emptied.
    int32_t smin = kInf;
    for (int i = threadIdx.x; i < nB; i += blockDim.x) {
      if (i != b % nB && ld_vol(P.slot_cnt[i]) > 0u) {
        const int32_t rel = ((i - lo % nB) % nB + nB) % nB;
        smin = min(smin, lo + rel);
      }
    }
    smin = block_min_i32(smin, s_int);
    if (threadIdx.x == 0) s_int[32] = smin;
    __syncthreads();
    smin = s_int[32];
    const uint32_t oc = ld_vol(ctl->ovf_cnt[cur]);
    const int32_t om = oc ? ld_vol(ctl->ovf_min[cur]) : kInf;
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st_vol(ctl->mcnt[(t + 1) & 1], 0u);
      st_vol(ctl->gmin[(t + 1) & 1], kInf);
      st_vol(ctl->fr[t & 1], 0ull);
      if (t > 1) st_vol(P.slot_cnt[b % nB], 0u);
      st_vol(ctl->ovf_cnt[cur ^ 1], 0u);
      st_vol(ctl->ovf_min[cur ^ 1], kInf);
      atomicAdd(&ctl->rounds, 1);
    }
    int32_t gmin = kInf;
    if (cnt > 0) {
      const bool dense = P.dense && P.pull_divisor > 0 &&
                         (unsigned long long)D * (unsigned)P.pull_divisor > g.m;
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicAdd(dense ? &ctl->pull_rounds : &ctl->push_rounds, 1);
        if (!dense) {
          scanned += D;
          expanded += cnt;
        }
      }
      if (dense) {
        dense_relax(P, b, t, gmin, relax, scanned);
      } else {
        QueueIn in{P.q, P.qoff, P.cs, cnt, D};
        RelaxFn fn{g.w, P.dist, P.stamp, b, t, kInf, 0};
        ListSink sink{P.moved[t & 1], &ctl->mcnt[t & 1], (uint32_t)g.n, ctl};
        blocked_edge_map(g, in, chunk_shift(D, P.log2_bmax_fine), S, fn, sink, ctl);
        gmin = fn.gmin;
        relax += fn.relax;
      }
    }
    {
      const int m = block_min_i32(gmin, s_int);
      if (threadIdx.x == 0 && m != kInf) atomicMin(&ctl->gmin[t & 1], m);
    }
    if (!grid_sync(ctl, bar, &s_flag)) break;

    // ---------------- E phase: Reset + updateBuckets + nextBucket
    const int32_t gm = ld_vol(ctl->gmin[t & 1]);
    const uint32_t mc = min(ld_vol(ctl->mcnt[t & 1]), (uint32_t)g.n);
    const int32_t bn = min(gm, min(smin, om));
    if (bn == kInf) break;  // nextBucket returned nullbkt
    const bool refill = oc > 0 && bn >= lo + nB;
    const int32_t lo_new = (oc == 0 || refill) ? bn : lo;
    const int32_t *mlist = P.moved[t & 1];
    QueueOut fout{P.q, P.qoff, P.cs, &ctl->fr[t & 1], (uint32_t)g.n, P.cs_cap};
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t wbase = gt & ~31u;  // warp-uniform loop start

    if (refill) {
      // Refill the window [bn, bn + nB) from the overflow bucket (stale
      // entries dropped), then file Moved under the new window.
      const uint32_t ocap = min(oc, P.ovf_cap);
      for (uint32_t base = wbase; base < ocap; base += stride) {
        const uint32_t i = base + (threadIdx.x & 31);
        const bool valid = i < ocap;
        const int2 e = valid ? P.ovf[cur][i] : make_int2(0, 0);
        const bool live = valid && P.dist[e.x] == e.y;
        const bool into_slot = live && e.y < lo_new + nB;
        slot_insert(P, into_slot ? (e.y % nB) : -1, e.x, inserts);
        ovf_insert(P, cur ^ 1, live && !into_slot, e.x, e.y, inserts);
      }
      for (uint32_t base = wbase; base < mc; base += stride) {
        const uint32_t i = base + (threadIdx.x & 31);
        const bool valid = i < mc;
        const int32_t v = valid ? mlist[i] : 0;
        const int32_t d = valid ? P.dist[v] : kInf;
        const bool keep = valid && (__ldg(g.off + v + 1) - __ldg(g.off + v)) >= 2u;
        const bool into_slot = keep && d < lo_new + nB;
        slot_insert(P, into_slot ? (d % nB) : -1, v, inserts);
        ovf_insert(P, cur ^ 1, keep && !into_slot, v, d, inserts);
      }
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&ctl->refills, 1);
      if (!grid_sync(ctl, bar, &s_flag)) break;
      cur ^= 1;
    } else {
      // File Moved: members of the next bucket go straight to the frontier.
      for (uint32_t base = blockIdx.x * blockDim.x; base < mc; base += stride) {
        const uint32_t i = base + threadIdx.x;
        const bool valid = i < mc;
        const int32_t v = valid ? mlist[i] : 0;
        const int32_t d = valid ? P.dist[v] : kInf;
        const uint32_t deg = valid ? (__ldg(g.off + v + 1) - __ldg(g.off + v)) : 0u;
        const bool keep = valid && deg >= 2u;
        const bool to_f = keep && d == bn;
        const bool into_slot = keep && !to_f && d < lo_new + nB;
        const bool into_ovf = keep && !to_f && !into_slot;
        slot_insert(P, into_slot ? (d % nB) : -1, v, inserts);
        ovf_insert(P, cur, into_ovf, v, d, inserts);
        stage_append(S, to_f, v, deg);
        __syncthreads();
        if (S.misc[0] + blockDim.x > S.cap_out) stage_flush(S, fout, ctl);
      }
    }
    // Extract the live entries of bucket bn; entries whose distance changed
    // after they were filed are stale and dropped (lazy deletion).
    {
      const int32_t slot = bn % nB;
      const uint32_t scnt = min(ld_vol(P.slot_cnt[slot]), (uint32_t)g.n);
      const int32_t *sl = P.slots + (size_t)slot * (size_t)g.n;
      for (uint32_t base = blockIdx.x * blockDim.x; base < scnt; base += stride) {
        const uint32_t i = base + threadIdx.x;
        bool live = false;
        int32_t v = 0;
        uint32_t deg = 0;
        if (i < scnt) {
          v = sl[i];
          if (P.dist[v] == bn) {
            deg = __ldg(g.off + v + 1) - __ldg(g.off + v);
            live = deg >= 2u;
          }
        }
        stage_append(S, live, v, deg);
        __syncthreads();
        if (S.misc[0] + blockDim.x > S.cap_out) stage_flush(S, fout, ctl);
      }
    }
    stage_flush(S, fout, ctl);
    lo = lo_new;
    b = bn;
    if (!grid_sync(ctl, bar, &s_flag)) break;
  }
  // statistics: reached vertices are counted by the host from dist.
  unsigned long long tt;
  tt = block_sum64(scanned, S.misc64);
  if (threadIdx.x == 0 && tt) atomicAdd(&ctl->edges_scanned, tt);
  tt = block_sum64(relax, S.misc64);
  if (threadIdx.x == 0 && tt) atomicAdd(&ctl->relax, tt);
  tt = block_sum64(inserts, S.misc64);
  if (threadIdx.x == 0 && tt) atomicAdd(&ctl->inserts, tt);
  tt = block_sum64(expanded, S.misc64);
  if (threadIdx.x == 0 && tt) atomicAdd(&ctl->expanded, tt);

}

gbf_status launch_wbfs(Graph &g, Workspace &ws, int32_t src, int32_t *dist, const Opts &o,
                       cudaStream_t st) {
  WbfsParams P;
  P.g = g.dev();
  P.src = src;
  P.dist = dist;
  P.stamp = ws.stamp;
  P.moved[0] = ws.moved[0];
  P.moved[1] = ws.moved[1];
  P.slots = ws.slots;
  P.slot_cnt = ws.slot_cnt;
  P.nB = ws.nB;
  P.ovf[0] = ws.ovf[0];
  P.ovf[1] = ws.ovf[1];
  P.ovf_cap = (uint32_t)ws.ovf_cap;
  P.q = ws.q[0];
  P.qoff = ws.qoff[0];
  P.cs = ws.cs[0];
  P.cs_cap = (uint32_t)(((uint64_t)g.m + kFine - 1) / kFine + 2);
  P.ctl = ws.ctl;
  P.pull_divisor = o.pull_divisor;
  P.dense = o.dense_wbfs;
  P.bmax = o.heavy_cutoff;
  int l = 0;
  while ((kFine << l) < (uint32_t)o.heavy_cutoff) l++;
  P.log2_bmax_fine = l;
  P.pull_serial = o.pull_serial;
  P.inject_wait = o.inject_wait;
  P.cap_ns = o.spin_cap_ns;
  const size_t smem = push_smem_bytes(o.heavy_cutoff);
  GBF_CUDA(cudaFuncSetAttribute(wbfs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  int per_sm = 0;
  GBF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wbfs_kernel, o.block, smem));
  if (per_sm < 1) {
    set_error("wbfs kernel does not fit on an SM with this block size");
    return GBF_ERR_INVALID;
  }
  int grid = per_sm * g.num_sms;
  if (o.ctas > 0 && o.ctas < grid) grid = o.ctas;
  GBF_CUDA(cudaMemsetAsync(ws.ctl, 0, sizeof(Ctl), st));
  void *args[] = {&P};
  GBF_CUDA(cudaLaunchCooperativeKernel((const void *)wbfs_kernel, dim3(grid), dim3(o.block), args,
                                       smem, st));
  ws.last_kind = 2;
  ws.last_grid = grid;
  ws.last_block = o.block;
  return GBF_OK;
}

}  // namespace gbf
