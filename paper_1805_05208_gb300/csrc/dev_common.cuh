// Device building blocks shared by the persistent traversal kernels:
//   - a bounded, time-limited grid barrier for cooperative launches,
//   - warp/block scans and warp-aggregated appends,
//   - the blocked sparse edgeMap (edgeMapBlocked, Alg. 2 and §6.2): frontier
//     edges are cut into equal chunks through a prefix sum of frontier
//     degrees; each CTA walks one chunk with its warps on consecutive edges
//     (coalesced target loads) and stages live neighbours in shared memory,
//   - the staged flush that writes the next frontier as a compact queue with
//     its own degree prefix (qoff) and chunk-start table (cs), reserving its
//     range with one 64-bit atomicAdd per CTA.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gbf.h"
#include "gbf_dev.h"

namespace gbf {
namespace dev {

constexpr int32_t kInf = 0x7fffffff;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kFineLog = 8;  // chunk-start table granularity: 256 frontier edges
constexpr uint32_t kFine = 1u << kFineLog;

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(unsigned *p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// L2 eviction priorities (per access, no device setting): the graph's
// arrays are streamed once per query and should leave L2 first; the small
// per-vertex state they index (distances, bitmaps) should stay.
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// read-only (non-coherent) load with an L2 policy
__device__ __forceinline__ uint32_t ldg_pol(const void *p, uint64_t pol) {
  uint32_t v;
  asm volatile("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
// coherent load at L2 (.cg) with an L2 policy
__device__ __forceinline__ uint32_t ldcg_pol(const void *p, uint64_t pol) {
  uint32_t v;
  asm volatile("ld.global.cg.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
// coherent load with an L2 policy
__device__ __forceinline__ uint32_t ld_pol(const void *p, uint64_t pol) {
  uint32_t v;
  asm volatile("ld.global.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol) : "memory");
  return v;
}
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}
__device__ __forceinline__ unsigned lanemask_le() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_le;" : "=r"(m));
  return m;
}
template <class T>
__device__ __forceinline__ T ld_vol(const T &x) {
  return *(const volatile T *)&x;
}
template <class T>
__device__ __forceinline__ void st_vol(T &x, T v) {
  *(volatile T *)&x = v;
}

__device__ __forceinline__ void raise_error(Ctl *ctl, int code, int where) {
  if (atomicCAS(&ctl->err, 0, code) == 0) ctl->err_where = where;
}

// ---------------------------------------------------------------- grid barrier
// Monotone arrival counter: the k-th barrier of a launch completes when the
// counter reaches k * gridDim.x.  Thread 0 of each CTA arrives with a release
// reduction and polls with acquire loads; the wait is bounded by cap_ns of
// %globaltimer time, after which it raises GBF_ERR_TIMEOUT and returns.
// Returns true (uniformly across the CTA) if no error has been raised.
struct Barrier {
  unsigned epoch;
  long long cap_ns;
};

__device__ __forceinline__ bool grid_sync(Ctl *ctl, Barrier &b, int *s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    b.epoch += gridDim.x;
    fence_acq_rel();
    red_release_add(&ctl->bar, 1u);
    unsigned long long t0 = 0;
    unsigned spins = 0;
    while ((int)(ld_acquire(&ctl->bar) - b.epoch) < 0) {
      if ((++spins & 255u) == 0) {
        unsigned long long t = globaltimer();
        if (t0 == 0) t0 = t;
        else if ((long long)(t - t0) > b.cap_ns) {
          raise_error(ctl, GBF_ERR_TIMEOUT, 1);
          break;
        }
      }
    }
    fence_acq_rel();
    *s_flag = ld_vol(ctl->err);
  }
  __syncthreads();
  return *s_flag == 0;
}

// Fault injection: wait on a flag nothing sets, bounded like a barrier; when
// the limit runs out, report the timeout as a stalled barrier would.
__device__ __forceinline__ void injected_wait(Ctl *ctl, long long cap_ns) {
  unsigned long long t0 = globaltimer();
  while (ld_vol(ctl->stop) == 0) {
    if ((long long)(globaltimer() - t0) > cap_ns) {
      raise_error(ctl, GBF_ERR_TIMEOUT, 9);
      break;
    }
    __nanosleep(1000);
  }
}

// ------------------------------------------------------------------- scans
// Exclusive block scan of one uint32 per thread; returns the exclusive prefix
// and writes the block total to *total.  s_tmp needs 33 words.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t *s_tmp, uint32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t y = __shfl_up_sync(kFull, inc, d);
    if (lane >= d) inc += y;
  }
  if (lane == 31) s_tmp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = (lane < nw) ? s_tmp[lane] : 0u;
    uint32_t si = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      uint32_t y = __shfl_up_sync(kFull, si, d);
      if (lane >= d) si += y;
    }
    s_tmp[lane] = si - s;  // exclusive warp offsets
    if (lane == 31) s_tmp[32] = si;
  }
  __syncthreads();
  uint32_t r = s_tmp[warp] + inc - x;
  *total = s_tmp[32];
  __syncthreads();
  return r;
}

// Block-wide sum of a 64-bit value (result valid in thread 0).
__device__ __forceinline__ unsigned long long block_sum64(unsigned long long x,
                                                          unsigned long long *s_tmp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) x += __shfl_down_sync(kFull, x, d);
  if (lane == 0) s_tmp[warp] = x;
  __syncthreads();
  unsigned long long r = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < nw; i++) r += s_tmp[i];
  __syncthreads();
  return r;
}

__device__ __forceinline__ int block_min_i32(int x, int *s_tmp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) x = min(x, __shfl_down_sync(kFull, x, d));
  if (lane == 0) s_tmp[warp] = x;
  __syncthreads();
  int r = kInf;
  if (threadIdx.x == 0)
    for (int i = 0; i < nw; i++) r = min(r, s_tmp[i]);
  __syncthreads();
  return r;
}

// ---------------------------------------------------- shared-memory layout
constexpr int kU = 4;  // 32-edge windows a warp keeps in flight per step

// Dynamic shared memory of the frontier kernels:
//   base/u/adj  [Bmax+2]   per frontier vertex of the current chunk: start in
//                          the chunk's edge space, vertex id, CSR offset of
//                          its first arc
//   out_v/out_d [cap]      staged next-frontier vertices and their degrees
//   pref        [cap]      exclusive prefix of out_d (or ranks) during a flush
//   out_a       [cap]      CSR offset of each staged vertex's first arc (only
//                          for queues that carry it)
//   fv/fs       [cap]      staged bucket filings: vertex, slot (<0: overflow)
//   hist/gbase  [nB]       per-slot counts and reserved positions of a flush
struct PushSmem {
  uint32_t *base;
  int32_t *u;
  uint32_t *adj;
  int32_t *out_v;
  uint32_t *out_d;
  uint32_t *pref;
  uint32_t *out_a;
  int32_t *fv;
  int32_t *fs;
  uint32_t *hist;
  uint32_t *gbase;
  uint32_t *misc;  // [0] n_out [1] pos [2] dpos [3] flag [4] n_filed [5] n_ovf [6] ovf pos [7] ovf min,
                   // [8..41] scan tmp, [48..49] next chunk of the blocked edgeMap
  unsigned long long *misc64;  // 32 entries
  uint32_t cap_out;
};

// Staging capacity for a CTA of `block` threads: room for two passes of kU
// appends per thread, capped (entries beyond it spill to global memory), and
// never below two appends per thread (the conversion and update loops add up
// to one entry per thread between flush checks).
__host__ __device__ inline int stage_capacity(int block) {
  const int c = 2 * kU * block;
  return c < 8192 ? c : (8192 > 2 * block ? 8192 : 2 * block);
}

struct SmemShape {
  int bmax;   // largest piece of the blocked edgeMap
  int cap;    // staging capacity (stage_capacity(blockDim))
  int filed;  // 1: reserve the bucket-filing stage
  int nB;     // bucket slots (histogram size)
  int adj;    // 1: stage first-arc offsets (queues with an adj array)
};

__host__ __device__ inline size_t push_smem_bytes(const SmemShape &sh) {
  size_t w = 64 + 3 * (size_t)(sh.bmax + 2) + (sh.adj ? 4 : 3) * (size_t)sh.cap;
  if (sh.filed) w += 2 * (size_t)sh.cap + 2 * (size_t)sh.nB;
  return 8 * 32 + 4 * w + 16;
}

__device__ __forceinline__ PushSmem carve_push_smem(void *raw, const SmemShape &sh) {
  PushSmem S;
  unsigned long long *p64 = (unsigned long long *)raw;
  S.misc64 = p64;
  uint32_t *p = (uint32_t *)(p64 + 32);
  S.misc = p;
  p += 64;
  S.base = p;
  p += sh.bmax + 2;
  S.u = (int32_t *)p;
  p += sh.bmax + 2;
  S.adj = p;
  p += sh.bmax + 2;
  S.out_v = (int32_t *)p;
  p += sh.cap;
  S.out_d = p;
  p += sh.cap;
  S.pref = p;
  p += sh.cap;
  S.out_a = nullptr;
  if (sh.adj) {
    S.out_a = p;
    p += sh.cap;
  }
  S.fv = S.fs = nullptr;
  S.hist = S.gbase = nullptr;
  if (sh.filed) {
    S.fv = (int32_t *)p;
    p += sh.cap;
    S.fs = (int32_t *)p;
    p += sh.cap;
    S.hist = p;
    p += sh.nB;
    S.gbase = p;
  }
  S.cap_out = (uint32_t)sh.cap;
  return S;
}

// Warp-collective: append the lanes with emit set to the CTA staging buffer
// (vertex, degree, CSR offset of its first arc).
__device__ __forceinline__ void stage_append(PushSmem &S, bool emit, int32_t v, uint32_t d,
                                             uint32_t a) {
  unsigned bal = __ballot_sync(kFull, emit);
  if (bal == 0) return;
  const int lane = threadIdx.x & 31;
  int leader = __ffs(bal) - 1;
  uint32_t pos = 0;
  if (lane == leader) pos = atomicAdd(&S.misc[0], (uint32_t)__popc(bal));
  pos = __shfl_sync(kFull, pos, leader);
  if (emit) {
    uint32_t r = pos + __popc(bal & lanemask_lt());
    S.out_v[r] = v;
    S.out_d[r] = d;
    if (S.out_a) S.out_a[r] = a;
  }
}

// Output frontier description (sparse vertexSubset with degree prefix and,
// if adj is set, the CSR offset of every entry's first arc).
struct QueueOut {
  int32_t *q;
  uint32_t *qoff;
  uint32_t *adj;
  uint32_t *cs;
  unsigned long long *counter;  // (count << 32) | degree sum, reserved per flush
  uint32_t q_cap;
  uint32_t cs_cap;
};

// CTA-collective: write the staged entries to the output queue.  One 64-bit
// atomicAdd reserves both the queue range and the edge-space range, so the
// per-entry degree prefix (qoff) is globally consistent; every chunk start
// (multiple of 256 edges) falling in an entry's range records the entry.
// With off given, the entries were staged as vertices only and their degree
// and first-arc offset are read here, many loads in flight at once.
__device__ __forceinline__ void stage_flush(PushSmem &S, const QueueOut &out, Ctl *ctl,
                                            const uint32_t *off = nullptr) {
  __syncthreads();
  const uint32_t k = min(S.misc[0], S.cap_out);  // entries beyond cap were spilled
  if (k == 0) return;
  const uint32_t tid = threadIdx.x, bd = blockDim.x;
  if (off) {
    for (uint32_t i = tid; i < k; i += bd) {
      const int32_t v = S.out_v[i];
      const uint32_t a = __ldg(off + v);
      S.out_d[i] = __ldg(off + v + 1) - a;
      if (S.out_a) S.out_a[i] = a;
    }
    __syncthreads();
  }
  const uint32_t per = (k + bd - 1) / bd;
  const uint32_t lo = min(k, tid * per), hi = min(k, lo + per);
  uint32_t loc = 0;
  for (uint32_t i = lo; i < hi; i++) loc += S.out_d[i];
  uint32_t total;
  uint32_t ex = block_excl_scan(loc, S.misc + 8, &total);
  for (uint32_t i = lo; i < hi; i++) {
    S.pref[i] = ex;
    ex += S.out_d[i];
  }
  if (tid == 0) {
    unsigned long long old = atomicAdd(out.counter, ((unsigned long long)k << 32) | total);
    uint32_t pos = (uint32_t)(old >> 32);
    if ((unsigned long long)pos + k > out.q_cap) {
      raise_error(ctl, GBF_ERR_OVERFLOW, 2);
      S.misc[3] = 1;
    } else {
      S.misc[3] = 0;
    }
    S.misc[1] = pos;
    S.misc[2] = (uint32_t)old;
  }
  __syncthreads();
  if (S.misc[3] == 0) {
    const uint32_t pos = S.misc[1], dpos = S.misc[2];
    for (uint32_t i = tid; i < k; i += bd) {
      out.q[pos + i] = S.out_v[i];
      out.qoff[pos + i] = dpos + S.pref[i];
      if (out.adj) out.adj[pos + i] = S.out_a[i];
    }
    // chunk starts (multiples of 256) inside [dpos, dpos + total), spread over
    // the CTA: each finds its entry by binary search of the staged prefix
    const uint32_t c0 = (dpos + kFine - 1) >> kFineLog;
    const uint32_t c1 = (uint32_t)(((unsigned long long)dpos + total + kFine - 1) >> kFineLog);
    for (uint32_t c = c0 + tid; c < c1; c += bd) {
      const uint32_t rel = (c << kFineLog) - dpos;
      uint32_t lo = 0, hi = k;  // largest i with pref[i] <= rel
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (S.pref[mid] <= rel) lo = mid;
        else hi = mid;
      }
      if (c < out.cs_cap) out.cs[c] = pos + lo;
    }
  }
  __syncthreads();
  if (tid == 0) S.misc[0] = 0;
  __syncthreads();
}

// CTA-collective, called right after a __syncthreads that follows the last
// appends: flush unless `room` more entries fit.  The barrier between the
// read and the flush keeps every thread's read of the count ahead of any
// thread's next append, so all threads take the same decision.
__device__ __forceinline__ void stage_make_room(PushSmem &S, const QueueOut &out, Ctl *ctl,
                                                uint32_t room) {
  const bool full = S.misc[0] + room > S.cap_out;
  __syncthreads();
  if (full) stage_flush(S, out, ctl);
}

// Input frontier description.
struct QueueIn {
  const int32_t *q;
  const uint32_t *qoff;
  const uint32_t *adj;
  const uint32_t *cs;
  uint32_t cnt;  // entries
  uint32_t D;    // degree sum (frontier edges)
};

// Largest k with base[k] <= x, for base[0] <= x < base[nv].
__device__ __forceinline__ uint32_t smem_upper(const uint32_t *base, uint32_t nv, uint32_t x) {
  uint32_t lo = 0, hi = nv;
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (base[mid] <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

// CTA-collective walk over the edges [e_lo, e_hi) of a chunk whose nv
// frontier vertices (each with at least one edge) are described by
// S.base/u/adj, base[nv] being the end of the last one.  Each warp takes a
// contiguous run of K windows of 32 consecutive edges (coalesced target
// loads); it locates the vertex of each lane from the boundaries falling in
// the window (one shared load per lane and a warp OR).  Every step hands kU
// windows to fn.batch, which issues all their loads before using them.
// Warps do not synchronise inside the walk: appends that find the shared
// staging buffer full take the sink's direct path to global memory.
template <class Fn, class Sink>
__device__ __forceinline__ void walk_chunk(PushSmem &S, uint32_t m, uint32_t nv, uint32_t e_lo,
                                           uint32_t e_hi, Fn &fn, Sink &sink) {
  constexpr int U = Fn::kWin;  // windows per step
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t nwin = (e_hi - e_lo + 31) >> 5;
  uint32_t K = (nwin + nw - 1) / nw;
  K = (K + U - 1) / U * U;
  const uint32_t w_lo = e_lo + (uint32_t)warp * K * 32;
  const uint32_t w_hi = min(w_lo + K * 32, e_hi);
  uint32_t j = (w_lo < w_hi) ? smem_upper(S.base, nv, w_lo) : 0u;
  // vertex j (the owner of the next window's first edge), kept in registers
  // while windows stay inside it: start in the chunk's edge space, first arc,
  // id, and the start of vertex j + 1 (base[nv] is the end of the last one)
  uint32_t jb = S.base[j], ja = S.adj[j], jn = S.base[j + 1];
  int32_t ju = S.u[j];
  for (uint32_t st = 0; st < K; st += U) {
    bool val[U];
    int32_t uu[U];
    uint32_t idx[U];
#pragma unroll
    for (int r = 0; r < U; r++) {
      const uint32_t b = w_lo + (st + r) * 32;
      const bool live = b < w_hi;  // warp-uniform
      const uint32_t e = b + lane;
      val[r] = live && e < w_hi;
      idx[r] = 0u;
      uu[r] = 0;
      if (live) {
        if (jn >= b + 32) {
          // no vertex starts inside the window: all of it belongs to j
          idx[r] = ja + (e - jb);
          uu[r] = ju;
        } else {
          // vertices j+1.. that start inside the window, one bit per offset
          unsigned bpos = 0;
          const uint32_t k = j + 1 + lane;
          if (k <= nv) {
            const uint32_t bb = S.base[k];
            if (bb < b + 32) bpos = 1u << (bb - b);
          }
          const unsigned mask = __reduce_or_sync(kFull, bpos);
          const uint32_t jj = min(j + __popc(mask & lanemask_le()), nv - 1);
          idx[r] = S.adj[jj] + (e - S.base[jj]);
          uu[r] = S.u[jj];
          j += __popc(mask);  // the owner of the window's last edge
          jb = S.base[j];
          ja = S.adj[j];
          ju = S.u[j];
          jn = S.base[j + 1];
        }
        if (jn == b + 32 && j < nv) {  // the next vertex starts with the next window
          j++;
          jb = jn;
          ja = S.adj[j];
          ju = S.u[j];
          jn = S.base[j + 1];
        }
        if (val[r]) val[r] = idx[r] < m;
      }
    }
    fn.batch(val, uu, idx, sink, S);
  }
  fn.drain(sink, S);
}

// Blocked sparse edgeMap over the frontier `in` with chunks of B = 256 << s
// edges located through the chunk-start table (edgeMapBlocked, Alg. 2).  A
// chunk's frontier vertices are loaded into the shared arrays bmax at a time
// and each piece's share of the chunk's edges is walked before the next
// piece is loaded, so the chunk size does not depend on the degrees.  Each
// CTA starts with chunk blockIdx.x and then takes chunks from a global
// counter, so CTAs that finish early take up the slack of slow ones before
// the round's barrier.  `inv` numbers the calls of a launch (identically in
// every CTA): call inv uses counter ctl->work[inv % 4] and clears
// ctl->work[(inv + 2) % 4], whose last user finished before at least one
// grid barrier.
template <class Fn, class Sink>
__device__ __forceinline__ void blocked_edge_map(const DevGraph &g, const QueueIn &in, int s,
                                                 uint32_t bmax, PushSmem &S, Fn &fn, Sink &sink,
                                                 Ctl *ctl, int inv) {
  const uint32_t B = kFine << s;
  const uint32_t nfine = (in.D + kFine - 1) >> kFineLog;
  const uint32_t nch = (in.D + B - 1) / B;
  unsigned int *work = &ctl->work[inv & 3];
  if (blockIdx.x == 0 && threadIdx.x == 0) st_vol(ctl->work[(inv + 2) & 3], 0u);
  uint32_t c = blockIdx.x;
  for (uint32_t it = 0; c < nch; it++) {
    const uint32_t e_lo = c * B, e_hi = min(e_lo + B, in.D);
    const uint32_t f1 = (c + 1) << s;
    const uint32_t i0 = in.cs[c << s];
    const uint32_t i1 = (f1 < nfine) ? in.cs[f1] : in.cnt - 1;
    const bool bad = i1 < i0 || i1 >= in.cnt;  // never expected
    if (bad && threadIdx.x == 0) raise_error(ctl, GBF_ERR_OVERFLOW, 3);
    // The next chunk for this CTA, taken while the current one is walked.
    // Two slots: a thread may still be reading the previous chunk's slot
    // when thread 0 writes this one (at most one chunk apart, as every
    // piece holds a __syncthreads).
    if (threadIdx.x == 0) S.misc[48 + (it & 1)] = gridDim.x + atomicAdd(work, 1u);
    const uint32_t iend = bad ? i0 : i1 + 1;
    for (uint32_t p0 = i0; p0 < iend; p0 += bmax) {  // CTA-uniform
      const uint32_t nv = min(bmax, iend - p0);
      for (uint32_t j = threadIdx.x; j < nv; j += blockDim.x) {
        const int32_t u = in.q[p0 + j];
        S.base[j] = in.qoff[p0 + j];
        S.u[j] = u;
        S.adj[j] = in.adj ? in.adj[p0 + j] : __ldg(g.off + u);
      }
      if (threadIdx.x == 0) S.base[nv] = (p0 + nv < in.cnt) ? in.qoff[p0 + nv] : in.D;
      __syncthreads();
      const uint32_t lo = max(e_lo, S.base[0]), hi = min(e_hi, S.base[nv]);
      if (lo < hi) walk_chunk(S, g.m, nv, lo, hi, fn, sink);
      sink.chunk_end(S);  // starts with __syncthreads
    }
    if (iend == i0) __syncthreads();  // the slot write above is read below
    c = S.misc[48 + (it & 1)];
  }
}

// One entry that found the stage full, written straight to the output
// queue: it reserves its own count and edge range, then its chunk starts.
__device__ __forceinline__ void stage_spill_one(PushSmem &, int32_t v, uint32_t d, uint32_t a,
                                                const QueueOut &out, Ctl *ctl, const uint32_t *off) {
  if (off) {
    a = __ldg(off + v);
    d = __ldg(off + v + 1) - a;
  }
  const unsigned long long old = atomicAdd(out.counter, (1ull << 32) | d);
  const uint32_t qp = (uint32_t)(old >> 32), e0 = (uint32_t)old;
  if (qp >= out.q_cap) {
    raise_error(ctl, GBF_ERR_OVERFLOW, 11);
    return;
  }
  out.q[qp] = v;
  out.qoff[qp] = e0;
  if (out.adj) out.adj[qp] = a;
  for (uint32_t c = (e0 + kFine - 1) >> kFineLog; (c << kFineLog) < e0 + d; c++)
    if (c < out.cs_cap) out.cs[c] = qp;
}

// Warp-collective: stage the lanes with emit set; an entry that finds the
// stage full is written straight to the output queue (reserving its own
// count and edge range, then its chunk starts).  With off given the entry's
// degree and first-arc offset are read from the CSR (at flush time for
// staged entries, here for spilled ones) and d, a are ignored.
__device__ __forceinline__ void stage_append_or_spill(PushSmem &S, bool emit, int32_t v,
                                                      uint32_t d, uint32_t a,
                                                      const QueueOut &out, Ctl *ctl,
                                                      const uint32_t *off) {
  const unsigned bal = __ballot_sync(kFull, emit);
  if (bal == 0) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(bal) - 1;
  uint32_t pos = 0;
  if (lane == leader) pos = atomicAdd(&S.misc[0], (uint32_t)__popc(bal));
  pos = __shfl_sync(kFull, pos, leader);
  if (!emit) return;
  const uint32_t r = pos + __popc(bal & lanemask_lt());
  if (r < S.cap_out) {
    S.out_v[r] = v;
    S.out_d[r] = d;
    if (S.out_a) S.out_a[r] = a;
    return;
  }
  stage_spill_one(S, v, d, a, out, ctl, off);
}

// Sink that stages into shared memory and flushes into a QueueOut.  With
// off given, callers append vertices only (d, a ignored) and the degrees and
// first-arc offsets are read when the stage is flushed.
struct StagedSink {
  QueueOut out;
  Ctl *ctl;
  const uint32_t *off;
  __device__ __forceinline__ void append(PushSmem &S, bool emit, int32_t v, uint32_t d,
                                         uint32_t a) {
    stage_append_or_spill(S, emit, v, d, a, out, ctl, off);
  }
  // Warp-collective: the U appends of one walk step with one shared-memory
  // atomic for the whole warp.
  template <int U>
  __device__ __forceinline__ void append_n(PushSmem &S, const bool *emit, const int32_t *v,
                                           const uint32_t *d, const uint32_t *a) {
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
    if (lane == 0) pos = atomicAdd(&S.misc[0], tot);
    pos = __shfl_sync(kFull, pos, 0);
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int r = 0; r < U; r++) {
      if (emit[r]) {
        const uint32_t i = pos + __popc(bal[r] & lt);
        if (i < S.cap_out) {
          S.out_v[i] = v[r];
          S.out_d[i] = d[r];
          if (S.out_a) S.out_a[i] = a[r];
        } else {
          stage_spill_one(S, v[r], d[r], a[r], out, ctl, off);
        }
      }
      pos += __popc(bal[r]);
    }
  }
  // CTA-collective, between chunks
  __device__ __forceinline__ void chunk_end(PushSmem &S) {
    __syncthreads();
    if (S.misc[0] > (S.cap_out >> 1)) stage_flush(S, out, ctl, off);
  }
  __device__ __forceinline__ void finish(PushSmem &S) { stage_flush(S, out, ctl, off); }
};

// Chunk exponent s (chunk = 256 << s edges) for a frontier of D edges:
// about `per_cta` chunks per CTA (the counter balances them), s <= max_s.
__device__ __forceinline__ int chunk_shift(uint32_t D, uint32_t per_cta, int max_s) {
  const uint32_t per = D / (per_cta * gridDim.x);
  int s = 0;
  while (s < max_s && (kFine << s) < per) s++;
  return s;
}

// Largest s with chunks of 256 << s edges not above `edges` (and 2^16).
__device__ __forceinline__ int chunk_shift_cap(uint32_t edges) {
  int s = 0;
  while (s < 8 && (kFine << (s + 1)) <= edges) s++;
  return s;
}

}  // namespace dev
}  // namespace gbf
