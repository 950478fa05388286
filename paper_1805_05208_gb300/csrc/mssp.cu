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
// Lane width.  A query first runs with 16-bit lanes (16 bytes per vertex, so
// the lanes of an RMAT 22 graph, 64 MB, stay in L2), lowered with a 32-bit
// compare-and-swap on the word of two lanes.  A proposal above 65534 is not
// written: it raises a flag, the rounds stop, and the same launch runs the
// query again with 32-bit lanes (written with atomicMin).  Without the flag
// no proposal was dropped, so the 16-bit result is exact.  A workspace whose
// 16-bit run overflowed once remembers it (a device word) and starts with
// 32-bit lanes from then on.
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
  void *dd;          // n x kMsspLanes distances, vertex-major (16- or 32-byte rows)
  unsigned *imp[3];  // lanes improved in round r % 3: byte v & 3 of word v >> 2
  unsigned *wide;    // device word: a 16-bit run on this workspace overflowed once
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

// The improved-lane byte of frontier vertex u, from the previous round's
// masks: final at this round's start, so an L1 copy is current (the grid
// barrier's acquire drops older ones); the arcs of one vertex read it once
// from L2.
__device__ __forceinline__ unsigned lane_byte(const unsigned *words, uint32_t u) {
  return (words[u >> 2] >> (8u * (u & 3u))) & 0xffu;
}

// Loads of the 8 lanes of vertex v.  kL2: at L2, for targets, which other
// SMs lower during the round; otherwise through L1, for the frontier vertex
// whose arcs are walked: a copy from the round's start may miss a lowering
// made during the round, which only proposes a larger (still valid)
// distance, and the lowering marks the vertex improved, so its new value is
// propagated next round.
template <bool kL2>
__device__ __forceinline__ int4 ld16(const int4 *p) {
  return kL2 ? __ldcg(p) : *p;
}

// 32-bit lanes: two 16-byte words per vertex, written with atomicMin.
struct Lanes32 {
  static constexpr uint32_t kWords4 = 2;  // 16-byte words per vertex
  template <bool kL2>
  __device__ __forceinline__ static void load(const void *dd, uint32_t v, int32_t (&x)[kMsspLanes]) {
    const int4 *p = reinterpret_cast<const int4 *>(dd) + (size_t)v * 2;
    const int4 a = ld16<kL2>(p), b = ld16<kL2>(p + 1);
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
    x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
  }
  __device__ __forceinline__ static int4 inf4() { return make_int4(kInf, kInf, kInf, kInf); }
  __device__ __forceinline__ static void set_zero(void *dd, uint32_t v, int i) {
    reinterpret_cast<int32_t *>(dd)[(size_t)v * kMsspLanes + i] = 0;
  }
  // writeMin of c[i] into lane i of v for the lanes in `want`; returns the
  // lanes it lowered
  __device__ __forceinline__ static unsigned relax(void *dd, uint32_t v, unsigned want,
                                                   const int32_t *c, const int32_t *, Ctl *) {
    int32_t *row = reinterpret_cast<int32_t *>(dd) + (size_t)v * kMsspLanes;
    unsigned better = 0;
#pragma unroll
    for (int i = 0; i < kMsspLanes; i++)
      if (((want >> i) & 1u) && atomicMin(row + i, c[i]) > c[i]) better |= 1u << i;
    return better;
  }
};

// 16-bit lanes: one 16-byte word per vertex, 0xffff = unreached, at most
// 65,534 (lowered by MsspFn::lower).
struct Lanes16 {
  static constexpr uint32_t kWords4 = 1;
  template <bool kL2>
  __device__ __forceinline__ static void load(const void *dd, uint32_t v, int32_t (&x)[kMsspLanes]) {
    const int4 a = ld16<kL2>(reinterpret_cast<const int4 *>(dd) + v);
    const uint32_t w4[4] = {(uint32_t)a.x, (uint32_t)a.y, (uint32_t)a.z, (uint32_t)a.w};
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const uint32_t lo = w4[j] & 0xffffu, hi = w4[j] >> 16;
      x[2 * j] = lo == 0xffffu ? kInf : (int32_t)lo;
      x[2 * j + 1] = hi == 0xffffu ? kInf : (int32_t)hi;
    }
  }
  __device__ __forceinline__ static int4 inf4() { return make_int4(-1, -1, -1, -1); }
  __device__ __forceinline__ static void set_zero(void *dd, uint32_t v, int i) {
    reinterpret_cast<uint16_t *>(dd)[(size_t)v * kMsspLanes + i] = 0;
  }
};

// 16-byte coherent load at L2 with an L2 policy (p 16-byte aligned)
__device__ __forceinline__ uint4 ldcg_pol_v4(const void *p, uint64_t pol) {
  uint4 v;
  asm volatile("ld.global.cg.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(pol));
  return v;
}

// Update of Alg. 4 for the lanes of kWin windows of frontier arcs.  The arcs
// stream through L2 first-out, the distance lanes stay (evict-last).
template <class L>
struct MsspFn {
  static constexpr int kWin = 2;  // windows per walk step (each carries 16 lane values)
  template <class Sink>
  __device__ __forceinline__ void drain(Sink &, PushSmem &) {}  // nothing deferred
  const uint32_t *off;
  const int32_t *tgt;
  const uint32_t *w;
  void *dd;
  const unsigned *lanes_in;
  unsigned *imp_out;
  Ctl *ctl;
  unsigned long long relax;
  uint64_t stream_pol, keep_pol;
  // the lanes of v that u (improved in lanes lm) lowers, with their writeMins
  __device__ __forceinline__ unsigned lower(uint32_t u, uint32_t v, unsigned lm, int32_t wt) {
    if constexpr (L::kWords4 == 1) {
      // 16-bit lanes, two per 32-bit word, with per-halfword SIMD: candidate
      // u + w (saturating at 0xffff), lanes of u that did not improve set to
      // 0xffff, compared with v's lanes and merged in with a compare-and-swap
      const uint4 a = reinterpret_cast<const uint4 *>(dd)[u];  // through L1 (see ld16)
      const uint4 b = ldcg_pol_v4(reinterpret_cast<const uint4 *>(dd) + v, keep_pol);
      const uint32_t du[4] = {a.x, a.y, a.z, a.w};
      uint32_t cur[4] = {b.x, b.y, b.z, b.w};
      // the weight in both halves, clamped (a weight above 0xffff saturates the
      // sum, and the overflow check below sends the query to 32-bit lanes)
      const uint32_t w2 = min((uint32_t)wt, 0xffffu) * 0x10001u;
      uint32_t cand[4], nw[4];
      bool act[4];
      unsigned ovf = 0;
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const uint32_t m = (((lm >> (2 * j)) & 1u) ? 0xffffu : 0u) |
                           (((lm >> (2 * j + 1)) & 1u) ? 0xffff0000u : 0u);
        cand[j] = __vaddus2(du[j], w2) | ~m;
        // a saturated proposal to an unreached lane: the distance does not fit
        ovf |= __vcmpeq2(cand[j], 0xffffffffu) & __vcmpeq2(cur[j], 0xffffffffu) & m;
        nw[j] = __vminu2(cur[j], cand[j]);
        act[j] = nw[j] != cur[j];
      }
      if (ovf) atomicOr(&ctl->lane_ovf, 1u);
      uint32_t prev[4];
      unsigned *row = reinterpret_cast<unsigned *>(dd) + (size_t)v * 4;
#pragma unroll
      for (int j = 0; j < 4; j++) prev[j] = act[j] ? atomicCAS(row + j, cur[j], nw[j]) : cur[j];
      unsigned better = 0;
#pragma unroll
      for (int j = 0; j < 4; j++) {
        if (!act[j]) continue;
        // a failed swap: another thread lowered the word; retry from its value
        // (lock-free: every failure means the word fell; capped all the same)
        for (int tries = 0; prev[j] != cur[j] && tries < (1 << 17); tries++) {
          cur[j] = prev[j];
          nw[j] = __vminu2(cur[j], cand[j]);
          if (nw[j] == cur[j]) break;
          prev[j] = atomicCAS(row + j, cur[j], nw[j]);
        }
        if (prev[j] == cur[j]) {
          const uint32_t lt = __vcmpltu2(nw[j], cur[j]);
          better |= ((lt & 1u) << (2 * j)) | (((lt >> 16) & 1u) << (2 * j + 1));
        } else {
          raise_error(ctl, GBF_ERR_TIMEOUT, 21);  // the cap: never expected
        }
      }
      return better;
    } else {
      int32_t du[kMsspLanes], dv[kMsspLanes], c[kMsspLanes];
      L::template load<false>(dd, u, du);
      L::template load<true>(dd, v, dv);
      unsigned want = 0;
#pragma unroll
      for (int i = 0; i < kMsspLanes; i++) {
        const bool li = (lm >> i) & 1u;  // u improved in lane i: du[i] < INF
        c[i] = li ? du[i] + wt : kInf;
        if (li && c[i] < dv[i]) want |= 1u << i;
      }
      return want ? L::relax(dd, v, want, c, dv, ctl) : 0u;
    }
  }
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
        v[r] = (int32_t)ldg_pol(tgt + idx[r], stream_pol);
        wt[r] = (int32_t)ldg_pol(w + idx[r], stream_pol);
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
        const unsigned better = lower((uint32_t)u[r], (uint32_t)v[r], lm[r], wt[r]);
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

struct MsspCounters {
  unsigned long long scanned, expanded, relax;
};

// One run of the query with lanes L: initialisation, sources, rounds, and
// (unless a 16-bit run overflowed) the output rows.  Returns false on a
// device error; *done is false when the run overflowed and must be redone
// with 32-bit lanes.
template <class L>
__device__ bool mssp_run(const MsspParams &P, PushSmem &S, Barrier &bar, int *s_flag,
                         MsspCounters &cnt, int &bem, bool *done, unsigned long long t_start) {
  Ctl *ctl = P.ctl;
  const DevGraph g = P.g;
  const uint32_t n = (uint32_t)g.n;
  const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  const uint32_t nw4 = (n + 3) >> 2;
  const int k = P.k;
  const bool l16 = L::kWords4 == 1;
  *done = false;
  // every lane unreached, no lane improved anywhere
  for (uint32_t i = gt; i < n * L::kWords4; i += gs) reinterpret_cast<int4 *>(P.dd)[i] = L::inf4();
  for (uint32_t i = gt; i < nw4; i += gs) {
    P.imp[0][i] = 0u;
    P.imp[1][i] = 0u;
    P.imp[2][i] = 0u;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st_vol(ctl->fr[0], 0ull);
    st_vol(ctl->fr[1], 0ull);
    st_vol(ctl->fr[2], 0ull);
  }
  bool ok = grid_sync(ctl, bar, s_flag);
  // sources: D_i[srcs[i]] = 0, lane i improved at its source in round 0; the
  // first frontier holds each distinct source with at least one arc
  if (ok && blockIdx.x == 0) {
    bool emit = false;
    int32_t s = 0;
    uint32_t d = 0, a = 0;
    if ((int)threadIdx.x < k) {
      s = P.srcs[threadIdx.x];
      L::set_zero(P.dd, (uint32_t)s, (int)threadIdx.x);
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
  ok = ok && grid_sync(ctl, bar, s_flag);

  int qb = 0;
  unsigned long long fr = ok ? ld_vol(ctl->fr[0]) : 0ull;
  bool ovf = false;
  for (int32_t round = 1; ok && round <= g.n; round++) {
    const uint32_t cnt_v = (uint32_t)(fr >> 32), D = (uint32_t)fr;
    if (cnt_v == 0) break;
    unsigned long long *outc = &ctl->fr[round % 3];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st_vol(ctl->fr[(round + 1) % 3], 0ull);
      atomicAdd(&ctl->rounds, 1);
      atomicAdd(&ctl->push_rounds, 1);
      cnt.scanned += D;
      cnt.expanded += cnt_v;
    }
    // ResetFlags: the lane masks of round r-2, last read in round r-1
    unsigned *stale = P.imp[(round + 1) % 3];
    for (uint32_t i = gt; i < nw4; i += gs) stale[i] = 0u;
    QueueIn in{P.q[qb], P.qoff[qb], P.qadj[qb], P.cs[qb], cnt_v, D};
    MsspFn<L> fn{g.off, g.tgt, g.w, P.dd, P.imp[(round - 1) % 3], P.imp[round % 3], ctl, 0,
                 l2_evict_first(), l2_evict_last()};
    StagedSink sink{QueueOut{P.q[qb ^ 1], P.qoff[qb ^ 1], P.qadj[qb ^ 1], P.cs[qb ^ 1], outc, n,
                             P.cs_cap},
                    ctl, nullptr};
    blocked_edge_map(g, in, chunk_shift(D, 4u, chunk_shift_cap(MsspFn<L>::kWin * blockDim.x)),
                     (uint32_t)P.bmax, S, fn, sink, ctl, bem++);
    sink.finish(S);
    cnt.relax += fn.relax;
    qb ^= 1;
    if (!grid_sync(ctl, bar, s_flag)) {
      ok = false;
      break;
    }
    fr = ld_vol(*outc);
    if (P.trace && blockIdx.x == 0 && threadIdx.x == 0 && round <= P.trace_cap)
      P.trace[round - 1] = TraceRec{round, 1, cnt_v, D, (long long)(globaltimer() - t_start), 0};
    if (l16 && ld_vol(ctl->lane_ovf)) {  // complete at the barrier: every CTA stops here
      ovf = true;
      break;
    }
  }
  if (!ok) return false;
  if (ovf) {
    if (blockIdx.x == 0 && threadIdx.x == 0) st_vol(*P.wide, 1u);
    return grid_sync(ctl, bar, s_flag);  // every CTA past its last use of this run's state
  }
  // each lane's row of the output (consecutive vertices: coalesced per row)
  if (ld_vol(ctl->err) == 0) {
    for (uint32_t v = gt; v < n; v += gs) {
      int32_t x[kMsspLanes];
      L::template load<true>(P.dd, v, x);
#pragma unroll
      for (int i = 0; i < kMsspLanes; i++)
        if (i < k) P.rows[i][v] = x[i];
    }
  }
  *done = true;
  return true;
}

}  // namespace

__global__ void __launch_bounds__(1024) mssp_kernel(MsspParams P) {
  extern __shared__ unsigned long long smem_raw[];
  __shared__ int s_flag;
  PushSmem S = carve_push_smem(smem_raw, SmemShape{P.bmax, P.cap, 0, 0, 1});
  if (threadIdx.x == 0) S.misc[0] = 0;
  Ctl *ctl = P.ctl;
  Barrier bar{0u, P.cap_ns};
  if (P.inject_wait && blockIdx.x == 0 && threadIdx.x == 0) injected_wait(ctl, P.cap_ns);
  MsspCounters cnt{0, 0, 0};
  int bem = 0;
  bool done = false;
  const unsigned long long t_start = globaltimer();
  // the device word is written only by earlier launches: the same in every CTA
  bool ok = true;
  if (ld_vol(*P.wide) == 0u) ok = mssp_run<Lanes16>(P, S, bar, &s_flag, cnt, bem, &done, t_start);
  if (ok && !done) ok = mssp_run<Lanes32>(P, S, bar, &s_flag, cnt, bem, &done, t_start);
  unsigned long long t;
  t = block_sum64(cnt.scanned, S.misc64);
  if (threadIdx.x == 0 && t) atomicAdd(&ctl->edges_scanned, t);
  t = block_sum64(cnt.expanded, S.misc64);
  if (threadIdx.x == 0 && t) atomicAdd(&ctl->expanded, t);
  t = block_sum64(cnt.relax, S.misc64);
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
    // three lane-mask arrays, then the word that records a 16-bit overflow
    const size_t w4 = (n + 3) / 4;
    e = cudaMalloc((void **)&ws.mssp_imp, sizeof(unsigned) * (3 * std::max<size_t>(w4, 1) + 4));
    if (e != cudaSuccess) {
      ws.mssp_imp = nullptr;
      return cuda_fail(e, "cudaMalloc");
    }
    e = cudaMemset(ws.mssp_imp, 0, sizeof(unsigned) * (3 * std::max<size_t>(w4, 1) + 4));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
    acc += sizeof(unsigned) * (3 * w4 + 4);
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
  P.wide = ws.mssp_imp + 3 * std::max<size_t>(w4, 1);
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
