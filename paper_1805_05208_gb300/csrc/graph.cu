// Graph residency (the CSR representation of §3), validation, workspaces and
// the C entry points of gbf.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "dev_common.cuh"
#include "gbf_impl.h"

namespace gbf {

// ------------------------------------------------------------ error reporting
static thread_local std::string t_last_error;

void set_error(const std::string &msg) { t_last_error = msg; }

gbf_status cuda_fail(cudaError_t e, const char *what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return GBF_ERR_OOM;
  }
  return GBF_ERR_CUDA;
}

gbf_status check_smem(size_t bytes, const char *kernel) {
  int dev = 0, optin = 0;
  GBF_CUDA(cudaGetDevice(&dev));
  GBF_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (bytes > (size_t)optin) {
    set_error(std::string(kernel) + ": block size / heavy_cutoff need " + std::to_string(bytes) +
              " bytes of shared memory per CTA, more than the device's " + std::to_string(optin));
    return GBF_ERR_INVALID;
  }
  return GBF_OK;
}

// ------------------------------------------------------------------ options
Opts resolve(const gbf_options *o, const Graph &g, int kind) {
  gbf_options d;
  gbf_options_default(&d);
  if (!o) o = &d;
  Opts r;
  // block 0: per-kind default (wBFS gains from wider CTAs: fewer barrier
  // arrivals per round and more warps per chunk)
  const int kind_block = kind == GBF_TUNE_WBFS ? 512 : 256;
  r.block = o->block ? o->block : kind_block;
  if (r.block != 128 && r.block != 256 && r.block != 512 && r.block != 1024) r.block = kind_block;
  r.pull_divisor = o->pull_divisor ? o->pull_divisor : d.pull_divisor;
  // heavy_cutoff 0: per-kind default
  r.heavy_cutoff = o->heavy_cutoff ? o->heavy_cutoff
                                   : (kind == GBF_TUNE_MSBFS ? 1024 : 512);
  int hc = 256;
  while (hc < r.heavy_cutoff && hc < 16384) hc <<= 1;
  r.heavy_cutoff = std::max(hc, r.block);  // staging buffer must hold one CTA pass
  r.bucket_window = o->bucket_window;
  r.dense_wbfs = o->dense_wbfs ? 1 : 0;
  // ctas 0: every CTA that fits, except on sparse graphs (fewer than 8 arcs
  // per vertex: high diameter, thin frontiers, thousands of rounds whose cost
  // is the grid barrier), where half the SMs' worth of CTAs is faster; the
  // 64-lane MS-BFS keeps the full grid
  const bool sparse = g.n > 0 && (uint64_t)g.m < 8ull * (uint64_t)g.n;
  r.ctas = o->ctas > 0 ? o->ctas : (sparse && kind != GBF_TUNE_MSBFS ? std::max(g.num_sms / 2, 1) : 0);
  // pull_serial 0: per-kind default (the BFS pull hands long scans to a warp
  // walk only rarely; the multi-source pull after a few arcs)
  r.pull_serial = o->pull_serial > 0 ? std::min(o->pull_serial, 1 << 20)
                                     : (kind == GBF_TUNE_MSBFS ? 8 : 128);
  r.inject_wait = o->inject_wait ? 1 : 0;
  // pull_stay 0: default 24 (after a dense level, the next stays dense while
  // the frontier holds more than n / 24 vertices); negative: off
  r.pull_stay = o->pull_stay > 0 ? o->pull_stay : (o->pull_stay < 0 ? 0 : 24);
  // local_arcs: off unless positive (below the 20-bit degree field)
  r.local_arcs = o->local_arcs > 0 ? std::min(o->local_arcs, (1 << 20) - 1) : 0;
  long long us = o->spin_cap_us > 0 ? o->spin_cap_us : d.spin_cap_us;
  r.spin_cap_ns = us * 1000LL;
  return r;
}

// ------------------------------------------------------------- validation
namespace {

enum : unsigned { kBadOffsets = 1, kBadTarget = 2, kSelfLoop = 4, kBadWeight = 8,
                  kUnsorted = 16, kAsymmetric = 32, kWeightAsym = 64 };

__global__ void k_validate_basic(int32_t n, uint32_t m, const uint32_t *off, const int32_t *tgt,
                                 const uint32_t *w, unsigned *flags) {
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t tw = (gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  unsigned f = 0;
  if (gw == 0 && lane == 0 && (off[0] != 0 || off[n] != m)) f |= kBadOffsets;
  for (uint32_t v = gw; v < (uint32_t)n; v += tw) {
    const uint32_t s = off[v], e = off[v + 1];
    if (e < s || e > m) {
      f |= kBadOffsets;
      continue;
    }
    for (uint32_t k = s + lane; k < e; k += 32) {
      const int32_t t = tgt[k];
      if (t < 0 || t >= n) f |= kBadTarget;
      else if ((uint32_t)t == v) f |= kSelfLoop;
      if (w && w[k] == 0) f |= kBadWeight;
    }
  }
  if (f) atomicOr(flags, f);
}

__global__ void k_validate_symmetric(int32_t n, const uint32_t *off, const int32_t *tgt,
                                     const uint32_t *w, unsigned *flags) {
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t tw = (gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  unsigned f = 0;
  for (uint32_t v = gw; v < (uint32_t)n; v += tw) {
    const uint32_t s = off[v], e = off[v + 1];
    for (uint32_t k = s + lane; k < e; k += 32) {
      const int32_t u = tgt[k];
      if (k + 1 < e && tgt[k + 1] <= u) f |= kUnsorted;
      // binary search v in N(u)
      uint32_t lo = off[u], hi = off[u + 1];
      bool found = false;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        const int32_t x = tgt[mid];
        if (x == (int32_t)v) {
          found = true;
          if (w && w[mid] != w[k]) f |= kWeightAsym;
          break;
        }
        if (x < (int32_t)v) lo = mid + 1;
        else hi = mid;
      }
      if (!found) f |= kAsymmetric;
    }
  }
  if (f) atomicOr(flags, f);
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  x += 0x9e3779b97f4a7c15ULL;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
  return x ^ (x >> 31);
}

// Order-independent fingerprint (sum of mixed arc hashes) and max weight.
__global__ void k_digest(int32_t n, uint32_t m, const uint32_t *off, const int32_t *tgt,
                         const uint32_t *w, unsigned long long *sum, unsigned *wmax) {
  unsigned long long h = 0;
  unsigned mw = 0;
  const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (uint32_t k = gt; k < m; k += gs) {
    const unsigned wk = w ? w[k] : 0u;
    h += mix64(((unsigned long long)k << 32) ^ (unsigned)tgt[k] ^ ((unsigned long long)wk << 40));
    mw = max(mw, wk);
  }
  for (uint32_t v = gt; v <= (uint32_t)n; v += gs) h += mix64(0xabcdefULL ^ ((unsigned long long)v << 32) ^ off[v]);
  for (int d = 16; d > 0; d >>= 1) {
    h += __shfl_down_sync(0xffffffffu, h, d);
    mw = max(mw, __shfl_down_sync(0xffffffffu, mw, d));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(sum, h);
    atomicMax(wmax, mw);
  }
}

// Each vertex's arc to its highest-degree neighbour is moved to the front of
// its list (swapped with the first arc; the lowest position wins ties), so
// that the first arc of every vertex, and the dense step's first-arc check
// (f1), lead to the neighbour most likely to be on an early frontier.  The
// order of a vertex's arcs carries no meaning for any query; the weights
// move with their arcs.  A warp per vertex.
__global__ void k_hub_first(int32_t n, const uint32_t *off, int32_t *tgt, uint32_t *w) {
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t tw = (gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (uint32_t v = gw; v < (uint32_t)n; v += tw) {
    const uint32_t s = off[v], e = off[v + 1];
    if (e - s < 2) continue;
    unsigned long long best = 0;  // (degree << 32) | ~position: larger is better
    for (uint32_t k = s + lane; k < e; k += 32) {
      const int32_t t = tgt[k];
      const uint32_t d = off[t + 1] - off[t];
      const unsigned long long key = ((unsigned long long)d << 32) | (0xffffffffu - (k - s));
      if (key > best) best = key;
    }
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long y = __shfl_xor_sync(0xffffffffu, best, o);
      if (y > best) best = y;
    }
    const uint32_t j = s + (0xffffffffu - (uint32_t)best);
    if (lane == 0 && j != s) {
      const int32_t t0 = tgt[s];
      tgt[s] = tgt[j];
      tgt[j] = t0;
      if (w) {
        const uint32_t w0 = w[s];
        w[s] = w[j];
        w[j] = w0;
      }
    }
  }
}

// Per-vertex arrays derived from the CSR: bit v of leaf[] is set iff vertex
// v has degree exactly 1, bit v of iso[] iff it has degree 0, and f1[v] is
// the target of v's first arc (-1 without arcs).
__global__ void k_leaf(int32_t n, const uint32_t *off, const int32_t *tgt, uint32_t *leaf,
                       uint32_t *iso, int32_t *f1) {
  const uint32_t nw = ((uint32_t)n + 31) >> 5;
  const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (uint32_t i = gt; i < nw * 32u; i += gs) {
    const uint32_t a = i < (uint32_t)n ? off[i] : 0u, z = i < (uint32_t)n ? off[i + 1] : 0u;
    const bool in = i < (uint32_t)n;
    const unsigned b1 = __ballot_sync(0xffffffffu, in && z - a == 1u);
    const unsigned b0 = __ballot_sync(0xffffffffu, in && z == a);
    if ((threadIdx.x & 31) == 0) {
      leaf[i >> 5] = b1;
      iso[i >> 5] = b0;
    }
    if (in) f1[i] = z > a ? tgt[a] : -1;
  }
}

template <class T>
gbf_status dmalloc(T **p, size_t count, size_t &acc) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void **)p, sizeof(T) * count);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e, "cudaMalloc");
  }
  acc += sizeof(T) * count;
  return GBF_OK;
}

#define GBF_TRY(x)                      \
  do {                                  \
    gbf_status _s = (x);                \
    if (_s != GBF_OK) return _s;        \
  } while (0)

// The first nonzero device status of a batch of launches.
__global__ void k_keep_error(int *acc, const int *err) {
  if (*acc == 0) *acc = *err;
}

}  // namespace

// ------------------------------------------------------------- workspaces
gbf_status ws_ensure_base(Graph &g, Workspace &ws) {
  if (ws.ctl) return GBF_OK;
  const size_t n = (size_t)g.n, nw = (n + 31) / 32;
  const size_t cs = ((size_t)g.m + dev::kFine - 1) / dev::kFine + 2;
  size_t acc = 0;
  ws.n = g.n;
  ws.m = g.m;
  GBF_TRY(dmalloc(&ws.visited, nw, acc));
  GBF_TRY(dmalloc(&ws.fbm[2], nw, acc));
  ws.lb_count = 8;
  GBF_TRY(dmalloc(&ws.lb, nw * (size_t)ws.lb_count, acc));
  for (int i = 0; i < 2; i++) {
    GBF_TRY(dmalloc(&ws.fbm[i], nw, acc));
    GBF_TRY(dmalloc(&ws.q[i], n, acc));
    GBF_TRY(dmalloc(&ws.qoff[i], n, acc));
    GBF_TRY(dmalloc(&ws.qadj[i], n, acc));
    GBF_TRY(dmalloc(&ws.cs[i], cs, acc));
  }
  GBF_TRY(dmalloc(&ws.dist_tmp, n, acc));
  GBF_TRY(dmalloc(&ws.parent_tmp, n, acc));
  GBF_TRY(dmalloc(&ws.ctl, 1, acc));
  ws.trace_cap = 1 << 16;
  GBF_TRY(dmalloc(&ws.trace, (size_t)ws.trace_cap, acc));
  GBF_CUDA(cudaMallocHost((void **)&ws.ctl_host, sizeof(Ctl)));
  memset(ws.ctl_host, 0, sizeof(Ctl));
  ws.bytes += acc;
  return GBF_OK;
}

gbf_status ws_ensure_wbfs(Graph &g, Workspace &ws, int nB, int dl) {
  GBF_TRY(ws_ensure_base(g, ws));
  const size_t n = (size_t)g.n;
  size_t acc = 0;
  if (ws.nB != nB) {
    if (ws.slots) {
      cudaFree(ws.slots);
      cudaFree(ws.slot_cnt);
      ws.bytes -= sizeof(int32_t) * (size_t)ws.nB * n + sizeof(uint32_t) * (size_t)ws.nB;
      ws.slots = nullptr;
      ws.slot_cnt = nullptr;
      ws.nB = 0;
    }
    GBF_TRY(dmalloc(&ws.slots, (size_t)nB * n, acc));
    GBF_TRY(dmalloc(&ws.slot_cnt, (size_t)nB, acc));
    ws.nB = nB;
  }
  // The overflow bucket is only reachable when the window is narrower than
  // the largest bucket step of one relaxation; each live (vertex, value) pair
  // is filed at most once, bounded by the number of successful relaxations
  // (<= m in exact wBFS) plus n.  Δ-stepping can exceed it on adversarial
  // inputs; the kernel then reports GBF_ERR_OVERFLOW.
  const uint32_t jump = (((1u << dl) - 1u) + g.w_max) >> dl;
  const bool need_ovf = (uint32_t)nB <= jump;
  if (dl > 0 && !ws.side[0]) {
    GBF_TRY(dmalloc(&ws.side[0], n, acc));
    GBF_TRY(dmalloc(&ws.side[1], n, acc));
    GBF_TRY(dmalloc(&ws.xround, n, acc));
  }
  const uint64_t cap = need_ovf ? (uint64_t)g.m + n : 1;
  if (ws.ovf_cap < cap) {
    for (int i = 0; i < 2; i++)
      if (ws.ovf[i]) cudaFree(ws.ovf[i]);
    ws.bytes -= sizeof(int2) * 2 * ws.ovf_cap;
    ws.ovf[0] = ws.ovf[1] = nullptr;
    ws.ovf_cap = 0;
    GBF_TRY(dmalloc(&ws.ovf[0], cap, acc));
    GBF_TRY(dmalloc(&ws.ovf[1], cap, acc));
    ws.ovf_cap = cap;
  }
  ws.bytes += acc;
  return GBF_OK;
}

gbf_status ws_ensure_msbfs(Graph &g, Workspace &ws, bool host_out) {
  GBF_TRY(ws_ensure_base(g, ws));
  const size_t n = (size_t)g.n;
  const size_t cs = ((size_t)g.m + dev::kFine - 1) / dev::kFine + 2;
  size_t acc = 0;
  if (!ws.ms_seen) {
    GBF_TRY(dmalloc(&ws.ms_seen, n, acc));
    GBF_TRY(dmalloc(&ws.ms_visit, 2 * n, acc));
    GBF_TRY(dmalloc(&ws.ms_next, n, acc));
    GBF_TRY(dmalloc(&ws.ms_q[2], n, acc));
    GBF_TRY(dmalloc(&ws.ms_qoff[2], n, acc));
    GBF_TRY(dmalloc(&ws.ms_qadj[2], n, acc));
    GBF_TRY(dmalloc(&ws.ms_cs[2], cs, acc));
    GBF_TRY(dmalloc(&ws.ms_touched, n, acc));
    char *call = nullptr;
    GBF_TRY(dmalloc(&call, 1024, acc));
    ws.ms_call = call;
    for (int i = 0; i < 2; i++) {
      ws.ms_q[i] = ws.q[i];
      ws.ms_qoff[i] = ws.qoff[i];
      ws.ms_qadj[i] = ws.qadj[i];
      ws.ms_cs[i] = ws.cs[i];
    }
    GBF_CUDA(cudaMallocHost(&ws.ms_call_host, 1024));
    GBF_CUDA(cudaStreamCreateWithFlags(&ws.ms_stream, cudaStreamNonBlocking));
    GBF_CUDA(cudaEventCreateWithFlags(&ws.ms_ready, cudaEventDisableTiming));
    GBF_CUDA(cudaEventCreateWithFlags(&ws.ms_done, cudaEventDisableTiming));
  }
  if (host_out && !ws.ms_dist_tmp) GBF_TRY(dmalloc(&ws.ms_dist_tmp, 64 * n, acc));
  ws.bytes += acc;
  return GBF_OK;
}

gbf_status ws_ensure_bc(Graph &g, Workspace &ws) {
  GBF_TRY(ws_ensure_base(g, ws));
  if (ws.bc_paths) return GBF_OK;
  const size_t n = (size_t)g.n;
  size_t acc = 0;
  ws.bc_max_levels = 1 << 16;
  ws.bc_cs_total = (uint32_t)(((uint64_t)g.m + dev::kFine - 1) / dev::kFine + 2 * (uint64_t)ws.bc_max_levels + 2);
  GBF_TRY(dmalloc(&ws.bc_paths, n, acc));
  GBF_TRY(dmalloc(&ws.bc_lvl, n, acc));
  GBF_TRY(dmalloc(&ws.bc_cs, (size_t)ws.bc_cs_total, acc));
  uint4 *info = nullptr;
  GBF_TRY(dmalloc(&info, (size_t)ws.bc_max_levels, acc));
  ws.bc_info = info;
  GBF_TRY(dmalloc(&ws.bc_out_tmp, n, acc));
  ws.bytes += acc;
  return GBF_OK;
}

void ws_free(Workspace &ws) {
  void *ptrs[] = {ws.visited, ws.lb, ws.fbm[0], ws.fbm[1], ws.fbm[2], ws.q[0], ws.q[1], ws.qoff[0], ws.qoff[1],
                  ws.qadj[0], ws.qadj[1], ws.ms_qadj[2],
                  ws.cs[0], ws.cs[1], ws.ctl, ws.dist_tmp, ws.parent_tmp, ws.trace, ws.slots,
                  ws.slot_cnt, ws.ovf[0], ws.ovf[1], ws.ms_seen, ws.ms_visit, ws.ms_next,
                  ws.ms_q[2], ws.ms_qoff[2], ws.ms_cs[2], ws.ms_touched, ws.ms_call,
                  ws.ms_dist_tmp, ws.bc_paths, ws.bc_lvl, ws.bc_cs, ws.bc_info,
                  ws.bc_out_tmp, ws.side[0], ws.side[1], ws.xround, ws.mssp_dd, ws.mssp_imp,
                  ws.mssp_out_tmp, ws.dist_tmp2, ws.parent_tmp2, ws.hb_err};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (ws.ctl_host) cudaFreeHost(ws.ctl_host);
  if (ws.ms_call_host) cudaFreeHost(ws.ms_call_host);
  if (ws.ms_exec) cudaGraphExecDestroy(ws.ms_exec);
  if (ws.ms_ready) cudaEventDestroy(ws.ms_ready);
  if (ws.ms_done) cudaEventDestroy(ws.ms_done);
  if (ws.ms_stream) cudaStreamDestroy(ws.ms_stream);
  if (ws.hb_err_host) cudaFreeHost(ws.hb_err_host);
  for (int i = 0; i < 2; i++) {
    if (ws.hb_kern_done[i]) cudaEventDestroy(ws.hb_kern_done[i]);
    if (ws.hb_copy_done[i]) cudaEventDestroy(ws.hb_copy_done[i]);
  }
  if (ws.hb_stream) cudaStreamDestroy(ws.hb_stream);
  ws = Workspace();
}

gbf_status ws_collect(Workspace &ws, cudaStream_t st, gbf_stats *stats) {
  GBF_CUDA(cudaMemcpyAsync(ws.ctl_host, ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  GBF_CUDA(cudaStreamSynchronize(st));
  const Ctl &c = *ws.ctl_host;
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->rounds = c.rounds;
    stats->push_rounds = c.push_rounds;
    stats->pull_rounds = c.pull_rounds;
    stats->edges_scanned = (int64_t)c.edges_scanned;
    stats->vertices_expanded = (int64_t)c.expanded;
    stats->vertices_reached = (int64_t)c.reached;
    stats->relaxations = (int64_t)c.relax;
    stats->bucket_inserts = (int64_t)c.inserts;
    stats->refills = c.refills;
    stats->heavy_vertices = (int64_t)c.heavy;
    stats->vertices_pulled = (int64_t)c.pulled;
    stats->device_ns = c.t_end_ns;
    stats->grid_ctas = ws.last_grid;
    stats->block = ws.last_block;
    stats->device_error = c.err;
    stats->local_rounds = c.local_rounds;
  }
  if (c.err != 0) {
    char buf[128];
    snprintf(buf, sizeof(buf), "device reported status %d (site %d)", c.err, c.err_where);
    set_error(buf);
    return (gbf_status)c.err;
  }
  return GBF_OK;
}

}  // namespace gbf

using namespace gbf;

// ================================================================ C entry points
extern "C" {

gbf_status gbf_options_default(gbf_options *opt) {
  if (!opt) return GBF_ERR_INVALID;
  memset(opt, 0, sizeof(*opt));
  opt->block = 0;
  opt->pull_divisor = 20;
  opt->heavy_cutoff = 0;
  opt->bucket_window = 0;
  opt->dense_wbfs = 0;
  opt->spin_cap_us = 5000000;
  opt->ctas = 0;
  opt->pull_serial = 0;
  opt->inject_wait = 0;
  opt->pull_stay = 0;
  return GBF_OK;
}

size_t gbf_last_error(char *buf, size_t len) {
  const std::string &s = t_last_error;
  if (buf && len) {
    size_t k = std::min(len - 1, s.size());
    memcpy(buf, s.data(), k);
    buf[k] = 0;
  }
  return s.size();
}

const char *gbf_version(void) { return "0.1.0"; }

gbf_status gbf_graph_create(int32_t n, const uint32_t *off, const int32_t *tgt, const uint32_t *w,
                            int mem, uint32_t validate_flags, void *cuda_stream, gbf_graph **out) {
  if (!out) return set_error("out is NULL"), GBF_ERR_INVALID;
  *out = nullptr;
  if (n < 1 || !off) return set_error("n must be >= 1 and off non-NULL"), GBF_ERR_INVALID;
  if (mem != GBF_HOST && mem != GBF_DEVICE) return set_error("bad mem"), GBF_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  uint32_t m = 0, off0 = 0;
  if (mem == GBF_HOST) {
    m = off[n];
    off0 = off[0];
  } else {
    GBF_CUDA(cudaMemcpy(&m, off + n, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    GBF_CUDA(cudaMemcpy(&off0, off, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  }
  if (off0 != 0) return set_error("off[0] must be 0"), GBF_ERR_INVALID;
  if (m > 0 && !tgt) return set_error("tgt is NULL"), GBF_ERR_INVALID;
  gbf_graph *h = new (std::nothrow) gbf_graph();
  if (!h) return set_error("host allocation failed"), GBF_ERR_OOM;
  Graph &g = h->g;
  g.n = n;
  g.m = m;
  GBF_CUDA(cudaGetDevice(&g.device));
  GBF_CUDA(cudaDeviceGetAttribute(&g.num_sms, cudaDevAttrMultiProcessorCount, g.device));
  auto fail = [&](gbf_status s) {
    gbf_graph_destroy(h);
    return s;
  };
  size_t acc = 0;
  gbf_status s;
  if ((s = dmalloc(&g.off, (size_t)n + 1, acc)) != GBF_OK) return fail(s);
  if ((s = dmalloc(&g.tgt, (size_t)m, acc)) != GBF_OK) return fail(s);
  if (w && (s = dmalloc(&g.w, (size_t)m, acc)) != GBF_OK) return fail(s);
  if ((s = dmalloc(&g.leaf, ((size_t)n + 31) / 32, acc)) != GBF_OK) return fail(s);
  if ((s = dmalloc(&g.iso, ((size_t)n + 31) / 32, acc)) != GBF_OK) return fail(s);
  if ((s = dmalloc(&g.f1, (size_t)n, acc)) != GBF_OK) return fail(s);
  g.bytes = acc;
  const cudaMemcpyKind kind = mem == GBF_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(g.off, off, sizeof(uint32_t) * ((size_t)n + 1), kind, st)) != cudaSuccess)
    return fail(cuda_fail(e, "upload off"));
  if (m && (e = cudaMemcpyAsync(g.tgt, tgt, sizeof(int32_t) * (size_t)m, kind, st)) != cudaSuccess)
    return fail(cuda_fail(e, "upload tgt"));
  if (w && m && (e = cudaMemcpyAsync(g.w, w, sizeof(uint32_t) * (size_t)m, kind, st)) != cudaSuccess)
    return fail(cuda_fail(e, "upload w"));
  // digest + validation flags in one small device buffer
  struct Aux {
    unsigned long long sum;
    unsigned wmax;
    unsigned flags;
  };
  Aux *aux = nullptr, haux;
  if ((e = cudaMalloc((void **)&aux, sizeof(Aux))) != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc"));
  cudaMemsetAsync(aux, 0, sizeof(Aux), st);
  const int grid = g.num_sms * 8;
  if (validate_flags & GBF_VALIDATE_SYMMETRIC) validate_flags |= GBF_VALIDATE_BASIC;
  if (validate_flags & GBF_VALIDATE_BASIC)
    k_validate_basic<<<grid, 256, 0, st>>>(n, m, g.off, g.tgt, g.w, &aux->flags);
  e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) {
    e = cudaMemcpy(&haux, aux, sizeof(Aux), cudaMemcpyDeviceToHost);
  }
  if (e != cudaSuccess) {
    cudaFree(aux);
    return fail(cuda_fail(e, "validate"));
  }
  if (haux.flags == 0 && (validate_flags & GBF_VALIDATE_SYMMETRIC)) {
    k_validate_symmetric<<<grid, 256, 0, st>>>(n, g.off, g.tgt, g.w, &aux->flags);
  }
  if (haux.flags == 0) {
    k_digest<<<grid, 256, 0, st>>>(n, m, g.off, g.tgt, g.w, &aux->sum, &aux->wmax);
    k_hub_first<<<grid, 256, 0, st>>>(n, g.off, g.tgt, g.w);
    k_leaf<<<grid, 256, 0, st>>>(n, g.off, g.tgt, g.leaf, g.iso, g.f1);
  }
  e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpy(&haux, aux, sizeof(Aux), cudaMemcpyDeviceToHost);
  cudaFree(aux);
  if (e != cudaSuccess) return fail(cuda_fail(e, "digest"));
  if (haux.flags) {
    std::string msg = "invalid graph:";
    if (haux.flags & kBadOffsets) msg += " offsets";
    if (haux.flags & kBadTarget) msg += " target-range";
    if (haux.flags & kSelfLoop) msg += " self-loop";
    if (haux.flags & kBadWeight) msg += " zero-weight";
    if (haux.flags & kUnsorted) msg += " unsorted-or-duplicate";
    if (haux.flags & kAsymmetric) msg += " asymmetric";
    if (haux.flags & kWeightAsym) msg += " weight-asymmetric";
    set_error(msg);
    return fail(GBF_ERR_INVALID);
  }
  g.w_max = haux.wmax;
  g.fingerprint = haux.sum ^ ((unsigned long long)n << 32) ^ m;
  if (w && (uint64_t)(n - 1) * (uint64_t)g.w_max >= 0x7fffffffULL) {
    set_error("(n-1) * max weight does not fit int32 distances");
    return fail(GBF_ERR_OVERFLOW);
  }
  *out = h;
  return GBF_OK;
}

gbf_status gbf_graph_destroy(gbf_graph *h) {
  if (!h) return GBF_OK;
  Graph &g = h->g;
  ws_free(g.ws);
  if (g.off) cudaFree(g.off);
  if (g.tgt) cudaFree(g.tgt);
  if (g.w) cudaFree(g.w);
  if (g.leaf) cudaFree(g.leaf);
  if (g.iso) cudaFree(g.iso);
  if (g.f1) cudaFree(g.f1);
  delete h;
  return GBF_OK;
}

gbf_status gbf_graph_info(const gbf_graph *h, int32_t *n, uint64_t *m, uint32_t *w_max,
                          uint64_t *fingerprint) {
  if (!h) return set_error("graph is NULL"), GBF_ERR_INVALID;
  if (n) *n = h->g.n;
  if (m) *m = h->g.m;
  if (w_max) *w_max = h->g.w_max;
  if (fingerprint) *fingerprint = h->g.fingerprint;
  return GBF_OK;
}

gbf_status gbf_graph_device_bytes(const gbf_graph *h, size_t *bytes) {
  if (!h || !bytes) return set_error("NULL argument"), GBF_ERR_INVALID;
  *bytes = h->g.bytes + h->g.ws.bytes;
  return GBF_OK;
}

gbf_status gbf_bfs(gbf_graph *h, int32_t src, int32_t *dist, int32_t *parent, int mem,
                   const gbf_options *opt, void *cuda_stream) {
  if (!h || !dist) return set_error("graph or dist is NULL"), GBF_ERR_INVALID;
  Graph &g = h->g;
  if (src < 0 || src >= g.n) return set_error("src out of range"), GBF_ERR_INVALID;
  if (mem != GBF_HOST && mem != GBF_DEVICE) return set_error("bad mem"), GBF_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  std::lock_guard<std::mutex> lk(g.mu);
  GBF_TRY(ws_ensure_base(g, g.ws));
  const Opts o = resolve(opt, g, GBF_TUNE_BFS);
  int32_t *dd = mem == GBF_HOST ? g.ws.dist_tmp : dist;
  int32_t *pp = parent ? (mem == GBF_HOST ? g.ws.parent_tmp : parent) : nullptr;
  GBF_TRY(launch_bfs(g, g.ws, src, dd, pp, o, st));
  if (mem == GBF_DEVICE) return GBF_OK;
  GBF_CUDA(cudaMemcpyAsync(dist, dd, sizeof(int32_t) * (size_t)g.n, cudaMemcpyDeviceToHost, st));
  if (parent)
    GBF_CUDA(cudaMemcpyAsync(parent, pp, sizeof(int32_t) * (size_t)g.n, cudaMemcpyDeviceToHost, st));
  return ws_collect(g.ws, st, nullptr);
}

gbf_status gbf_bfs_host_batch(gbf_graph *h, const int32_t *srcs, int32_t k, int32_t *dist,
                              int32_t *parent, const gbf_options *opt, void *cuda_stream) {
  if (!h || !srcs || !dist) return set_error("graph, srcs or dist is NULL"), GBF_ERR_INVALID;
  Graph &g = h->g;
  if (k < 1) return set_error("k must be at least 1"), GBF_ERR_INVALID;
  for (int32_t i = 0; i < k; i++)
    if (srcs[i] < 0 || srcs[i] >= g.n) return set_error("source out of range"), GBF_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  std::lock_guard<std::mutex> lk(g.mu);
  GBF_TRY(ws_ensure_base(g, g.ws));
  Workspace &ws = g.ws;
  const size_t n = (size_t)g.n;
  if (!ws.dist_tmp2) {
    size_t acc = 0;
    GBF_TRY(dmalloc(&ws.dist_tmp2, n, acc));
    GBF_TRY(dmalloc(&ws.parent_tmp2, n, acc));
    GBF_TRY(dmalloc(&ws.hb_err, 1, acc));
    GBF_CUDA(cudaMallocHost((void **)&ws.hb_err_host, sizeof(int)));
    GBF_CUDA(cudaStreamCreateWithFlags(&ws.hb_stream, cudaStreamNonBlocking));
    for (int i = 0; i < 2; i++) {
      GBF_CUDA(cudaEventCreateWithFlags(&ws.hb_kern_done[i], cudaEventDisableTiming));
      GBF_CUDA(cudaEventCreateWithFlags(&ws.hb_copy_done[i], cudaEventDisableTiming));
    }
    ws.bytes += acc;
  }
  const Opts o = resolve(opt, g, GBF_TUNE_BFS);
  int32_t *dbuf[2] = {ws.dist_tmp, ws.dist_tmp2}, *pbuf[2] = {ws.parent_tmp, ws.parent_tmp2};
  // enqueue every query; on a failure, wait for the copies already issued,
  // so that none writes into the caller's buffers after this call returns
  auto enqueue = [&]() -> gbf_status {
    GBF_CUDA(cudaMemsetAsync(ws.hb_err, 0, sizeof(int), st));
    for (int b = 0; b < 2; b++) GBF_CUDA(cudaEventRecord(ws.hb_copy_done[b], st));
    for (int32_t i = 0; i < k; i++) {
      const int b = i & 1;
      // result buffer b is free once the read-back of query i - 2 is done
      GBF_CUDA(cudaStreamWaitEvent(st, ws.hb_copy_done[b], 0));
      GBF_TRY(launch_bfs(g, ws, srcs[i], dbuf[b], parent ? pbuf[b] : nullptr, o, st));
      // the query's device status, kept past the next launch's reset of the control block
      k_keep_error<<<1, 1, 0, st>>>(ws.hb_err, &ws.ctl->err);
      GBF_CUDA(cudaGetLastError());
      GBF_CUDA(cudaEventRecord(ws.hb_kern_done[b], st));
      // read-back on the second stream, while the next query computes
      GBF_CUDA(cudaStreamWaitEvent(ws.hb_stream, ws.hb_kern_done[b], 0));
      GBF_CUDA(cudaMemcpyAsync(dist + (size_t)i * n, dbuf[b], sizeof(int32_t) * n,
                               cudaMemcpyDeviceToHost, ws.hb_stream));
      if (parent)
        GBF_CUDA(cudaMemcpyAsync(parent + (size_t)i * n, pbuf[b], sizeof(int32_t) * n,
                                 cudaMemcpyDeviceToHost, ws.hb_stream));
      GBF_CUDA(cudaEventRecord(ws.hb_copy_done[b], ws.hb_stream));
    }
    return GBF_OK;
  };
  const gbf_status es = enqueue();
  if (es != GBF_OK) {
    cudaStreamSynchronize(ws.hb_stream);
    cudaStreamSynchronize(st);
    return es;
  }
  for (int b = 0; b < 2; b++) GBF_CUDA(cudaStreamWaitEvent(st, ws.hb_copy_done[b], 0));
  GBF_CUDA(cudaMemcpyAsync(ws.hb_err_host, ws.hb_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  const gbf_status s = ws_collect(ws, st, nullptr);  // synchronises st
  if (s != GBF_OK) return s;
  if (*ws.hb_err_host != 0) {
    set_error("a query of the batch reported a device error");
    return (gbf_status)*ws.hb_err_host;
  }
  return GBF_OK;
}

gbf_status gbf_wbfs(gbf_graph *h, int32_t src, int32_t *dist, int mem, const gbf_options *opt,
                    void *cuda_stream) {
  if (!h || !dist) return set_error("graph or dist is NULL"), GBF_ERR_INVALID;
  Graph &g = h->g;
  if (!g.w) return set_error("graph has no weights"), GBF_ERR_INVALID;
  if (src < 0 || src >= g.n) return set_error("src out of range"), GBF_ERR_INVALID;
  if (mem != GBF_HOST && mem != GBF_DEVICE) return set_error("bad mem"), GBF_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  std::lock_guard<std::mutex> lk(g.mu);
  const Opts o = resolve(opt, g, GBF_TUNE_WBFS);
  int nB = o.bucket_window > 0 ? o.bucket_window : (int)std::max<uint32_t>(g.w_max + 1, 2);
  nB = std::min(nB, 256);
  GBF_TRY(ws_ensure_wbfs(g, g.ws, nB));
  int32_t *dd = mem == GBF_HOST ? g.ws.dist_tmp : dist;
  GBF_TRY(launch_wbfs(g, g.ws, src, dd, o, st));
  if (mem == GBF_DEVICE) return GBF_OK;
  GBF_CUDA(cudaMemcpyAsync(dist, dd, sizeof(int32_t) * (size_t)g.n, cudaMemcpyDeviceToHost, st));
  return ws_collect(g.ws, st, nullptr);
}

gbf_status gbf_delta_stepping(gbf_graph *h, int32_t src, int32_t delta, int32_t *dist, int mem,
                              const gbf_options *opt, void *cuda_stream) {
  if (!h || !dist) return set_error("graph or dist is NULL"), GBF_ERR_INVALID;
  Graph &g = h->g;
  if (!g.w) return set_error("graph has no weights"), GBF_ERR_INVALID;
  if (src < 0 || src >= g.n) return set_error("src out of range"), GBF_ERR_INVALID;
  if (mem != GBF_HOST && mem != GBF_DEVICE) return set_error("bad mem"), GBF_ERR_INVALID;
  int dl = 0;
  while (dl <= 20 && (1 << dl) < delta) dl++;
  if (delta < 1 || dl > 20 || (1 << dl) != delta)
    return set_error("delta must be a power of two in [1, 2^20]"), GBF_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  std::lock_guard<std::mutex> lk(g.mu);
  const Opts o = resolve(opt, g, GBF_TUNE_WBFS);
  // a window one wider than the largest bucket step slides without overflow
  const uint32_t jump = (((1u << dl) - 1u) + g.w_max) >> dl;
  int nB = o.bucket_window > 0 ? o.bucket_window : (int)std::max<uint32_t>(jump + 1, 2);
  nB = std::min(nB, 256);
  GBF_TRY(ws_ensure_wbfs(g, g.ws, nB, dl));
  int32_t *dd = mem == GBF_HOST ? g.ws.dist_tmp : dist;
  GBF_TRY(launch_wbfs(g, g.ws, src, dd, o, st, dl));
  if (mem == GBF_DEVICE) return GBF_OK;
  GBF_CUDA(cudaMemcpyAsync(dist, dd, sizeof(int32_t) * (size_t)g.n, cudaMemcpyDeviceToHost, st));
  return ws_collect(g.ws, st, nullptr);
}

gbf_status gbf_trace(gbf_graph *h, gbf_round_trace *out, int32_t cap, int32_t *count) {
  if (!h || !count || (cap > 0 && !out)) return set_error("NULL argument"), GBF_ERR_INVALID;
  Workspace &ws = h->g.ws;
  *count = 0;
  if (!ws.trace) return GBF_OK;
  const int rounds = std::min(ws.ctl_host ? ws.ctl_host->rounds : 0, ws.trace_cap);
  const int k = std::min(rounds, std::max(cap, 0));
  if (k > 0) {
    static_assert(sizeof(TraceRec) == sizeof(gbf_round_trace), "trace record layout");
    GBF_CUDA(cudaMemcpy(out, ws.trace, sizeof(TraceRec) * (size_t)k, cudaMemcpyDeviceToHost));
  }
  *count = k;
  return GBF_OK;
}

gbf_status gbf_msbfs(gbf_graph *h, const int32_t *srcs, int32_t k, int32_t *dist, int mem,
                     const gbf_options *opt, void *cuda_stream) {
  if (!h || !srcs || !dist) return set_error("graph, srcs or dist is NULL"), GBF_ERR_INVALID;
  Graph &g = h->g;
  if (k < 1 || k > 64) return set_error("k must be in [1, 64]"), GBF_ERR_INVALID;
  for (int i = 0; i < k; i++)
    if (srcs[i] < 0 || srcs[i] >= g.n) return set_error("source out of range"), GBF_ERR_INVALID;
  if (mem != GBF_HOST && mem != GBF_DEVICE) return set_error("bad mem"), GBF_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  std::lock_guard<std::mutex> lk(g.mu);
  GBF_TRY(ws_ensure_msbfs(g, g.ws, mem == GBF_HOST));
  const Opts o = resolve(opt, g, GBF_TUNE_MSBFS);
  int32_t *dd = mem == GBF_HOST ? g.ws.ms_dist_tmp : dist;
  GBF_TRY(launch_msbfs(g, g.ws, srcs, k, dd, o, st));
  if (mem == GBF_DEVICE) return GBF_OK;
  GBF_CUDA(cudaMemcpyAsync(dist, dd, sizeof(int32_t) * (size_t)k * (size_t)g.n,
                           cudaMemcpyDeviceToHost, st));
  return ws_collect(g.ws, st, nullptr);
}

gbf_status gbf_wait(gbf_graph *h, void *cuda_stream, gbf_stats *stats) {
  if (!h) return set_error("graph is NULL"), GBF_ERR_INVALID;
  Graph &g = h->g;
  if (!g.ws.ctl) {
    if (stats) memset(stats, 0, sizeof(*stats));
    return GBF_OK;
  }
  return ws_collect(g.ws, (cudaStream_t)cuda_stream, stats);
}

}  // extern "C"
