// gbf_bfs_noalloc: BFS for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: their device memory is owned by
// another allocator that has already reserved it (a framework's caching
// allocator, a fixed-budget deployment), or they run in a latency-critical
// loop where cudaMalloc/cudaFree, which may synchronise the whole device, are
// not acceptable.  This entry point runs the same persistent BFS kernel as
// gbf_bfs, but its scratch (visited and frontier bitmaps, frontier queues
// with their degree prefixes and chunk-start tables, the control block) lives
// in one file-scope device array of fixed size that the CUDA module holds from
// load until process exit, on every GPU that loads the library.  The call
// itself allocates nothing.
#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "gbf_impl.h"

namespace gbf {
namespace {

constexpr int32_t kMaxN = 1 << 20;          // vertices
constexpr uint64_t kMaxM = 1ull << 25;      // arcs
constexpr size_t words256(size_t words) { return (words + 63) & ~size_t(63); }  // 256-byte regions
constexpr size_t kBitW = words256((size_t)kMaxN / 32);
constexpr size_t kQW = words256((size_t)kMaxN);
constexpr size_t kCsW = words256((size_t)(kMaxM / dev::kFine) + 2);
constexpr size_t kCtlW = words256((sizeof(Ctl) + 3) / 4);
constexpr size_t kFlagW = 64;  // the CSR check's flag word
constexpr size_t kScratchWords = 4 * kBitW + 6 * kQW + 2 * kCsW + kCtlW + kFlagW;  // ~26.7 MB

static __device__ __align__(256) uint32_t g_scratch[kScratchWords];

// The caller's CSR, checked before the search so that a malformed graph is
// rejected instead of sending the BFS out of bounds: off[0] = 0, off[n] = m,
// offsets non-decreasing, targets in [0, n).  Every read stays inside off[0..n]
// and tgt[0..m), whatever the offsets hold.
__global__ void k_noalloc_check(int32_t n, uint32_t m, const uint32_t *off, const int32_t *tgt,
                                uint32_t *flag) {
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t tw = (gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  uint32_t bad = 0;
  if (gw == 0 && lane == 0 && (off[0] != 0u || off[n] != m)) bad = 1;
  for (uint32_t v = gw; v < (uint32_t)n; v += tw) {
    const uint32_t s = off[v], e = off[v + 1];
    if (e < s || e > m) {
      bad = 1;
      continue;
    }
    for (uint32_t k = s + lane; k < e; k += 32) {
      const int32_t t = tgt[k];
      if (t < 0 || t >= n) bad = 1;
    }
  }
  if (bad) atomicOr(flag, 1u);
}

// Device address of g_scratch on the current device.  In host code the
// symbol's name is only a host-side stand-in, so the address is looked up
// with the device current, on every call: a context that was reset and
// created again may hold the array elsewhere.
gbf_status scratch_on_device(uint32_t **out) {
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_scratch)");
  *out = (uint32_t *)p;
  return GBF_OK;
}

}  // namespace
}  // namespace gbf

using namespace gbf;

extern "C" gbf_status gbf_bfs_noalloc(int32_t n, uint32_t m, const uint32_t *off, const int32_t *tgt,
                                      int32_t src, int32_t *dist, int32_t *parent,
                                      const gbf_options *opt, void *cuda_stream) {
  if (n < 1 || n > kMaxN) {
    set_error("gbf_bfs_noalloc: n must be in [1, 1048576]");
    return GBF_ERR_INVALID;
  }
  if ((uint64_t)m > kMaxM) {
    set_error("gbf_bfs_noalloc: m must be at most 33554432 arcs");
    return GBF_ERR_INVALID;
  }
  if (!off || (m > 0 && !tgt) || !dist) {
    set_error("gbf_bfs_noalloc: off, tgt and dist must be device pointers");
    return GBF_ERR_INVALID;
  }
  if (src < 0 || src >= n) {
    set_error("gbf_bfs_noalloc: src out of range");
    return GBF_ERR_INVALID;
  }
  int dev = 0;
  GBF_CUDA(cudaGetDevice(&dev));
  uint32_t *base = nullptr;
  gbf_status s = scratch_on_device(&base);
  if (s != GBF_OK) return s;
  cudaStream_t st = (cudaStream_t)cuda_stream;

  Graph g;
  g.n = n;
  g.m = m;
  g.off = const_cast<uint32_t *>(off);
  g.tgt = const_cast<int32_t *>(tgt);
  g.w = nullptr;
  g.device = dev;
  GBF_CUDA(cudaDeviceGetAttribute(&g.num_sms, cudaDevAttrMultiProcessorCount, dev));

  // Carve the workspace out of the static array; every region starts on a
  // 256-byte boundary.  Everything the kernel reads before writing is reset
  // by the launch (control block memset, bitmaps initialised in-kernel).
  Workspace ws;
  uint32_t *p = base;
  ws.visited = p;
  p += kBitW;
  ws.fbm[0] = p;
  p += kBitW;
  ws.fbm[1] = p;
  p += kBitW;
  ws.fbm[2] = p;
  p += kBitW;
  ws.q[0] = (int32_t *)p;
  p += kQW;
  ws.q[1] = (int32_t *)p;
  p += kQW;
  ws.qoff[0] = p;
  p += kQW;
  ws.qoff[1] = p;
  p += kQW;
  ws.qadj[0] = p;
  p += kQW;
  ws.qadj[1] = p;
  p += kQW;
  ws.cs[0] = p;
  p += kCsW;
  ws.cs[1] = p;
  p += kCsW;
  ws.ctl = (Ctl *)p;
  p += kCtlW;
  uint32_t *flag = p;
  ws.n = n;
  ws.m = m;

  // the CSR check (its flag word starts at zero on every call)
  uint32_t bad = 0;
  GBF_CUDA(cudaMemsetAsync(flag, 0, sizeof(uint32_t), st));
  k_noalloc_check<<<g.num_sms * 4, 256, 0, st>>>(n, m, off, tgt, flag);
  GBF_CUDA(cudaGetLastError());
  GBF_CUDA(cudaMemcpyAsync(&bad, flag, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  GBF_CUDA(cudaStreamSynchronize(st));
  if (bad) {
    set_error("gbf_bfs_noalloc: invalid CSR (off[0] != 0, off[n] != m, decreasing offsets or a "
              "target outside [0, n))");
    return GBF_ERR_INVALID;
  }

  const Opts o = resolve(opt, g, GBF_TUNE_BFS);
  s = launch_bfs(g, ws, src, dist, parent, o, st);
  if (s != GBF_OK) return s;
  int err = 0;
  GBF_CUDA(cudaMemcpyAsync(&err, &ws.ctl->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  GBF_CUDA(cudaStreamSynchronize(st));
  if (err != 0) {
    set_error("gbf_bfs_noalloc: device reported an error");
    return (gbf_status)err;
  }
  return GBF_OK;
}
