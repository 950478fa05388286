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

#include <mutex>

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
constexpr size_t kScratchWords = 4 * kBitW + 6 * kQW + 2 * kCsW + kCtlW;  // ~26.7 MB

static __device__ __align__(256) uint32_t g_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint32_t *g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device.  In host code the
// symbol's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
gbf_status scratch_on_device(int dev, uint32_t **out) {
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal out of range");
    return GBF_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_scratch)");
    g_scratch_addr[dev] = (uint32_t *)p;
  }
  *out = g_scratch_addr[dev];
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
  gbf_status s = scratch_on_device(dev, &base);
  if (s != GBF_OK) return s;

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
  ws.n = n;
  ws.m = m;

  const Opts o = resolve(opt, g, GBF_TUNE_BFS);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  s = launch_bfs(g, ws, src, dist, parent, o, st);
  if (s != GBF_OK) return s;
  GBF_CUDA(cudaStreamSynchronize(st));
  int err = 0;
  GBF_CUDA(cudaMemcpy(&err, &ws.ctl->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err != 0) {
    set_error("gbf_bfs_noalloc: device reported an error");
    return (gbf_status)err;
  }
  return GBF_OK;
}
