// Autotuner: picks the persistent kernels' block size, push/pull divisor and
// heavy cutoff for one resident graph by timing real queries (median of
// repeats over a few seeded sources), by coordinate descent over the knob
// grid.  Results are cached per (graph fingerprint, device, query kind) in
// the process and, if GBF_TUNE_CACHE names a file, across processes.
// Distances never depend on the knobs; only time does.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "gbf_impl.h"

namespace gbf {
namespace {

std::mutex g_tune_mu;
std::map<std::tuple<uint64_t, std::string, int>, gbf_options> g_tune_cache;

std::string device_key(int dev) {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
  char buf[64];
  std::string s = p.name;
  for (int i = 0; i < 16; i++) {
    snprintf(buf, sizeof(buf), "%02x", (unsigned char)p.uuid.bytes[i]);
    s += (i == 0 ? ":" : "") + std::string(buf);
  }
  for (char &c : s)
    if (c == ' ') c = '_';
  return s;
}

bool file_lookup(uint64_t fp, const std::string &dev, int kind, gbf_options *out) {
  const char *path = getenv("GBF_TUNE_CACHE");
  if (!path || !*path) return false;
  FILE *f = fopen(path, "r");
  if (!f) return false;
  char dbuf[256];
  unsigned long long ffp;
  int fk, b, d, h;
  bool found = false;
  while (fscanf(f, "%llx %255s %d %d %d %d", &ffp, dbuf, &fk, &b, &d, &h) == 6) {
    if (ffp == fp && dev == dbuf && fk == kind) {
      gbf_options_default(out);
      out->block = b;
      out->pull_divisor = d;
      out->heavy_cutoff = h;
      found = true;
    }
  }
  fclose(f);
  return found;
}

void file_store(uint64_t fp, const std::string &dev, int kind, const gbf_options &o) {
  const char *path = getenv("GBF_TUNE_CACHE");
  if (!path || !*path) return;
  FILE *f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%llx %s %d %d %d %d\n", (unsigned long long)fp, dev.c_str(), kind, o.block,
          o.pull_divisor, o.heavy_cutoff);
  fclose(f);
}

uint64_t mix(uint64_t x) {
  x += 0x9e3779b97f4a7c15ULL;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
  return x ^ (x >> 31);
}

}  // namespace
}  // namespace gbf

using namespace gbf;

extern "C" gbf_status gbf_autotune(gbf_graph *h, int32_t kind, gbf_options *out) {
  if (!h || !out) return set_error("graph or out is NULL"), GBF_ERR_INVALID;
  if (kind < GBF_TUNE_BFS || kind > GBF_TUNE_WBFS) return set_error("bad kind"), GBF_ERR_INVALID;
  Graph &g = h->g;
  if (kind == GBF_TUNE_WBFS && !g.w) return set_error("graph has no weights"), GBF_ERR_INVALID;
  const std::string dev = device_key(g.device);
  const auto key = std::make_tuple(g.fingerprint, dev, (int)kind);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      *out = it->second;
      return GBF_OK;
    }
    gbf_options o;
    if (file_lookup(g.fingerprint, dev, kind, &o)) {
      g_tune_cache[key] = o;
      *out = o;
      return GBF_OK;
    }
  }
  // seeded sources with at least one edge (read degrees from the device CSR)
  std::vector<int32_t> srcs;
  {
    uint64_t x = g.fingerprint ^ 0x7475ULL;
    for (int tries = 0; tries < 4096 && srcs.size() < 64; tries++) {
      x = mix(x);
      const int32_t v = (int32_t)(x % (uint64_t)g.n);
      uint32_t o2[2];
      GBF_CUDA(cudaMemcpy(o2, g.off + v, sizeof(o2), cudaMemcpyDeviceToHost));
      if (o2[1] > o2[0]) srcs.push_back(v);
    }
    if (srcs.empty()) srcs.push_back(0);
    while (srcs.size() < 64) srcs.push_back(srcs[srcs.size() % srcs.size()]);
  }
  std::lock_guard<std::mutex> lk(g.mu);
  Workspace &ws = g.ws;
  gbf_status s = GBF_OK;
  if (kind == GBF_TUNE_MSBFS) s = ws_ensure_msbfs(g, ws, true);
  else if (kind == GBF_TUNE_WBFS) {
    const int nB = (int)std::min<uint32_t>(std::max<uint32_t>(g.w_max + 1, 2), 256);
    s = ws_ensure_wbfs(g, ws, nB);
  } else s = ws_ensure_base(g, ws);
  if (s != GBF_OK) return s;
  cudaStream_t st;
  GBF_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int nsrc = kind == GBF_TUNE_MSBFS ? 1 : 3;
  const int reps = kind == GBF_TUNE_MSBFS ? 3 : 5;

  // median time of one configuration (ms); +inf if it fails
  auto measure = [&](const gbf_options &opt, float *ms_out) -> gbf_status {
    const Opts o = resolve(&opt, g, kind);
    std::vector<float> t;
    for (int si = 0; si < nsrc; si++) {
      for (int r = 0; r < reps + 1; r++) {
        cudaEventRecord(e0, st);
        gbf_status ls;
        if (kind == GBF_TUNE_BFS)
          ls = launch_bfs(g, ws, srcs[si], ws.dist_tmp, ws.parent_tmp, o, st);
        else if (kind == GBF_TUNE_WBFS)
          ls = launch_wbfs(g, ws, srcs[si], ws.dist_tmp, o, st);
        else
          ls = launch_msbfs(g, ws, srcs.data(), 64, ws.ms_dist_tmp, o, st);
        if (ls != GBF_OK) return ls;
        cudaEventRecord(e1, st);
        GBF_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0) t.push_back(ms);  // first run warms up
      }
      gbf_stats sts;
      gbf_status cs = ws_collect(ws, st, &sts);
      if (cs != GBF_OK) return cs;
    }
    std::sort(t.begin(), t.end());
    *ms_out = t[t.size() / 2];
    return GBF_OK;
  };

  gbf_options best;
  gbf_options_default(&best);
  {
    const Opts d0 = resolve(&best, g, kind);  // the kind's defaults, made explicit
    best.heavy_cutoff = d0.heavy_cutoff;
    best.block = d0.block;
  }
  float best_ms = 0;
  s = measure(best, &best_ms);
  if (s == GBF_OK) {
    const int blocks[] = {128, 256, 512, 1024};
    const int divisors[] = {10, 14, 20, 28, 40};
    const int heavies[] = {256, 512, 1024, 2048, 4096, 8192, 16384};
    for (int pass = 0; pass < 2 && s == GBF_OK; pass++) {
      for (int dim = 0; dim < 3 && s == GBF_OK; dim++) {
        const int *vals = dim == 0 ? blocks : dim == 1 ? divisors : heavies;
        const int nv = dim == 0 ? 4 : dim == 1 ? 5 : 7;
        for (int i = 0; i < nv; i++) {
          gbf_options c = best;
          if (dim == 0) c.block = vals[i];
          else if (dim == 1) c.pull_divisor = vals[i];
          else c.heavy_cutoff = vals[i];
          if (c.block == best.block && c.pull_divisor == best.pull_divisor &&
              c.heavy_cutoff == best.heavy_cutoff)
            continue;
          float ms = 0;
          s = measure(c, &ms);
          if (s == GBF_ERR_INVALID) {  // does not fit this device (shared memory): skip it
            s = GBF_OK;
            continue;
          }
          if (s != GBF_OK) break;
          if (ms < best_ms * 0.97f) {
            best = c;
            best_ms = ms;
          }
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  if (s != GBF_OK) return s;
  {
    std::lock_guard<std::mutex> lk2(g_tune_mu);
    g_tune_cache[key] = best;
  }
  file_store(g.fingerprint, dev, kind, best);
  *out = best;
  return GBF_OK;
}
