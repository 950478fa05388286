// Continuous-batching query server over several resident graphs.
//
// Requests (BFS or weighted BFS from one source on one graph) are admitted
// while a result slot of device memory is free (the slots are carved once
// from an HBM budget) and the pending queue has room; otherwise submit
// returns GBF_ERR_BUSY.  A dispatcher thread keeps a set of engines busy,
// each with its own CUDA stream and workspace:
//   - BFS engines take the pending BFS requests of one graph (the graph whose
//     oldest request is oldest): up to max_batch of them as one multi-source
//     BFS launch (8-bit lanes for 2..8 requests, 64-bit lanes above) whose
//     lane i writes straight into request i's result slot, or a few as
//     single-source launches back to back;
//   - wBFS engines likewise: up to 8 weighted requests of one graph as one
//     multi-source SSSP launch (distance lanes advanced by shared
//     Bellman-Ford rounds), or single weighted BFS launches.
// Whether to batch is decided per graph and kind from the GPU time each way
// has taken per query so far (CUDA events around every launch, weighted to
// the recent ones; a batch size class not yet measured is tried), so a
// batch runs only where it is cheaper per query: on the large graphs a few
// weighted queries cost more together than apart, on the small ones far
// less.  Batches smaller than min_batch never run, and max_batch = 1 gives
// one query per launch.
// Engines run concurrently; each persistent launch gets a share of the GPU's
// resident CTAs (equal shares, or wbfs_share percent for the weighted
// engines together), and the shares add up to what fits at once, so all
// engines' CTAs can be co-resident.
// Results stay in their device slots until polled (copied to the caller or
// dropped), which frees the slot.  Latency is measured from submit to the
// dispatcher observing the launch's completion event.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gbf_impl.h"

namespace gbf {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket;
  int graph;
  int kind;
  int32_t src;
  int slot;
  Clock::time_point t_submit;
  Clock::time_point t_done;
  int state;  // 0 pending, 1 running, 2 done, 3 failed
  gbf_status status;
};

struct Engine {
  int kind;  // GBF_QUERY_BFS or GBF_QUERY_WBFS
  Graph shape;  // sizing descriptor (max n, m, w) for the workspace
  Workspace ws;
  cudaStream_t st = nullptr;
  cudaEvent_t start = nullptr, done = nullptr;
  bool busy = false;
  int graph = -1;
  int cls = 0;       // cost class of the running work (see CostModel)
  int launches = 1;  // launches it took
  std::vector<uint64_t> batch;
};

// Measured GPU time per launch (ms, exponentially weighted) of each way a
// graph's queries of one kind can run: class 0 one query per launch, class
// j >= 1 one multi-source launch of 2^(j-1) < k <= 2^j queries.
constexpr int kCostClasses = 7;
struct CostModel {
  double ms[kCostClasses] = {0, 0, 0, 0, 0, 0, 0};
  int seen[kCostClasses] = {0, 0, 0, 0, 0, 0, 0};
  void add(int c, double v) {
    ms[c] = seen[c] ? 0.7 * ms[c] + 0.3 * v : v;
    seen[c]++;
  }
};
inline int cost_class(int k) {
  int j = 0;
  while ((1 << j) < k) j++;
  return k <= 1 ? 0 : j;
}

}  // namespace
}  // namespace gbf

struct gbf_server {
  std::vector<gbf::Graph *> graphs;
  gbf_server_options opt;
  gbf::Opts kopt_bfs, kopt_single, kopt_wbfs, kopt_mssp;
  int32_t max_n = 0;
  char *slot_mem = nullptr;
  size_t slot_bytes = 0;
  std::vector<int> free_slots;
  std::vector<gbf::Engine *> engines;
  std::mutex mu;
  std::condition_variable cv;
  std::unordered_map<uint64_t, gbf::Request> reqs;
  std::vector<std::deque<uint64_t>> bfs_q;  // per graph
  std::vector<std::deque<uint64_t>> wbfs_q;  // per graph
  std::vector<gbf::CostModel> cost[2];        // per kind, per graph
  uint64_t next_ticket = 1;
  size_t pending = 0;
  std::thread worker;
  std::atomic<bool> stop{false};
  // statistics
  uint64_t completed = 0, failed = 0, batches = 0, batched_queries = 0;
  int device = 0;
};

namespace gbf {
namespace {

int32_t *slot_ptr(gbf_server *s, int slot) {
  return (int32_t *)(s->slot_mem + (size_t)slot * s->slot_bytes);
}

// Launch work on an idle engine; caller holds s->mu.
void dispatch(gbf_server *s, Engine *e) {
  // the graph whose oldest pending request of this engine's kind is oldest
  auto &queues = e->kind == GBF_QUERY_WBFS ? s->wbfs_q : s->bfs_q;
  int best = -1;
  Clock::time_point oldest = Clock::time_point::max();
  for (size_t gi = 0; gi < queues.size(); gi++) {
    if (queues[gi].empty()) continue;
    const Request &r = s->reqs[queues[gi].front()];
    if (r.t_submit < oldest) {
      oldest = r.t_submit;
      best = (int)gi;
    }
  }
  if (best < 0) return;
  auto &q = queues[best];
  Graph &g = *s->graphs[best];
  const bool wk = e->kind == GBF_QUERY_WBFS;
  // Batch or not: the largest batch the queue allows (up to 8 weighted, 64
  // BFS queries), against one query per launch, by the measured GPU time
  // per query of each on this graph; a way not measured yet is tried first.
  const int cap = std::max(1, std::min(wk ? 8 : 64, s->opt.max_batch));
  const int kb = std::min<int>(cap, (int)q.size());
  bool batch = false;
  if (kb >= std::max(2, s->opt.min_batch)) {
    const CostModel &cm = s->cost[wk ? 1 : 0][best];
    const int cb = cost_class(kb);
    if (s->opt.always_batch || !cm.seen[cb]) batch = true;
    else if (!cm.seen[0]) batch = false;
    else batch = cm.ms[cb] / kb < cm.ms[0];
  }
  const int k = batch ? kb : std::min<int>((int)q.size(), 4);  // singles: a few back to back
  e->batch.clear();
  int32_t srcs[64];
  int32_t *rows[64];
  while ((int)e->batch.size() < k) {
    const uint64_t t = q.front();
    q.pop_front();
    Request &r = s->reqs[t];
    r.state = 1;
    srcs[e->batch.size()] = r.src;
    rows[e->batch.size()] = slot_ptr(s, r.slot);
    e->batch.push_back(t);
  }
  e->graph = best;
  e->cls = batch ? cost_class(k) : 0;
  e->launches = batch ? 1 : k;
  cudaEventRecord(e->start, e->st);
  gbf_status st = GBF_OK;
  if (batch) {
    st = wk ? launch_mssp_rows(g, e->ws, srcs, (int32_t)k, rows, s->kopt_mssp, e->st)
            : launch_msbfs_rows(g, e->ws, srcs, (int32_t)k, rows, s->kopt_bfs, e->st);
  } else {
    for (int i = 0; i < k && st == GBF_OK; i++)
      st = wk ? launch_wbfs(g, e->ws, srcs[i], rows[i], s->kopt_wbfs, e->st)
              : launch_bfs(g, e->ws, srcs[i], rows[i], nullptr, s->kopt_single, e->st);
  }
  if (st != GBF_OK) {
    for (uint64_t t : e->batch) {
      Request &r = s->reqs[t];
      r.state = 3;
      r.status = st;
      r.t_done = Clock::now();
      s->failed++;
      s->pending--;
    }
    e->batch.clear();
    return;
  }
  if (!wk) {
    s->batches += batch ? 1 : k;
    s->batched_queries += e->batch.size();
  }
  cudaEventRecord(e->done, e->st);
  e->busy = true;
}

void worker_loop(gbf_server *s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop.load()) {
    bool progress = false;
    for (Engine *e : s->engines) {
      if (!e->busy) continue;
      const cudaError_t q = cudaEventQuery(e->done);
      if (q == cudaErrorNotReady) continue;
      const Clock::time_point now = Clock::now();
      gbf_status st = GBF_OK;
      if (q != cudaSuccess) {
        cuda_fail(q, "engine completion");
        st = GBF_ERR_CUDA;
      } else {
        gbf_stats sts;
        st = ws_collect(e->ws, e->st, &sts);
        float ms = 0.f;
        if (st == GBF_OK && cudaEventElapsedTime(&ms, e->start, e->done) == cudaSuccess)
          s->cost[e->kind == GBF_QUERY_WBFS ? 1 : 0][e->graph].add(e->cls, ms / e->launches);
      }
      for (uint64_t t : e->batch) {
        auto it = s->reqs.find(t);
        if (it == s->reqs.end()) continue;
        it->second.state = st == GBF_OK ? 2 : 3;
        it->second.status = st;
        it->second.t_done = now;
        if (st == GBF_OK) s->completed++;
        else s->failed++;
        s->pending--;
      }
      e->batch.clear();
      e->busy = false;
      progress = true;
    }
    for (Engine *e : s->engines) {
      if (e->busy) continue;
      dispatch(s, e);
      if (e->busy) progress = true;
    }
    if (progress) s->cv.notify_all();
    if (!progress) {
      // idle: sleep until a submit arrives or a short poll interval passes
      s->cv.wait_for(lk, std::chrono::microseconds(20));
    }
  }
}

void destroy_engine(Engine *e) {
  if (e->st) cudaStreamSynchronize(e->st);
  ws_free(e->ws);
  if (e->done) cudaEventDestroy(e->done);
  if (e->start) cudaEventDestroy(e->start);
  if (e->st) cudaStreamDestroy(e->st);
  delete e;
}

}  // namespace
}  // namespace gbf

using namespace gbf;

extern "C" {

gbf_status gbf_server_options_default(gbf_server_options *o) {
  if (!o) return GBF_ERR_INVALID;
  memset(o, 0, sizeof(*o));
  o->bfs_engines = 2;
  o->wbfs_engines = 2;
  o->max_batch = 64;
  o->min_batch = 2;
  o->max_queue = 1 << 16;
  o->hbm_budget = 0;
  gbf_options_default(&o->kernel);
  return GBF_OK;
}

gbf_status gbf_server_create(gbf_graph *const *graphs, int32_t ngraphs,
                             const gbf_server_options *opt, gbf_server **out) {
  if (!out || !graphs || ngraphs < 1) return set_error("bad arguments"), GBF_ERR_INVALID;
  *out = nullptr;
  gbf_server *s = new (std::nothrow) gbf_server();
  if (!s) return set_error("host allocation failed"), GBF_ERR_OOM;
  gbf_server_options_default(&s->opt);
  if (opt) s->opt = *opt;
  if (s->opt.bfs_engines < 0 || s->opt.wbfs_engines < 0 || s->opt.bfs_engines + s->opt.wbfs_engines < 1) {
    delete s;
    return set_error("need at least one engine"), GBF_ERR_INVALID;
  }
  s->opt.max_batch = std::max(1, std::min(64, s->opt.max_batch ? s->opt.max_batch : 64));
  if (s->opt.max_queue <= 0) s->opt.max_queue = 1 << 16;
  s->opt.min_batch = std::max(0, std::min(65, s->opt.min_batch));
  uint32_t max_m = 0, max_w = 0;
  bool any_w = false;
  for (int i = 0; i < ngraphs; i++) {
    if (!graphs[i]) {
      delete s;
      return set_error("NULL graph"), GBF_ERR_INVALID;
    }
    Graph *g = &graphs[i]->g;
    s->graphs.push_back(g);
    s->max_n = std::max(s->max_n, g->n);
    max_m = std::max(max_m, g->m);
    if (g->w) {
      any_w = true;
      max_w = std::max(max_w, g->w_max);
    }
  }
  s->device = s->graphs[0]->device;
  s->bfs_q.resize(ngraphs);
  s->wbfs_q.resize(ngraphs);
  s->cost[0].resize(ngraphs);
  s->cost[1].resize(ngraphs);
  auto fail = [&](gbf_status st) {
    gbf_server_destroy(s);
    return st;
  };
  // result slots from the HBM budget
  s->slot_bytes = ((size_t)s->max_n * sizeof(int32_t) + 255) & ~(size_t)255;
  size_t budget = s->opt.hbm_budget;
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    budget = fr / 4;
  }
  const size_t nslots = std::min<size_t>(budget / s->slot_bytes, 1 << 20);
  if (nslots < 1) return fail((set_error("HBM budget below one result slot"), GBF_ERR_OOM));
  cudaError_t e = cudaMalloc((void **)&s->slot_mem, nslots * s->slot_bytes);
  if (e != cudaSuccess) return fail(cuda_fail(e, "result slots"));
  s->free_slots.reserve(nslots);
  for (size_t i = 0; i < nslots; i++) s->free_slots.push_back((int)(nslots - 1 - i));
  // engines: an equal share of the resident CTAs each
  const int nengines = s->opt.bfs_engines + (any_w ? s->opt.wbfs_engines : 0);
  int sms = s->graphs[0]->num_sms;
  for (int i = 0; i < nengines; i++) {
    Engine *en = new (std::nothrow) Engine();
    if (!en) return fail((set_error("host allocation failed"), GBF_ERR_OOM));
    en->kind = i < s->opt.bfs_engines ? GBF_QUERY_BFS : GBF_QUERY_WBFS;
    s->engines.push_back(en);
    Graph &sh = en->shape;
    sh.n = s->max_n;
    sh.m = max_m;
    sh.w_max = max_w;
    sh.device = s->device;
    sh.num_sms = sms;
    if ((e = cudaStreamCreateWithFlags(&en->st, cudaStreamNonBlocking)) != cudaSuccess)
      return fail(cuda_fail(e, "engine stream"));
    if ((e = cudaEventCreate(&en->start)) != cudaSuccess || (e = cudaEventCreate(&en->done)) != cudaSuccess)
      return fail(cuda_fail(e, "engine event"));
    gbf_status st;
    if (en->kind == GBF_QUERY_WBFS) {
      st = ws_ensure_wbfs(sh, en->ws, (int)std::min<uint32_t>(std::max<uint32_t>(max_w + 1, 2), 256));
      if (st == GBF_OK && s->opt.max_batch > 1) st = ws_ensure_mssp(sh, en->ws, false);
    }
    else if (s->opt.max_batch > 1) st = ws_ensure_msbfs(sh, en->ws, false);
    else st = ws_ensure_base(sh, en->ws);
    if (st != GBF_OK) return fail(st);
  }
  // kernel knobs: every engine gets an equal share of the CTAs the GPU can
  // hold at once (the smallest residency among the kernels in use), so all
  // engines' persistent launches are co-resident whatever runs together
  gbf_options ko = s->opt.kernel;
  s->kopt_bfs = resolve(&ko, *s->graphs[0], s->opt.max_batch > 1 ? GBF_TUNE_MSBFS : GBF_TUNE_BFS);
  s->kopt_single = resolve(&ko, *s->graphs[0], GBF_TUNE_BFS);
  s->kopt_wbfs = resolve(&ko, *s->graphs[0], GBF_TUNE_WBFS);
  s->kopt_mssp = resolve(&ko, *s->graphs[0], GBF_TUNE_BFS);
  {
    int per_sm = resident_ctas_per_sm_bfs(s->kopt_single);
    if (s->opt.max_batch > 1) per_sm = std::min(per_sm, resident_ctas_per_sm_msbfs(s->kopt_bfs));
    if (any_w && s->opt.wbfs_engines > 0) {
      const int nB = (int)std::min<uint32_t>(std::max<uint32_t>(max_w + 1, 2), 256);
      per_sm = std::min(per_sm, resident_ctas_per_sm_wbfs(s->kopt_wbfs, nB));
      if (s->opt.max_batch > 1) per_sm = std::min(per_sm, resident_ctas_per_sm_mssp(s->kopt_mssp));
    }
    if (per_sm < 1) return fail((set_error("kernels do not fit on an SM"), GBF_ERR_INVALID));
    const int total = sms * per_sm;
    int bshare = std::max(1, total / nengines), wshare = bshare;
    const int nw = any_w ? s->opt.wbfs_engines : 0, nb = s->opt.bfs_engines;
    if (s->opt.wbfs_share > 0 && nw > 0 && nb > 0) {
      // the weighted engines together get wbfs_share percent, the rest goes
      // to the BFS engines; the shares still add up to what fits at once
      const int wtot = std::min(total - nb, std::max(nw, total * std::min(s->opt.wbfs_share, 99) / 100));
      wshare = std::max(1, wtot / nw);
      bshare = std::max(1, (total - wshare * nw) / nb);
    }
    if (s->kopt_bfs.ctas == 0 || s->kopt_bfs.ctas > bshare) s->kopt_bfs.ctas = bshare;
    if (s->kopt_single.ctas == 0 || s->kopt_single.ctas > bshare) s->kopt_single.ctas = bshare;
    if (s->kopt_wbfs.ctas == 0 || s->kopt_wbfs.ctas > wshare) s->kopt_wbfs.ctas = wshare;
    if (s->kopt_mssp.ctas == 0 || s->kopt_mssp.ctas > wshare) s->kopt_mssp.ctas = wshare;
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return GBF_OK;
}

gbf_status gbf_server_submit(gbf_server *s, int32_t graph_idx, int32_t kind, int32_t src,
                             uint64_t *ticket) {
  if (!s || !ticket) return set_error("NULL argument"), GBF_ERR_INVALID;
  if (graph_idx < 0 || graph_idx >= (int32_t)s->graphs.size())
    return set_error("graph index out of range"), GBF_ERR_INVALID;
  if (kind != GBF_QUERY_BFS && kind != GBF_QUERY_WBFS) return set_error("bad kind"), GBF_ERR_INVALID;
  Graph &g = *s->graphs[graph_idx];
  if (src < 0 || src >= g.n) return set_error("src out of range"), GBF_ERR_INVALID;
  if (kind == GBF_QUERY_WBFS && !g.w) return set_error("graph has no weights"), GBF_ERR_INVALID;
  bool has_engine = false;
  for (Engine *e : s->engines) has_engine |= e->kind == kind;
  if (!has_engine) return set_error("no engine for this kind"), GBF_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->free_slots.empty() || s->pending >= (size_t)s->opt.max_queue) {
    set_error("server busy: no free result slot or queue full");
    return GBF_ERR_BUSY;
  }
  Request r;
  r.ticket = s->next_ticket++;
  r.graph = graph_idx;
  r.kind = kind;
  r.src = src;
  r.slot = s->free_slots.back();
  s->free_slots.pop_back();
  r.t_submit = Clock::now();
  r.state = 0;
  r.status = GBF_OK;
  s->reqs.emplace(r.ticket, r);
  if (kind == GBF_QUERY_BFS) s->bfs_q[graph_idx].push_back(r.ticket);
  else s->wbfs_q[graph_idx].push_back(r.ticket);
  s->pending++;
  *ticket = r.ticket;
  s->cv.notify_all();
  return GBF_OK;
}

gbf_status gbf_server_poll(gbf_server *s, uint64_t ticket, int32_t *dist_host, int32_t *done,
                           double *latency_us) {
  if (!s || !done) return set_error("NULL argument"), GBF_ERR_INVALID;
  *done = 0;
  int slot = -1, gi = 0;
  gbf_status st = GBF_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error("unknown ticket"), GBF_ERR_NOT_FOUND;
    Request &r = it->second;
    if (r.state < 2) return GBF_OK;
    *done = 1;
    if (latency_us)
      *latency_us = std::chrono::duration<double, std::micro>(r.t_done - r.t_submit).count();
    slot = r.slot;
    gi = r.graph;
    st = r.state == 2 ? GBF_OK : r.status;
    s->reqs.erase(it);
  }
  gbf_status cst = GBF_OK;
  if (st == GBF_OK && dist_host) {
    cudaError_t e = cudaMemcpy(dist_host, slot_ptr(s, slot), sizeof(int32_t) * (size_t)s->graphs[gi]->n,
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) cst = cuda_fail(e, "result copy");
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->free_slots.push_back(slot);
  }
  return st != GBF_OK ? st : cst;
}

gbf_status gbf_server_collect(gbf_server *s, uint64_t *tickets, double *latency_us,
                              int32_t *status, int32_t cap, int32_t *count) {
  if (!s || !count || cap < 0 || (cap > 0 && !tickets)) return set_error("bad arguments"), GBF_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  int32_t k = 0;
  for (auto it = s->reqs.begin(); it != s->reqs.end() && k < cap;) {
    const Request &r = it->second;
    if (r.state < 2) {
      ++it;
      continue;
    }
    tickets[k] = r.ticket;
    if (latency_us) latency_us[k] = std::chrono::duration<double, std::micro>(r.t_done - r.t_submit).count();
    if (status) status[k] = r.state == 2 ? GBF_OK : r.status;
    k++;
    s->free_slots.push_back(r.slot);
    it = s->reqs.erase(it);
  }
  *count = k;
  return GBF_OK;
}

gbf_status gbf_server_stats(gbf_server *s, gbf_server_counters *out) {
  if (!s || !out) return set_error("NULL argument"), GBF_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  memset(out, 0, sizeof(*out));
  out->completed = s->completed;
  out->failed = s->failed;
  out->pending = s->pending;
  out->batches = s->batches;
  out->batched_queries = s->batched_queries;
  out->free_slots = s->free_slots.size();
  out->engines = (int32_t)s->engines.size();
  return GBF_OK;
}

gbf_status gbf_server_destroy(gbf_server *s) {
  if (!s) return GBF_OK;
  if (s->worker.joinable()) {
    s->stop.store(true);
    s->cv.notify_all();
    s->worker.join();
  }
  for (Engine *e : s->engines) destroy_engine(e);
  if (s->slot_mem) cudaFree(s->slot_mem);
  delete s;
  return GBF_OK;
}

}  // extern "C"
