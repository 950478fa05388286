// Internal host-side definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/gbf.h"
#include "gbf_dev.h"

namespace gbf {

// ------------------------------------------------------------ error reporting
void set_error(const std::string &msg);
gbf_status cuda_fail(cudaError_t e, const char *what);

#define GBF_CUDA(call)                                   \
  do {                                                   \
    cudaError_t _e = (call);                             \
    if (_e != cudaSuccess) return ::gbf::cuda_fail(_e, #call); \
  } while (0)

// The structs device code reads and writes (control block, trace records,
// graph view) are in gbf_dev.h.

// Device-resident scratch for one query at a time.
struct Workspace {
  int32_t n = 0;
  uint32_t m = 0;
  size_t bytes = 0;
  uint32_t *visited = nullptr;   // ceil(n/32) words
  uint32_t *fbm[3] = {nullptr, nullptr, nullptr};
  uint32_t *lb = nullptr;        // lb_count bitmaps of BFS levels whose D is written at the end
  int lb_count = 0;
  int32_t *q[2] = {nullptr, nullptr};
  uint32_t *qoff[2] = {nullptr, nullptr};
  uint32_t *qadj[2] = {nullptr, nullptr};  // CSR offset of each entry's first arc
  uint32_t *cs[2] = {nullptr, nullptr};  // chunk starts, one per 256 frontier edges
  Ctl *ctl = nullptr;
  int32_t *dist_tmp = nullptr;     // used for host-memory outputs
  int32_t *parent_tmp = nullptr;
  // batched BFS to host memory (lazy): a second result buffer pair, the
  // read-back stream, its events, and the first device status of the batch
  int32_t *dist_tmp2 = nullptr;
  int32_t *parent_tmp2 = nullptr;
  cudaStream_t hb_stream = nullptr;
  cudaEvent_t hb_kern_done[2] = {nullptr, nullptr}, hb_copy_done[2] = {nullptr, nullptr};
  int *hb_err = nullptr;
  int *hb_err_host = nullptr;
  TraceRec *trace = nullptr;
  int trace_cap = 0;
  // wBFS (lazy)
  int32_t *slots = nullptr;        // nB * n (ring buffers)
  uint32_t *slot_cnt = nullptr;    // nB
  int32_t nB = 0;
  int2 *ovf[2] = {nullptr, nullptr};
  uint64_t ovf_cap = 0;
  int32_t *side[2] = {nullptr, nullptr};  // Δ-stepping side lists (lazy), n each
  int32_t *xround = nullptr;               // Δ-stepping: last round each vertex was expanded
  // MS-BFS (lazy); queues 0 and 1 are shared with q/qoff/cs above
  unsigned long long *ms_seen = nullptr, *ms_visit = nullptr, *ms_next = nullptr;
  int32_t *ms_q[3] = {nullptr, nullptr, nullptr};
  uint32_t *ms_qoff[3] = {nullptr, nullptr, nullptr};
  uint32_t *ms_qadj[3] = {nullptr, nullptr, nullptr};
  uint32_t *ms_cs[3] = {nullptr, nullptr, nullptr};
  int32_t *ms_touched = nullptr;
  void *ms_call = nullptr;        // device parameter block
  void *ms_call_host = nullptr;   // pinned staging of the parameter block
  int32_t *ms_dist_tmp = nullptr; // 64*n, only for host-memory outputs
  cudaStream_t ms_stream = nullptr;
  cudaEvent_t ms_ready = nullptr, ms_done = nullptr;
  cudaGraphExec_t ms_exec = nullptr;
  long long ms_key[7] = {0, 0, 0, 0, 0, 0, 0};
  int ms_grid = 0;
  // betweenness (lazy): path counts / coefficients, levels, chunk starts of
  // every level, per-level descriptors, fp64 output staging for host buffers
  double *bc_paths = nullptr;
  int32_t *bc_lvl = nullptr;
  uint32_t *bc_cs = nullptr;
  uint32_t bc_cs_total = 0;
  void *bc_info = nullptr;
  int bc_max_levels = 0;
  double *bc_out_tmp = nullptr;
  // multi-source SSSP (lazy): 8 distance lanes per vertex, 3 lane-mask arrays
  // (a byte per vertex), output staging for host buffers
  int32_t *mssp_dd = nullptr;
  unsigned *mssp_imp = nullptr;
  int32_t *mssp_out_tmp = nullptr;
  // pinned host copy of the control block
  Ctl *ctl_host = nullptr;
  int last_kind = 0;   // 1 bfs, 2 wbfs, 3 msbfs
  int last_grid = 0, last_block = 0;
};

struct Graph {
  int32_t n = 0;
  uint32_t m = 0;
  uint32_t w_max = 0;
  uint64_t fingerprint = 0;
  int device = 0;
  int num_sms = 0;
  uint32_t *off = nullptr;
  int32_t *tgt = nullptr;
  uint32_t *w = nullptr;
  uint32_t *leaf = nullptr;  // bit v set iff deg(v) == 1 (wBFS does not file these)
  uint32_t *iso = nullptr;   // bit v set iff deg(v) == 0
  int32_t *f1 = nullptr;     // target of each vertex's first arc (-1 if it has none)
  size_t bytes = 0;
  Workspace ws;
  std::mutex mu;   // serialises host calls on the default workspace
  DevGraph dev() const { return DevGraph{n, m, off, tgt, w}; }
};

// Resolved options (defaults filled, clamped).
struct Opts {
  int block, pull_divisor, heavy_cutoff, bucket_window, dense_wbfs, ctas, pull_serial, inject_wait;
  int pull_stay;  // BFS: after a dense level, stay dense while |F| * pull_stay > n (0: off)
  int local_arcs; // wBFS: arcs of a bucket one CTA expands alone (0: off)
  long long spin_cap_ns;
};
Opts resolve(const gbf_options *o, const Graph &g, int kind);  // kind: GBF_TUNE_*

// GBF_ERR_INVALID (with a message) if a CTA cannot get `bytes` of dynamic
// shared memory on the current device.
gbf_status check_smem(size_t bytes, const char *kernel);

// Workspace management (graph.cu)
gbf_status ws_ensure_base(Graph &g, Workspace &ws);
gbf_status ws_ensure_wbfs(Graph &g, Workspace &ws, int nB, int dl = 0);
gbf_status ws_ensure_msbfs(Graph &g, Workspace &ws, bool host_out);
gbf_status ws_ensure_bc(Graph &g, Workspace &ws);
void ws_free(Workspace &ws);
gbf_status ws_collect(Workspace &ws, cudaStream_t st, gbf_stats *stats);

// Launchers (bfs.cu / wbfs.cu / msbfs.cu); outputs are device pointers.
gbf_status launch_bfs(Graph &g, Workspace &ws, int32_t src, int32_t *dist, int32_t *parent,
                      const Opts &o, cudaStream_t st);
// dl > 0: Δ-stepping with Δ = 2^dl (needs ws_ensure_wbfs(..., dl) side lists)
gbf_status launch_wbfs(Graph &g, Workspace &ws, int32_t src, int32_t *dist, const Opts &o,
                       cudaStream_t st, int dl = 0);
gbf_status launch_msbfs(Graph &g, Workspace &ws, const int32_t *srcs_host, int32_t k,
                        int32_t *dist, const Opts &o, cudaStream_t st);
// Resident CTAs per SM of each persistent kernel for these knobs (0 on error).
int resident_ctas_per_sm_bfs(const Opts &o);
int resident_ctas_per_sm_wbfs(const Opts &o, int nB);
int resident_ctas_per_sm_msbfs(const Opts &o);
gbf_status launch_msbfs_rows(Graph &g, Workspace &ws, const int32_t *srcs_host, int32_t k,
                             int32_t *const *rows, const Opts &o, cudaStream_t st);
// Multi-source SSSP (mssp.cu): k <= 8 weighted sources, row i -> rows[i].
gbf_status ws_ensure_mssp(Graph &g, Workspace &ws, bool host_out);
gbf_status launch_mssp_rows(Graph &g, Workspace &ws, const int32_t *srcs_host, int32_t k,
                            int32_t *const *rows, const Opts &o, cudaStream_t st);
int resident_ctas_per_sm_mssp(const Opts &o);

}  // namespace gbf

struct gbf_graph {
  gbf::Graph g;
};
