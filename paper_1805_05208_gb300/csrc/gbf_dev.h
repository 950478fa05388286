// The structs the persistent kernels read and write: the control block of a
// launch, the per-round trace record and the device view of a graph.  Kept
// apart from the host-side definitions (gbf_impl.h) so that a kernel's
// sources are its .cu file, the device helpers and this header.
#pragma once

#include <cstdint>

namespace gbf {

// Control block of one persistent launch.  Zeroed by the host before every
// launch; every field is touched by the device only through atomics or
// volatile accesses.
struct Ctl {
  unsigned int bar;            // monotone grid-barrier arrival counter
  int err;                     // gbf_status raised on the device (0 = ok)
  int err_where;               // where it was raised (debug)
  int stop;                    // fault injection flag nobody sets
  unsigned int done;           // CTAs past their last phase (BFS end-of-kernel time stamp)
  long long t_end_ns;          // BFS: %globaltimer time of the last CTA's end, since its start
  unsigned long long fr[3];    // frontier counters (count << 32 | degree sum), by round % 3
  unsigned long long conv;     // conversion cursor (same packing)
  unsigned long long cv[3];    // BFS bitmap -> queue conversions (same packing), by level % 3
  // wBFS
  unsigned int mcnt[2];        // moved-list counts, by round parity
  int gmin[3];                 // k-core: smallest remaining degree of the next bucket, by bucket % 3
  unsigned int scnt[3];        // Δ-stepping: side-list counts, by round % 3
  unsigned int ovf_cnt[2];     // overflow bucket counts
  int ovf_min[2];              // overflow bucket minimum value
  unsigned int imask[3][32];   // buckets filed into during round t, by t % 3 (one bit per slot)
  unsigned int work[4];        // dynamic chunk counters of the blocked edgeMap, by invocation % 4
  // statistics
  unsigned long long edges_scanned;
  unsigned long long expanded;
  unsigned long long reached;
  unsigned long long relax;
  unsigned long long inserts;
  unsigned long long heavy;
  unsigned long long pulled;   // dense-round candidates
  int rounds, push_rounds, pull_rounds, refills, local_rounds;
  unsigned int lane_ovf;       // multi-source SSSP: a 16-bit lane could not hold a distance
  // wBFS: bucket state CTA 0 hands back after a run of CTA-local rounds
  int loc_t, loc_lo;
  unsigned int loc_pend[8];
  unsigned int loc_base[256];
};

// One record per round of a persistent launch, written by CTA 0 after the
// round's last barrier (kind: 1 sparse, 2 dense, 3 sparse + heavy pass,
// 4 conversion, 5 k-core bucket pass, 6 / 7 BFS levels writing a bitmap,
// 8 wBFS round of one CTA alone); t_ns is %globaltimer time since the
// kernel started.
struct TraceRec {
  int32_t round;
  int32_t kind;
  uint32_t frontier;
  uint32_t frontier_edges;
  long long t_ns;
  long long t_mid_ns;  // end of the round's first phase (0 if single-phase)
};

struct DevGraph {
  int32_t n;
  uint32_t m;
  const uint32_t *off;
  const int32_t *tgt;
  const uint32_t *w;
};

}  // namespace gbf
