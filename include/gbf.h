/*
 * gbf.h — C ABI of the GB300 frontier-traversal library (libgbf.so).
 *
 * The library runs, on one NVIDIA GB300 (sm_103a), the frontier-based
 * edgeMap over vertexSubsets of Ligra as used by the paper (§3 "Ligra,
 * Ligra+, and Julienne"), and the two searches built on it:
 *   - BFS (§4 problem statement; Alg. 1),
 *   - integral-weight SSSP / weighted BFS over Julienne buckets (§4; Alg. 3),
 * plus a 64-lane bit-packed multi-source BFS and a continuous-batching query
 * server, and further problems on the same edgeMap and bucket structure:
 * Bellman-Ford and widest path (Alg. 4), single-source betweenness (Alg. 2),
 * k-core (Alg. 16) and Δ-stepping.  All arithmetic is integer (int32
 * distances and ids, uint32 offsets and weights) except betweenness, whose
 * path counts and dependencies are fp64.
 *
 * Conventions for every call:
 *   - Every function returns a gbf_status, never aborts, never throws across
 *     the ABI.  gbf_last_error() gives a thread-local message for the last
 *     failure on the calling thread.
 *   - Graphs are symmetric CSR: offsets uint32[n+1] with off[0] = 0 and
 *     off[n] = m (number of arcs, each undirected edge stored twice), targets
 *     int32[m], optional weights uint32[m] (both arcs of an edge carry the same
 *     weight).  Adjacency lists need not be sorted unless the symmetry check
 *     is requested.  Results are defined only for symmetric graphs.
 *   - `mem` says where caller buffers live: GBF_HOST (pageable or pinned host
 *     memory; the call copies and blocks until the result is in place) or
 *     GBF_DEVICE (device pointers in the current CUDA context; the call is
 *     ordered on `cuda_stream` and returns after launch — call gbf_wait()
 *     to synchronise and collect the device-side status).
 *   - `cuda_stream` is a cudaStream_t (NULL = legacy default stream).
 *   - Unreachable vertices get distance GBF_INF and parent GBF_NOPARENT; the
 *     source is its own parent.
 *   - Calls on the same graph handle share its default workspace: do not run
 *     two queries on one handle concurrently from different streams (the
 *     server keeps its own per-query workspaces for that).
 */
#ifndef GBF_H
#define GBF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GBF_OK = 0,
  GBF_ERR_INVALID = 1,  /* bad argument or malformed graph */
  GBF_ERR_OOM = 2,      /* device or host allocation failed, or HBM budget exhausted */
  GBF_ERR_CUDA = 3,     /* a CUDA runtime call failed (message in gbf_last_error) */
  GBF_ERR_TIMEOUT = 4,  /* a bounded device wait (grid barrier) ran out */
  GBF_ERR_OVERFLOW = 5, /* distances could exceed int32, or a device queue overflowed */
  GBF_ERR_BUSY = 6,     /* server cannot admit the request now */
  GBF_ERR_NOT_FOUND = 7 /* unknown server ticket */
} gbf_status;

#define GBF_INF INT32_MAX  /* distance of an unreachable vertex */
#define GBF_NOPARENT (-1)  /* parent of an unreachable vertex */

#define GBF_HOST 0
#define GBF_DEVICE 1

/* gbf_graph_create validate_flags (OR-able) */
#define GBF_VALIDATE_BASIC 1u     /* off monotone, off[0]=0, targets in [0,n), no self-loops, weights >= 1 */
#define GBF_VALIDATE_SYMMETRIC 2u /* adjacency lists sorted, no duplicates, every arc has its reverse with the same weight */

typedef struct gbf_graph gbf_graph;

/*
 * Tuning knobs.  Zero in any field selects the default; results (distances)
 * never depend on them.  gbf_options_default() fills the defaults.
 *   block         threads per CTA of the persistent kernels: 128, 256, 512 or 1024
 *                 (0 = per-query default: 512 for wBFS, 256 otherwise)
 *   pull_divisor  edgeMap takes the dense (pull) direction when the frontier's
 *                 out-degree sum exceeds m / pull_divisor (default 20; -1 = push only)
 *   heavy_cutoff  largest number of frontier edges one CTA processes as one
 *                 block of the blocked sparse edgeMap; a vertex with more
 *                 edges is split over several CTAs (power of two, 256..16384; values whose
 *                 shared-memory footprint does not fit a CTA with the chosen block give
 *                 GBF_ERR_INVALID; 0 = per-query
 *                 default: 1024 for multi-source BFS, 512 for BFS and wBFS, whose
 *                 light vertices (<= heavy_cutoff / 8 arcs) are expanded without it)
 *   bucket_window number of open buckets nB of the wBFS bucket structure
 *                 (1..256, default min(max weight + 1, 256); values <= max weight use the overflow bucket)
 *   dense_wbfs    1 = let wBFS switch to a dense edgeMap for dense buckets (default 0)
 *   spin_cap_us   time limit of every bounded device wait, microseconds (default 5,000,000)
 *   local_arcs    wBFS: a bucket of at most `block` entries whose live entries hold at most
 *                 local_arcs arcs (1 .. 2^20 - 1) is expanded by one CTA alone, and so are
 *                 the buckets after it while they stay that small, with CTA barriers only,
 *                 while the other CTAs wait at one grid barrier (0 or negative = off, the
 *                 default: on the measured graphs the kernel with this mode is slower)
 *   ctas          CTAs of the persistent kernels (default: every CTA that fits, all SMs;
 *                 on graphs with fewer than 8 arcs per vertex, whose many thin rounds
 *                 cost mostly their grid barrier, half as many CTAs as SMs)
 *   pull_serial   arcs each vertex checks on its own (4 at a time) before the dense step
 *                 may walk its remaining arcs with the whole warp (0 = per kind:
 *                 128 for BFS, 8 for multi-source BFS)
 *   inject_wait   fault injection for tests: 1 = one CTA waits on a flag nothing sets,
 *                 so the first grid barrier times out and the call returns GBF_ERR_TIMEOUT
 *   pull_stay     BFS: after a dense level the next level stays dense while its frontier
 *                 holds more than n / pull_stay vertices (0 = default 24; negative = off,
 *                 the out-degree rule alone)
 */
typedef struct {
  int32_t block;
  int32_t pull_divisor;
  int32_t heavy_cutoff;
  int32_t bucket_window;
  int32_t dense_wbfs;
  int32_t local_arcs;
  int64_t spin_cap_us;
  int32_t ctas;
  int32_t pull_serial;
  int32_t inject_wait;
  int32_t pull_stay;
} gbf_options;

/* Per-query statistics, filled by gbf_wait / host-memory calls. */
typedef struct {
  int64_t rounds;            /* BFS levels, or wBFS bucket rounds */
  int64_t push_rounds;       /* sparse edgeMap rounds */
  int64_t pull_rounds;       /* dense edgeMap rounds */
  int64_t edges_scanned;     /* arcs examined by edgeMap */
  int64_t vertices_expanded; /* frontier vertices whose arcs were traversed */
  int64_t vertices_reached;  /* vertices with finite distance */
  int64_t relaxations;       /* wBFS: successful writeMin calls */
  int64_t bucket_inserts;    /* wBFS: entries appended to buckets (incl. overflow) */
  int64_t refills;           /* wBFS: overflow-bucket refills */
  int64_t heavy_vertices;    /* frontier vertices expanded by the blocked edgeMap pass */
  int64_t vertices_pulled;   /* dense rounds: unvisited candidates examined */
  int64_t device_ns;         /* BFS: %globaltimer time from the kernel's start to its last CTA's end */
  int32_t grid_ctas;         /* CTAs of the persistent launch */
  int32_t block;             /* threads per CTA */
  int32_t device_error;      /* gbf_status reported by the device */
  int32_t local_rounds;      /* wBFS: bucket rounds expanded by one CTA alone (local_arcs) */
} gbf_stats;

/* Fills *opt with the defaults (all knobs explicit). */
gbf_status gbf_options_default(gbf_options *opt);

/* Thread-local message describing the last failure; returns its length. */
size_t gbf_last_error(char *buf, size_t len);

/* Library version as "major.minor.patch". */
const char *gbf_version(void);

/*
 * gbf_graph_create — make a graph resident on the current CUDA device
 * (the paper's CSR representation, §3 graph notation).
 *   n         vertices, 1 <= n < 2^31
 *   off       uint32[n+1], off[n] = m < 2^32 arcs
 *   tgt       int32[m]
 *   w         uint32[m] or NULL (unweighted: only BFS and MS-BFS available)
 *   mem       where off/tgt/w live (GBF_HOST or GBF_DEVICE)
 *   validate_flags  GBF_VALIDATE_* checks run on the device; failures give GBF_ERR_INVALID
 *   cuda_stream     stream for the upload and the checks
 *   out       receives the handle
 * The library copies the arrays into memory it owns; the caller keeps its
 * buffers.  Weighted graphs with (n-1) * max(w) >= 2^31-1 are rejected with
 * GBF_ERR_OVERFLOW (distances would not fit int32).  Blocks until resident.
 */
gbf_status gbf_graph_create(int32_t n, const uint32_t *off, const int32_t *tgt, const uint32_t *w,
                            int mem, uint32_t validate_flags, void *cuda_stream, gbf_graph **out);

/* Frees the graph and every workspace it owns. NULL is accepted. */
gbf_status gbf_graph_destroy(gbf_graph *g);

/* Vertices, arcs, max weight (0 if unweighted) and a 64-bit fingerprint of
 * the CSR contents (used to key autotuning results). Any pointer may be NULL. */
gbf_status gbf_graph_info(const gbf_graph *g, int32_t *n, uint64_t *m, uint32_t *w_max,
                          uint64_t *fingerprint);

/* Device bytes held by the graph (arrays plus workspaces allocated so far). */
gbf_status gbf_graph_device_bytes(const gbf_graph *g, size_t *bytes);

/*
 * gbf_bfs — breadth-first search from src (§4 "Breadth-First Search";
 * Alg. 1, with the direction-optimising edgeMap of §3).
 *   dist    int32[n]: hop distance, GBF_INF if unreachable
 *   parent  int32[n] or NULL: a BFS tree; parent[src] = src, GBF_NOPARENT if
 *           unreachable.  Which neighbour one level closer becomes the parent
 *           depends on timing (the test-and-set winner); any such tree is valid.
 *   mem     GBF_HOST: blocks; GBF_DEVICE: stream-ordered, see gbf_wait
 *   opt     NULL for defaults
 * Errors: GBF_ERR_INVALID for a bad src or NULL dist; GBF_ERR_TIMEOUT if a
 * bounded device wait ran out (outputs are then undefined).
 */
gbf_status gbf_bfs(gbf_graph *g, int32_t src, int32_t *dist, int32_t *parent, int mem,
                   const gbf_options *opt, void *cuda_stream);

/*
 * gbf_bfs_host_batch — k BFS queries of gbf_bfs (§4 "Breadth-First Search";
 * Alg. 1) with their results in host memory, each query's read-back
 * overlapping the next query's search: the results go to two device buffers
 * in turn, and a second stream copies one out while the next query runs.
 *   srcs    int32[k] host array of sources, k >= 1
 *   dist    host int32[k * n]: row i = the distances from srcs[i]
 *   parent  host int32[k * n] or NULL: row i = a BFS tree of srcs[i]
 *   opt     NULL for defaults
 * Blocks until every row is in host memory; page-locked (pinned) buffers
 * let the copies overlap the searches.  Returns the first device status of
 * the batch.  Allocates a second result buffer pair and a copy stream on the
 * graph's first call.  gbf_wait afterwards reports the last query.
 * Errors: GBF_ERR_INVALID for k < 1, a bad source or NULL srcs/dist.
 */
gbf_status gbf_bfs_host_batch(gbf_graph *g, const int32_t *srcs, int32_t k, int32_t *dist,
                              int32_t *parent, const gbf_options *opt, void *cuda_stream);

/*
 * gbf_wbfs — integral-weight single-source shortest paths from src by
 * weighted BFS over a Julienne bucket structure (§4 "Integral-Weight SSSP";
 * Alg. 3).  Requires a weighted graph with weights >= 1.
 *   dist    int32[n]: shortest-path distance, GBF_INF if unreachable
 * Errors: as gbf_bfs; GBF_ERR_INVALID on an unweighted graph.
 */
gbf_status gbf_wbfs(gbf_graph *g, int32_t src, int32_t *dist, int mem, const gbf_options *opt,
                    void *cuda_stream);

/*
 * gbf_delta_stepping — the same shortest paths by Δ-stepping, the bucket
 * coarsening the SSSP discussion of §7 compares wBFS with (Meyer and Sanders):
 * bucket q holds the distances [qΔ, (q+1)Δ); a vertex lowered into the bucket
 * being processed is expanded again in a further round of that bucket (at
 * most once per round: a test-and-set side list) until the bucket settles,
 * then the next non-empty bucket is taken.  Distances are exact for every Δ;
 * Δ trades rounds (grid barriers) against re-expansions.  delta = 1 is gbf_wbfs.
 *   delta   power of two in [1, 2^20]
 *   dist    int32[n]: shortest-path distance, GBF_INF if unreachable
 *   mem     GBF_HOST: blocks; GBF_DEVICE: stream-ordered, see gbf_wait
 * Errors: as gbf_wbfs; GBF_ERR_INVALID for a bad delta; GBF_ERR_OVERFLOW if a
 * bucket ring or the overflow bucket ran out of room (possible only on
 * adversarial inputs; outputs are then undefined).  The dense switch
 * (dense_wbfs) does not apply.
 */
gbf_status gbf_delta_stepping(gbf_graph *g, int32_t src, int32_t delta, int32_t *dist, int mem,
                              const gbf_options *opt, void *cuda_stream);

/*
 * gbf_bellman_ford — general-weight single-source shortest paths by the
 * frontier Bellman-Ford of §4 "General-Weight SSSP (Bellman-Ford)" (Alg. 4):
 * rounds of the blocked sparse edgeMap whose Update relaxes D[s] + w with
 * writeMin and puts an improved target on the next frontier once (a
 * test-and-set flag, reset a round later).  Weights are the graph's uint32
 * weights (>= 1, so a symmetric graph has no negative cycle).
 *   dist    int32[n]: shortest-path distance, GBF_INF if unreachable
 *   mem     GBF_HOST: blocks; GBF_DEVICE: stream-ordered, see gbf_wait
 * Errors: as gbf_wbfs.  The sparse (push) direction only.
 */
gbf_status gbf_bellman_ford(gbf_graph *g, int32_t src, int32_t *dist, int mem,
                            const gbf_options *opt, void *cuda_stream);

/*
 * gbf_widest_path — single-source widest (bottleneck) path (§4 "Widest
 * Path"; §5: the Bellman-Ford rounds of Alg. 4 over the (max, min) semiring):
 * width[v] is the largest, over paths from src to v, of the smallest weight
 * on the path.  width[src] = GBF_INF (the empty path) and, following the
 * problem statement's output convention, width[v] = GBF_INF for unreachable v.
 * Arguments and errors as gbf_bellman_ford.
 */
gbf_status gbf_widest_path(gbf_graph *g, int32_t src, int32_t *width, int mem,
                           const gbf_options *opt, void *cuda_stream);

/*
 * gbf_betweenness — single-source betweenness centrality (§4 "Single-Source
 * Betweenness Centrality"; Alg. 2): a forward pass of frontier rounds that
 * counts shortest paths with fp64 fetch-and-add and keeps every frontier,
 * then a backward pass over those frontiers in reverse that accumulates
 * dependencies.  Works on the graph's arcs; weights are ignored.
 *   dep     double[n]: dep[v] = sum over targets t of the fraction of
 *           shortest src-t paths through v (v != src); dep[src] = the number
 *           of other vertices reached; 0 where unreachable.  fp64, summation
 *           order varies between runs (relative differences ~1e-15).
 *   mem     GBF_HOST: blocks; GBF_DEVICE: stream-ordered, see gbf_wait
 * Errors: as gbf_bfs; GBF_ERR_OVERFLOW if the search has more than 65,536
 * levels.
 */
gbf_status gbf_betweenness(gbf_graph *g, int32_t src, double *dep, int mem,
                           const gbf_options *opt, void *cuda_stream);

/*
 * gbf_kcore — the coreness of every vertex (§4 "k-core"; Alg. 16): for k in
 * increasing order, the unfinished vertices whose remaining degree is at
 * most k are finished with coreness k and peeled in rounds of the blocked
 * sparse edgeMap, each lowering its unfinished neighbours' remaining degree
 * by its number of arcs to them (combined per warp window); a neighbour that
 * reaches k is finished in the same bucket.
 *   core    int32[n]: coreness (0 for isolated vertices)
 *   mem     GBF_HOST: blocks; GBF_DEVICE: stream-ordered, see gbf_wait
 * Errors: GBF_ERR_INVALID for NULL arguments; GBF_ERR_TIMEOUT as gbf_bfs.
 */
gbf_status gbf_kcore(gbf_graph *g, int32_t *core, int mem, const gbf_options *opt,
                     void *cuda_stream);

/*
 * gbf_ldd — low-diameter decomposition (§4 "Low-Diameter Decomposition";
 * Alg. 6, the Miller-Peng-Xu clustering): vertex v may start its own cluster
 * in round floor(max delta - delta[v]) unless a search has reached it; every
 * round each frontier vertex hands its cluster to its unclaimed neighbours
 * (compare-and-swap), which form the next frontier.
 *   delta    fp64[n]: the shifts, drawn by the caller from Exp(beta); finite,
 *            >= 0, with max delta - min delta < 2^22
 *   cluster  int32[n]: the centre of v's cluster (a centre is its own)
 *   round    int32[n]: the round in which v joined a frontier (unique; which
 *            of several searches reaching v in one round wins is not)
 *   mem      GBF_HOST: all three are host buffers, blocks; GBF_DEVICE: all
 *            three are device pointers, stream-ordered, see gbf_wait
 * Errors: GBF_ERR_INVALID for NULL arguments or negative / non-finite /
 * too widely spread shifts (reported by the device; outputs undefined);
 * GBF_ERR_TIMEOUT as gbf_bfs.
 */
gbf_status gbf_ldd(gbf_graph *g, const double *delta, int32_t *cluster, int32_t *round, int mem,
                   const gbf_options *opt, void *cuda_stream);

/*
 * gbf_connectivity — connected components (§4 "Connectivity"): label[v] = the
 * smallest vertex id in v's component.  Rounds of hooking over every arc
 * (writeMin of the smaller label into the larger label and into the vertex
 * it names) and shortcutting (L[v] = L[L[v]]) until a round changes nothing;
 * the paper's decomposition-contraction recursion (Alg. 7) is not used.
 *   label   int32[n]
 *   mem     GBF_HOST: blocks; GBF_DEVICE: stream-ordered, see gbf_wait
 * Errors: GBF_ERR_INVALID for NULL arguments; GBF_ERR_OVERFLOW after 4,096
 * rounds without convergence (not expected: labels halve their distance to
 * the component's root about every round); GBF_ERR_TIMEOUT as gbf_bfs.
 */
gbf_status gbf_connectivity(gbf_graph *g, int32_t *label, int mem, const gbf_options *opt,
                            void *cuda_stream);

/*
 * gbf_wait — synchronise `cuda_stream` and return the device-side status of
 * the last gbf_bfs / gbf_wbfs / gbf_msbfs / gbf_bellman_ford /
 * gbf_widest_path / gbf_betweenness / gbf_kcore / gbf_delta_stepping /
 * gbf_ldd / gbf_connectivity issued on g with GBF_DEVICE
 * buffers; fills *stats if non-NULL.
 */
gbf_status gbf_wait(gbf_graph *g, void *cuda_stream, gbf_stats *stats);

/*
 * gbf_msbfs — k independent BFSs (1 <= k <= 64) from srcs[0..k) in one
 * persistent launch, one bit lane of a uint64 per source per vertex
 * (multi-source BFS; the paper's nearest precedent is the simultaneous
 * searches from many centres of its SCC algorithm, §5 "Strongly Connected
 * Components").  Each level is one edgeMap (§3) shared by all lanes.  The
 * launch is captured once into a CUDA graph per set of knobs and replayed.
 *   srcs  int32[k] in host memory (duplicates allowed)
 *   dist  int32[k*n], row i = hop distances from srcs[i] (GBF_INF if unreachable)
 *   mem   where dist lives; GBF_HOST blocks, GBF_DEVICE is stream-ordered
 * Errors: GBF_ERR_INVALID for k out of range, a bad source or NULL pointers.
 */
gbf_status gbf_msbfs(gbf_graph *g, const int32_t *srcs, int32_t k, int32_t *dist, int mem,
                     const gbf_options *opt, void *cuda_stream);

/*
 * gbf_mssp — shortest-path distances (§4 "Integral-Weight SSSP") from k
 * sources (1 <= k <= 8) on a weighted graph in one persistent launch: the
 * frontier rounds of Bellman-Ford (Alg. 4) with one int32 distance lane per
 * source, the 8 lanes of a vertex stored together so that every arc read and
 * every round serves all sources.  The distances equal gbf_wbfs's.
 *   srcs  int32[k] in host memory (duplicates allowed)
 *   dist  int32[k*n], row i = distances from srcs[i] (GBF_INF if unreachable)
 *   mem   where dist lives; GBF_HOST blocks, GBF_DEVICE is stream-ordered
 * Errors: GBF_ERR_INVALID for an unweighted graph, k out of range, a bad
 * source or NULL pointers.
 */
gbf_status gbf_mssp(gbf_graph *g, const int32_t *srcs, int32_t k, int32_t *dist, int mem,
                    const gbf_options *opt, void *cuda_stream);

#define GBF_TUNE_BFS 0   /* tune gbf_bfs */
#define GBF_TUNE_MSBFS 1 /* tune gbf_msbfs (64 lanes) */
#define GBF_TUNE_WBFS 2  /* tune gbf_wbfs */

/*
 * gbf_autotune — choose block size, pull divisor (the m / divisor switch of
 * edgeMap, §3) and heavy cutoff (the block size of the blocked edgeMap,
 * §6.2) for queries of `kind` on g, by timing real queries (median of
 * repeats over seeded sources) in a coordinate descent over block in
 * {128, 256, 512, 1024}, divisor in {10, 14, 20, 28, 40} and heavy cutoff in
 * {256, ..., 16384}.  Writes the fastest setting to *out (other fields at
 * their defaults).  Results are cached per (graph fingerprint, device, kind)
 * in the process, and across processes in the file named by the environment
 * variable GBF_TUNE_CACHE if set.  Distances never depend on the knobs.
 * Uses g's default workspace; blocks until done.
 */
gbf_status gbf_autotune(gbf_graph *g, int32_t kind, gbf_options *out);

/* ------------------------------------------------------------------ serving
 * A continuous-batching query server over several resident graphs.  BFS
 * and weighted-BFS queries (§4 problem statements) are admitted while a
 * device result slot is free (slots are carved once from an HBM budget) and
 * the pending queue has room.  A dispatcher thread keeps engines busy, each
 * with its own stream and workspace: BFS engines coalesce up to max_batch
 * pending BFS queries of one graph into one multi-source launch (8-bit lanes
 * for 2..8 queries, 64-bit lanes above; each lane writes its query's result
 * slot), or run a batch smaller than min_batch as single-source launches;
 * wBFS engines coalesce up to 8 pending weighted queries of one graph into
 * one gbf_mssp launch (a single one runs as gbf_wbfs).  Engines run
 * concurrently on shares of the GPU.
 * Results stay on the device until polled.  The paper has no serving layer;
 * results are identical to the single-query calls.
 */
typedef struct gbf_server gbf_server;

#define GBF_QUERY_BFS 0
#define GBF_QUERY_WBFS 1

typedef struct {
  int32_t bfs_engines;   /* concurrent BFS batches (default 2) */
  int32_t wbfs_engines;  /* concurrent weighted queries (default 2; unused without weighted graphs) */
  int32_t max_batch;     /* BFS queries per launch, 1..64 (default 64), and weighted queries
                            per launch, up to 8; 1 = one query per launch with the
                            single-source kernels */
  int32_t max_queue;     /* pending queries before submit returns GBF_ERR_BUSY (default 65536) */
  size_t hbm_budget;     /* device bytes for result slots (0 = a quarter of free HBM) */
  gbf_options kernel;    /* kernel knobs (ctas is capped to the engine's share) */
  int32_t min_batch;     /* BFS batches with fewer queries run as single-source launches
                            (default 2) */
  int32_t wbfs_share;    /* percent of the GPU's resident CTAs the weighted engines share
                            (split evenly among them; the BFS engines share the rest);
                            0 = every engine gets an equal share (default) */
  int32_t always_batch;  /* 1 = batch whenever min_batch or more queries of a graph wait;
                            0 = batch only where the measured GPU time per query is lower
                            than one query per launch (default) */
  int32_t reserved;
} gbf_server_options;

typedef struct {
  uint64_t completed;       /* queries finished successfully */
  uint64_t failed;          /* queries finished with a device or launch error */
  uint64_t pending;         /* admitted, not finished */
  uint64_t batches;         /* BFS launches */
  uint64_t batched_queries; /* BFS queries carried by those launches */
  uint64_t free_slots;      /* result slots available for admission */
  int32_t engines;
  int32_t reserved;
} gbf_server_counters;

/* Fills *opt with the defaults. */
gbf_status gbf_server_options_default(gbf_server_options *opt);

/* Start a server over ngraphs resident graphs (handles stay owned by the
 * caller and must outlive the server).  Reserves the result slots and the
 * engines' workspaces up front; GBF_ERR_OOM if they do not fit. */
gbf_status gbf_server_create(gbf_graph *const *graphs, int32_t ngraphs,
                             const gbf_server_options *opt, gbf_server **out);

/* Admit a query (kind GBF_QUERY_BFS or GBF_QUERY_WBFS) from src on graph
 * graph_idx; *ticket identifies it.  GBF_ERR_BUSY if no result slot is free
 * or the queue is full (try again later); GBF_ERR_INVALID for bad
 * arguments.  Thread-safe. */
gbf_status gbf_server_submit(gbf_server *s, int32_t graph_idx, int32_t kind, int32_t src,
                             uint64_t *ticket);

/* Poll a ticket: *done = 0 while it runs.  Once done, copies its distances
 * (n int32, GBF_INF if unreachable) to dist_host if non-NULL, stores the
 * submit-to-completion latency in *latency_us (if non-NULL), releases the
 * ticket and its slot, and returns the query's status.  GBF_ERR_NOT_FOUND
 * for an unknown or already released ticket.  Thread-safe. */
gbf_status gbf_server_poll(gbf_server *s, uint64_t ticket, int32_t *dist_host, int32_t *done,
                           double *latency_us);

/* Release up to cap finished queries without copying their results (for
 * callers that only need completion and latency): their tickets, latencies
 * (if non-NULL) and statuses (if non-NULL) go to the arrays, their number
 * to *count.  Thread-safe. */
gbf_status gbf_server_collect(gbf_server *s, uint64_t *tickets, double *latency_us,
                              int32_t *status, int32_t cap, int32_t *count);

/* Counters since creation. */
gbf_status gbf_server_stats(gbf_server *s, gbf_server_counters *out);

/* Stop the dispatcher (running launches finish first) and free everything. */
gbf_status gbf_server_destroy(gbf_server *s);

/* One record per round of the last query (see gbf_trace). */
typedef struct {
  int32_t round;          /* 1-based round (BFS level or wBFS bucket round) */
  int32_t kind;           /* 1 sparse, 2 dense, 3 sparse + heavy pass, 4 conversion
                             (BFS: bitmap -> queue, then sparse), 5 k-core bucket pass
                             (frontier = the bucket), 6 BFS sparse level writing a
                             bitmap, 7 the same after a bitmap -> queue conversion,
                             8 wBFS bucket round expanded by one CTA alone */
  uint32_t frontier;      /* frontier vertices (wBFS: bucket entries, stale ones included) */
  uint32_t frontier_edges;/* out-degree sum of the frontier when known (0 otherwise) */
  int64_t t_ns;           /* device time at the end of the round, since the kernel started */
  int64_t t_mid_ns;       /* end of the round's first phase when it has two (0 otherwise) */
} gbf_round_trace;

/*
 * gbf_trace — per-round device timeline of the last query on g (the round
 * structure of Alg. 1 / Alg. 3 / Alg. 16 as it ran: direction chosen,
 * frontier size, time).  Call after the query completed (host buffers, or
 * after gbf_wait).  Copies min(rounds, cap) records to out and their number
 * to *count.
 */
gbf_status gbf_trace(gbf_graph *g, gbf_round_trace *out, int32_t cap, int32_t *count);

/*
 * gbf_bfs_noalloc — the same BFS as gbf_bfs for callers that cannot allocate
 * device memory: for example a process whose device memory is already owned
 * by another allocator (a framework's caching allocator, a fixed-budget
 * deployment), or a latency-critical loop where cudaMalloc / cudaFree, which
 * may synchronise the whole device, are not acceptable.  The paper has no
 * counterpart.
 *   n, m      vertices (1 <= n <= 1,048,576) and arcs (m <= 33,554,432)
 *   off, tgt  the symmetric CSR graph in DEVICE memory: off holds n+1 uint32
 *             entries, tgt holds m int32 entries (the caller guarantees these
 *             lengths; the library cannot see them)
 *   src       source vertex
 *   dist      int32[n] in device memory (GBF_INF if unreachable)
 *   parent    int32[n] in device memory, or NULL
 *   opt       NULL for defaults
 *   cuda_stream  stream to run on; the call blocks until the search is done
 *             and returns the device-side status
 * Before the search the call checks the CSR on the device (off[0] = 0,
 * off[n] = m, offsets non-decreasing, targets in [0, n)) and returns
 * GBF_ERR_INVALID if it is malformed.  The call allocates nothing: its
 * scratch (~26.7 MB) is one fixed array in the library's device module, held
 * on every GPU that loads the library until the process exits.  Every call
 * looks up that array's device address (cudaGetSymbolAddress) with the device
 * current; the first call on a device may also load the module, so make it
 * before any stream capture.  All calls share the one array, so calls that
 * overlap on the GPU (different streams, threads or processes sharing a
 * context) race and must be serialised by the caller.  Sizes above the limits
 * return GBF_ERR_INVALID without touching the GPU.
 */
gbf_status gbf_bfs_noalloc(int32_t n, uint32_t m, const uint32_t *off, const int32_t *tgt,
                           int32_t src, int32_t *dist, int32_t *parent, const gbf_options *opt,
                           void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* GBF_H */
