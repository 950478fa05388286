/*
 * oracle.c — TEST INFRASTRUCTURE.  A plain, serial, obviously-correct CPU
 * statement of what the traversal path computes.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the product path
 * never does.  It shares no code, header, table or helper with the CUDA
 * library.
 *
 * What it computes (problem statements of the benchmark section, §4):
 *   - BFS: D[v] = hop distance from src, "infinity" if unreachable.
 *   - Integral-weight SSSP (weighted BFS): D[v] = shortest-path distance with
 *     positive integer edge weights, "infinity" if unreachable.
 * Both results are unique, so the oracle computes the plain definitions —
 * a FIFO-queue BFS and a binary-heap Dijkstra — with no frontier or bucket
 * machinery.
 *   - General-weight SSSP by Bellman-Ford (Alg. 4) and single-source widest
 *     path (the same rounds over the (max, min) semiring, §5 "Widest Path"):
 *     these follow the algorithm's rounds in order (frontier, Update with a
 *     flag per vertex, ResetFlags), since their answers are pinned by other
 *     methods (Dijkstra, Floyd–Warshall, maximum spanning trees).
 *   - Single-source betweenness centrality (Alg. 2): a forward pass of
 *     frontier rounds counting shortest paths (NumPaths, fetch-and-add) and
 *     recording each round's frontier, then a backward pass over the
 *     recorded frontiers in reverse accumulating dependencies, in fp64; it
 *     is pinned against the definition (sums of path-count ratios over all
 *     targets) computed by brute force.
 *   - k-core (coreness, §4 "k-core"; Alg. 16): the coreness of v is the
 *     largest k such that v lies in a subgraph whose vertices all have
 *     degree >= k.  The oracle is the textbook bucket peeling (repeatedly
 *     remove a vertex of minimum current degree; its coreness is the largest
 *     minimum seen so far), pinned against the definition by brute force.
 *   - Connectivity (§4 "Connectivity"): label[v] = the smallest vertex id in
 *     v's connected component, a canonical form of the unique partition (the
 *     paper's Alg. 7 reaches the partition through low-diameter
 *     decompositions; any labelling of it maps to this one).  Computed by a
 *     FIFO search from each vertex, in increasing id, not yet labelled.
 *   - Low-diameter decomposition (§4; Alg. 6, Miller–Peng–Xu): given the
 *     shifts delta[v] ~ Exp(beta) as an input, vertex v may start its own
 *     cluster in round floor(max delta - delta[v]) if nothing has reached it;
 *     each round every frontier vertex hands its cluster to its unclaimed
 *     neighbours.  The round T[v] in which v joins a frontier is unique;
 *     which cluster wins a tie is not, so C is one valid assignment (the
 *     first claimant in frontier order) and tests check T exactly and C by
 *     its invariants.
 * Floyd–Warshall is included as a brute-force check for tiny graphs.  Infinity is INT32_MAX; unreachable parents are -1; the parent of
 * the source is the source itself.
 *
 * The validators state the invariants that any correct BFS tree / shortest-
 * path labelling satisfies (used where several outputs are correct, e.g.
 * parents chosen by whichever test-and-set wins, Alg. 1).
 *
 * Inputs: symmetric CSR, uint32 offsets off[0..n], int32 targets tgt[0..m),
 * optional uint32 weights w[0..m).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_INF INT32_MAX

/* ------------------------------------------------------------------ BFS */
/* Hop distances and one BFS tree (FIFO order, neighbours in CSR order).
 * Returns the number of reached vertices, or -1 on a bad argument. */
int64_t or_bfs(int32_t n, const uint32_t *off, const int32_t *tgt, int32_t src,
               int32_t *dist, int32_t *parent) {
  if (n <= 0 || src < 0 || src >= n) return -1;
  for (int32_t v = 0; v < n; v++) {
    dist[v] = OR_INF;
    if (parent) parent[v] = -1;
  }
  int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  if (!queue) return -1;
  int64_t head = 0, tail = 0;
  dist[src] = 0;
  if (parent) parent[src] = src;
  queue[tail++] = src;
  while (head < tail) {
    int32_t u = queue[head++];
    for (uint32_t k = off[u]; k < off[u + 1]; k++) {
      int32_t v = tgt[k];
      if (dist[v] == OR_INF) {
        dist[v] = dist[u] + 1;
        if (parent) parent[v] = u;
        queue[tail++] = v;
      }
    }
  }
  free(queue);
  return tail;
}

/* ------------------------------------------------------------- Dijkstra */
typedef struct {
  int64_t d;
  int32_t v;
} heap_item;

static void heap_push(heap_item *h, int64_t *size, heap_item x) {
  int64_t i = (*size)++;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (h[p].d <= x.d) break;
    h[i] = h[p];
    i = p;
  }
  h[i] = x;
}

static heap_item heap_pop(heap_item *h, int64_t *size) {
  heap_item top = h[0];
  heap_item last = h[--(*size)];
  int64_t i = 0, s = *size;
  for (;;) {
    int64_t c = 2 * i + 1;
    if (c >= s) break;
    if (c + 1 < s && h[c + 1].d < h[c].d) c++;
    if (h[c].d >= last.d) break;
    h[i] = h[c];
    i = c;
  }
  if (s > 0) h[i] = last;
  return top;
}

/* Shortest-path distances with non-negative integer weights (int64
 * accumulation, int32 result).  Binary heap with lazy deletion: a vertex may
 * be pushed once per improvement; stale pops are skipped.  Returns the number
 * of reached vertices, -1 on a bad argument, -2 if a distance exceeds int32. */
int64_t or_dijkstra(int32_t n, const uint32_t *off, const int32_t *tgt, const uint32_t *w,
                    int32_t src, int32_t *dist) {
  if (n <= 0 || src < 0 || src >= n || !w) return -1;
  int64_t m = off[n];
  int64_t *d = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  heap_item *h = (heap_item *)malloc(sizeof(heap_item) * (size_t)(m + 1));
  char *done = (char *)calloc((size_t)n, 1);
  if (!d || !h || !done) {
    free(d);
    free(h);
    free(done);
    return -1;
  }
  for (int32_t v = 0; v < n; v++) d[v] = INT64_MAX;
  int64_t size = 0, reached = 0;
  d[src] = 0;
  heap_item s0 = {0, src};
  heap_push(h, &size, s0);
  while (size > 0) {
    heap_item it = heap_pop(h, &size);
    int32_t u = it.v;
    if (done[u] || it.d != d[u]) continue;
    done[u] = 1;
    reached++;
    for (uint32_t k = off[u]; k < off[u + 1]; k++) {
      int32_t v = tgt[k];
      int64_t nd = d[u] + (int64_t)w[k];
      if (nd < d[v]) {
        d[v] = nd;
        heap_item x = {nd, v};
        heap_push(h, &size, x);
      }
    }
  }
  int64_t rc = reached;
  for (int32_t v = 0; v < n; v++) {
    if (d[v] == INT64_MAX) dist[v] = OR_INF;
    else if (d[v] >= OR_INF) { dist[v] = OR_INF; rc = -2; }
    else dist[v] = (int32_t)d[v];
  }
  free(d);
  free(h);
  free(done);
  return rc;
}

/* ------------------------------------------------ Bellman-Ford (Alg. 4) */
/* Frontier rounds: every frontier vertex s relaxes its arcs (s, d, w) in CSR
 * order; a d whose value improved joins the next frontier once (its flag);
 * the flags of the new frontier are then reset.  mode 0: D = min over paths
 * of the weight sum ((min, +)), D[src] = 0, unreachable = infinity.  mode 1:
 * widest path ((max, min)): D[v] = max over paths of the smallest weight on
 * the path; the empty path at the source has width infinity, and internally
 * 0 means "no path yet" (weights are >= 1).  The paper's output convention
 * gives unreachable vertices infinity as well.  Returns the number of rounds,
 * -1 on a bad argument, -2 if a sum exceeds int32 (mode 0). */
int64_t or_bellman_ford(int32_t n, const uint32_t *off, const int32_t *tgt, const uint32_t *w,
                        int32_t src, int mode, int32_t *out) {
  if (n <= 0 || src < 0 || src >= n || !w || (mode != 0 && mode != 1)) return -1;
  int64_t *D = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  char *fl = (char *)calloc((size_t)n, 1);
  int32_t *F = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t *F2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  if (!D || !fl || !F || !F2) {
    free(D);
    free(fl);
    free(F);
    free(F2);
    return -1;
  }
  const int64_t unset = mode == 0 ? INT64_MAX : 0;
  for (int32_t v = 0; v < n; v++) D[v] = unset;
  D[src] = mode == 0 ? 0 : INT64_MAX;
  int64_t nf = 1, rounds = 0;
  F[0] = src;
  while (nf > 0 && rounds < (int64_t)n) {
    int64_t nf2 = 0;
    for (int64_t i = 0; i < nf; i++) {
      const int32_t s = F[i];
      for (uint32_t k = off[s]; k < off[s + 1]; k++) {
        const int32_t d = tgt[k];
        const int64_t c = mode == 0 ? D[s] + (int64_t)w[k]
                                    : (D[s] < (int64_t)w[k] ? D[s] : (int64_t)w[k]);
        const int better = mode == 0 ? c < D[d] : c > D[d];
        if (better) {
          D[d] = c;
          if (!fl[d]) {
            fl[d] = 1;
            F2[nf2++] = d;
          }
        }
      }
    }
    for (int64_t i = 0; i < nf2; i++) fl[F2[i]] = 0; /* ResetFlags over the new frontier */
    int32_t *t = F;
    F = F2;
    F2 = t;
    nf = nf2;
    rounds++;
  }
  int64_t rc = rounds;
  for (int32_t v = 0; v < n; v++) {
    if (mode == 0) {
      if (D[v] == INT64_MAX) out[v] = OR_INF;
      else if (D[v] >= OR_INF) { out[v] = OR_INF; rc = -2; }
      else out[v] = (int32_t)D[v];
    } else {
      out[v] = (D[v] == 0 || D[v] >= OR_INF) ? OR_INF : (int32_t)D[v];
    }
  }
  free(D);
  free(fl);
  free(F);
  free(F2);
  return rc;
}

/* ------------------------------------------- betweenness (Alg. 2) */
/* Readings: NumPaths[r] = 1 and r is visited before the first round (the
 * listing leaves the source's path count and flag at 0); NumPaths and the
 * dependencies are fp64.  Forward: the frontier's vertices s add
 * NumPaths[s] to every unvisited neighbour d (in CSR order); d joins the
 * next frontier at its first contribution; the new frontier is recorded as a
 * level and marked visited.  Backward: the levels in reverse; each level is
 * marked visited, then every s in it adds NumPaths[d] / NumPaths[s] *
 * (1 + D[s]) to each neighbour d not yet visited (the level above).
 * Outputs: D (dependencies; 0 where unreachable), the path counts and the
 * hop levels (-1 where unreachable) for the tests.  Returns the number of
 * forward rounds, or -1 on a bad argument. */
int64_t or_betweenness(int32_t n, const uint32_t *off, const int32_t *tgt, int32_t src,
                       double *D, double *paths, int32_t *level) {
  if (n <= 0 || src < 0 || src >= n) return -1;
  char *vis = (char *)calloc((size_t)n, 1);
  int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int64_t *lo = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 2));
  if (!vis || !order || !lo) {
    free(vis);
    free(order);
    free(lo);
    return -1;
  }
  for (int32_t v = 0; v < n; v++) {
    D[v] = 0.0;
    paths[v] = 0.0;
    level[v] = -1;
  }
  paths[src] = 1.0;
  vis[src] = 1;
  level[src] = 0;
  order[0] = src;
  int64_t nl = 0, end = 1;  /* levels[k] = order[lo[k] .. lo[k+1]) */
  lo[0] = 0;
  lo[1] = 1;
  int64_t fb = 0, fe = 1;   /* current frontier */
  while (fe > fb) {
    int64_t ne = end;
    for (int64_t i = fb; i < fe; i++) {
      const int32_t s = order[i];
      for (uint32_t k = off[s]; k < off[s + 1]; k++) {
        const int32_t d = tgt[k];
        if (vis[d]) continue;
        const double prev = paths[d];
        paths[d] = prev + paths[s];
        if (prev == 0.0) order[ne++] = d;
      }
    }
    for (int64_t i = end; i < ne; i++) {
      vis[order[i]] = 1;
      level[order[i]] = (int32_t)(nl + 1);
    }
    nl++;
    lo[nl + 1] = ne;
    fb = end;
    fe = ne;
    end = ne;
  }
  /* lo[0..nl]: levels 0..nl-1 nonempty (the last recorded frontier is
   * empty); backward over levels nl-1 .. 1 */
  memset(vis, 0, (size_t)n);
  for (int64_t L = nl - 1; L >= 1; L--) {
    for (int64_t i = lo[L]; i < lo[L + 1]; i++) vis[order[i]] = 1;
    for (int64_t i = lo[L]; i < lo[L + 1]; i++) {
      const int32_t s = order[i];
      for (uint32_t k = off[s]; k < off[s + 1]; k++) {
        const int32_t d = tgt[k];
        if (vis[d]) continue;
        D[d] += paths[d] / paths[s] * (1.0 + D[s]);
      }
    }
  }
  free(vis);
  free(order);
  free(lo);
  return nl;
}

/* ------------------------------------------------------- coreness */
/* Bucket peeling: vertices sit in buckets by current degree; repeatedly take
 * a vertex from the lowest non-empty bucket (never below the running k),
 * give it coreness k = max(k, its degree), and lower each remaining
 * neighbour's degree by one, moving it one bucket down.  Buckets are doubly
 * linked lists.  Returns the largest coreness, or -1 on a bad argument. */
/* Connected components: label[v] = smallest id in v's component.  Returns
 * the number of components, or -1 on a bad argument / allocation failure. */
int64_t or_components(int32_t n, const uint32_t *off, const int32_t *tgt, int32_t *label) {
  if (n < 0) return -1;
  if (n == 0) return 0;
  int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  if (!queue) return -1;
  for (int32_t v = 0; v < n; v++) label[v] = -1;
  int64_t comps = 0;
  for (int32_t s = 0; s < n; s++) {
    if (label[s] >= 0) continue;
    /* every smaller id is labelled already, so s is its component's minimum */
    comps++;
    label[s] = s;
    int64_t head = 0, tail = 0;
    queue[tail++] = s;
    while (head < tail) {
      const int32_t u = queue[head++];
      for (uint32_t e = off[u]; e < off[u + 1]; e++) {
        const int32_t v = tgt[e];
        if (label[v] < 0) {
          label[v] = s;
          queue[tail++] = v;
        }
      }
    }
  }
  free(queue);
  return comps;
}

/* Low-diameter decomposition rounds (Alg. 6).  C[v] = centre of v's cluster,
 * T[v] = round in which v joined a frontier.  Returns the number of
 * clusters, or -1 on a bad argument / allocation failure. */
int64_t or_ldd(int32_t n, const uint32_t *off, const int32_t *tgt, const double *delta,
               int32_t *C, int32_t *T) {
  if (n < 0) return -1;
  if (n == 0) return 0;
  double dmax = delta[0];
  for (int32_t v = 1; v < n; v++)
    if (delta[v] > dmax) dmax = delta[v];
  /* start round of v: the first round r with Start[v] = dmax - delta[v] < r + 1 */
  int64_t *start = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t *F = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t *F2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int64_t maxs = 0;
  if (!start || !order || !F || !F2) {
    free(start); free(order); free(F); free(F2);
    return -1;
  }
  for (int32_t v = 0; v < n; v++) {
    const double s = floor(dmax - delta[v]);
    start[v] = s < 0 ? 0 : (int64_t)s;
    if (start[v] > maxs) maxs = start[v];
  }
  /* vertices by start round (counting sort; ties by id) */
  int64_t *cnt = (int64_t *)calloc((size_t)maxs + 2, sizeof(int64_t));
  if (!cnt) {
    free(start); free(order); free(F); free(F2);
    return -1;
  }
  for (int32_t v = 0; v < n; v++) cnt[start[v] + 1]++;
  for (int64_t r = 0; r <= maxs; r++) cnt[r + 1] += cnt[r];
  for (int32_t v = 0; v < n; v++) order[cnt[start[v]]++] = v;
  free(cnt);
  for (int32_t v = 0; v < n; v++) C[v] = T[v] = -1;
  int64_t visited = 0, clusters = 0, fs = 0, next = 0;
  for (int64_t r = 0; visited < n; r++) {
    /* vertices whose start round has come and that nothing has reached */
    while (next < n && start[order[next]] <= r) {
      const int32_t v = order[next++];
      if (C[v] < 0) {
        C[v] = v;
        T[v] = (int32_t)r;
        F[fs++] = v;
        visited++;
        clusters++;
      }
    }
    /* edgeMap: the frontier hands its clusters to unclaimed neighbours */
    int64_t fs2 = 0;
    for (int64_t i = 0; i < fs; i++) {
      const int32_t u = F[i];
      for (uint32_t e = off[u]; e < off[u + 1]; e++) {
        const int32_t d = tgt[e];
        if (C[d] < 0) {
          C[d] = C[u];
          T[d] = (int32_t)(r + 1);
          F2[fs2++] = d;
          visited++;
        }
      }
    }
    int32_t *tmp = F;
    F = F2;
    F2 = tmp;
    fs = fs2;
  }
  free(start); free(order); free(F); free(F2);
  return clusters;
}

int64_t or_coreness(int32_t n, const uint32_t *off, const int32_t *tgt, int32_t *core) {
  if (n <= 0) return -1;
  int32_t maxd = 0;
  for (int32_t v = 0; v < n; v++) {
    const int32_t d = (int32_t)(off[v + 1] - off[v]);
    if (d > maxd) maxd = d;
  }
  int32_t *deg = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t *head = (int32_t *)malloc(sizeof(int32_t) * ((size_t)maxd + 1));
  int32_t *nxt = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t *prv = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  char *done = (char *)calloc((size_t)n, 1);
  if (!deg || !head || !nxt || !prv || !done) {
    free(deg); free(head); free(nxt); free(prv); free(done);
    return -1;
  }
  for (int32_t d = 0; d <= maxd; d++) head[d] = -1;
  for (int32_t v = 0; v < n; v++) {
    deg[v] = (int32_t)(off[v + 1] - off[v]);
    prv[v] = -1;
    nxt[v] = head[deg[v]];
    if (head[deg[v]] >= 0) prv[head[deg[v]]] = v;
    head[deg[v]] = v;
  }
  int32_t k = 0, lo = 0;
  for (int32_t removed = 0; removed < n; removed++) {
    while (head[lo] < 0) lo++;
    const int32_t v = head[lo];
    head[lo] = nxt[v];
    if (nxt[v] >= 0) prv[nxt[v]] = -1;
    done[v] = 1;
    if (deg[v] > k) k = deg[v];
    core[v] = k;
    for (uint32_t e = off[v]; e < off[v + 1]; e++) {
      const int32_t u = tgt[e];
      if (done[u] || deg[u] <= lo) continue;  /* never below the current minimum */
      const int32_t d = deg[u];
      /* unlink u from bucket d, relink in d - 1 */
      if (prv[u] >= 0) nxt[prv[u]] = nxt[u];
      else head[d] = nxt[u];
      if (nxt[u] >= 0) prv[nxt[u]] = prv[u];
      deg[u] = d - 1;
      prv[u] = -1;
      nxt[u] = head[d - 1];
      if (head[d - 1] >= 0) prv[head[d - 1]] = u;
      head[d - 1] = u;
    }
  }
  free(deg); free(head); free(nxt); free(prv); free(done);
  return k;
}

/* --------------------------------------------------------- Floyd–Warshall */
/* All-pairs shortest paths by brute force, for tiny graphs only.  d is
 * n*n int64, row-major, INT64_MAX = unreachable.  w == NULL means unit
 * weights (hop distances). */
int or_floyd_warshall(int32_t n, const uint32_t *off, const int32_t *tgt, const uint32_t *w,
                      int64_t *d) {
  if (n <= 0 || n > 4096) return -1;
  for (int64_t i = 0; i < (int64_t)n * n; i++) d[i] = INT64_MAX;
  for (int32_t u = 0; u < n; u++) {
    d[(int64_t)u * n + u] = 0;
    for (uint32_t k = off[u]; k < off[u + 1]; k++) {
      int64_t c = w ? (int64_t)w[k] : 1;
      int64_t *e = &d[(int64_t)u * n + tgt[k]];
      if (c < *e) *e = c;
    }
  }
  for (int32_t k = 0; k < n; k++)
    for (int32_t i = 0; i < n; i++) {
      int64_t dik = d[(int64_t)i * n + k];
      if (dik == INT64_MAX) continue;
      for (int32_t j = 0; j < n; j++) {
        int64_t dkj = d[(int64_t)k * n + j];
        if (dkj == INT64_MAX) continue;
        if (dik + dkj < d[(int64_t)i * n + j]) d[(int64_t)i * n + j] = dik + dkj;
      }
    }
  return 0;
}

/* ------------------------------------------------------------ validators */
static int has_arc(const uint32_t *off, const int32_t *tgt, int32_t u, int32_t v) {
  for (uint32_t k = off[u]; k < off[u + 1]; k++)
    if (tgt[k] == v) return 1;
  return 0;
}

/* Error codes written to *code by the validators. */
enum {
  OR_OK = 0,
  OR_BAD_SOURCE = 1,     /* dist[src] != 0 or parent[src] != src */
  OR_EDGE_GAP = 2,       /* an arc (u,v) with |D[u]-D[v]| > 1 (BFS) or D[v] > D[u]+w (SSSP) */
  OR_REACH_MISMATCH = 3, /* an arc joining a reached and an unreached vertex */
  OR_BAD_PARENT = 4,     /* parent out of range, not adjacent, or D[parent] != D[v]-1 */
  OR_UNREACHED_PARENT = 5, /* unreached vertex with parent != -1 */
  OR_NO_TIGHT_ARC = 6,   /* reached v != src with no arc u->v where D[u]+w == D[v] */
  OR_NEGATIVE = 7        /* a negative distance */
};

/* BFS output invariants: D[src]=0, P[src]=src; for every arc, both ends are
 * reached or neither, and |D[u]-D[v]| <= 1; for reached v != src, P[v] is a
 * neighbour of v with D[P[v]] = D[v]-1; unreached v has P[v] = -1.  Together
 * with D[src]=0 these imply D is exactly the hop distance.  parent may be NULL
 * (distances only).  Returns -1 if all hold, else the first failing vertex
 * (code in *code). */
int64_t or_check_bfs(int32_t n, const uint32_t *off, const int32_t *tgt, int32_t src,
                     const int32_t *dist, const int32_t *parent, int32_t *code) {
  *code = OR_OK;
  if (dist[src] != 0 || (parent && parent[src] != src)) {
    *code = OR_BAD_SOURCE;
    return src;
  }
  for (int32_t v = 0; v < n; v++) {
    int32_t dv = dist[v];
    if (dv < 0) {
      *code = OR_NEGATIVE;
      return v;
    }
    for (uint32_t k = off[v]; k < off[v + 1]; k++) {
      int32_t u = tgt[k];
      int32_t du = dist[u];
      if ((du == OR_INF) != (dv == OR_INF)) {
        *code = OR_REACH_MISMATCH;
        return v;
      }
      if (dv != OR_INF && (du - dv > 1 || dv - du > 1)) {
        *code = OR_EDGE_GAP;
        return v;
      }
    }
    if (v == src) continue;
    if (dv == OR_INF) {
      if (parent && parent[v] != -1) {
        *code = OR_UNREACHED_PARENT;
        return v;
      }
      continue;
    }
    if (parent) {
      int32_t p = parent[v];
      if (p < 0 || p >= n || dist[p] != dv - 1 || !has_arc(off, tgt, v, p)) {
        *code = OR_BAD_PARENT;
        return v;
      }
    } else {
      /* Without parents, some neighbour must be one level closer. */
      int ok = 0;
      for (uint32_t k = off[v]; k < off[v + 1] && !ok; k++)
        if (dist[tgt[k]] == dv - 1) ok = 1;
      if (!ok) {
        *code = OR_NO_TIGHT_ARC;
        return v;
      }
    }
  }
  return -1;
}

/* SSSP output invariants (positive integer weights): D[src]=0; every arc
 * joins two reached or two unreached vertices and satisfies
 * D[v] <= D[u] + w(u,v); every reached v != src has a tight arc
 * D[u] + w(u,v) == D[v].  With positive weights these characterise the
 * shortest-path distances. */
int64_t or_check_sssp(int32_t n, const uint32_t *off, const int32_t *tgt, const uint32_t *w,
                      int32_t src, const int32_t *dist, int32_t *code) {
  *code = OR_OK;
  if (dist[src] != 0) {
    *code = OR_BAD_SOURCE;
    return src;
  }
  for (int32_t v = 0; v < n; v++) {
    int64_t dv = dist[v];
    if (dv < 0) {
      *code = OR_NEGATIVE;
      return v;
    }
    int tight = (v == src);
    for (uint32_t k = off[v]; k < off[v + 1]; k++) {
      int32_t u = tgt[k];
      int64_t du = dist[u];
      if ((du == OR_INF) != (dv == OR_INF)) {
        *code = OR_REACH_MISMATCH;
        return v;
      }
      if (dv == OR_INF) continue;
      if (dv > du + (int64_t)w[k]) {
        *code = OR_EDGE_GAP;
        return v;
      }
      if (du + (int64_t)w[k] == dv) tight = 1;
    }
    if (dv != OR_INF && !tight) {
      *code = OR_NO_TIGHT_ARC;
      return v;
    }
  }
  return -1;
}
