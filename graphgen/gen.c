/*
 * graphgen — seeded synthetic graph inputs shared by the tests, the benchmark
 * and the oracle's callers.  It holds none of the traversal arithmetic: it only
 * draws graphs, weights and source vertices.
 *
 * Inputs stand in for the paper's datasets (Table 2 of the experiments
 * section): power-law RMAT graphs for the web/social inputs and a 2D grid for
 * the high-diameter 3D-Torus.  Weights follow the experiments' convention of
 * integers drawn uniformly from a half-open range [lo, hi) (the paper uses
 * [1, log n)), one weight per undirected edge so both arcs agree.
 *
 * Every random draw is a counter-based hash (splitmix64 finaliser) of
 * (seed, counter), so outputs do not depend on the number of threads.
 *
 * Output format: symmetric CSR, vertices 0..n-1, adjacency lists sorted
 * ascending, no self-loops, no duplicate arcs; uint32 offsets (n+1), int32
 * targets (off[n] arcs).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef struct {
  int32_t n;
  uint64_t m;        /* arcs (directed), = off[n] */
  uint32_t *off;     /* n+1 */
  int32_t *tgt;      /* m */
} gg_csr;

/* ------------------------------------------------------------------ hashing */
static inline uint64_t mix64(uint64_t x) {
  x += 0x9e3779b97f4a7c15ULL;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
  return x ^ (x >> 31);
}
static inline uint64_t hash3(uint64_t seed, uint64_t a, uint64_t b) {
  return mix64(mix64(mix64(seed) ^ a) ^ (b * 0xd1b54a32d192ed03ULL));
}
/* uniform integer in [0, k) from 64 random bits (multiply-high). */
static inline uint64_t below(uint64_t r, uint64_t k) {
  return (uint64_t)(((unsigned __int128)r * k) >> 64);
}

/* --------------------------------------------------------------- threading */
typedef void (*range_fn)(void *ctx, uint64_t lo, uint64_t hi);
typedef struct {
  range_fn fn;
  void *ctx;
  uint64_t total, grain;
  uint64_t next; /* atomic */
} pool_job;

static void *pool_worker(void *p) {
  pool_job *j = (pool_job *)p;
  for (;;) {
    uint64_t lo = __atomic_fetch_add(&j->next, j->grain, __ATOMIC_RELAXED);
    if (lo >= j->total) break;
    uint64_t hi = lo + j->grain;
    if (hi > j->total) hi = j->total;
    j->fn(j->ctx, lo, hi);
  }
  return NULL;
}

static int g_threads = 0;
static int nthreads(void) {
  if (g_threads > 0) return g_threads;
  long c = sysconf(_SC_NPROCESSORS_ONLN);
  return c > 0 ? (int)c : 1;
}

/* Run fn over [0,total) in chunks of `grain` with dynamic scheduling. */
static void parallel_for(uint64_t total, uint64_t grain, range_fn fn, void *ctx) {
  pool_job job = {fn, ctx, total, grain ? grain : 1, 0};
  int t = nthreads();
  if (t <= 1 || total <= grain) {
    pool_worker(&job);
    return;
  }
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)t);
  int started = 0;
  for (int i = 0; i < t; i++)
    if (pthread_create(&th[i], NULL, pool_worker, &job) == 0) started++;
    else break;
  if (started == 0) pool_worker(&job);
  for (int i = 0; i < started; i++) pthread_join(th[i], NULL);
  free(th);
}

void gg_set_threads(int t) { g_threads = t; }
int gg_get_threads(void) { return nthreads(); }

/* --------------------------------------------------- arc buffer to CSR */
/* Arcs are gathered into per-vertex buckets sized by a first counting pass,
 * then each bucket is sorted and deduplicated, then compacted. */
typedef struct {
  int32_t n;
  uint32_t *deg;      /* raw degree incl. duplicates (atomic counters) */
  uint64_t *raw_off;  /* n+1 prefix of raw degrees */
  uint64_t *cursor;   /* n fill cursors */
  int32_t *raw;       /* raw arcs */
  uint32_t *ndeg;     /* deduplicated degrees */
} builder;

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

static void sort_small(int32_t *a, uint64_t k) {
  if (k > 48) {
    qsort(a, (size_t)k, sizeof(int32_t), cmp_i32);
    return;
  }
  for (uint64_t i = 1; i < k; i++) {
    int32_t x = a[i];
    uint64_t j = i;
    while (j > 0 && a[j - 1] > x) {
      a[j] = a[j - 1];
      j--;
    }
    a[j] = x;
  }
}

static void sort_dedup_range(void *ctx, uint64_t lo, uint64_t hi) {
  builder *b = (builder *)ctx;
  for (uint64_t v = lo; v < hi; v++) {
    int32_t *a = b->raw + b->raw_off[v];
    uint64_t k = b->raw_off[v + 1] - b->raw_off[v];
    sort_small(a, k);
    uint64_t w = 0;
    for (uint64_t i = 0; i < k; i++)
      if (w == 0 || a[i] != a[w - 1]) a[w++] = a[i];
    b->ndeg[v] = (uint32_t)w;
  }
}

typedef struct {
  builder *b;
  gg_csr *out;
} compact_ctx;

static void compact_range(void *ctx, uint64_t lo, uint64_t hi) {
  compact_ctx *c = (compact_ctx *)ctx;
  for (uint64_t v = lo; v < hi; v++) {
    memcpy(c->out->tgt + c->out->off[v], c->b->raw + c->b->raw_off[v],
           sizeof(int32_t) * c->b->ndeg[v]);
  }
}

/* Returns 0 on success, -1 on allocation failure, -2 if arcs exceed uint32. */
static int finish_builder(builder *b, gg_csr *out) {
  int32_t n = b->n;
  b->ndeg = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  if (!b->ndeg) return -1;
  parallel_for((uint64_t)n, 2048, sort_dedup_range, b);
  out->n = n;
  out->off = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n + 1));
  if (!out->off) return -1;
  uint64_t s = 0;
  for (int32_t v = 0; v < n; v++) {
    out->off[v] = (uint32_t)s;
    s += b->ndeg[v];
    if (s > 0xffffffffULL) return -2;
  }
  out->off[n] = (uint32_t)s;
  out->m = s;
  out->tgt = (int32_t *)malloc(sizeof(int32_t) * (s ? s : 1));
  if (!out->tgt) return -1;
  compact_ctx cc = {b, out};
  parallel_for((uint64_t)n, 4096, compact_range, &cc);
  return 0;
}

static void free_builder(builder *b) {
  free(b->deg);
  free(b->raw_off);
  free(b->cursor);
  free(b->raw);
  free(b->ndeg);
}

/* ------------------------------------------------------------------- RMAT */
typedef struct {
  int scale;
  uint64_t seed;
  uint32_t ta, tab, tabc; /* quadrant thresholds in 2^-32 units */
  int permute;
  uint64_t pk[3], pc[3];
  builder *b;
  int pass; /* 0: count degrees, 1: fill */
} rmat_ctx;

/* Bijective scramble of [0, 2^scale): odd multiplies, additions and
 * xor-shifts, each invertible modulo 2^scale. */
static inline uint32_t scramble(const rmat_ctx *c, uint32_t x) {
  uint64_t mask = (c->scale >= 32) ? 0xffffffffULL : ((1ULL << c->scale) - 1);
  uint64_t y = x;
  int sh = c->scale / 2 + 1;
  for (int r = 0; r < 3; r++) {
    y = (y * c->pk[r]) & mask;
    y = (y + c->pc[r]) & mask;
    y ^= (y >> sh);
  }
  return (uint32_t)y;
}

static inline void rmat_edge(const rmat_ctx *c, uint64_t i, uint32_t *pu, uint32_t *pv) {
  uint64_t st = mix64(c->seed ^ (i * 0x9e3779b97f4a7c15ULL));
  uint32_t u = 0, v = 0;
  uint64_t r = 0;
  for (int l = 0; l < c->scale; l++) {
    uint32_t x;
    if ((l & 1) == 0) {
      st += 0x9e3779b97f4a7c15ULL;
      r = mix64(st);
      x = (uint32_t)r;
    } else {
      x = (uint32_t)(r >> 32);
    }
    uint32_t bit = 1u << (c->scale - 1 - l);
    if (x < c->ta) {
    } else if (x < c->tab) {
      v |= bit;
    } else if (x < c->tabc) {
      u |= bit;
    } else {
      u |= bit;
      v |= bit;
    }
  }
  if (c->permute) {
    u = scramble(c, u);
    v = scramble(c, v);
  }
  *pu = u;
  *pv = v;
}

static void rmat_range(void *ctx, uint64_t lo, uint64_t hi) {
  rmat_ctx *c = (rmat_ctx *)ctx;
  builder *b = c->b;
  for (uint64_t i = lo; i < hi; i++) {
    uint32_t u, v;
    rmat_edge(c, i, &u, &v);
    if (u == v) continue;
    if (c->pass == 0) {
      __atomic_fetch_add(&b->deg[u], 1u, __ATOMIC_RELAXED);
      __atomic_fetch_add(&b->deg[v], 1u, __ATOMIC_RELAXED);
    } else {
      uint64_t pu = __atomic_fetch_add(&b->cursor[u], 1ULL, __ATOMIC_RELAXED);
      uint64_t pv = __atomic_fetch_add(&b->cursor[v], 1ULL, __ATOMIC_RELAXED);
      b->raw[pu] = (int32_t)v;
      b->raw[pv] = (int32_t)u;
    }
  }
}

/*
 * RMAT graph with 2^scale vertices and edgefactor * 2^scale edge draws; each
 * draw descends `scale` quadrant levels with probabilities (a, b, c, 1-a-b-c).
 * Self-loops are dropped, both directions of each draw are stored, duplicates
 * removed.  permute != 0 relabels vertices by a seeded bijection so that hubs
 * are not clustered at low ids.  Returns 0 on success.
 */
int gg_rmat(int scale, int edgefactor, double a, double b, double c, uint64_t seed,
            int permute, gg_csr *out) {
  memset(out, 0, sizeof(*out));
  if (scale < 1 || scale > 30 || edgefactor < 1) return -3;
  int32_t n = (int32_t)(1u << scale);
  rmat_ctx ctx;
  memset(&ctx, 0, sizeof(ctx));
  ctx.scale = scale;
  ctx.seed = mix64(seed ^ 0x5bd1e995ULL);
  ctx.ta = (uint32_t)(a * 4294967296.0);
  ctx.tab = (uint32_t)((a + b) * 4294967296.0);
  double abc = a + b + c;
  ctx.tabc = abc >= 1.0 ? 0xffffffffu : (uint32_t)(abc * 4294967296.0);
  ctx.permute = permute;
  for (int r = 0; r < 3; r++) {
    ctx.pk[r] = mix64(seed * 31 + 7 + (uint64_t)r) | 1ULL;
    ctx.pc[r] = mix64(seed * 37 + 11 + (uint64_t)r);
  }
  builder bl;
  memset(&bl, 0, sizeof(bl));
  bl.n = n;
  ctx.b = &bl;
  uint64_t draws = (uint64_t)edgefactor * (uint64_t)n;
  bl.deg = (uint32_t *)calloc((size_t)n, sizeof(uint32_t));
  bl.raw_off = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)n + 1));
  bl.cursor = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
  if (!bl.deg || !bl.raw_off || !bl.cursor) {
    free_builder(&bl);
    return -1;
  }
  ctx.pass = 0;
  parallel_for(draws, 1 << 16, rmat_range, &ctx);
  uint64_t s = 0;
  for (int32_t v = 0; v < n; v++) {
    bl.raw_off[v] = s;
    bl.cursor[v] = s;
    s += bl.deg[v];
  }
  bl.raw_off[n] = s;
  bl.raw = (int32_t *)malloc(sizeof(int32_t) * (s ? s : 1));
  if (!bl.raw) {
    free_builder(&bl);
    return -1;
  }
  ctx.pass = 1;
  parallel_for(draws, 1 << 16, rmat_range, &ctx);
  int rc = finish_builder(&bl, out);
  free_builder(&bl);
  return rc;
}

/* ------------------------------------------------------------------- grid */
typedef struct {
  int32_t R, C;
  uint64_t seed, thresh;
  gg_csr *out;
  uint32_t *deg;
} grid_ctx;

/* Edge ids: right edge of (r,c) = 2*(r*C+c), down edge = 2*(r*C+c)+1. */
static inline int grid_keep(const grid_ctx *g, uint64_t eid) {
  return hash3(g->seed, eid, 0x67726964ULL) >= g->thresh;
}

static void grid_deg_range(void *ctx, uint64_t lo, uint64_t hi) {
  grid_ctx *g = (grid_ctx *)ctx;
  for (uint64_t id = lo; id < hi; id++) {
    int32_t r = (int32_t)(id / (uint64_t)g->C), c = (int32_t)(id % (uint64_t)g->C);
    uint32_t d = 0;
    if (r > 0 && grid_keep(g, 2 * (id - (uint64_t)g->C) + 1)) d++;
    if (c > 0 && grid_keep(g, 2 * (id - 1))) d++;
    if (c + 1 < g->C && grid_keep(g, 2 * id)) d++;
    if (r + 1 < g->R && grid_keep(g, 2 * id + 1)) d++;
    g->deg[id] = d;
  }
}

static void grid_fill_range(void *ctx, uint64_t lo, uint64_t hi) {
  grid_ctx *g = (grid_ctx *)ctx;
  for (uint64_t id = lo; id < hi; id++) {
    int32_t r = (int32_t)(id / (uint64_t)g->C), c = (int32_t)(id % (uint64_t)g->C);
    int32_t *t = g->out->tgt + g->out->off[id];
    if (r > 0 && grid_keep(g, 2 * (id - (uint64_t)g->C) + 1)) *t++ = (int32_t)(id - (uint64_t)g->C);
    if (c > 0 && grid_keep(g, 2 * (id - 1))) *t++ = (int32_t)(id - 1);
    if (c + 1 < g->C && grid_keep(g, 2 * id)) *t++ = (int32_t)(id + 1);
    if (r + 1 < g->R && grid_keep(g, 2 * id + 1)) *t++ = (int32_t)(id + (uint64_t)g->C);
  }
}

/* R x C 4-neighbour grid, vertex id r*C+c, each undirected edge deleted
 * independently with probability delete_frac (seeded). */
int gg_grid(int32_t R, int32_t C, double delete_frac, uint64_t seed, gg_csr *out) {
  memset(out, 0, sizeof(*out));
  if (R < 1 || C < 1 || (int64_t)R * C > 0x7fffffffLL) return -3;
  int32_t n = R * C;
  grid_ctx g;
  g.R = R;
  g.C = C;
  g.seed = seed;
  g.thresh = delete_frac <= 0 ? 0 : (delete_frac >= 1 ? ~0ULL : (uint64_t)(delete_frac * 18446744073709551616.0));
  g.out = out;
  g.deg = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  out->off = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n + 1));
  if (!g.deg || !out->off) {
    free(g.deg);
    return -1;
  }
  parallel_for((uint64_t)n, 1 << 14, grid_deg_range, &g);
  uint64_t s = 0;
  for (int32_t v = 0; v < n; v++) {
    out->off[v] = (uint32_t)s;
    s += g.deg[v];
  }
  out->off[n] = (uint32_t)s;
  out->n = n;
  out->m = s;
  out->tgt = (int32_t *)malloc(sizeof(int32_t) * (s ? s : 1));
  if (!out->tgt) {
    free(g.deg);
    return -1;
  }
  parallel_for((uint64_t)n, 1 << 14, grid_fill_range, &g);
  free(g.deg);
  return 0;
}

/* Release one array handed out by gg_rmat / gg_grid. */
void gg_release(void *p) { free(p); }

void gg_free(gg_csr *g) {
  free(g->off);
  free(g->tgt);
  memset(g, 0, sizeof(*g));
}

/* ---------------------------------------------------------------- weights */
typedef struct {
  const uint32_t *off;
  const int32_t *tgt;
  uint32_t *w;
  uint64_t seed;
  uint32_t lo, span;
} wctx;

static void weight_range(void *ctx, uint64_t lo, uint64_t hi) {
  wctx *c = (wctx *)ctx;
  for (uint64_t u = lo; u < hi; u++) {
    for (uint64_t k = c->off[u]; k < c->off[u + 1]; k++) {
      uint64_t v = (uint64_t)(uint32_t)c->tgt[k];
      uint64_t a = u < v ? u : v, b = u < v ? v : u;
      c->w[k] = c->lo + (uint32_t)below(hash3(c->seed, a, b), c->span);
    }
  }
}

/* w[k] for arc k=(u,v): uniform integer in [lo, hi), a function of the
 * unordered pair {u,v} so both directions carry the same weight. */
int gg_weights(int32_t n, const uint32_t *off, const int32_t *tgt, uint32_t lo, uint32_t hi,
               uint64_t seed, uint32_t *w) {
  if (hi <= lo) return -3;
  wctx c = {off, tgt, w, mix64(seed ^ 0x77656967ULL), lo, hi - lo};
  parallel_for((uint64_t)n, 4096, weight_range, &c);
  return 0;
}

/* ---------------------------------------------------------------- sources */
/* k seeded sources, each uniform over the vertices with degree > 0
 * (redrawn until one is found). Returns the number written (0 if the graph
 * has no arcs). */
int gg_sources(int32_t n, const uint32_t *off, uint64_t seed, int32_t k, int32_t *out) {
  if (n <= 0 || off[n] == 0) return 0;
  for (int32_t i = 0; i < k; i++) {
    for (uint64_t j = 0;; j++) {
      uint64_t v = below(hash3(seed, (uint64_t)i, j), (uint64_t)n);
      if (off[v + 1] > off[v]) {
        out[i] = (int32_t)v;
        break;
      }
    }
  }
  return k;
}

/* Highest-degree vertex, ties broken by the lowest id. */
int32_t gg_max_degree_vertex(int32_t n, const uint32_t *off) {
  int32_t best = 0;
  uint32_t bd = 0;
  for (int32_t v = 0; v < n; v++) {
    uint32_t d = off[v + 1] - off[v];
    if (d > bd) {
      bd = d;
      best = v;
    }
  }
  return best;
}
