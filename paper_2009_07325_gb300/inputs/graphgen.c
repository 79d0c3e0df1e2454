/*
 * Seeded synthetic graph generators (input fixtures only).
 *
 * These produce the directed graphs on which influence maximisation is run:
 * a directed Erdos-Renyi graph with an exact edge count, R-MAT (Chakrabarti,
 * Zhan, Faloutsos 2004) with per-level quadrant probabilities (a, b, c, d),
 * Chung-Lu power-law graphs, and Barabasi-Albert preferential attachment
 * (the scalability graphs of the paper's Sec. IV-F). Every graph is returned
 * as an in-edge CSR indexed by target vertex: row v lists the sources u of
 * the edges u->v in ascending order, with duplicate edges and self-loops
 * dropped.
 *
 * This file holds no part of the influence-maximisation method. It is used
 * by the tests, the benchmark and the oracle alike, so that both sides read
 * identical bytes. All randomness comes from a counter-based mix of
 * (seed, stream, index) built on the SplitMix64 finaliser (Steele, Lea,
 * Flood, OOPSLA 2014), so results do not depend on the thread count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* One 64-bit draw for (seed, stream, idx); a pure function of its inputs. */
static inline uint64_t gen64(uint64_t seed, uint64_t stream, uint64_t idx) {
  uint64_t s = mix64(seed * 0x9E3779B97F4A7C15ull + stream * 0xD1B54A32D192ED03ull + 0x632BE59BD9B4E019ull);
  return mix64(s + (idx + 1) * 0x9E3779B97F4A7C15ull);
}

static inline uint32_t below(uint64_t r, uint32_t n) {  /* r scaled to [0, n) */
  return (uint32_t)(((unsigned __int128)r * n) >> 64);
}

static inline double unit53(uint64_t r) { return (double)(r >> 11) * 0x1p-53; }

static int cmp_u32(const void *a, const void *b) {
  uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
  return (x > y) - (x < y);
}

/*
 * Builds the deduplicated in-edge CSR of the D directed edges src[i]->dst[i]
 * on n vertices. off receives n+1 offsets; out receives the sources (at most
 * D entries, so out must hold D). Returns the number of edges kept, or -1 if
 * scratch memory could not be allocated.
 */
int64_t gg_build_in_csr(uint32_t n, uint64_t D, const uint32_t *src, const uint32_t *dst,
                        uint64_t *off, uint32_t *out) {
  uint64_t *cur = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
  uint32_t *tmp = (uint32_t *)malloc((D ? D : 1) * sizeof(uint32_t));
  uint64_t *len = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
  if (!cur || !tmp || !len) { free(cur); free(tmp); free(len); return -1; }

#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)D; ++i) __atomic_fetch_add(&cur[dst[i] + 1], 1, __ATOMIC_RELAXED);
  for (uint32_t v = 0; v < n; ++v) cur[v + 1] += cur[v];          /* row starts */
  uint64_t *start = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
  if (!start) { free(cur); free(tmp); free(len); return -1; }
  memcpy(start, cur, ((size_t)n + 1) * sizeof(uint64_t));

#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)D; ++i) {
    uint64_t p = __atomic_fetch_add(&cur[dst[i]], 1, __ATOMIC_RELAXED);
    tmp[p] = src[i];
  }

  /* sort each row, drop duplicates and self-loops (in place) */
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t v = 0; v < (int64_t)n; ++v) {
    uint64_t s = start[v], e = start[v + 1];
    if (e - s > 1) qsort(tmp + s, e - s, sizeof(uint32_t), cmp_u32);
    uint64_t w = s;
    for (uint64_t i = s; i < e; ++i) {
      uint32_t u = tmp[i];
      if (u == (uint32_t)v) continue;
      if (w > s && tmp[w - 1] == u) continue;
      tmp[w++] = u;
    }
    len[v] = w - s;
  }
  off[0] = 0;
  for (uint32_t v = 0; v < n; ++v) off[v + 1] = off[v] + len[v];
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t v = 0; v < (int64_t)n; ++v)
    memcpy(out + off[v], tmp + start[v], len[v] * sizeof(uint32_t));

  int64_t m = (int64_t)off[n];
  free(cur); free(tmp); free(len); free(start);
  return m;
}

/*
 * R-MAT: D recursive quadrant draws on 2^scale vertices. At each of the
 * `scale` levels the (source bit, target bit) pair is (0,0) with probability
 * a, (0,1) with b, (1,0) with c and (1,1) with d = 1-a-b-c, most significant
 * bit first, with no noise and no vertex relabelling. Edge i is src[i]->dst[i].
 */
void gg_rmat_edges(uint32_t scale, uint64_t D, double a, double b, double c, uint64_t seed,
                   uint32_t *src, uint32_t *dst) {
  const double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)D; ++i) {
    uint32_t u = 0, v = 0;
    uint64_t r = 0;
    for (uint32_t l = 0; l < scale; ++l) {
      double x;
      if ((l & 1) == 0) { r = gen64(seed, 1000 + l / 2, (uint64_t)i); x = (double)(r >> 32) * 0x1p-32; }
      else x = (double)(r & 0xFFFFFFFFu) * 0x1p-32;
      uint32_t sb, db;
      if (x < a) { sb = 0; db = 0; }
      else if (x < ab) { sb = 0; db = 1; }
      else if (x < abc) { sb = 1; db = 0; }
      else { sb = 1; db = 1; }
      u = (u << 1) | sb;
      v = (v << 1) | db;
    }
    src[i] = u;
    dst[i] = v;
  }
}

/*
 * Directed Erdos-Renyi graph with exactly m distinct edges and no self-loops:
 * uniform endpoint pairs are drawn in sequence; self-loops and pairs already
 * drawn are skipped until m distinct edges exist. Requires m <= n(n-1).
 * Returns 0, or -1 on bad arguments or allocation failure.
 */
int gg_er_edges(uint32_t n, uint64_t m, uint64_t seed, uint32_t *src, uint32_t *dst) {
  if (n < 2 || m > (uint64_t)n * (n - 1)) return -1;
  uint64_t cap = 16;
  while (cap < 2 * m + 16) cap <<= 1;
  uint64_t *tab = (uint64_t *)malloc(cap * sizeof(uint64_t));
  if (!tab) return -1;
  memset(tab, 0xFF, cap * sizeof(uint64_t));
  uint64_t got = 0;
  for (uint64_t i = 0; got < m; ++i) {
    uint32_t u = below(gen64(seed, 1, i), n), v = below(gen64(seed, 2, i), n);
    if (u == v) continue;
    uint64_t key = (uint64_t)u * n + v, h = mix64(key) & (cap - 1);
    int fresh = 1;
    while (tab[h] != UINT64_MAX) {
      if (tab[h] == key) { fresh = 0; break; }
      h = (h + 1) & (cap - 1);
    }
    if (!fresh) continue;
    tab[h] = key;
    src[got] = u;
    dst[got] = v;
    ++got;
  }
  free(tab);
  return 0;
}

/*
 * Chung-Lu power-law graph: vertex i has weight (i+1)^(-1/(gamma-1)); D
 * (source, target) pairs are drawn with each endpoint chosen with probability
 * proportional to its weight (inverse-CDF search). Returns 0, or -1 on
 * allocation failure.
 */
int gg_chung_lu_edges(uint32_t n, uint64_t D, double gamma, uint64_t seed, uint32_t *src, uint32_t *dst) {
  double *cdf = (double *)malloc((size_t)n * sizeof(double));
  if (!cdf) return -1;
  double acc = 0.0, ex = -1.0 / (gamma - 1.0);
  for (uint32_t i = 0; i < n; ++i) { acc += pow((double)i + 1.0, ex); cdf[i] = acc; }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)D; ++i) {
    for (int side = 0; side < 2; ++side) {
      double x = unit53(gen64(seed, 3 + side, (uint64_t)i)) * acc;
      uint32_t lo = 0, hi = n - 1;            /* first index with cdf > x */
      while (lo < hi) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (cdf[mid] > x) hi = mid; else lo = mid + 1;
      }
      if (side == 0) src[i] = lo; else dst[i] = lo;
    }
  }
  free(cdf);
  return 0;
}

/*
 * Barabasi-Albert preferential attachment (the paper's Sec. IV-F): start from
 * a clique on r0 vertices, then add vertices r0..n-1 one at a time, each
 * joined to r distinct earlier vertices chosen with probability proportional
 * to their current degree. The graph is undirected, so every edge is emitted
 * in both directions. src/dst must hold 2*(r0*(r0-1)/2 + (n-r0)*r) entries.
 * Returns the number of directed edges written, or -1 on bad arguments.
 */
int64_t gg_barabasi_albert_edges(uint32_t n, uint32_t r0, uint32_t r, uint64_t seed,
                                 uint32_t *src, uint32_t *dst) {
  if (r0 < 2 || r < 1 || r > r0 || n < r0) return -1;
  uint64_t ends_cap = (uint64_t)r0 * (r0 - 1) + 2ull * (n - r0) * r;
  uint32_t *ends = (uint32_t *)malloc(ends_cap * sizeof(uint32_t));  /* one entry per edge end */
  uint32_t *pick = (uint32_t *)malloc((size_t)r * sizeof(uint32_t));
  if (!ends || !pick) { free(ends); free(pick); return -1; }
  uint64_t ne = 0, E = 0;
  for (uint32_t i = 0; i < r0; ++i)
    for (uint32_t j = i + 1; j < r0; ++j) {
      src[E] = i; dst[E++] = j; src[E] = j; dst[E++] = i;
      ends[ne++] = i; ends[ne++] = j;
    }
  uint64_t draw = 0;
  for (uint32_t v = r0; v < n; ++v) {
    uint32_t got = 0;
    while (got < r) {
      uint32_t u = ends[(uint64_t)(((unsigned __int128)gen64(seed, 5, draw++) * ne) >> 64)];
      int dup = 0;
      for (uint32_t t = 0; t < got; ++t) dup |= (pick[t] == u);
      if (!dup) pick[got++] = u;
    }
    for (uint32_t t = 0; t < r; ++t) {
      src[E] = v; dst[E++] = pick[t]; src[E] = pick[t]; dst[E++] = v;
      ends[ne++] = v; ends[ne++] = pick[t];
    }
  }
  free(ends); free(pick);
  return (int64_t)E;
}

/* Uniform 64-bit draws for other seeded choices (query mixes, arrival times). */
void gg_u64(uint64_t seed, uint64_t stream, uint64_t count, uint64_t *out) {
  for (uint64_t i = 0; i < count; ++i) out[i] = gen64(seed, stream, i);
}
