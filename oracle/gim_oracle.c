/*
 * CPU ORACLE for IMM on RR sets (gIM, Shahrouz, Salehkaleybar, Hashemi,
 * IEEE TPDS; arXiv 2009.07325).
 *
 * TEST INFRASTRUCTURE ONLY. This file is a plain, slow, sequential statement
 * of what the GPU path computes. Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may build, load or run it; the library path
 * never does. It shares no code, header, table or helper with the CUDA
 * sources: its Philox, its LT thresholds, its BFS, its greedy and its IMM
 * driver are written here from the paper and the published definitions.
 *
 * Readings of points the paper leaves open (each one also holds for the GPU):
 *  - Randomness: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with key
 *    (seed_lo, seed_hi) and counter (idx, tag, j_lo, j_hi) for RR set j.
 *    tag 0 = root draw (idx 0, 64-bit word w1:w0, root = high half of
 *    word * n); tag 1 = IC coin of in-edge e (idx e/4, word e%4);
 *    tag 2 = LT draw at vertex x (idx x, word 0).
 *  - IC coin: edge e is live iff float(word >> 8) * 2^-24 < w[e] (fp32);
 *    for w[e] <= 2^-8 the 24-bit uniform is drawn as a zero-test byte (16
 *    per draw) and a 16-bit residual (see orc_ic_live).
 *  - LT thresholds: cum[e_i] = min(2^32, llround(P_i * 2^32)) with P_i the
 *    fp64 running sum of the row's weights in CSR order; a row whose total
 *    is within 1e-6 of 1 has its last threshold set to 2^32.
 *  - The root is marked visited (Alg. 3 omits it; Sec. III-A forbids
 *    expanding a vertex twice). Visited state is fresh for every RR set.
 *  - Greedy ties go to the lowest vertex id; once every RR set is covered
 *    the greedy keeps taking the lowest unselected id with gain 0.
 *  - IMM's f, lambda and ell come from Tang, Shi, Xiao (SIGMOD 2015); the
 *    paper defers to that work (Sec. II-E, Alg. 2). Sampling stops once
 *    |R| >= ceil(theta) (Alg. 2 and Alg. 6 print the loop condition
 *    inverted). RR sets drawn during the lower-bound search are reused.
 *  - Multi-round IM (Sec. IV-H): round t of multi-round RR set j uses
 *    rr_id t * 2^32 + j with the root of RR set j; elements t * n + v; the
 *    greedy picks k per round; the constants use T ln C(n, k) and the
 *    partition-matroid guarantee 1/2 (Sun et al.'s own rules are not in
 *    the paper; that choice of N_S and ratio is a reading).
 *
 * Pins: everything here is pinned by the CPU tests against exhaustive
 * enumeration, brute force, library routines and invariants. The IMM
 * constants (ell', lambda', lambda*) are pinned by the concentration
 * bounds they are derived from in IMM's analysis: each tail bound, at the
 * constants' sample sizes, comes out at exactly its failure-probability
 * target, and the error budget eps is spent exactly; the same conditions
 * pin the multi-round constants under the reading above.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, as defined by Salmon et al. (SC'11): ten rounds of two     */
/* 32x32->64 multiplies with a Weyl-sequence key bump after each round.     */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(prod1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)prod1;
    uint32_t n2 = (uint32_t)(prod0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)prod0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw4(uint64_t seed, uint64_t j, uint32_t tag, uint32_t idx, uint32_t out[4]) {
  uint32_t ctr[4] = {idx, tag, (uint32_t)j, (uint32_t)(j >> 32)};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}

/* randSelect(V) of Alg. 3: a uniform root for RR set j. */
uint32_t orc_root(uint64_t seed, uint64_t j, uint32_t n) {
  uint32_t w[4];
  draw4(seed, j, 0, 0, w);
  uint64_t r = ((uint64_t)w[1] << 32) | w[0];
  return (uint32_t)(((unsigned __int128)r * n) >> 64);
}

/*
 * The coin of Alg. 3 ("p = U(0,1)", "p < p_uv") for in-edge e of RR set j.
 * Edges with p > 2^-8: u = word (e mod 4) of draw (tag 1, idx e/4), reduced
 * to its top 24 bits, live iff u 2^-24 < p. Edges with p <= 2^-8 draw the
 * same 24-bit uniform in two independent parts: its top 8 bits are byte
 * (e mod 16) of draw (tag 1, idx 2^31 + e/16) and must be zero (otherwise
 * u >= 2^-8 >= p), and its low 16 bits h are half-word (e mod 8) of draw
 * (tag 1, idx 2^30 + e/8); then live iff h 2^-24 < p. Both give
 * Pr[live] = ceil(p 2^24) / 2^24, independently per edge; the second form
 * spends one draw per 16 edges where almost every edge is dead. The three
 * idx ranges are disjoint for e < 2^32.
 */
int orc_ic_live(uint64_t seed, uint64_t j, uint64_t e, float p) {
  uint32_t w[4];
  if (p > 0x1p-8f) {
    draw4(seed, j, 1, (uint32_t)(e >> 2), w);
    uint32_t word = w[e & 3];
    float u = (float)(word >> 8) * 0x1p-24f;
    return u < p;
  }
  draw4(seed, j, 1, 0x80000000u | (uint32_t)(e >> 4), w);
  const uint32_t top = (w[(e >> 2) & 3] >> (8 * (e & 3))) & 0xFFu;
  if (top != 0) return 0;
  draw4(seed, j, 1, 0x40000000u | (uint32_t)(e >> 3), w);
  const uint32_t h = (w[(e >> 1) & 3] >> (16 * (e & 1))) & 0xFFFFu;
  return (float)h * 0x1p-24f < p;
}

/* The single uniform drawn at vertex x of an LT walk (Sec. III-G). */
uint32_t orc_lt_draw(uint64_t seed, uint64_t j, uint32_t x) {
  uint32_t w[4];
  draw4(seed, j, 2, x, w);
  return w[0];
}

/* ------------------------------------------------------------------------ */
/* Oracle state: a graph (in-edge CSR) plus the RR collection R in rr_id     */
/* order, members sorted within each set.                                   */
/* ------------------------------------------------------------------------ */
typedef struct orc {
  uint32_t n;
  uint64_t m;
  uint64_t *off;       /* n+1 */
  uint32_t *src;       /* m   */
  float *w;            /* m   */
  uint64_t *cum;       /* m, LT thresholds */
  int lt_ok;           /* every row sum <= 1 + 1e-6 */
  /* RR collection */
  int model;           /* -1 while empty */
  uint64_t seed;
  uint64_t count;      /* |R| */
  uint64_t ctr_base;   /* RR set at position j is drawn with rr_id ctr_base + j (0 except in a fresh final phase) */
  uint32_t rounds;     /* T: 1 for IM; T > 1 for multi-round IM, whose elements are t*n + v */
  uint64_t cap_sets, cap_members;
  uint64_t *rr_off;    /* count+1 */
  uint32_t *members;   /* rr_off[count] */
} orc;

/*
 * LT cumulative thresholds for every row (Sec. III-G: the scan over in-edge
 * weights whose consecutive outputs bracket the uniform draw), in 2^-32
 * units so that the bracket test is an exact integer compare.
 */
static void lt_thresholds(const orc *g, uint64_t *cum, int *lt_ok) {
  int ok = 1;
  for (uint32_t v = 0; v < g->n; ++v) {
    double P = 0.0;
    for (uint64_t e = g->off[v]; e < g->off[v + 1]; ++e) {
      P += (double)g->w[e];
      long long c = llround(P * 4294967296.0);
      if (c > 4294967296LL) c = 4294967296LL;
      if (c < 0) c = 0;
      cum[e] = (uint64_t)c;
    }
    if (g->off[v + 1] > g->off[v] && fabs(P - 1.0) <= 1e-6) cum[g->off[v + 1] - 1] = 4294967296ull;
    if (P > 1.0 + 1e-6) ok = 0;
  }
  *lt_ok = ok;
}

orc *orc_create(uint32_t n, uint64_t m, const uint64_t *off, const uint32_t *src, const float *w) {
  orc *g = (orc *)calloc(1, sizeof(orc));
  if (!g) return NULL;
  g->n = n;
  g->m = m;
  g->off = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
  g->src = (uint32_t *)malloc((m ? m : 1) * sizeof(uint32_t));
  g->w = (float *)malloc((m ? m : 1) * sizeof(float));
  g->cum = (uint64_t *)malloc((m ? m : 1) * sizeof(uint64_t));
  g->cap_sets = 1024;
  g->rr_off = (uint64_t *)calloc(g->cap_sets + 1, sizeof(uint64_t));
  g->cap_members = 1 << 16;
  g->members = (uint32_t *)malloc(g->cap_members * sizeof(uint32_t));
  if (!g->off || !g->src || !g->w || !g->cum || !g->rr_off || !g->members) {
    free(g->off); free(g->src); free(g->w); free(g->cum); free(g->rr_off); free(g->members); free(g);
    return NULL;
  }
  memcpy(g->off, off, ((size_t)n + 1) * sizeof(uint64_t));
  if (m) { memcpy(g->src, src, m * sizeof(uint32_t)); memcpy(g->w, w, m * sizeof(float)); }
  lt_thresholds(g, g->cum, &g->lt_ok);
  g->model = -1;
  g->rounds = 1;
  return g;
}

void orc_destroy(orc *g) {
  if (!g) return;
  free(g->off); free(g->src); free(g->w); free(g->cum); free(g->rr_off); free(g->members); free(g);
}

int orc_lt_valid(const orc *g) { return g->lt_ok; }
void orc_lt_export(const orc *g, uint64_t *cum) { memcpy(cum, g->cum, g->m * sizeof(uint64_t)); }

static int cmp_u32(const void *a, const void *b) {
  uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
  return (x > y) - (x < y);
}

/*
 * IC RR set j (Sec. II-E definition; Alg. 3): every vertex u from which the
 * root can be reached along live edges. A FIFO reverse BFS over in-edges
 * expands each vertex once and flips each in-edge's coin once. `visited`
 * (n bytes, all zero on entry and on return) and `out` (n entries) are
 * caller scratch. Returns |RR_j|; out holds the members in ascending order.
 */
static uint32_t rr_ic_from(const orc *g, uint64_t seed, uint32_t root, uint64_t j, uint8_t *visited,
                           uint32_t *out) {
  uint32_t head = 0, tail = 0;
  out[tail++] = root;
  visited[root] = 1;
  while (head < tail) {
    uint32_t v = out[head++];
    for (uint64_t e = g->off[v]; e < g->off[v + 1]; ++e) {
      uint32_t u = g->src[e];
      if (visited[u]) continue;            /* the coin of e does not matter then */
      if (orc_ic_live(seed, j, e, g->w[e])) {
        visited[u] = 1;
        out[tail++] = u;
      }
    }
  }
  for (uint32_t i = 0; i < tail; ++i) visited[out[i]] = 0;
  qsort(out, tail, sizeof(uint32_t), cmp_u32);
  return tail;
}

static uint32_t rr_ic(const orc *g, uint64_t seed, uint64_t j, uint8_t *visited, uint32_t *out) {
  return rr_ic_from(g, seed, orc_root(seed, j, g->n), j, visited, out);
}

/*
 * LT RR set j (Sec. III-G): at each vertex one uniform draw selects at most
 * one live in-edge (the edge whose threshold interval contains the draw);
 * the walk moves to its source and stops when no edge is selected or the
 * source was already visited. Same scratch contract as rr_ic.
 */
static uint32_t rr_lt_from(const orc *g, uint64_t seed, uint32_t root, uint64_t j, uint8_t *visited,
                           uint32_t *out) {
  uint32_t x = root;
  uint32_t size = 0;
  out[size++] = x;
  visited[x] = 1;
  for (;;) {
    uint32_t U = orc_lt_draw(seed, j, x);
    uint64_t chosen = UINT64_MAX;
    for (uint64_t e = g->off[x]; e < g->off[x + 1]; ++e)
      if ((uint64_t)U < g->cum[e]) { chosen = e; break; }
    if (chosen == UINT64_MAX) break;
    uint32_t u = g->src[chosen];
    if (visited[u]) break;
    visited[u] = 1;
    out[size++] = u;
    x = u;
  }
  for (uint32_t i = 0; i < size; ++i) visited[out[i]] = 0;
  qsort(out, size, sizeof(uint32_t), cmp_u32);
  return size;
}

static uint32_t rr_lt(const orc *g, uint64_t seed, uint64_t j, uint8_t *visited, uint32_t *out) {
  return rr_lt_from(g, seed, orc_root(seed, j, g->n), j, visited, out);
}

/*
 * Multi-round RR set j (Sec. IV-H, CR-NAIMM of Sun et al.): one root, drawn as
 * for RR set j, and T independent reverse traversals from it, round t in the
 * live-edge world of rr_id t * 2^32 + j (round 0 is RR set j itself). The
 * elements are (vertex, round) pairs, numbered t * n + v; out (T * n entries)
 * receives them in ascending order (round-major, then vertex).
 */
static uint32_t rr_multi(const orc *g, int model, uint64_t seed, uint64_t j, uint32_t T, uint8_t *visited,
                         uint32_t *out) {
  const uint32_t root = orc_root(seed, j, g->n);
  uint32_t size = 0;
  for (uint32_t t = 0; t < T; ++t) {
    const uint64_t id = ((uint64_t)t << 32) | j;
    const uint32_t s = model == 0 ? rr_ic_from(g, seed, root, id, visited, out + size)
                                  : rr_lt_from(g, seed, root, id, visited, out + size);
    for (uint32_t i = 0; i < s; ++i) out[size + i] += t * g->n;
    size += s;
  }
  return size;
}

/* One multi-round RR set on its own (T * n entries of out). */
int64_t orc_mrim_one(const orc *g, int model, uint32_t T, uint64_t seed, uint64_t j, uint32_t *out) {
  if ((model == 1 && !g->lt_ok) || T < 1 || j >= (1ull << 32)) return -1;
  uint8_t *visited = (uint8_t *)calloc(g->n, 1);
  if (!visited) return -2;
  uint32_t s = rr_multi(g, model, seed, j, T, visited, out);
  free(visited);
  return s;
}

/* One RR set, computed on its own (used for sampled parity at full size). */
int64_t orc_rr_one(const orc *g, int model, uint64_t seed, uint64_t j, uint32_t *out) {
  if (model == 1 && !g->lt_ok) return -1;
  uint8_t *visited = (uint8_t *)calloc(g->n, 1);
  if (!visited) return -2;
  uint32_t s = model == 0 ? rr_ic(g, seed, j, visited, out) : rr_lt(g, seed, j, visited, out);
  free(visited);
  return s;
}

static int grow_sets(orc *g, uint64_t need) {
  if (need <= g->cap_sets) return 0;
  uint64_t c = g->cap_sets;
  while (c < need) c *= 2;
  uint64_t *p = (uint64_t *)realloc(g->rr_off, (c + 1) * sizeof(uint64_t));
  if (!p) return -1;
  g->rr_off = p;
  g->cap_sets = c;
  return 0;
}

static int grow_members(orc *g, uint64_t need) {
  if (need <= g->cap_members) return 0;
  uint64_t c = g->cap_members;
  while (c < need) c *= 2;
  uint32_t *p = (uint32_t *)realloc(g->members, c * sizeof(uint32_t));
  if (!p) return -1;
  g->members = p;
  g->cap_members = c;
  return 0;
}

typedef struct { uint64_t n_sets, n_members, cap; uint32_t *mem; uint32_t *sizes; } chunk_buf;

/*
 * Appends RR sets |R| .. |R|+count-1 to R (the sampling steps of Alg. 1 and Alg. 2).
 * With threads > 1 the rr_id range is split into contiguous chunks, one per
 * thread, and the chunks are concatenated in order, so R is the same as with
 * one thread. Returns 0, -1 (model/seed differ from the stored collection,
 * or LT on a graph whose rows sum above 1) or -2 (out of memory).
 */
int orc_sample(orc *g, int model, uint64_t seed, uint64_t count, int threads) {
  if (g->count > 0 && (g->model != model || g->seed != seed)) return -1;
  if (g->rounds > 1 && (g->ctr_base != 0 || g->count + count > (1ull << 32))) return -1;
  if (model == 1 && !g->lt_ok) return -1;
  if (count == 0) return 0;
  g->model = model;
  g->seed = seed;
  if (threads < 1) threads = 1;
  if ((uint64_t)threads > count) threads = (int)count;
  uint64_t j0 = g->count;
  chunk_buf *cb = (chunk_buf *)calloc((size_t)threads, sizeof(chunk_buf));
  if (!cb) return -2;
  int fail = 0;
#pragma omp parallel for num_threads(threads) schedule(static, 1)
  for (int t = 0; t < threads; ++t) {
    uint64_t a = j0 + count * (uint64_t)t / (uint64_t)threads;
    uint64_t b = j0 + count * (uint64_t)(t + 1) / (uint64_t)threads;
    uint8_t *visited = (uint8_t *)calloc(g->n, 1);
    uint32_t *out = (uint32_t *)malloc((size_t)g->n * g->rounds * sizeof(uint32_t));
    chunk_buf *c = &cb[t];
    c->cap = 1 << 16;
    c->mem = (uint32_t *)malloc(c->cap * sizeof(uint32_t));
    c->sizes = (uint32_t *)malloc((b - a) * sizeof(uint32_t) + 4);
    if (!visited || !out || !c->mem || !c->sizes) { fail = 1; }
    for (uint64_t j = a; j < b && !fail; ++j) {
      const uint64_t id = g->ctr_base + j;
      uint32_t s = g->rounds > 1 ? rr_multi(g, model, seed, j, g->rounds, visited, out)
                   : model == 0  ? rr_ic(g, seed, id, visited, out)
                                 : rr_lt(g, seed, id, visited, out);
      if (c->n_members + s > c->cap) {
        uint64_t nc = c->cap;
        while (nc < c->n_members + s) nc *= 2;
        uint32_t *p = (uint32_t *)realloc(c->mem, nc * sizeof(uint32_t));
        if (!p) { fail = 1; break; }
        c->mem = p;
        c->cap = nc;
      }
      memcpy(c->mem + c->n_members, out, (size_t)s * sizeof(uint32_t));
      c->n_members += s;
      c->sizes[c->n_sets++] = s;
    }
    free(visited);
    free(out);
  }
  uint64_t add_members = 0;
  for (int t = 0; t < threads; ++t) add_members += cb[t].n_members;
  if (!fail && (grow_sets(g, g->count + count) || grow_members(g, g->rr_off[g->count] + add_members))) fail = 2;
  if (!fail) {
    for (int t = 0; t < threads; ++t) {
      uint64_t base = g->rr_off[g->count];
      memcpy(g->members + base, cb[t].mem, cb[t].n_members * sizeof(uint32_t));
      for (uint64_t i = 0; i < cb[t].n_sets; ++i) {
        g->rr_off[g->count + 1] = g->rr_off[g->count] + cb[t].sizes[i];
        g->count++;
      }
    }
  }
  for (int t = 0; t < threads; ++t) { free(cb[t].mem); free(cb[t].sizes); }
  free(cb);
  return fail ? -2 : 0;
}

/*
 * Replaces R with a caller-built collection (tests of the greedy on
 * hand-made set systems): count sets, offsets[count+1], members[offsets[count]].
 * Returns 0, -1 (a member >= n) or -2 (out of memory).
 */
int orc_load_collection(orc *g, uint64_t count, const uint64_t *offsets, const uint32_t *members) {
  const uint64_t universe = (uint64_t)g->n * g->rounds;
  for (uint64_t z = 0; z < offsets[count]; ++z)
    if (members[z] >= universe) return -1;
  if (grow_sets(g, count) || grow_members(g, offsets[count])) return -2;
  memcpy(g->rr_off, offsets, (count + 1) * sizeof(uint64_t));
  memcpy(g->members, members, offsets[count] * sizeof(uint32_t));
  g->count = count;
  g->ctr_base = 0;
  g->model = -2;
  g->seed = 0;
  return 0;
}

void orc_reset(orc *g) { g->count = 0; g->rr_off[0] = 0; g->model = -1; g->ctr_base = 0; g->rounds = 1; }

/* Sets T for an empty collection (multi-round sets, or a multi-round collection to load). */
int orc_set_rounds(orc *g, uint32_t T) {
  if (g->count != 0 || T < 1 || (uint64_t)g->n * T >= 0xFFFFFFFFull) return -1;
  g->rounds = T;
  return 0;
}
uint32_t orc_rounds(const orc *g) { return g->rounds; }
uint64_t orc_rr_count(const orc *g) { return g->count; }
uint64_t orc_store_size(const orc *g) { return g->rr_off[g->count]; }

void orc_export(const orc *g, uint64_t *offsets, uint32_t *members) {
  memcpy(offsets, g->rr_off, (g->count + 1) * sizeof(uint64_t));
  memcpy(members, g->members, g->rr_off[g->count] * sizeof(uint32_t));
}

/* Occur of Sec. III-B: the number of RR sets each vertex belongs to. */
void orc_counts(const orc *g, uint32_t *cnt) {
  memset(cnt, 0, (size_t)g->n * g->rounds * sizeof(uint32_t));
  for (uint64_t z = 0; z < g->rr_off[g->count]; ++z) cnt[g->members[z]]++;
}

/*
 * Greedy maximum coverage over R (the maximum-coverage step of Alg. 1; Sec. III-H): k times,
 * take the unselected vertex that lies in the most uncovered RR sets (lowest
 * id on ties), record that number as its marginal gain, and remove every RR
 * set containing it, lowering the counts of all their members. The sets that
 * contain a vertex are found through a per-vertex list of set ids built
 * once up front. Returns the number of covered RR sets, or -1 on allocation
 * failure / k out of range.
 *
 * With T = rounds > 1 (multi-round IM, Sec. IV-H) the elements are the T*n
 * (vertex, round) pairs and the seed sets are constrained to k per round (a
 * partition matroid): k*T picks, each the best element among the rounds that
 * still have fewer than k seeds, the same tie rule. seeds/gains hold k*T
 * entries in pick order.
 */
int64_t orc_greedy(const orc *g, uint32_t k, uint32_t *seeds, uint32_t *gains) {
  const uint32_t n = g->n, T = g->rounds;
  const uint64_t U = (uint64_t)n * T;
  const uint64_t R = g->count, Z = g->rr_off[R];
  if (k < 1 || k > n) return -1;
  uint32_t *cnt = (uint32_t *)calloc(U, sizeof(uint32_t));
  uint64_t *lst_off = (uint64_t *)calloc((size_t)U + 1, sizeof(uint64_t));
  uint64_t *fill = (uint64_t *)malloc(((size_t)U + 1) * sizeof(uint64_t));
  uint64_t *lst = (uint64_t *)malloc((Z ? Z : 1) * sizeof(uint64_t));
  uint8_t *covered = (uint8_t *)calloc(R ? R : 1, 1);
  uint8_t *selected = (uint8_t *)calloc(U, 1);
  uint32_t *per_round = (uint32_t *)calloc(T, sizeof(uint32_t));
  if (!cnt || !lst_off || !fill || !lst || !covered || !selected || !per_round) {
    free(cnt); free(lst_off); free(fill); free(lst); free(covered); free(selected); free(per_round);
    return -1;
  }
  for (uint64_t z = 0; z < Z; ++z) cnt[g->members[z]]++;
  for (uint64_t x = 0; x < U; ++x) lst_off[x + 1] = lst_off[x] + cnt[x];
  memcpy(fill, lst_off, ((size_t)U + 1) * sizeof(uint64_t));
  for (uint64_t j = 0; j < R; ++j)
    for (uint64_t z = g->rr_off[j]; z < g->rr_off[j + 1]; ++z) lst[fill[g->members[z]]++] = j;

  int64_t n_covered = 0;
  for (uint32_t t = 0; t < k * T; ++t) {
    uint64_t best = UINT64_MAX;
    for (uint64_t x = 0; x < U; ++x) {
      if (selected[x] || per_round[x / n] == k) continue;
      if (best == UINT64_MAX || cnt[x] > cnt[best]) best = x;
    }
    seeds[t] = (uint32_t)best;
    if (gains) gains[t] = cnt[best];
    selected[best] = 1;
    per_round[best / n]++;
    for (uint64_t i = lst_off[best]; i < lst_off[best + 1]; ++i) {
      uint64_t j = lst[i];
      if (covered[j]) continue;
      covered[j] = 1;
      n_covered++;
      for (uint64_t z = g->rr_off[j]; z < g->rr_off[j + 1]; ++z) cnt[g->members[z]]--;
    }
  }
  free(cnt); free(lst_off); free(fill); free(lst); free(covered); free(selected); free(per_round);
  return n_covered;
}

/* ------------------------------------------------------------------------ */
/* IMM (Tang, Shi, Xiao 2015), the algorithm gIM runs (Alg. 1, Alg. 2).     */
/* ------------------------------------------------------------------------ */

/* ln C(n, k) as a fixed-order sum, i = 0..k-1 of ln(n-i) - ln(i+1). */
double orc_log_binom(uint32_t n, uint32_t k) {
  double s = 0.0;
  for (uint32_t i = 0; i < k; ++i) s += log((double)(n - i)) - log((double)(i + 1));
  return s;
}

/*
 * The IMM constants for (n, k, eps, ell): out = {ell', eps', lambda',
 * lambda*, i_max}. ell' = ell (1 + ln2 / ln n) gives success probability
 * 1 - 1/n^ell; eps' = sqrt(2) eps is the (1 + sqrt(2) eps) of Alg. 2.
 */
/*
 * The same constants for multi-round IM with T rounds of k seeds (CR-NAIMM,
 * Sec. IV-H). The paper leaves them to Sun et al.; reading: the number of
 * feasible seed sets is C(n, k)^T, so ln C(n, k) becomes T ln C(n, k), and the
 * greedy's guarantee over the partition matroid is 1/2, which takes the place
 * of 1 - 1/e in lambda* (alpha, beta). With T = 1 they are IMM's constants
 * exactly. The estimate stays n F_R(S): one root per set, drawn over V.
 */
void orc_mrim_constants(uint32_t n, uint32_t k, uint32_t T, double eps, double ell, double out[5]) {
  const double ln_n = log((double)n);
  const double ellp = ell * (1.0 + log(2.0) / ln_n);
  const double epsp = sqrt(2.0) * eps;
  const double lnC = (double)T * orc_log_binom(n, k);
  const double lam_prime = (2.0 + 2.0 * epsp / 3.0) * (lnC + ellp * ln_n + log(log2((double)n))) * (double)n /
                           (epsp * epsp);
  const double gamma = T == 1 ? 1.0 - exp(-1.0) : 0.5;
  const double alpha = sqrt(ellp * ln_n + log(2.0));
  const double beta = sqrt(gamma * (lnC + ellp * ln_n + log(2.0)));
  const double t = gamma * alpha + beta;
  const double lam_star = 2.0 * (double)n * t * t / (eps * eps);
  int lg = 0;
  while (((uint64_t)n >> (lg + 1)) != 0) lg++; /* floor(log2 n), shift kept below 64 bits */
  out[0] = ellp; out[1] = epsp; out[2] = lam_prime; out[3] = lam_star; out[4] = (double)(lg - 1);
}

void orc_imm_constants(uint32_t n, uint32_t k, double eps, double ell, double out[5]) {
  orc_mrim_constants(n, k, 1, eps, ell, out);
}

/*
 * IMM end to end: the lower-bound search of Alg. 2 (x = n/2^i, theta_i =
 * ceil(lambda'/x), sample until |R| >= theta_i, greedy, test
 * n F_R(S) >= (1 + eps') x), then theta = ceil(lambda* / LB), sample until
 * |R| >= theta and return the greedy seeds over R (Alg. 1). The store must
 * start empty. trace (nullable, 4 doubles per lower-bound round, at most
 * 64 rounds): {x, theta_i, covered, |R|}. Returns the number of lower-bound
 * rounds, or a negative error.
 */
/*
 * "Sample until |R| >= target": draw fresh sets (avail == 0), or, when the
 * collection was preloaded with avail sets, expose its first target sets.
 */
static int grow_to(orc *g, int model, uint64_t seed, int threads, uint64_t avail, uint64_t target) {
  if (g->count >= target) return 0;
  if (!avail) return orc_sample(g, model, seed, target - g->count, threads);
  if (target > avail) return -4;
  g->count = target;
  return 0;
}

static int imm_core(orc *g, int model, uint32_t k, double eps, double ell, uint64_t seed, int threads,
                    uint64_t avail, int fresh, uint32_t *seeds, uint64_t *theta_out, double *lb_out,
                    double *trace) {
  double c[5];
  orc_mrim_constants(g->n, k, g->rounds, eps, ell, c);
  const double epsp = c[1], lam_prime = c[2], lam_star = c[3];
  const int i_max = (int)c[4];
  double LB = 1.0;
  int rounds = 0;
  for (int i = 1; i <= i_max; ++i) {
    const double x = (double)g->n / ldexp(1.0, i);
    const uint64_t theta_i = (uint64_t)ceil(lam_prime / x);
    int rc = grow_to(g, model, seed, threads, avail, theta_i);
    if (rc) return rc;
    int64_t cov = orc_greedy(g, k, seeds, NULL);
    if (cov < 0) return -2;
    if (trace && rounds < 64) {
      trace[4 * rounds + 0] = x;
      trace[4 * rounds + 1] = (double)theta_i;
      trace[4 * rounds + 2] = (double)cov;
      trace[4 * rounds + 3] = (double)g->count;
    }
    rounds++;
    const double est = ((double)g->n * (double)cov) / (double)g->count;
    if (est >= (1.0 + epsp) * x) {
      LB = est / (1.0 + epsp);
      break;
    }
  }
  const uint64_t theta = (uint64_t)ceil(lam_star / LB);
  if (fresh) {
    /* the final phase on theta new RR sets, drawn with rr_ids 2^63 + j, independent of the
       sets the lower-bound search used */
    g->count = 0;
    g->rr_off[0] = 0;
    g->ctr_base = 1ull << 63;   /* kept: the collection left in place is that stream's prefix */
    int rc = orc_sample(g, model, seed, theta, threads);
    if (rc) return rc;
  } else {
    int rc = grow_to(g, model, seed, threads, avail, theta);
    if (rc) return rc;
  }
  if (orc_greedy(g, k, seeds, NULL) < 0) return -2;
  if (theta_out) *theta_out = theta;
  if (lb_out) *lb_out = LB;
  return rounds;
}

int orc_imm(orc *g, int model, uint32_t k, double eps, double ell, uint64_t seed, int threads,
            uint32_t *seeds, uint64_t *theta_out, double *lb_out, double *trace) {
  if (k < 1 || k > g->n || !(eps > 0.0 && eps < 1.0) || !(ell > 0.0) || g->n < 2) return -3;
  if (g->count != 0) return -1;
  g->rounds = 1;
  return imm_core(g, model, k, eps, ell, seed, threads, 0, 0, seeds, theta_out, lb_out, trace);
}

/*
 * IMM with a fresh final phase: the lower-bound search of orc_imm, then theta
 * new RR sets (rr_ids 2^63, 2^63 + 1, ..., independent of the search's sets)
 * replace the collection and the greedy runs over them. This is the variant
 * that avoids reusing the search's sets in the final estimate (a later
 * correction to IMM's analysis; the paper runs IMM as published). Afterwards
 * |R| = theta.
 */
int orc_imm_fresh(orc *g, int model, uint32_t k, double eps, double ell, uint64_t seed, int threads,
                  uint32_t *seeds, uint64_t *theta_out, double *lb_out, double *trace) {
  if (k < 1 || k > g->n || !(eps > 0.0 && eps < 1.0) || !(ell > 0.0) || g->n < 2) return -3;
  if (g->count != 0) return -1;
  g->rounds = 1;
  return imm_core(g, model, k, eps, ell, seed, threads, 0, 1, seeds, theta_out, lb_out, trace);
}

/*
 * IMM over a preloaded collection: the same steps as orc_imm, with every
 * "sample until |R| >= t" served by the first t sets of the collection that
 * orc_load_collection installed (which must hold RR sets 0, 1, ... of one
 * (model, seed) in rr_id order). Afterwards |R| is the prefix IMM used.
 * Returns the lower-bound rounds, -4 if the collection is too short for the
 * theta it needs, or another negative error.
 */
int orc_imm_replay(orc *g, uint32_t k, double eps, double ell, uint32_t *seeds, uint64_t *theta_out,
                   double *lb_out, double *trace) {
  if (k < 1 || k > g->n || !(eps > 0.0 && eps < 1.0) || !(ell > 0.0) || g->n < 2) return -3;
  const uint64_t avail = g->count;
  if (!avail) return -1;
  g->count = 0;
  const int rc = imm_core(g, 0, k, eps, ell, 0, 1, avail, 0, seeds, theta_out, lb_out, trace);
  if (rc < 0) g->count = avail;
  return rc;
}

/*
 * Multi-round IM (Sec. IV-H, CR-NAIMM): IMM's steps over multi-round RR sets
 * (rr_multi) with the constants of orc_mrim_constants and the greedy under k
 * seeds per round. seeds: k*T element ids t*n + v in pick order. The store
 * must start empty; afterwards it holds the multi-round collection (T stays
 * set until orc_reset). Returns the lower-bound rounds or a negative error.
 */
int orc_mrim(orc *g, int model, uint32_t T, uint32_t k, double eps, double ell, uint64_t seed, int threads,
             uint32_t *seeds, uint64_t *theta_out, double *lb_out, double *trace) {
  if (k < 1 || k > g->n || !(eps > 0.0 && eps < 1.0) || !(ell > 0.0) || g->n < 2) return -3;
  if (g->count != 0 || orc_set_rounds(g, T) != 0) return -1;
  return imm_core(g, model, k, eps, ell, seed, threads, 0, 0, seeds, theta_out, lb_out, trace);
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
