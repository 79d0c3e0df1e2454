/*
 * gim.h - C ABI of the GB300 IMM library (libgim.so).
 *
 * IMM on reverse-reachable (RR) sets, as accelerated by gIM (Shahrouz,
 * Salehkaleybar, Hashemi, "gIM: GPU Accelerated RIS-based Influence
 * Maximization Algorithm", IEEE TPDS; arXiv 2009.07325):
 *   - RR-set sampling under the IC and LT diffusion models (Sec. III-B,
 *     Alg. 3 and 6; Sec. III-G),
 *   - greedy maximum coverage over the RR sets (the maximum-coverage step of Alg. 1,
 *     Sec. III-H, Alg. 7),
 *   - IMM's lower-bound search and theta in FP64 on the host (Alg. 2).
 *
 * Conventions shared by every entry point:
 *   - Every call returns a gim_status; none throws, aborts or exits. On an
 *     error, gim_last_error_string(ctx) describes it.
 *   - All pointer arguments are HOST pointers unless a name says otherwise.
 *     Inputs are copied before the call returns; the caller keeps ownership
 *     of every buffer it passes. Outputs are written into caller-owned
 *     buffers of the stated length.
 *   - A context owns all of its device memory and runs its work on one CUDA
 *     stream of one device. A context must not be used from two threads at
 *     once; distinct contexts are independent.
 *   - Vertex ids are uint32 in [0, n); edge counts and RR-set ids are uint64.
 *   - Randomness: RR set j is a pure function of (graph, model, seed, j).
 *     It is drawn with Philox4x32-10 (Salmon et al., SC'11) keyed by the
 *     64-bit seed, with counter (idx, tag, j_lo, j_hi): tag 0 draws the root
 *     (idx 0), tag 1 the IC coin of in-edge e (idx e/4, word e%4), tag 2 the
 *     LT draw at vertex x (idx x, word 0). Results therefore do not depend
 *     on thread counts, launch shapes or the order in which RR sets finish.
 */
#ifndef GIM_H_
#define GIM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gim_ctx gim_ctx;

/* Diffusion models of Sec. II-B. */
typedef enum { GIM_IC = 0, GIM_LT = 1 } gim_model;

typedef enum {
  GIM_OK = 0,
  GIM_ERR_ARG = 1,      /* an argument is out of range or inconsistent      */
  GIM_ERR_OOM = 2,      /* device or host memory could not be obtained      */
  GIM_ERR_CUDA = 3,     /* a CUDA call failed (message has the CUDA error)  */
  GIM_ERR_TIMEOUT = 4,  /* a bounded device-side wait gave up               */
  GIM_ERR_STATE = 5     /* call not valid in the context's current state    */
} gim_status;

/*
 * Creates a context on CUDA device `device` (0-based). If `stream` is not
 * NULL it must be a cudaStream_t of that device, owned by the caller and
 * alive for the context's lifetime; all work of the context is issued on
 * it. With NULL the context creates and owns a non-blocking stream.
 * *out receives the context. Errors: GIM_ERR_ARG (out NULL, bad device),
 * GIM_ERR_CUDA, GIM_ERR_OOM.
 */
gim_status gim_create(gim_ctx **out, int device, void *stream);

/* Frees every resource of the context. NULL is accepted. */
void gim_destroy(gim_ctx *ctx);

/*
 * Loads graph G = (V, E) with n = |V| vertices and m = |E| directed edges as
 * an in-edge CSR (the CSR of Sec. III-B, indexed by target): the sources u
 * of the edges u->v are in_sources[in_offsets[v] .. in_offsets[v+1]), in
 * ascending order without repeats, and in_weights holds p(u,v) of Sec. II-A
 * for the same positions (fp32, in [0, 1]).
 *   in_offsets: n+1 entries, in_offsets[0] = 0, non-decreasing, last = m.
 *   in_sources: m entries, each < n, strictly ascending within a row.
 *   in_weights: m entries.
 * Precomputes the IC coin thresholds; the LT cumulative thresholds
 * (Sec. III-G) are built on the first LT use (gim_graph_lt_valid, an LT
 * call, gim_server_start), so IC work never waits for them. The graph is
 * usable under LT only if every row's weights sum to at most 1 + 1e-6
 * (Sec. II-B); gim_graph_lt_valid reports it. The weights stay on the
 * device (4m bytes) for that purpose.
 * Replaces any previous graph and empties the RR collection.
 * Limits: 2 <= n < 2^32 - 1, m < 2^32 - 4.
 * Errors: GIM_ERR_ARG (violated layout or range; the context is unchanged),
 * GIM_ERR_OOM, GIM_ERR_CUDA.
 */
gim_status gim_graph_load(gim_ctx *ctx, uint32_t n, uint64_t m, const uint64_t *in_offsets,
                          const uint32_t *in_sources, const float *in_weights);

/* *out = 1 if the loaded graph satisfies the LT weight condition, else 0
   (builds the LT thresholds if no LT call has yet). */
gim_status gim_graph_lt_valid(gim_ctx *ctx, int *out);

/*
 * Appends `count` random RR sets with ids |R| .. |R|+count-1 to the
 * context's collection R (the sampling step of Alg. 1; Alg. 6), drawn under `model` with
 * the 64-bit `seed`. IC: the vertices from which the root reaches along
 * live edges, each in-edge live with its probability (Sec. II-E, Alg. 3).
 * LT: the walk that, at each vertex, picks at most one in-edge with
 * probability equal to its weight (Sec. III-G). The occurrence counts
 * (Occur of Sec. III-B) are updated.
 * Errors: GIM_ERR_STATE (no graph; or model/seed differ from those of a
 * non-empty collection: call gim_reset_rr first), GIM_ERR_ARG (LT on a
 * graph whose weights are not LT-valid), GIM_ERR_OOM, GIM_ERR_CUDA.
 * On error the collection is left as it was before the call.
 */
gim_status gim_sample_rr(gim_ctx *ctx, gim_model model, uint64_t count, uint64_t seed);

/* Empties the RR collection (keeps the graph); it becomes a plain (1-round) collection. */
gim_status gim_reset_rr(gim_ctx *ctx);

/*
 * Makes the empty collection a multi-round collection of T rounds
 * (multi-round IM, Sec. IV-H; CR-NAIMM of Sun et al.). Multi-round RR set j
 * has the root of RR set j and T independent reverse traversals from it
 * (BFS under IC, walk under LT): round t runs in the live-edge world of
 * rr_id t * 2^32 + j (Philox counter words j_lo = j, j_hi = t; round 0 is RR
 * set j itself), and its vertices v are stored as elements t * n + v. Then
 * gim_sample_rr appends such sets, gim_select_seeds takes k seeds per round,
 * gim_coverage_export copies T * n element counts and the exports return
 * element ids. T = 1 is a plain collection.
 * Errors: GIM_ERR_STATE (no graph, or the collection is not empty),
 * GIM_ERR_ARG (T = 0, T > 32, or n * T >= 2^32 - 1), GIM_ERR_OOM, GIM_ERR_CUDA.
 */
gim_status gim_rr_set_rounds(gim_ctx *ctx, uint32_t rounds);

/* T of the collection (1 for plain RR sets). Errors: GIM_ERR_ARG (null argument). */
gim_status gim_rr_rounds(gim_ctx *ctx, uint32_t *rounds_out);

/*
 * Greedy maximum coverage over the collection (the maximum-coverage step of Alg. 1;
 * Sec. III-H): k rounds, each taking the vertex outside the seed set that
 * lies in the most RR sets not yet covered (lowest id on ties), then
 * removing the RR sets it covers. Once all sets are covered, the remaining
 * rounds take the lowest unselected ids with gain 0.
 *   seeds_out:   k entries, the seeds in selection order (required).
 *   covered_out: nullable; the number of RR sets covered by all k seeds.
 *   gains_out:   nullable, k entries; the marginal coverage of each seed.
 * The collection is not modified. Errors: GIM_ERR_ARG (k = 0, k > n, or
 * seeds_out NULL), GIM_ERR_STATE (no graph), GIM_ERR_OOM, GIM_ERR_CUDA.
 * On a multi-round collection of T rounds the candidates are the T * n
 * elements, a round takes at most k seeds, and there are k * T picks (each
 * the best element among the rounds not yet full); seeds_out and gains_out
 * then hold k * T entries (element ids t * n + v).
 */
gim_status gim_select_seeds(gim_ctx *ctx, uint32_t k, uint32_t *seeds_out, uint64_t *covered_out,
                            uint32_t *gains_out);

/*
 * IMM end to end (Alg. 2 then Alg. 1, with IMM's constants from Tang, Shi
 * and Xiao, SIGMOD 2015): ell' = ell (1 + ln 2 / ln n), eps' = sqrt(2) eps;
 * for i = 1 .. floor(log2 n) - 1: x = n / 2^i, sample until
 * |R| >= ceil(lambda' / x), select k seeds, and stop with
 * LB = n F_R(S) / (1 + eps') once n F_R(S) >= (1 + eps') x (LB = 1 if
 * never); then sample until |R| >= theta = ceil(lambda* / LB) and return
 * the greedy seeds over R. RR sets drawn during the search are reused.
 * Empties the collection first; leaves the final collection in place.
 *   seeds_out: k entries (required). theta_out, lb_out: nullable.
 * Errors: GIM_ERR_ARG (k = 0 or k > n, eps not in (0, 1), ell <= 0,
 * LT on a graph that is not LT-valid), GIM_ERR_STATE (no graph),
 * GIM_ERR_OOM, GIM_ERR_CUDA.
 */
gim_status gim_imm(gim_ctx *ctx, gim_model model, uint32_t k, double eps, double ell, uint64_t seed,
                   uint32_t *seeds_out, uint64_t *theta_out, double *lb_out);

/*
 * Multi-round IM (Sec. IV-H; the CR-NAIMM algorithm of Sun et al., KDD
 * 2018): gim_imm's steps over multi-round RR sets of `rounds` = T rounds
 * (see gim_rr_set_rounds), every selection taking k seeds per round. The
 * paper defers the constants to Sun et al.; this library's reading: the
 * number of feasible seed sets is C(n, k)^T, so ln C(n, k) becomes
 * T ln C(n, k), and the greedy's guarantee over that partition matroid, 1/2,
 * replaces 1 - 1/e in lambda*. LB and theta are as in gim_imm; the estimate
 * is n F_R(S), F_R the covered fraction of the multi-round sets. T = 1 is
 * gim_imm exactly. GIM_OPT_FRESH_FINAL does not apply (sets are reused).
 * Empties the collection first and leaves the final multi-round collection.
 *   seeds_out: k * T entries (required), element ids t * n + v in pick order.
 *   theta_out, lb_out: nullable.
 * Errors: as gim_imm, plus GIM_ERR_ARG (T = 0, T > 32, n * T >= 2^32 - 1).
 */
gim_status gim_mrim(gim_ctx *ctx, gim_model model, uint32_t rounds, uint32_t k, double eps, double ell,
                    uint64_t seed, uint32_t *seeds_out, uint64_t *theta_out, double *lb_out);

/*
 * Greedy maximum coverage that allocates no memory. The paper has no
 * counterpart: this entry point exists for callers that cannot let a
 * library allocate device memory - processes whose device memory is
 * reserved up front by their own pool or arena, where a foreign cudaMalloc
 * would fail or break their budget, and latency-critical paths that cannot
 * afford the synchronisation an allocation may bring. It returns the same
 * seeds, gains and covered count as gim_select_seeds (same tie rule: lowest
 * id), over an RR collection the caller holds in device memory, and needs
 * no context. It runs the k rounds as a per-round pair of kernels (argmax,
 * then cover), not gim_select_seeds's persistent greedy kernel.
 *   n:             number of vertices, 1 <= n <= 65536.
 *   num_sets:      number of RR sets R, <= 262144.
 *   num_members:   total members Z = d_rr_offsets[R], <= 1048576.
 *   d_rr_offsets:  DEVICE pointer, R+1 entries: set j is
 *                  d_rr_members[d_rr_offsets[j] .. d_rr_offsets[j+1]).
 *   d_rr_members:  DEVICE pointer, Z vertex ids < n (a set lists each
 *                  vertex at most once).
 *   k:             1 <= k <= min(n, 1024).
 *   d_seeds_out:   DEVICE pointer, k entries (required).
 *   d_gains_out:   DEVICE pointer, k entries, nullable.
 *   d_covered_out: DEVICE pointer, one uint64, nullable.
 *   stream:        cudaStream_t of the current device (NULL: legacy default).
 *   msg, msg_len:  nullable caller buffer for an error description.
 * Scratch: one fixed array of about 6.6 MB in the library's device image,
 * present on every device that loads the library until the process exits.
 * The first call on a device looks up the array's device address (set-up,
 * done once per device under a lock) and keeps it for the life of the
 * process, so that first call should come before any stream capture begins,
 * and the call must not be used on a device after cudaDeviceReset (the
 * kept address would be stale). Every call on a device shares the array and finds it as
 * the previous call left it (the call clears what must start at zero), so
 * calls whose work overlaps on the GPU - concurrent streams, or concurrent
 * host threads on one device - race and must be serialised by the caller.
 * The call synchronises `stream` twice to validate its inputs and returns
 * with the greedy rounds enqueued on `stream`.
 * Errors: GIM_ERR_ARG (a size above the limits, k > n, a null required
 * pointer, offsets not starting at 0 / decreasing / not ending at
 * num_members, a member >= n), GIM_ERR_CUDA.
 */
gim_status gim_select_seeds_noalloc(uint32_t n, uint64_t num_sets, uint64_t num_members,
                                    const uint64_t *d_rr_offsets, const uint32_t *d_rr_members, uint32_t k,
                                    uint32_t *d_seeds_out, uint32_t *d_gains_out, uint64_t *d_covered_out,
                                    void *stream, char *msg, size_t msg_len);

/* Parameters of one IMM instance of a batch (as the arguments of gim_imm). */
typedef struct {
  gim_model model;
  uint32_t k;
  double eps;
  double ell;
  uint64_t seed;
} gim_imm_params;

/* Outcome of one IMM instance of a batch. */
typedef struct {
  uint64_t theta;       /* final theta = ceil(lambda* / LB)                  */
  double lb;            /* the lower bound LB of Alg. 2 (1 if never raised)  */
  uint64_t rr_count;    /* |R| at the end                                    */
  uint32_t lb_rounds;   /* lower-bound rounds run                            */
  gim_status status;    /* GIM_OK                                            */
} gim_imm_result;

/*
 * Batched IMM: runs gim_imm's algorithm (Alg. 2 then Alg. 1) on n_inst
 * contexts at once, instance i on ctxs[i]'s graph with params[i]. The
 * instances advance in lockstep: each round, the RR sets every unfinished
 * instance still needs are drawn in one launch per diffusion model whose
 * device work queue holds (instance, rr_id) items, and the greedy selections
 * of all unfinished instances run as one replay of a CUDA graph of
 * multi-instance kernels. Instance i's seeds, theta, LB and final RR
 * collection are exactly those gim_imm(ctxs[i], params[i]...) gives.
 *   ctxs:      n_inst distinct contexts of one device, each with a graph;
 *              the work is issued on ctxs[0]'s stream.
 *   params:    n_inst entries (validated as in gim_imm).
 *   seeds_out: n_inst host pointers, seeds_out[i] holding params[i].k entries.
 *   results:   n_inst entries.
 * Errors: GIM_ERR_ARG (n_inst = 0, a repeated or null context, contexts on
 * different devices, a parameter gim_imm would reject), GIM_ERR_STATE (a
 * context without a graph), GIM_ERR_OOM, GIM_ERR_CUDA; the description is
 * on ctxs[0] (gim_last_error_string).
 */
gim_status gim_batch_imm(gim_ctx *const *ctxs, uint32_t n_inst, const gim_imm_params *params,
                         uint32_t *const *seeds_out, gim_imm_result *results);

/*
 * Query server over one resident graph: continuous batching with resident
 * RR stores. Not in the paper; it serves many IMM queries (gim_imm's
 * algorithm) on the graph loaded in graph_ctx.
 *
 * RR set j depends only on (graph, model, seed, j) and an IMM run uses the
 * first |R| sets of its sequence, so the server keeps one RR store per
 * (model, seed) on the device and answers each query from the prefix its
 * run needs: every query's seeds, theta and LB equal those of
 * gim_imm(model, k, eps, ell, seed) run alone, while RR sets are sampled once
 * for all queries sharing a (model, seed). A worker thread advances the
 * admitted queries together, one IMM round at a time (one sampling launch
 * per model, then one batched greedy selection); queries that arrive
 * meanwhile wait in a FIFO and are admitted at the next round when one of
 * max_active slots is free and their projected RR-store bytes (theta times
 * the mean RR-set size) fit the memory budget.
 *
 * gim_server_start: graph_ctx must hold a graph and must not be changed or
 *   destroyed until gim_server_stop; the server only reads it.
 *   max_active in [1, 1024] slots; max_k in [1, n] is the largest k a query
 *   may ask for; mem_budget_bytes = 0 takes 60% of the free device memory.
 * gim_server_submit: queues one query; *ticket_out identifies it. Errors:
 *   GIM_ERR_ARG (k > max_k or a parameter gim_imm would reject),
 *   GIM_ERR_STATE (the server is stopping).
 * gim_server_poll: *done = 1 once the query finished (waits up to timeout_ms
 *   for it); then seeds_out (k entries, nullable), result (nullable) and
 *   latency_ms (submit to finish, nullable) are filled. Returns the query's
 *   error if it failed.
 * gim_server_stats: out[8] = {completed queries, rounds, busy ms, sampling
 *   ms, selection ms, most queries admitted at once, queries waiting,
 *   RR sets resident in the pools}.
 * gim_server_stop: lets admitted queries finish, fails the waiting ones with
 *   GIM_ERR_STATE, frees the server. Submit/poll/stats are thread-safe.
 */
typedef struct gim_server gim_server;
gim_status gim_server_start(gim_server **out, gim_ctx *graph_ctx, uint32_t max_active, uint32_t max_k,
                            uint64_t mem_budget_bytes);
gim_status gim_server_submit(gim_server *srv, const gim_imm_params *params, uint64_t *ticket_out);
gim_status gim_server_poll(gim_server *srv, uint64_t ticket, uint32_t timeout_ms, int *done, uint32_t *seeds_out,
                           gim_imm_result *result, double *latency_ms);
gim_status gim_server_stats(gim_server *srv, double out[8]);
void gim_server_stop(gim_server *srv);

/* Options of a context. GIM_OPT_GROUP_BUDGET, GIM_OPT_LARGE_PASS_BYTES,
   GIM_OPT_FRONTIER_BATCH, GIM_OPT_CHUNK_GROUPS and GIM_OPT_QUEUE_CAP are
   tuning knobs: they change speed, never results (every RR set is a function
   of (graph, model, seed, rr_id) alone). GIM_OPT_FRESH_FINAL selects a
   variant of IMM and changes its results. A launch that serves several
   contexts (gim_batch_imm, the server) takes the knobs of its first
   context. */
typedef enum {
  /* In-edge groups (4 in-edges each) one RR set may scan in the warp-per-set
     IC pass before it is handed to the block-per-set pass. Default 16384. */
  GIM_OPT_GROUP_BUDGET = 0,
  /* Device bytes for the scratch of the block-per-set pass (an n-bit visited
     bitmap and an n-entry queue per heavy RR set in flight; per device,
     shared by its contexts). Heavy sets in flight = min(bytes / (n/8 + 4n),
     8 x SM count), at least 1. Default 16 GiB; lower it to leave room for
     other work on the GPU. */
  GIM_OPT_LARGE_PASS_BYTES = 1,
  /* 1: gim_imm and gim_batch_imm run IMM's final phase on fresh RR sets.
     After the lower-bound search (Alg. 2) the collection is emptied and
     theta new sets are drawn with rr_ids 2^63, 2^63 + 1, ... (Philox
     counter words j_lo = j, j_hi = 2^31), stored at positions 0 .. theta-1;
     the greedy (Alg. 1) runs over them, so the final estimate does not
     reuse the sets the search selected on. The paper reuses them (IMM as
     published); this is the later correction of IMM's analysis. theta and
     LB are unchanged; rr_count = theta. The collection keeps its counter
     base until it is reset. The server always runs IMM as published.
     0 (default): reuse. Values other than 0 and 1 are rejected. */
  GIM_OPT_FRESH_FINAL = 2,
  /* Frontier vertices the block-per-set IC pass expands per block step (a
     level-synchronous batch): 32 .. 256, a multiple of 32; values above the
     pass's block size (128 threads, one frontier row each) act as 128.
     Default 128. */
  GIM_OPT_FRONTIER_BATCH = 3,
  /* In-edge groups (4 in-edges) per work chunk of the block-per-set IC
     pass: 64 .. 4096, a multiple of 64. A row with p <= 2^-8 is cut into
     chunks of half as many super-groups (16 in-edges), i.e. twice the
     in-edges. Default 512 (2048 in-edges; 4096 in screened rows). */
  GIM_OPT_CHUNK_GROUPS = 4,
  /* Members an RR set may reach in the warp-per-set IC pass before it is
     handed to the block-per-set pass (the warp's queue): 256 .. 4096, a
     multiple of 32. Default 4096. */
  GIM_OPT_QUEUE_CAP = 5,
  /* 1: compact collections for gim_imm (T = 1, IC or LT). The greedy's first
     pick (the vertex in the most RR sets, lowest id on ties; Alg. 1) covers
     every set that holds it, so the later rounds never read those sets'
     members. After its first selection gim_imm keeps, for every set it draws
     from then on that holds that first pick, only the set's size and its
     occurrence counts, not its members. Where one vertex lies in nearly all
     of the large sets (IC with a giant component, e.g. p = 0.01 on R-MAT)
     this shrinks the collection by orders of magnitude. Results are those of
     the plain run: each later selection checks on the device that its first
     pick is still that vertex and fails with GIM_ERR_STATE otherwise (never a
     different answer). A sampling call that fails empties a compact
     collection instead of rolling it back. gim_rr_export then fails on such
     sets (gim_rr_export_compact, gim_rr_info read them). gim_batch_imm, the
     server and multi-round IM ignore it. 0 (default): every set is kept. */
  GIM_OPT_COMPACT_FIRST_PICK = 6
} gim_option;

/* Sets an option. Errors: GIM_ERR_ARG (unknown option, value 0 for the
   tuning knobs or outside a knob's stated range, value above 1 for
   GIM_OPT_FRESH_FINAL or GIM_OPT_COMPACT_FIRST_PICK). */
gim_status gim_set_option(gim_ctx *ctx, gim_option opt, uint64_t value);

/* Reads a tuning knob into *value. */
gim_status gim_get_option(gim_ctx *ctx, gim_option opt, uint64_t *value);

/*
 * Autotuner: picks the sampling schedule of a workload - GIM_OPT_GROUP_BUDGET
 * (how long one warp keeps an RR set before a 128-thread block takes it
 * over, i.e. warps per RR set for heavy sets), then GIM_OPT_CHUNK_GROUPS
 * (the block pass's work chunk), GIM_OPT_FRONTIER_BATCH (its frontier batch)
 * and GIM_OPT_QUEUE_CAP (the warp pass's frontier buffer), one knob at a time
 * with the others at their best so far - by timing the sampling of
 * `sample_sets` RR sets per instance under each candidate exactly as
 * gim_batch_imm (n_inst > 1) or gim_imm (n_inst = 1) would launch it (the
 * paper sizes its shared queue and grid by hand, Sec. III-F and IV-G). The
 * choice is cached for the process under the workload's degree profile
 * (log2 of n, of mean and of maximum in-degree, the model, log2 of n_inst),
 * so later calls with the same profile only read the cache. The chosen
 * values are set on every context; their RR collections are emptied.
 *   ctxs, n_inst, params: as for gim_batch_imm (params give model and seed).
 *   budget_out: nullable; the chosen budget (the other knobs: gim_get_option).
 *   measured_out: nullable; 1 if this call timed the candidates, 0 if it
 *   used the cache.
 */
gim_status gim_autotune(gim_ctx *const *ctxs, uint32_t n_inst, const gim_imm_params *params, uint64_t sample_sets,
                        uint64_t *budget_out, int *measured_out);

/* ---- introspection (tests, tools) ------------------------------------- */

/* *count_out = |R|; *members_out (nullable) = total members over all sets
   whose members are kept (a compact collection's sets that hold the compact
   vertex count none: see GIM_OPT_COMPACT_FIRST_PICK). */
gim_status gim_rr_count(gim_ctx *ctx, uint64_t *count_out, uint64_t *members_out);

/*
 * Copies R out in rr_id order as a CSR: offsets_out has |R|+1 entries,
 * members_out has gim_rr_count's members_out entries; the members of each
 * set are written in ascending vertex order. GIM_ERR_STATE if a set is kept
 * without its members (compact collections: use gim_rr_export_compact).
 */
gim_status gim_rr_export(gim_ctx *ctx, uint64_t *offsets_out, uint32_t *members_out);

/*
 * As gim_rr_export, for a compact collection: a set kept without its members
 * (it holds the compact vertex) is exported with none, and compact_out[j]
 * (|R| bytes) is 1 for it, 0 for every other set. Its size: gim_rr_info.
 */
gim_status gim_rr_export_compact(gim_ctx *ctx, uint64_t *offsets_out, uint32_t *members_out, uint8_t *compact_out);

/* Size of RR set rr_id (rr_id < |R|) and *stored_out = 1 if its members are
   kept, 0 if it is a compact collection's set that holds the compact vertex. */
gim_status gim_rr_info(gim_ctx *ctx, uint64_t rr_id, uint32_t *len_out, int *stored_out);

/*
 * Copies RR set rr_id (rr_id < |R|) in ascending vertex order into
 * members_out (cap entries) and its size into *len_out. A set larger than cap
 * gives GIM_ERR_ARG with *len_out set, so a caller can retry with room; a set
 * kept without its members (compact collections) gives GIM_ERR_STATE.
 */
gim_status gim_rr_get(gim_ctx *ctx, uint64_t rr_id, uint32_t *members_out, uint32_t cap, uint32_t *len_out);

/* Copies the occurrence counts (RR sets containing each vertex): n entries,
   or T * n (one per element) for a multi-round collection of T rounds. */
gim_status gim_coverage_export(gim_ctx *ctx, uint32_t *cnt_out);

/*
 * Per-phase device times of the last gim_imm / gim_sample_rr /
 * gim_select_seeds call, in milliseconds, from CUDA events on the
 * context's stream: out[0] sampling, out[1] selection (index build +
 * greedy rounds), out[2] host wall time of the call, out[3] lower-bound
 * rounds run by gim_imm. Accumulated since gim_reset_timings (or context
 * creation): out[4] time inside the common-case sampling kernel and out[5]
 * its launches; out[6], out[7] the same for the large-set pass.
 * out must hold 8 doubles.
 */
gim_status gim_last_timings(gim_ctx *ctx, double out[8]);

/* Zeroes the accumulated kernel counters of gim_last_timings (out[4..7])
   and of gim_selection_stats. */
gim_status gim_reset_timings(gim_ctx *ctx);

/*
 * Greedy selections (the maximum-coverage step of Alg. 1, Sec. III-H) run
 * with this context since gim_reset_timings, accumulated: out[0] device time
 * of the selection kernels in ms (CUDA events on the stream around the index
 * build and the k rounds), out[1] their algorithmic bytes (8 per store
 * member for reading the store and writing the index, 4 per vertex for the
 * count scan, per round 4 per vertex for the argmax and 4 per word of the
 * seed's list or bitmap row, 12 per member of each newly covered set, and
 * the covered bitmap), out[2] selections, out[3] members of newly covered
 * sets. out must hold 4 doubles. Batched and served selections are
 * accounted to the first context of the batch or the server's graph context.
 */
gim_status gim_selection_stats(gim_ctx *ctx, double out[4]);

/*
 * Diagnostic: the device's throughput of Philox4x32-10 blocks (the coin
 * generator of Alg. 3's "p = U(0,1)") measured by a kernel that does nothing
 * else, in calls per second (best of three timed launches after a warm-up).
 * This is the integer-ALU ceiling of the IC sampler's coin work.
 */
gim_status gim_diag_philox_rate(gim_ctx *ctx, double *calls_per_s);

/*
 * Diagnostic of the failure path of the greedy selection's bounded waits (the
 * paper has no counterpart): runs the persistent greedy kernel on a tiny
 * instance whose block group is declared as two blocks while only one is
 * launched, so its group barrier can never be met. The wait gives up after
 * about 2 s; the call then returns GIM_ERR_TIMEOUT and *waited_ms (nullable)
 * holds the kernel's time. No fault is raised and the context stays usable.
 */
gim_status gim_diag_barrier_timeout(gim_ctx *ctx, double *waited_ms);

/* Number of kernels this context has launched since it was created. */
gim_status gim_launch_count(gim_ctx *ctx, uint64_t *out);

/* Human-readable description of the context's last error ("" if none). */
const char *gim_last_error_string(gim_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* GIM_H_ */
