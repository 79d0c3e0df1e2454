// Query server: IMM queries over one resident graph, with continuous
// batching and resident RR stores.
//
// RR set j is a pure function of (graph, model, seed, j), and an IMM run
// only ever uses the first |R| sets of its sequence. So the server keeps one
// RR store per (model, seed) resident on the device - a pool - and answers
// each query from the prefix of its pool that its own run needs: the query's
// collection at every step is exactly the one gim_imm would build alone, so
// its seeds, theta and LB are identical to a lone run, while the pool's sets
// are sampled once for all queries that share it.
//
// A worker thread advances all admitted queries together, one round at a
// time (the rounds of Alg. 2 / Alg. 1): grow every pool to the largest
// prefix its queries now need (one sampling launch per model), then run the
// greedy selection of every admitted query over its own prefix as one
// batched selection (a replayed CUDA graph). Queries that arrive while
// others are on the GPU wait in a FIFO and are admitted at the next round
// as soon as a slot is free and their projected RR-store bytes fit the
// memory budget; finished queries free their slots at once.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "gim_internal.cuh"

using namespace gim;

namespace {

using Clock = std::chrono::steady_clock;

struct Query {
  uint64_t ticket = 0;
  gim_imm_params p{};
  ImmState st;
  gim_ctx *pool = nullptr;
  int slot = -1;
  uint64_t Rq = 0;                 // the prefix of the pool this query's run has reached
  uint64_t counted = 0;            // sets [0, counted) are already in the slot's occurrence counts
  uint64_t projected = 0;          // admission bytes
  std::vector<uint32_t> seeds;
  gim_imm_result res{};
  bool done = false;
  gim_status status = GIM_OK;
  Clock::time_point t_submit, t_admit, t_done;
};

}  // namespace

struct gim_server {
  gim_ctx *graph = nullptr;        // the caller's context holding the resident graph (only read)
  gim_ctx *self = nullptr;         // the server's own view of the graph: errors, launches, selection
  cudaStream_t stream = nullptr;
  uint32_t max_active = 0;
  uint32_t max_k = 0;
  uint64_t budget = 0;
  std::map<std::pair<int, uint64_t>, gim_ctx *> pools;   // (model, seed) -> RR pool sharing the graph
  std::map<gim_ctx *, uint64_t> pool_used;               // pool -> the last round a query read it
  std::vector<SelectBuffers> slot_buf;
  std::vector<Query *> slot_q;
  // shared indexes: instance max_active + i of ms builds the index of pool
  // index_pool[i] over its first index_R[i] sets
  std::vector<SelectBuffers> index_buf;
  std::vector<gim_ctx *> index_pool;
  std::vector<uint64_t> index_R;
  MultiSelect ms;
  std::deque<Query *> waiting;
  std::map<uint64_t, std::unique_ptr<Query>> all;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stopping = false;
  uint64_t next_ticket = 1;
  gim_status fatal = GIM_OK;
  std::string fatal_msg;
  double cover_frac[2] = {0.05, 0.05};   // running coverage fraction per model (admission estimate)
  // statistics
  uint64_t rounds = 0, completed = 0;
  double busy_ms = 0, sample_ms = 0, select_ms = 0;
  uint64_t peak_active = 0;
};

namespace {

uint64_t pool_bytes(gim_ctx *c) { return c->st.cap * 4 + c->rr_cap * 12 + (uint64_t)c->g.n * 4; }

uint64_t slot_bytes(const SelectBuffers &b) {
  return b.n_cap * 29 + b.z_cap * 4 + b.r_cap * 4 + b.k_cap * 16 + b.scan_cap * 8;
}

// Projected device bytes a query adds: its share of pool growth plus its
// selection buffers, from theta = lambda* / LB with LB estimated from the
// coverage seen by earlier queries of its model.
uint64_t projected_bytes(gim_server *S, const Query &q) {
  const uint32_t n = S->graph->g.n;
  const ImmConst c = imm_constants(n, q.p.k, q.p.eps, q.p.ell);
  const double lb = std::max(1.0, n * S->cover_frac[q.p.model] / (1.0 + c.epsp));
  const double theta = c.lam2 / lb;
  double mean_rr = 32.0;
  for (auto &kv : S->pools)
    if (kv.second->R > 0) mean_rr = std::max(mean_rr, (double)kv.second->Z / (double)kv.second->R);
  return (uint64_t)(theta * mean_rr * 8.0 + theta * 13.0) + (uint64_t)n * 24;
}

// A context that uses the resident graph without owning it.
gim_status make_view(gim_server *S, gim_ctx **out) {
  gim_ctx *c = nullptr;
  gim_status st = gim_create(&c, S->graph->device, S->stream);
  if (st != GIM_OK) return st;
  c->g = S->graph->g;
  c->owns_graph = false;
  c->has_graph = true;
  c->lt_ok = S->graph->lt_ok;
  c->max_indeg = S->graph->max_indeg;
  c->group_budget = S->graph->group_budget;
  c->frontier_batch = S->graph->frontier_batch;
  c->chunk_groups = S->graph->chunk_groups;
  c->queue_cap = S->graph->queue_cap;
  *out = c;
  return GIM_OK;
}

// Pools no admitted query reads, least recently used first.
std::vector<std::pair<std::pair<int, uint64_t>, gim_ctx *>> idle_pools(gim_server *S,
                                                                       const std::vector<Query *> &active) {
  std::vector<std::pair<std::pair<int, uint64_t>, gim_ctx *>> out;
  for (auto &kv : S->pools) {
    bool used = false;
    for (const Query *q : active) used |= q->pool == kv.second;
    if (!used) out.push_back(kv);
  }
  std::sort(out.begin(), out.end(), [&](const auto &a, const auto &b) { return S->pool_used[a.second] < S->pool_used[b.second]; });
  return out;
}

// A pool leaves the server: its shared index (if any) is dropped with it.
void forget_pool(gim_server *S, gim_ctx *c) {
  for (size_t i = 0; i < S->index_pool.size(); ++i)
    if (S->index_pool[i] == c) {
      S->index_pool[i] = nullptr;
      S->index_R[i] = 0;
    }
  S->pool_used.erase(c);
}

gim_status get_pool(gim_server *S, int model, uint64_t seed, const std::vector<Query *> &active, uint64_t used,
                    gim_ctx **out) {
  auto key = std::make_pair(model, seed);
  auto it = S->pools.find(key);
  if (it != S->pools.end()) {
    *out = it->second;
    return GIM_OK;
  }
  // A new (model, seed): once the server holds as many pools as slots, or
  // half its memory budget, the least recently used idle pool is emptied
  // and reused (its store, counts and tables stay allocated), so queries
  // with their own seeds do not allocate a pool each.
  if (S->pools.size() >= S->max_active || used > S->budget / 2) {
    auto idle = idle_pools(S, active);
    if (!idle.empty()) {
      gim_ctx *c = idle.front().second;
      S->pools.erase(idle.front().first);
      forget_pool(S, c);
      const gim_status st = gim_reset_rr(c);
      if (st != GIM_OK) {
        gim_destroy(c);
        return st;
      }
      S->pools[key] = c;
      S->pool_used[c] = S->rounds;
      *out = c;
      return GIM_OK;
    }
  }
  gim_ctx *c = nullptr;
  gim_status st = make_view(S, &c);
  if (st != GIM_OK) return st;
  if (cudaMalloc(&c->st.cnt, (uint64_t)c->g.n * 4 + 16) != cudaSuccess ||
      cudaMemsetAsync(c->st.cnt, 0, (uint64_t)c->g.n * 4 + 16, S->stream) != cudaSuccess) {
    cudaGetLastError();
    gim_destroy(c);
    return GIM_ERR_OOM;
  }
  S->pools[key] = c;
  S->pool_used[c] = S->rounds;
  *out = c;
  return GIM_OK;
}

// One round over the admitted queries. Returns GIM_OK or a fatal error.
gim_status round_once(gim_server *S, std::vector<Query *> &active) {
  const uint32_t n = S->graph->g.n;
  // 1. each query's next prefix; each pool's target
  std::map<gim_ctx *, uint64_t> target;
  for (Query *q : active) {
    const uint64_t t = imm_target(q->st, n);
    if (t >= 0xFFFFFFFFull) return set_err(S->self, GIM_ERR_ARG, "query %llu: theta above 2^32-2 RR sets",
                                           (unsigned long long)q->ticket);
    q->Rq = std::max(q->Rq, t);
    uint64_t &pt = target[q->pool];
    pt = std::max(pt, q->Rq);
    S->pool_used[q->pool] = S->rounds;
  }
  const auto t0 = Clock::now();
  std::vector<SampleJobH> jobs;
  for (auto &kv : target)
    if (kv.second > kv.first->R)
      jobs.push_back(SampleJobH{kv.first, kv.first->model >= 0 ? kv.first->model : 0, kv.first->seed,
                                kv.second - kv.first->R});
  // a new pool has model -1: take model and seed from its queries
  for (auto &jb : jobs)
    for (Query *q : active)
      if (q->pool == jb.ctx) {
        jb.model = q->p.model;
        jb.seed = q->p.seed;
        break;
      }
  gim_status st = sample_jobs(jobs, S->stream);
  if (st != GIM_OK) {
    if (!jobs.empty()) S->self->last_error = jobs[0].ctx->last_error;
    return st;
  }
  const auto t1 = Clock::now();
  // 2. every admitted query's greedy selection over its own prefix. A pool
  // with room among the shared indexes gets one index over all its sets,
  // rebuilt only when the pool has grown; a query whose prefix is at least a
  // quarter of its pool uses it (its lists read up to the prefix) instead of
  // indexing its prefix itself. A pool read by one query only gets no shared
  // index: that query indexes its prefix itself, with the first pick taken
  // during the fill
  const uint32_t ni = (uint32_t)S->index_buf.size();
  std::vector<SelInput> in(S->max_active + ni);
  std::map<gim_ctx *, int> pool_index, readers;
  for (Query *q : active) readers[q->pool]++;
  for (Query *q : active) {
    if (pool_index.count(q->pool)) continue;
    if (readers[q->pool] < 2) {
      pool_index[q->pool] = -1;
      continue;
    }
    int ix = -1;
    for (uint32_t i = 0; i < ni; ++i)
      if (S->index_pool[i] == q->pool) ix = (int)i;
    for (uint32_t i = 0; i < ni && ix < 0; ++i) {
      bool used = false;   // a free entry: its pool has no admitted query now
      for (Query *o : active) used |= S->index_pool[i] == o->pool;
      if (!used) {
        ix = (int)i;
        S->index_pool[i] = q->pool;
        S->index_R[i] = 0;
      }
    }
    pool_index[q->pool] = ix;
    if (ix >= 0 && S->index_R[ix] != q->pool->R) {
      SelInput &x = in[S->max_active + ix];
      x.active = true;
      x.index_only = true;
      x.R = q->pool->R;
      x.Z = q->pool->Z;
      x.members = q->pool->st.members;
      x.rr_start = q->pool->st.rr_start;
      x.rr_len = q->pool->st.rr_len;
      x.cnt = q->pool->st.cnt;   // the pool's occurrence counts over all its sets
      x.k = 1;
      x.buf = &S->index_buf[ix];
    }
  }
  for (Query *q : active) {
    SelInput &x = in[q->slot];
    x.active = true;
    x.R = q->Rq;
    x.Z = q->pool->Z;          // bounds the prefix's members
    x.members = q->pool->st.members;
    x.rr_start = q->pool->st.rr_start;
    x.rr_len = q->pool->st.rr_len;
    x.cnt = nullptr;           // counted over the prefix, incrementally across the query's rounds
    x.count_from = q->counted;
    x.k = q->p.k;
    x.buf = &S->slot_buf[q->slot];
    const int ix = pool_index[q->pool];
    if (ix >= 0 && 4 * q->Rq >= q->pool->R) {
      x.index = &S->index_buf[ix];
      x.index_R = q->pool->R;
    }
  }
  std::vector<unsigned long long> cov;
  std::vector<uint32_t> seeds;
  if ((st = S->ms.run(S->self, in, S->stream, cov, seeds)) != GIM_OK) return st;
  for (auto &kv : pool_index)
    if (kv.second >= 0) S->index_R[kv.second] = kv.first->R;
  const auto t2 = Clock::now();
  S->sample_ms += std::chrono::duration<double, std::milli>(t1 - t0).count();
  S->select_ms += std::chrono::duration<double, std::milli>(t2 - t1).count();
  // 3. advance the state machines
  for (Query *q : active) {
    q->counted = q->Rq;
    const bool final_round = q->st.phase == 1;
    imm_advance(q->st, n, q->Rq, cov[q->slot]);
    if (final_round) {
      q->seeds.assign(seeds.begin() + S->ms.seed_offset(q->slot), seeds.begin() + S->ms.seed_offset(q->slot) + q->p.k);
      q->res.theta = q->st.theta;
      q->res.lb = q->st.LB;
      q->res.rr_count = q->Rq;
      q->res.lb_rounds = q->st.rounds;
      q->res.status = GIM_OK;
      const double f = (double)cov[q->slot] / (double)std::max<uint64_t>(q->Rq, 1);
      S->cover_frac[q->p.model] = 0.5 * S->cover_frac[q->p.model] + 0.5 * f;
    }
  }
  S->rounds++;
  return GIM_OK;
}

void worker_main(gim_server *S) {
  cudaSetDevice(S->graph->device);
  std::vector<Query *> active;
  for (;;) {
    {
      std::unique_lock<std::mutex> lock(S->mu);
      S->cv_work.wait(lock, [&] { return S->stopping || !S->waiting.empty() || !active.empty(); });
      if (S->stopping && active.empty()) return;
      // admission: FIFO, a free slot and room in the memory budget
      uint64_t used = 0;
      for (auto &kv : S->pools) used += pool_bytes(kv.second);
      for (const SelectBuffers &b : S->slot_buf) used += slot_bytes(b);
      while (!S->waiting.empty() && !S->stopping) {
        int free_slot = -1;
        for (uint32_t i = 0; i < S->max_active; ++i)
          if (!S->slot_q[i]) {
            free_slot = (int)i;
            break;
          }
        if (free_slot < 0) break;
        Query *q = S->waiting.front();
        q->projected = projected_bytes(S, *q);
        uint64_t pending = 0;
        for (Query *a : active) pending += a->projected;
        if (!active.empty() && used + pending + q->projected > S->budget) {
          // free idle pools (least recently used first) before holding the query back
          auto idle = idle_pools(S, active);
          for (auto &kv : idle) {
            if (kv.first == std::make_pair((int)q->p.model, q->p.seed)) continue;   // the query's own pool
            used -= std::min(used, pool_bytes(kv.second));
            S->pools.erase(kv.first);
            forget_pool(S, kv.second);
            gim_destroy(kv.second);
            if (used + pending + q->projected <= S->budget) break;
          }
          if (used + pending + q->projected > S->budget) break;
        }
        S->waiting.pop_front();
        gim_ctx *pool = nullptr;
        const gim_status st = get_pool(S, q->p.model, q->p.seed, active, used, &pool);
        if (st != GIM_OK) {
          q->status = st;
          q->done = true;
          q->t_done = Clock::now();
          S->cv_done.notify_all();
          continue;
        }
        q->pool = pool;
        q->slot = free_slot;
        q->t_admit = Clock::now();
        S->slot_q[free_slot] = q;
        active.push_back(q);
      }
      S->peak_active = std::max<uint64_t>(S->peak_active, active.size());
    }
    if (active.empty()) continue;
    const auto t0 = Clock::now();
    const gim_status st = round_once(S, active);
    std::lock_guard<std::mutex> lock(S->mu);
    S->busy_ms += std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
    if (st != GIM_OK) {   // fail every admitted query, keep serving the rest
      S->fatal = st;
      S->fatal_msg = S->self->last_error;
      for (Query *q : active) {
        q->status = st;
        q->done = true;
        q->t_done = Clock::now();
        S->slot_q[q->slot] = nullptr;
      }
      active.clear();
      S->cv_done.notify_all();
      continue;
    }
    std::vector<Query *> still;
    for (Query *q : active) {
      if (q->st.phase == 2) {
        q->done = true;
        q->t_done = Clock::now();
        S->slot_q[q->slot] = nullptr;
        S->completed++;
      } else {
        still.push_back(q);
      }
    }
    if (still.size() != active.size()) S->cv_done.notify_all();
    active.swap(still);
  }
}

}  // namespace

extern "C" {

gim_status gim_server_start(gim_server **out, gim_ctx *graph_ctx, uint32_t max_active, uint32_t max_k,
                            uint64_t mem_budget_bytes) {
  if (!out || !graph_ctx) return GIM_ERR_ARG;
  *out = nullptr;
  if (!graph_ctx->has_graph) return set_err(graph_ctx, GIM_ERR_STATE, "no graph loaded");
  if (max_active == 0 || max_active > 1024 || max_k == 0 || max_k > graph_ctx->g.n)
    return set_err(graph_ctx, GIM_ERR_ARG, "need 1 <= max_active <= 1024 and 1 <= max_k <= n");
  if (cudaSetDevice(graph_ctx->device) != cudaSuccess) return cuda_err(graph_ctx, cudaGetLastError(), "device");
  {   // LT queries are served from the shared graph's thresholds: build them now
    const gim_status lt = ensure_lt(graph_ctx);
    if (lt != GIM_OK) return lt;
  }
  auto S = std::make_unique<gim_server>();
  S->graph = graph_ctx;
  S->max_active = max_active;
  S->max_k = max_k;
  if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess)
    return cuda_err(graph_ctx, cudaGetLastError(), "server stream");
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  S->budget = mem_budget_bytes ? mem_budget_bytes : (uint64_t)(0.6 * (double)free_b);
  S->slot_buf.resize(max_active);
  S->slot_q.assign(max_active, nullptr);
  constexpr uint32_t kSharedIndexes = 4;
  S->index_buf.resize(kSharedIndexes);
  S->index_pool.assign(kSharedIndexes, nullptr);
  S->index_R.assign(kSharedIndexes, 0);
  gim_status st = make_view(S.get(), &S->self);
  if (st != GIM_OK) {
    cudaStreamDestroy(S->stream);
    return set_err(graph_ctx, st, "server context");
  }
  std::vector<uint32_t> ns(max_active + S->index_buf.size(), graph_ctx->g.n), ks(ns.size(), max_k);
  std::vector<bool> only(ns.size(), false);
  for (size_t i = max_active; i < ks.size(); ++i) {   // index-only instances
    ks[i] = 1;
    only[i] = true;
  }
  st = S->ms.configure(S->self, ns, ks, &only);
  if (st != GIM_OK) {
    graph_ctx->last_error = S->self->last_error;
    gim_destroy(S->self);
    cudaStreamDestroy(S->stream);
    return st;
  }
  gim_server *raw = S.release();
  raw->worker = std::thread(worker_main, raw);
  *out = raw;
  return GIM_OK;
}

gim_status gim_server_submit(gim_server *S, const gim_imm_params *p, uint64_t *ticket_out) {
  if (!S || !p || !ticket_out) return GIM_ERR_ARG;
  const uint32_t n = S->graph->g.n;
  if ((p->model != GIM_IC && p->model != GIM_LT) || p->k == 0 || p->k > S->max_k || !(p->eps > 0.0 && p->eps < 1.0) ||
      !(p->ell > 0.0) || (p->model == GIM_LT && !S->graph->lt_ok) || p->k > n)
    return GIM_ERR_ARG;
  auto q = std::make_unique<Query>();
  q->p = *p;
  imm_init(q->st, n, *p);
  q->t_submit = Clock::now();
  std::lock_guard<std::mutex> lock(S->mu);
  if (S->stopping) return GIM_ERR_STATE;
  q->ticket = S->next_ticket++;
  *ticket_out = q->ticket;
  S->waiting.push_back(q.get());
  S->all[q->ticket] = std::move(q);
  S->cv_work.notify_one();
  return GIM_OK;
}

gim_status gim_server_poll(gim_server *S, uint64_t ticket, uint32_t timeout_ms, int *done, uint32_t *seeds_out,
                           gim_imm_result *result, double *latency_ms) {
  if (!S || !done) return GIM_ERR_ARG;
  std::unique_lock<std::mutex> lock(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return GIM_ERR_ARG;
  Query *q = it->second.get();
  if (!q->done && timeout_ms)
    S->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), [&] { return q->done; });
  *done = q->done ? 1 : 0;
  if (!q->done) return GIM_OK;
  if (q->status != GIM_OK) return q->status;
  if (seeds_out) std::copy(q->seeds.begin(), q->seeds.end(), seeds_out);
  if (result) *result = q->res;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(q->t_done - q->t_submit).count();
  return GIM_OK;
}

gim_status gim_server_stats(gim_server *S, double out[8]) {
  if (!S || !out) return GIM_ERR_ARG;
  std::lock_guard<std::mutex> lock(S->mu);
  out[0] = (double)S->completed;
  out[1] = (double)S->rounds;
  out[2] = S->busy_ms;
  out[3] = S->sample_ms;
  out[4] = S->select_ms;
  out[5] = (double)S->peak_active;
  out[6] = (double)S->waiting.size();
  double pool_sets = 0;
  for (auto &kv : S->pools) pool_sets += (double)kv.second->R;
  out[7] = pool_sets;
  return GIM_OK;
}

void gim_server_stop(gim_server *S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stopping = true;
    for (Query *q : S->waiting) {   // never admitted
      q->status = GIM_ERR_STATE;
      q->done = true;
    }
    S->waiting.clear();
    S->cv_work.notify_all();
    S->cv_done.notify_all();
  }
  if (S->worker.joinable()) S->worker.join();
  cudaSetDevice(S->graph->device);
  cudaStreamSynchronize(S->stream);
  for (auto &kv : S->pools) gim_destroy(kv.second);
  gim_destroy(S->self);
  for (SelectBuffers &b : S->slot_buf) free_select_buffers(b);
  for (SelectBuffers &b : S->index_buf) free_select_buffers(b);
  cudaStreamDestroy(S->stream);
  delete S;
}

}  // extern "C"
