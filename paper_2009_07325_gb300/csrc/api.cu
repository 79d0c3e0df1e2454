// C ABI of libgim (declared in include/gim.h): context management, graph
// upload, RR sampling orchestration, greedy selection and the IMM driver.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "gim_internal.cuh"

using namespace gim;

namespace {

constexpr int kBlock = 256;
constexpr int kWarpsPerBlock = kBlock / 32;
constexpr uint32_t kIcQueueCap = 4096;        // per-worker queue of the common-case IC pass
constexpr uint32_t kLtPathCap = 1024;         // per-warp shared-memory path of the common-case LT pass
constexpr uint64_t kScratchBudget = 4ull << 30;   // bytes of visited bitmaps + queues per pass
constexpr uint64_t kInitialStore = 1ull << 26;    // store entries at first use

gim_status set_err(gim_ctx *ctx, gim_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->last_error = buf;
  return st;
}

gim_status cuda_err(gim_ctx *ctx, cudaError_t e, const char *what) {
  cudaGetLastError();   // clear a non-sticky error so the context stays usable
  if (e == cudaErrorMemoryAllocation) return set_err(ctx, GIM_ERR_OOM, "%s: out of device memory", what);
  return set_err(ctx, GIM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CU(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_err(ctx, e_, #call);   \
  } while (0)

template <typename T>
void dfree(T *&p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void free_graph(DevGraph &g) {
  dfree(g.off);
  dfree(g.src);
  dfree(g.thr);
  dfree(g.rthr);
  dfree(g.cum);
  g = DevGraph{};
}

void free_scratch(WorkerScratch &w) {
  dfree(w.bitmap);
  dfree(w.queue);
  w = WorkerScratch{};
}

void free_select(SelectBuffers &b) {
  dfree(b.cnt_work);
  dfree(b.inv_off);
  dfree(b.cursor);
  dfree(b.inv);
  dfree(b.covered);
  dfree(b.best);
  dfree(b.seeds);
  dfree(b.gains);
  dfree(b.covered_total);
  dfree(b.scan_tmp);
  b = SelectBuffers{};
}

// Allocates zeroed per-worker scratch: `workers` workers, each with a visited
// bitmap of n bits and a queue of qcap entries (either may be skipped).
cudaError_t alloc_scratch(WorkerScratch &w, uint32_t n, uint32_t workers, uint32_t qcap, bool bitmap, bool queue,
                          cudaStream_t s) {
  free_scratch(w);
  w.workers = workers;
  w.qcap = qcap;
  w.words_per_worker = bitmap ? ((uint64_t)n + 31) / 32 : 0;
  w.words_per_worker = (w.words_per_worker + 31) / 32 * 32;   // 128-byte aligned per worker
  cudaError_t e;
  if (bitmap) {
    if ((e = cudaMalloc(&w.bitmap, w.words_per_worker * workers * 4)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w.bitmap, 0, w.words_per_worker * workers * 4, s)) != cudaSuccess) return e;
  }
  if (queue) {
    if ((e = cudaMalloc(&w.queue, (uint64_t)qcap * workers * 4)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

uint32_t cap_workers(uint64_t per_worker_bytes, uint32_t want) {
  const uint64_t lim = std::max<uint64_t>(kWarpsPerBlock, kScratchBudget / std::max<uint64_t>(per_worker_bytes, 1));
  uint64_t w = std::min<uint64_t>(want, lim);
  w = w / kWarpsPerBlock * kWarpsPerBlock;
  return (uint32_t)std::max<uint64_t>(w, kWarpsPerBlock);
}

template <typename T>
cudaError_t grow_copy(T *&p, uint64_t &cap, uint64_t need, uint64_t keep, cudaStream_t s) {
  if (need <= cap && p) return cudaSuccess;
  const uint64_t c = std::max<uint64_t>(need, cap * 2);
  T *q = nullptr;
  cudaError_t e = cudaMalloc(&q, c * sizeof(T));
  if (e != cudaSuccess) return e;
  if (p && keep) {
    e = cudaMemcpyAsync(q, p, keep * sizeof(T), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
      cudaFree(q);
      return e;
    }
  }
  if (p) {
    cudaStreamSynchronize(s);
    cudaFree(p);
  }
  p = q;
  cap = c;
  return cudaSuccess;
}

double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// ---------------------------------------------------------------------------
// Sampling orchestration.
// ---------------------------------------------------------------------------
// Runs one sampling launch and reads its counters back.
gim_status run_pass(gim_ctx *ctx, int model, bool large, const WorkerScratch &ws, const SampleJob &job) {
  SampleCtl init{};
  init.store_tail = ctx->store_used;
  CU(cudaMemcpyAsync(ctx->ctl, &init, sizeof init, cudaMemcpyHostToDevice, ctx->stream));
  const uint32_t workers = large ? (uint32_t)std::min<uint64_t>(ws.workers, job.count) : ws.workers;
  WorkerScratch w = ws;
  w.workers = std::max<uint32_t>(workers, 1);
  const int grid = (int)((w.workers + kWarpsPerBlock - 1) / kWarpsPerBlock);
  CU(cudaEventRecord(ctx->ev[6], ctx->stream));
  CU(launch_sample(model, ctx->g, ctx->st, w, job, ctx->ctl, large, grid, kBlock, ctx->stream));
  CU(cudaEventRecord(ctx->ev[7], ctx->stream));
  ctx->launches++;
  CU(cudaMemcpyAsync(ctx->ctl_host, ctx->ctl, sizeof(SampleCtl), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  float ms = 0;
  cudaEventElapsedTime(&ms, ctx->ev[6], ctx->ev[7]);
  ctx->t_kernel_ms[large ? 1 : 0] += ms;
  ctx->n_kernel[large ? 1 : 0] += 1;
  return GIM_OK;
}

// After a pass: account stored members, grow the store if reservations ran past it.
gim_status settle_store(gim_ctx *ctx) {
  const SampleCtl &c = *ctx->ctl_host;
  if (c.err & kErrDeferredFull) return set_err(ctx, GIM_ERR_OOM, "deferred-set list overflow");
  ctx->Z += c.members;
  if (c.store_tail > ctx->st.cap) {
    const uint64_t old = ctx->st.cap;
    const uint64_t want = std::max<uint64_t>(old * 2, c.store_tail * 2);
    uint64_t cap = ctx->st.cap;
    CU(grow_copy(ctx->st.members, cap, want, ctx->st.cap, ctx->stream));
    ctx->st.cap = cap;
    ctx->store_used = old;   // the last partial reservation leaves a hole below the old end
  } else {
    ctx->store_used = c.store_tail;
  }
  return GIM_OK;
}

gim_status ensure_large_scratch(gim_ctx *ctx) {
  if (ctx->ws_large.workers) return GIM_OK;
  const uint32_t n = ctx->g.n;
  const uint64_t per = ((uint64_t)n + 31) / 32 * 4 + (uint64_t)n * 4;
  const uint32_t want = (uint32_t)ctx->sm_count * 16;
  CU(alloc_scratch(ctx->ws_large, n, cap_workers(per, want), n, true, true, ctx->stream));
  return GIM_OK;
}

// Appends RR sets [R, R + count) under (model, seed). On failure rolls the
// occurrence counts back so that the collection is as before.
gim_status sample_range(gim_ctx *ctx, int model, uint64_t seed, uint64_t count) {
  const uint64_t R0 = ctx->R, Z0 = ctx->Z, used0 = ctx->store_used;
  gim_status st = GIM_OK;
  auto rollback = [&]() {
    launch_uncount(ctx->st, R0, count, ctx->stream);
    ctx->launches++;
    cudaStreamSynchronize(ctx->stream);
    ctx->Z = Z0;
    ctx->store_used = used0;
  };
  // capacities
  {
    uint64_t cap = ctx->rr_cap, cap2 = ctx->rr_cap;
    CU(grow_copy(ctx->st.rr_start, cap, R0 + count, R0, ctx->stream));
    CU(grow_copy(ctx->st.rr_len, cap2, R0 + count, R0, ctx->stream));
    ctx->rr_cap = std::min(cap, cap2);
  }
  CU(cudaMemsetAsync(ctx->st.rr_start + R0, 0xFF, count * sizeof(uint64_t), ctx->stream));
  if (!ctx->st.members) {
    uint64_t cap = 0;
    CU(grow_copy(ctx->st.members, cap, kInitialStore, 0, ctx->stream));
    ctx->st.cap = cap;
  }
  {
    uint64_t dcap = ctx->deferred_cap;
    CU(grow_copy(ctx->deferred, dcap, 2 * count, 0, ctx->stream));
    ctx->deferred_cap = dcap;
  }
  uint64_t *list_a = ctx->deferred, *list_b = ctx->deferred + count;

  SampleJob job{};
  job.key = PhiloxKey{(uint32_t)seed, (uint32_t)(seed >> 32)};
  job.j_begin = R0;
  job.count = count;
  job.j_list = nullptr;
  job.deferred = list_a;
  job.deferred_cap = count;
  const WorkerScratch &ws = model == GIM_IC ? ctx->ws_small : ctx->ws_lt;
  if ((st = run_pass(ctx, model, false, ws, job)) != GIM_OK) return rollback(), st;
  if ((st = settle_store(ctx)) != GIM_OK) return rollback(), st;
  uint64_t pending = ctx->ctl_host->n_deferred;
  int rounds = 0;
  while (pending > 0) {
    if (++rounds > 40) {
      rollback();
      return set_err(ctx, GIM_ERR_OOM, "large-set pass did not converge");
    }
    if ((st = ensure_large_scratch(ctx)) != GIM_OK) return rollback(), st;
    SampleJob lj = job;
    lj.j_list = list_a;
    lj.count = pending;
    lj.deferred = list_b;
    lj.deferred_cap = count;
    if ((st = run_pass(ctx, model, true, ctx->ws_large, lj)) != GIM_OK) return rollback(), st;
    if ((st = settle_store(ctx)) != GIM_OK) return rollback(), st;
    pending = ctx->ctl_host->n_deferred;
    std::swap(list_a, list_b);
  }
  ctx->R = R0 + count;
  return GIM_OK;
}

gim_status check_ctx(gim_ctx *ctx) {
  if (!ctx) return GIM_ERR_ARG;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  ctx->last_error.clear();
  return GIM_OK;
}

gim_status do_select(gim_ctx *ctx, uint32_t k, uint32_t *seeds_out, uint64_t *covered_out, uint32_t *gains_out) {
  if (ctx->R >= 0xFFFFFFFFull) return set_err(ctx, GIM_ERR_ARG, "more than 2^32-2 RR sets");
  CU(run_select(ctx->g, ctx->st, ctx->R, ctx->Z, k, ctx->sel, ctx->sm_count, ctx->stream, &ctx->launches));
  CU(cudaMemcpyAsync(seeds_out, ctx->sel.seeds, k * sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
  if (gains_out)
    CU(cudaMemcpyAsync(gains_out, ctx->sel.gains, k * sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
  unsigned long long cov = 0;
  CU(cudaMemcpyAsync(&cov, ctx->sel.covered_total, sizeof cov, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  if (covered_out) *covered_out = cov;
  return GIM_OK;
}

// IMM constants (Tang, Shi, Xiao 2015) in a fixed evaluation order.
struct ImmConst {
  double ellp, epsp, lam1, lam2;
  int i_max;
};

ImmConst imm_constants(uint32_t n, uint32_t k, double eps, double ell) {
  ImmConst c;
  const double logn = std::log((double)n);
  c.ellp = ell * (1.0 + std::log(2.0) / logn);
  c.epsp = std::sqrt(2.0) * eps;
  double lnc = 0.0;
  for (uint32_t i = 0; i < k; ++i) lnc += std::log((double)(n - i)) - std::log((double)(i + 1));
  c.lam1 = (2.0 + 2.0 * c.epsp / 3.0) * (lnc + c.ellp * logn + std::log(std::log2((double)n))) * (double)n /
           (c.epsp * c.epsp);
  const double g = 1.0 - std::exp(-1.0);
  const double alpha = std::sqrt(c.ellp * logn + std::log(2.0));
  const double beta = std::sqrt(g * (lnc + c.ellp * logn + std::log(2.0)));
  const double t = g * alpha + beta;
  c.lam2 = 2.0 * (double)n * t * t / (eps * eps);
  c.i_max = (31 - __builtin_clz(n)) - 1;
  return c;
}

}  // namespace

// ===========================================================================
extern "C" {

gim_status gim_create(gim_ctx **out, int device, void *stream) {
  if (!out) return GIM_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return GIM_ERR_ARG;
  }
  gim_ctx *ctx = new (std::nothrow) gim_ctx();
  if (!ctx) return GIM_ERR_OOM;
  ctx->device = device;
  auto fail = [&](gim_status s) {
    gim_destroy(ctx);
    return s;
  };
  if (cudaSetDevice(device) != cudaSuccess) return fail(GIM_ERR_CUDA);
  if (cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return fail(GIM_ERR_CUDA);
  if (stream) {
    ctx->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(GIM_ERR_CUDA);
    ctx->own_stream = true;
  }
  for (auto &e : ctx->ev)
    if (cudaEventCreate(&e) != cudaSuccess) return fail(GIM_ERR_CUDA);
  if (cudaMalloc(&ctx->ctl, sizeof(SampleCtl)) != cudaSuccess) return fail(GIM_ERR_OOM);
  if (cudaMallocHost(&ctx->ctl_host, sizeof(SampleCtl)) != cudaSuccess) return fail(GIM_ERR_OOM);
  *out = ctx;
  return GIM_OK;
}

void gim_destroy(gim_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  free_graph(ctx->g);
  dfree(ctx->st.members);
  dfree(ctx->st.rr_start);
  dfree(ctx->st.rr_len);
  dfree(ctx->st.cnt);
  free_scratch(ctx->ws_small);
  free_scratch(ctx->ws_lt);
  free_scratch(ctx->ws_large);
  dfree(ctx->deferred);
  free_select(ctx->sel);
  dfree(ctx->ctl);
  if (ctx->ctl_host) cudaFreeHost(ctx->ctl_host);
  for (auto &e : ctx->ev)
    if (e) cudaEventDestroy(e);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char *gim_last_error_string(gim_ctx *ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

gim_status gim_graph_load(gim_ctx *ctx, uint32_t n, uint64_t m, const uint64_t *in_offsets, const uint32_t *in_sources,
                          const float *in_weights) {
  gim_status st = check_ctx(ctx);
  if (st) return st;
  if (n < 2 || n >= 0xFFFFFFFFu) return set_err(ctx, GIM_ERR_ARG, "n must be in [2, 2^32-2]");
  if (m >= 0xFFFFFFFCull) return set_err(ctx, GIM_ERR_ARG, "m must be below 2^32-4");
  if (!in_offsets || (m > 0 && (!in_sources || !in_weights))) return set_err(ctx, GIM_ERR_ARG, "null input array");
  if (in_offsets[0] != 0 || in_offsets[n] != m) return set_err(ctx, GIM_ERR_ARG, "offsets must start at 0 and end at m");
  std::vector<uint32_t> off32((size_t)n + 1);
  for (uint64_t v = 0; v <= n; ++v) {
    if (v > 0 && in_offsets[v] < in_offsets[v - 1]) return set_err(ctx, GIM_ERR_ARG, "offsets decrease at row %llu",
                                                                   (unsigned long long)v - 1);
    off32[v] = (uint32_t)in_offsets[v];
  }
  const uint64_t m_pad = (m + 3) / 4 * 4 + 4;
  DevGraph g;
  g.n = n;
  g.m = m;
  float *d_w = nullptr;
  unsigned int *d_flags = nullptr;
  unsigned int flags = 0;
  cudaError_t e = cudaSuccess;
  auto bail = [&](cudaError_t err, const char *what) {
    free_graph(g);
    dfree(d_w);
    dfree(d_flags);
    return cuda_err(ctx, err, what);
  };
  if ((e = cudaMalloc(&g.off, ((uint64_t)n + 1) * 4)) != cudaSuccess) return bail(e, "alloc offsets");
  if ((e = cudaMalloc(&g.src, m_pad * 4)) != cudaSuccess) return bail(e, "alloc sources");
  if ((e = cudaMalloc(&g.thr, m_pad * 4)) != cudaSuccess) return bail(e, "alloc thresholds");
  if ((e = cudaMalloc(&g.rthr, (uint64_t)n * 4)) != cudaSuccess) return bail(e, "alloc row thresholds");
  if ((e = cudaMalloc(&g.cum, std::max<uint64_t>(m, 1) * 8)) != cudaSuccess) return bail(e, "alloc lt thresholds");
  if ((e = cudaMalloc(&d_w, std::max<uint64_t>(m, 1) * 4)) != cudaSuccess) return bail(e, "alloc weights");
  if ((e = cudaMalloc(&d_flags, 4)) != cudaSuccess) return bail(e, "alloc flags");
  cudaStream_t s = ctx->stream;
  if ((e = cudaMemcpyAsync(g.off, off32.data(), ((uint64_t)n + 1) * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return bail(e, "upload offsets");
  if ((e = cudaMemsetAsync(g.src, 0, m_pad * 4, s)) != cudaSuccess) return bail(e, "clear sources");
  if (m) {
    if ((e = cudaMemcpyAsync(g.src, in_sources, m * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return bail(e, "upload sources");
    if ((e = cudaMemcpyAsync(d_w, in_weights, m * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return bail(e, "upload weights");
  }
  if ((e = cudaMemsetAsync(d_flags, 0, 4, s)) != cudaSuccess) return bail(e, "clear flags");
  if ((e = launch_graph_prep(g, d_w, d_flags, s)) != cudaSuccess) return bail(e, "graph preprocessing");
  ctx->launches += 2;
  if ((e = cudaMemcpyAsync(&flags, d_flags, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return bail(e, "flags");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return bail(e, "graph preprocessing");
  dfree(d_w);
  dfree(d_flags);
  if (flags & (kGraphBadSource | kGraphNotAscending | kGraphBadWeight)) {
    free_graph(g);
    return set_err(ctx, GIM_ERR_ARG, "%s%s%s", (flags & kGraphBadSource) ? "source id >= n; " : "",
                   (flags & kGraphNotAscending) ? "sources not strictly ascending within a row; " : "",
                   (flags & kGraphBadWeight) ? "weight outside [0, 1]; " : "");
  }

  // commit: replace the graph, empty the collection, size the scratch for n
  cudaStreamSynchronize(s);
  free_graph(ctx->g);
  ctx->g = g;
  ctx->has_graph = true;
  ctx->lt_ok = (flags & kGraphNotLT) ? 0 : 1;
  dfree(ctx->st.cnt);
  free_scratch(ctx->ws_small);
  free_scratch(ctx->ws_lt);
  free_scratch(ctx->ws_large);
  free_select(ctx->sel);
  ctx->R = ctx->Z = ctx->store_used = 0;
  ctx->model = -1;
  CU(cudaMalloc(&ctx->st.cnt, (uint64_t)n * 4 + 16));
  CU(cudaMemsetAsync(ctx->st.cnt, 0, (uint64_t)n * 4 + 16, s));
  {
    const uint64_t per = ((uint64_t)n + 31) / 32 * 4 + kIcQueueCap * 4;
    const uint32_t want = (uint32_t)ctx->sm_count * 64;   // up to 64 warps per SM
    CU(alloc_scratch(ctx->ws_small, n, cap_workers(per, want), kIcQueueCap, true, true, s));
    ctx->ws_lt = WorkerScratch{};
    ctx->ws_lt.workers = (uint32_t)ctx->sm_count * 48;   // 6 blocks of 8 warps with 32 KB shared memory each
    ctx->ws_lt.qcap = kLtPathCap;
  }
  CU(cudaStreamSynchronize(s));
  return GIM_OK;
}

gim_status gim_graph_lt_valid(gim_ctx *ctx, int *out) {
  gim_status st = check_ctx(ctx);
  if (st) return st;
  if (!out) return set_err(ctx, GIM_ERR_ARG, "out is null");
  if (!ctx->has_graph) return set_err(ctx, GIM_ERR_STATE, "no graph loaded");
  *out = ctx->lt_ok;
  return GIM_OK;
}

gim_status gim_sample_rr(gim_ctx *ctx, gim_model model, uint64_t count, uint64_t seed) {
  gim_status st = check_ctx(ctx);
  if (st) return st;
  const auto t0 = std::chrono::steady_clock::now();
  if (!ctx->has_graph) return set_err(ctx, GIM_ERR_STATE, "no graph loaded");
  if (model != GIM_IC && model != GIM_LT) return set_err(ctx, GIM_ERR_ARG, "unknown model");
  if (model == GIM_LT && !ctx->lt_ok) return set_err(ctx, GIM_ERR_ARG, "graph weights are not valid for LT");
  if (ctx->R > 0 && (ctx->model != (int)model || ctx->seed != seed))
    return set_err(ctx, GIM_ERR_STATE, "model/seed differ from the stored collection; call gim_reset_rr");
  if (ctx->R + count >= 0xFFFFFFFFull) return set_err(ctx, GIM_ERR_ARG, "more than 2^32-2 RR sets");
  if (count == 0) return GIM_OK;
  CU(cudaEventRecord(ctx->ev[0], ctx->stream));
  st = sample_range(ctx, model, seed, count);
  if (st) return st;
  ctx->model = model;
  ctx->seed = seed;
  CU(cudaEventRecord(ctx->ev[1], ctx->stream));
  CU(cudaEventSynchronize(ctx->ev[1]));
  float ms = 0;
  cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
  ctx->t_sample_ms = ms;
  ctx->t_select_ms = 0;
  ctx->t_wall_ms = ms_since(t0);
  ctx->lb_rounds = 0;
  return GIM_OK;
}

gim_status gim_reset_rr(gim_ctx *ctx) {
  gim_status st = check_ctx(ctx);
  if (st) return st;
  if (!ctx->has_graph) return GIM_OK;
  ctx->R = ctx->Z = ctx->store_used = 0;
  ctx->model = -1;
  CU(cudaMemsetAsync(ctx->st.cnt, 0, (uint64_t)ctx->g.n * 4, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return GIM_OK;
}

gim_status gim_select_seeds(gim_ctx *ctx, uint32_t k, uint32_t *seeds_out, uint64_t *covered_out,
                            uint32_t *gains_out) {
  gim_status st = check_ctx(ctx);
  if (st) return st;
  const auto t0 = std::chrono::steady_clock::now();
  if (!ctx->has_graph) return set_err(ctx, GIM_ERR_STATE, "no graph loaded");
  if (k == 0 || k > ctx->g.n || !seeds_out) return set_err(ctx, GIM_ERR_ARG, "need 1 <= k <= n and seeds_out");
  CU(cudaEventRecord(ctx->ev[2], ctx->stream));
  st = do_select(ctx, k, seeds_out, covered_out, gains_out);
  if (st) return st;
  CU(cudaEventRecord(ctx->ev[3], ctx->stream));
  CU(cudaEventSynchronize(ctx->ev[3]));
  float ms = 0;
  cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]);
  ctx->t_sample_ms = 0;
  ctx->t_select_ms = ms;
  ctx->t_wall_ms = ms_since(t0);
  ctx->lb_rounds = 0;
  return GIM_OK;
}

gim_status gim_imm(gim_ctx *ctx, gim_model model, uint32_t k, double eps, double ell, uint64_t seed,
                   uint32_t *seeds_out, uint64_t *theta_out, double *lb_out) {
  gim_status st = check_ctx(ctx);
  if (st) return st;
  const auto t0 = std::chrono::steady_clock::now();
  if (!ctx->has_graph) return set_err(ctx, GIM_ERR_STATE, "no graph loaded");
  if (model != GIM_IC && model != GIM_LT) return set_err(ctx, GIM_ERR_ARG, "unknown model");
  if (k == 0 || k > ctx->g.n || !seeds_out) return set_err(ctx, GIM_ERR_ARG, "need 1 <= k <= n and seeds_out");
  if (!(eps > 0.0 && eps < 1.0)) return set_err(ctx, GIM_ERR_ARG, "eps must be in (0, 1)");
  if (!(ell > 0.0)) return set_err(ctx, GIM_ERR_ARG, "ell must be > 0");
  if (model == GIM_LT && !ctx->lt_ok) return set_err(ctx, GIM_ERR_ARG, "graph weights are not valid for LT");
  if ((st = gim_reset_rr(ctx)) != GIM_OK) return st;

  const uint32_t n = ctx->g.n;
  const ImmConst c = imm_constants(n, k, eps, ell);
  double t_sample = 0, t_select = 0;
  auto timed = [&](double &acc, auto &&fn) -> gim_status {
    cudaEventRecord(ctx->ev[4], ctx->stream);
    gim_status r = fn();
    cudaEventRecord(ctx->ev[5], ctx->stream);
    cudaEventSynchronize(ctx->ev[5]);
    float ms = 0;
    cudaEventElapsedTime(&ms, ctx->ev[4], ctx->ev[5]);
    acc += ms;
    return r;
  };
  auto sample_to = [&](uint64_t target) -> gim_status {
    if (ctx->R >= target) return GIM_OK;
    if (target >= 0xFFFFFFFFull) return set_err(ctx, GIM_ERR_ARG, "theta above 2^32-2 RR sets");
    const uint64_t cnt = target - ctx->R;
    return timed(t_sample, [&] {
      gim_status r = sample_range(ctx, model, seed, cnt);
      if (r == GIM_OK) {
        ctx->model = model;
        ctx->seed = seed;
      }
      return r;
    });
  };
  double LB = 1.0;
  int rounds = 0;
  for (int i = 1; i <= c.i_max; ++i) {
    const double x = (double)n / std::ldexp(1.0, i);
    const uint64_t theta_i = (uint64_t)std::ceil(c.lam1 / x);
    if ((st = sample_to(theta_i)) != GIM_OK) return st;
    uint64_t cov = 0;
    if ((st = timed(t_select, [&] { return do_select(ctx, k, seeds_out, &cov, nullptr); })) != GIM_OK) return st;
    ++rounds;
    const double est = ((double)n * (double)cov) / (double)ctx->R;
    if (est >= (1.0 + c.epsp) * x) {
      LB = est / (1.0 + c.epsp);
      break;
    }
  }
  const uint64_t theta = (uint64_t)std::ceil(c.lam2 / LB);
  if ((st = sample_to(theta)) != GIM_OK) return st;
  if ((st = timed(t_select, [&] { return do_select(ctx, k, seeds_out, nullptr, nullptr); })) != GIM_OK) return st;
  if (theta_out) *theta_out = theta;
  if (lb_out) *lb_out = LB;
  ctx->t_sample_ms = t_sample;
  ctx->t_select_ms = t_select;
  ctx->t_wall_ms = ms_since(t0);
  ctx->lb_rounds = rounds;
  return GIM_OK;
}

gim_status gim_rr_count(gim_ctx *ctx, uint64_t *count_out, uint64_t *members_out) {
  gim_status st = check_ctx(ctx);
  if (st) return st;
  if (!count_out) return set_err(ctx, GIM_ERR_ARG, "count_out is null");
  *count_out = ctx->R;
  if (members_out) *members_out = ctx->Z;
  return GIM_OK;
}

gim_status gim_rr_export(gim_ctx *ctx, uint64_t *offsets_out, uint32_t *members_out) {
  gim_status st = check_ctx(ctx);
  if (st) return st;
  if (!offsets_out || (ctx->Z > 0 && !members_out)) return set_err(ctx, GIM_ERR_ARG, "null output");
  const uint64_t R = ctx->R;
  std::vector<uint64_t> start(R);
  std::vector<uint32_t> len(R);
  std::vector<uint32_t> store(ctx->store_used);
  if (R) {
    CU(cudaMemcpyAsync(start.data(), ctx->st.rr_start, R * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(len.data(), ctx->st.rr_len, R * 4, cudaMemcpyDeviceToHost, ctx->stream));
  }
  if (ctx->store_used)
    CU(cudaMemcpyAsync(store.data(), ctx->st.members, ctx->store_used * 4, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  offsets_out[0] = 0;
  for (uint64_t j = 0; j < R; ++j) {
    const uint64_t o = offsets_out[j];
    if (start[j] == kNoStart || start[j] + len[j] > ctx->store_used)
      return set_err(ctx, GIM_ERR_STATE, "RR set %llu is not stored", (unsigned long long)j);
    std::memcpy(members_out + o, store.data() + start[j], (size_t)len[j] * 4);
    std::sort(members_out + o, members_out + o + len[j]);
    offsets_out[j + 1] = o + len[j];
  }
  return GIM_OK;
}

gim_status gim_coverage_export(gim_ctx *ctx, uint32_t *cnt_out) {
  gim_status st = check_ctx(ctx);
  if (st) return st;
  if (!ctx->has_graph) return set_err(ctx, GIM_ERR_STATE, "no graph loaded");
  if (!cnt_out) return set_err(ctx, GIM_ERR_ARG, "cnt_out is null");
  CU(cudaMemcpyAsync(cnt_out, ctx->st.cnt, (uint64_t)ctx->g.n * 4, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return GIM_OK;
}

gim_status gim_last_timings(gim_ctx *ctx, double out[8]) {
  if (!ctx || !out) return GIM_ERR_ARG;
  out[0] = ctx->t_sample_ms;
  out[1] = ctx->t_select_ms;
  out[2] = ctx->t_wall_ms;
  out[3] = ctx->lb_rounds;
  out[4] = ctx->t_kernel_ms[0];
  out[5] = ctx->n_kernel[0];
  out[6] = ctx->t_kernel_ms[1];
  out[7] = ctx->n_kernel[1];
  return GIM_OK;
}

gim_status gim_reset_timings(gim_ctx *ctx) {
  if (!ctx) return GIM_ERR_ARG;
  ctx->t_kernel_ms[0] = ctx->t_kernel_ms[1] = 0;
  ctx->n_kernel[0] = ctx->n_kernel[1] = 0;
  return GIM_OK;
}

gim_status gim_diag_philox_rate(gim_ctx *ctx, double *calls_per_s) {
  gim_status st = check_ctx(ctx);
  if (st) return st;
  if (!calls_per_s) return set_err(ctx, GIM_ERR_ARG, "calls_per_s is null");
  uint32_t *sink = nullptr;
  CU(cudaMalloc(&sink, 1024 * 4));
  const int blocks = ctx->sm_count * 8;
  const uint32_t per_thread = 4096;
  float best = 0;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(ctx->ev[6], ctx->stream);
    cudaError_t e = launch_philox_rate(blocks, per_thread, sink, ctx->stream);
    cudaEventRecord(ctx->ev[7], ctx->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(ctx->ev[7]);
    if (e != cudaSuccess) {
      cudaFree(sink);
      return cuda_err(ctx, e, "philox rate kernel");
    }
    ctx->launches++;
    float ms = 0;
    cudaEventElapsedTime(&ms, ctx->ev[6], ctx->ev[7]);
    if (rep > 0 && (best == 0 || ms < best)) best = ms;
  }
  cudaFree(sink);
  *calls_per_s = (double)blocks * 256.0 * per_thread / (best / 1e3);
  return GIM_OK;
}

gim_status gim_launch_count(gim_ctx *ctx, uint64_t *out) {
  if (!ctx || !out) return GIM_ERR_ARG;
  *out = ctx->launches;
  return GIM_OK;
}

}  // extern "C"
