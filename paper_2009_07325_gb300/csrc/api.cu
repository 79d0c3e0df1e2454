// C ABI of libgim (declared in include/gim.h): context management, graph
// upload, RR sampling orchestration, greedy selection and the IMM driver.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "gim_internal.cuh"

using namespace gim;

namespace {

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
  dfree(g.rw);
  dfree(g.cum);
  dfree(g.w);
  dfree(g.off64);
  g = DevGraph{};
}

}  // namespace

void gim::free_select_buffers(SelectBuffers &b) {
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
  dfree(b.cnt_own);
  dfree(b.hslot);
  dfree(b.hbits);
  dfree(b.hmeta);
  b = SelectBuffers{};
}

namespace {

void free_select(SelectBuffers &b) { free_select_buffers(b); }

double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// Appends RR sets [R, R + count) of ctx under (model, seed).
gim_status sample_range(gim_ctx *ctx, int model, uint64_t seed, uint64_t count) {
  std::vector<SampleJobH> jobs{SampleJobH{ctx, model, seed, count}};
  return sample_jobs(jobs, ctx->stream);
}

gim_status check_ctx(gim_ctx *ctx) {
  if (!ctx) return GIM_ERR_ARG;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  ctx->last_error.clear();
  return GIM_OK;
}

// Greedy selection over the context's collection: k seeds, or k per round
// (k * T picks over the T * n elements) on a multi-round collection.
gim_status do_select(gim_ctx *ctx, uint32_t k, uint32_t *seeds_out, uint64_t *covered_out, uint32_t *gains_out) {
  if (ctx->R >= 0xFFFFFFFFull) return set_err(ctx, GIM_ERR_ARG, "more than 2^32-2 RR sets");
  const uint32_t T = ctx->rounds, U = ctx->g.n * T, picks = k * T;
  // a one-slot batched selection, configured for this universe and the most picks asked so far
  if (!ctx->msel || ctx->msel_n != U || ctx->msel_k < picks) {
    delete ctx->msel;
    ctx->msel = new (std::nothrow) MultiSelect();
    if (!ctx->msel) return set_err(ctx, GIM_ERR_OOM, "selection state");
    const uint32_t kc = std::max(picks, ctx->msel_n == U ? ctx->msel_k : 0u);
    ctx->msel_n = U;
    ctx->msel_k = 0;
    gim_status st = ctx->msel->configure(ctx, {U}, {kc});
    if (st != GIM_OK) return st;
    ctx->msel_k = kc;
  }
  SelInput x;
  x.active = true;
  x.R = ctx->R;
  x.Z = ctx->Z;
  x.members = ctx->st.members;
  x.rr_start = ctx->st.rr_start;
  x.rr_len = ctx->st.rr_len;
  x.cnt = ctx->st.cnt;
  x.buf = &ctx->sel;
  x.k = picks;
  x.skip = ctx->skip_vertex;
  if (T > 1) {
    x.part_n = ctx->g.n;
    x.part_k = k;
  }
  std::vector<unsigned long long> cov;
  std::vector<uint32_t> seeds, gains;
  gim_status st = ctx->msel->run(ctx, {x}, ctx->stream, cov, seeds, gains_out ? &gains : nullptr);
  if (st != GIM_OK) return st;
  std::memcpy(seeds_out, seeds.data(), picks * sizeof(uint32_t));
  if (gains_out) std::memcpy(gains_out, gains.data(), picks * sizeof(uint32_t));
  if (covered_out) *covered_out = cov[0];
  return GIM_OK;
}

// IMM (T = 1) or multi-round IM (CR-NAIMM, T > 1): Alg. 2's lower-bound
// search, then theta sets and the final greedy (Alg. 1). With T > 1 the sets
// are multi-round RR sets and every selection takes k seeds per round.
gim_status run_imm(gim_ctx *ctx, gim_model model, uint32_t T, uint32_t k, double eps, double ell, uint64_t seed,
                   uint32_t *seeds_out, uint64_t *theta_out, double *lb_out) {
  gim_status st = check_ctx(ctx);
  if (st) return st;
  const auto t0 = std::chrono::steady_clock::now();
  if (!ctx->has_graph) return set_err(ctx, GIM_ERR_STATE, "no graph loaded");
  if (model != GIM_IC && model != GIM_LT) return set_err(ctx, GIM_ERR_ARG, "unknown model");
  if (k == 0 || k > ctx->g.n || !seeds_out) return set_err(ctx, GIM_ERR_ARG, "need 1 <= k <= n and seeds_out");
  if (!(eps > 0.0 && eps < 1.0)) return set_err(ctx, GIM_ERR_ARG, "eps must be in (0, 1)");
  if (!(ell > 0.0)) return set_err(ctx, GIM_ERR_ARG, "ell must be > 0");
  if (model == GIM_LT && !lt_valid(ctx)) return set_err(ctx, GIM_ERR_ARG, "graph weights are not valid for LT");
  if ((st = gim_reset_rr(ctx)) != GIM_OK) return st;
  if (T > 1 && (st = gim_rr_set_rounds(ctx, T)) != GIM_OK) return st;

  const uint32_t n = ctx->g.n;
  const ImmConst c = mrim_constants(n, k, T, eps, ell);
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
      gim_status r = T > 1 ? mrim_sample(ctx, model, seed, cnt) : sample_range(ctx, model, seed, cnt);
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
    // compact collection: the sets drawn from now on that hold the first pick
    // keep only their size (every later selection checks that its first pick
    // is still this vertex, and fails otherwise)
    if (ctx->compact && T == 1 && ctx->skip_vertex == kNoSkip) ctx->skip_vertex = seeds_out[0];
    ++rounds;
    const double est = ((double)n * (double)cov) / (double)ctx->R;
    if (est >= (1.0 + c.epsp) * x) {
      LB = est / (1.0 + c.epsp);
      break;
    }
  }
  const uint64_t theta = (uint64_t)std::ceil(c.lam2 / LB);
  if (ctx->fresh_final && T == 1) {   // theta new sets, rr_ids 2^63 + j, replace the search's collection
    const uint32_t skip = ctx->skip_vertex;   // a compact collection stays compact
    if ((st = gim_reset_rr(ctx)) != GIM_OK) return st;
    ctx->jhi = ctx->rhi = 1u << 31;
    ctx->skip_vertex = skip;
  }
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

}  // namespace

// ===========================================================================
extern "C" {

gim_status gim_create(gim_ctx **out, int device, void *stream) {
  if (!out) return GIM_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev || device >= kMaxDevices) {
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
  {
    const gim_status st = shared_acquire(ctx);
    if (st != GIM_OK) return fail(st);
    ctx->shared_held = true;
  }
  *out = ctx;
  return GIM_OK;
}

void gim_destroy(gim_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  mrim_release(ctx);
  if (ctx->owns_graph) free_graph(ctx->g);
  free_graph(ctx->g_spare);
  dfree(ctx->d_info);
  dfree(ctx->st.members);
  dfree(ctx->st.rr_start);
  dfree(ctx->st.rr_len);
  dfree(ctx->st.cnt);
  free_select(ctx->sel);
  delete ctx->msel;
  ctx->msel = nullptr;
  if (ctx->shared_held) shared_release(ctx->device);
  ctx->shared_held = false;
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
  const uint64_t m_pad = (m + 3) / 4 * 4 + 4;
  cudaStream_t s = ctx->stream;
  // the arrays: those of the graph before the current one when they are large enough
  DevGraph g;
  if (ctx->g_spare.off && ctx->g_spare.n_cap >= n && ctx->g_spare.m_cap >= m_pad) {
    g = ctx->g_spare;
    ctx->g_spare = DevGraph{};
  } else {
    free_graph(ctx->g_spare);
  }
  unsigned int info[4] = {0, 0, 0, 0};   // flags, first decreasing row, largest in-degree, big-row count
  cudaError_t e = cudaSuccess;
  auto bail = [&](cudaError_t err, const char *what) {
    free_graph(g);
    return cuda_err(ctx, err, what);
  };
  if (!g.off) {
    g.n_cap = n;
    g.m_cap = m_pad;
    if ((e = cudaMalloc(&g.off, ((uint64_t)n + 1) * 4)) != cudaSuccess) return bail(e, "alloc offsets");
    if ((e = cudaMalloc(&g.off64, ((uint64_t)n + 1) * 8)) != cudaSuccess) return bail(e, "alloc offsets");
    if ((e = cudaMalloc(&g.src, m_pad * 4)) != cudaSuccess) return bail(e, "alloc sources");
    if ((e = cudaMalloc(&g.thr, m_pad * 4)) != cudaSuccess) return bail(e, "alloc thresholds");
    if ((e = cudaMalloc(&g.rthr, (uint64_t)n * 4)) != cudaSuccess) return bail(e, "alloc row thresholds");
    if ((e = cudaMalloc(&g.rw, (uint64_t)n * 4)) != cudaSuccess) return bail(e, "alloc row weights");
    if ((e = cudaMalloc(&g.w, m_pad * 4)) != cudaSuccess) return bail(e, "alloc weights");
  }
  g.n = n;
  g.m = m;
  if (!ctx->d_info && (e = cudaMalloc(&ctx->d_info, 4 * sizeof(unsigned int))) != cudaSuccess)
    return bail(e, "alloc flags");
  unsigned int *d_info = ctx->d_info;
  // a graph that fails validation leaves its arrays for the next load and the context as it was
  auto reject = [&]() { ctx->g_spare = g; };
  if ((e = cudaMemcpyAsync(g.off64, in_offsets, ((uint64_t)n + 1) * 8, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return bail(e, "upload offsets");
  if ((e = cudaMemsetAsync(g.src + m, 0, (m_pad - m) * 4, s)) != cudaSuccess) return bail(e, "clear padding");
  if (m) {
    if ((e = cudaMemcpyAsync(g.src, in_sources, m * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return bail(e, "upload sources");
    if ((e = cudaMemcpyAsync(g.w, in_weights, m * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return bail(e, "upload weights");
  }
  if ((e = cudaMemsetAsync(d_info, 0, 4, s)) != cudaSuccess) return bail(e, "clear flags");
  if ((e = cudaMemsetAsync(d_info + 1, 0xFF, 4, s)) != cudaSuccess) return bail(e, "clear flags");
  if ((e = cudaMemsetAsync(d_info + 2, 0, 8, s)) != cudaSuccess) return bail(e, "clear flags");
  if ((e = launch_offsets_prep(g, d_info, s)) != cudaSuccess) return bail(e, "offsets");
  if ((e = cudaMemcpyAsync(info, d_info, 3 * sizeof(unsigned int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return bail(e, "offsets");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return bail(e, "offsets");
  ctx->launches += 1;
  if (info[0] & kGraphBadOffsets) {
    reject();
    return set_err(ctx, GIM_ERR_ARG, "offsets decrease at row %u", info[1]);
  }
  const uint32_t max_indeg = info[2];
  // offsets are valid (non-decreasing from 0 to m): the edge and row passes stay in bounds
  if ((e = launch_graph_prep(g, d_info, s)) != cudaSuccess) return bail(e, "graph preprocessing");
  ctx->launches += 3;
  if ((e = cudaMemcpyAsync(info, d_info, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return bail(e, "flags");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return bail(e, "graph preprocessing");
  const unsigned int flags = info[0];
  if (flags & (kGraphBadSource | kGraphNotAscending | kGraphBadWeight)) {
    reject();
    return set_err(ctx, GIM_ERR_ARG, "%s%s%s", (flags & kGraphBadSource) ? "source id >= n; " : "",
                   (flags & kGraphNotAscending) ? "sources not strictly ascending within a row; " : "",
                   (flags & kGraphBadWeight) ? "weight outside [0, 1]; " : "");
  }

  // commit: replace the graph (its arrays are kept for the next load) and empty the collection
  if (ctx->owns_graph && ctx->g.off) {
    free_graph(ctx->g_spare);
    ctx->g_spare = ctx->g;
  }
  ctx->owns_graph = true;
  ctx->g = g;
  ctx->has_graph = true;
  ctx->lt_ok = -1;   // the LT thresholds are built on the first LT use
  ctx->max_indeg = max_indeg;
  ctx->R = ctx->Z = ctx->store_used = 0;
  ctx->model = -1;
  ctx->jhi = ctx->rhi = 0;
  ctx->rounds = 1;
  ctx->skip_vertex = kNoSkip;
  if (ctx->cnt_cap < (uint64_t)n + 4) {
    dfree(ctx->st.cnt);
    ctx->cnt_cap = 0;
    CU(cudaMalloc(&ctx->st.cnt, (uint64_t)n * 4 + 16));
    ctx->cnt_cap = (uint64_t)n + 4;
  }
  CU(cudaMemsetAsync(ctx->st.cnt, 0, (uint64_t)n * 4 + 16, s));
  CU(cudaStreamSynchronize(s));
  return GIM_OK;
}

gim_status gim_graph_lt_valid(gim_ctx *ctx, int *out) {
  gim_status st = check_ctx(ctx);
  if (st) return st;
  if (!out) return set_err(ctx, GIM_ERR_ARG, "out is null");
  if (!ctx->has_graph) return set_err(ctx, GIM_ERR_STATE, "no graph loaded");
  if ((st = ensure_lt(ctx)) != GIM_OK) return st;
  *out = ctx->lt_ok;
  return GIM_OK;
}

gim_status gim_sample_rr(gim_ctx *ctx, gim_model model, uint64_t count, uint64_t seed) {
  gim_status st = check_ctx(ctx);
  if (st) return st;
  const auto t0 = std::chrono::steady_clock::now();
  if (!ctx->has_graph) return set_err(ctx, GIM_ERR_STATE, "no graph loaded");
  if (model != GIM_IC && model != GIM_LT) return set_err(ctx, GIM_ERR_ARG, "unknown model");
  if (model == GIM_LT && !lt_valid(ctx)) return set_err(ctx, GIM_ERR_ARG, "graph weights are not valid for LT");
  if (ctx->R > 0 && (ctx->model != (int)model || ctx->seed != seed))
    return set_err(ctx, GIM_ERR_STATE, "model/seed differ from the stored collection; call gim_reset_rr");
  if (ctx->R + count >= 0xFFFFFFFFull) return set_err(ctx, GIM_ERR_ARG, "more than 2^32-2 RR sets");
  if (count == 0) return GIM_OK;
  CU(cudaEventRecord(ctx->ev[0], ctx->stream));
  st = ctx->rounds > 1 ? mrim_sample(ctx, model, seed, count) : sample_range(ctx, model, seed, count);
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
  ctx->jhi = ctx->rhi = 0;
  ctx->skip_vertex = kNoSkip;
  CU(cudaMemsetAsync(ctx->st.cnt, 0, (uint64_t)ctx->g.n * ctx->rounds * 4, ctx->stream));
  ctx->rounds = 1;
  CU(cudaStreamSynchronize(ctx->stream));
  return GIM_OK;
}

gim_status gim_rr_set_rounds(gim_ctx *ctx, uint32_t T) {
  gim_status st = check_ctx(ctx);
  if (st) return st;
  if (!ctx->has_graph) return set_err(ctx, GIM_ERR_STATE, "no graph loaded");
  if (ctx->R != 0) return set_err(ctx, GIM_ERR_STATE, "the collection is not empty; call gim_reset_rr");
  if (T < 1 || T > kMaxRounds) return set_err(ctx, GIM_ERR_ARG, "rounds must be in [1, %u]", kMaxRounds);
  const uint64_t U = (uint64_t)ctx->g.n * T;
  if (U >= 0xFFFFFFFFull) return set_err(ctx, GIM_ERR_ARG, "n * rounds must stay below 2^32 - 1");
  if (ctx->cnt_cap < U + 4) {
    uint32_t *c = nullptr;
    CU(cudaMalloc(&c, (U + 4) * 4));
    cudaFree(ctx->st.cnt);
    ctx->st.cnt = c;
    ctx->cnt_cap = U + 4;
  }
  CU(cudaMemsetAsync(ctx->st.cnt, 0, (U + 4) * 4, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  ctx->rounds = T;
  return GIM_OK;
}

gim_status gim_rr_rounds(gim_ctx *ctx, uint32_t *rounds_out) {
  if (!ctx || !rounds_out) return GIM_ERR_ARG;
  *rounds_out = ctx->rounds;
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
  return run_imm(ctx, model, 1, k, eps, ell, seed, seeds_out, theta_out, lb_out);
}

gim_status gim_mrim(gim_ctx *ctx, gim_model model, uint32_t rounds, uint32_t k, double eps, double ell,
                    uint64_t seed, uint32_t *seeds_out, uint64_t *theta_out, double *lb_out) {
  gim_status st = check_ctx(ctx);
  if (st) return st;
  if (rounds < 1 || rounds > kMaxRounds) return set_err(ctx, GIM_ERR_ARG, "rounds must be in [1, %u]", kMaxRounds);
  return run_imm(ctx, model, rounds, k, eps, ell, seed, seeds_out, theta_out, lb_out);
}

gim_status gim_batch_imm(gim_ctx *const *ctxs, uint32_t n_inst, const gim_imm_params *params,
                         uint32_t *const *seeds_out, gim_imm_result *results) {
  if (!ctxs || n_inst == 0 || !ctxs[0]) return GIM_ERR_ARG;
  gim_ctx *ctx = ctxs[0];
  gim_status st = check_ctx(ctx);
  if (st) return st;
  if (!params || !seeds_out || !results) return set_err(ctx, GIM_ERR_ARG, "null argument array");
  std::vector<gim_ctx *> seen(ctxs, ctxs + n_inst);
  std::sort(seen.begin(), seen.end());
  if (std::adjacent_find(seen.begin(), seen.end()) != seen.end() || !seen[0])
    return set_err(ctx, GIM_ERR_ARG, "contexts must be distinct and non-null");
  for (uint32_t i = 0; i < n_inst; ++i) {
    gim_ctx *c = ctxs[i];
    const gim_imm_params &p = params[i];
    if (c->device != ctx->device) return set_err(ctx, GIM_ERR_ARG, "instance %u: context on another device", i);
    if (!c->has_graph) return set_err(ctx, GIM_ERR_STATE, "instance %u: no graph loaded", i);
    if (p.model != GIM_IC && p.model != GIM_LT) return set_err(ctx, GIM_ERR_ARG, "instance %u: unknown model", i);
    if (p.k == 0 || p.k > c->g.n || !seeds_out[i]) return set_err(ctx, GIM_ERR_ARG, "instance %u: bad k or seeds", i);
    if (!(p.eps > 0.0 && p.eps < 1.0)) return set_err(ctx, GIM_ERR_ARG, "instance %u: eps not in (0, 1)", i);
    if (!(p.ell > 0.0)) return set_err(ctx, GIM_ERR_ARG, "instance %u: ell <= 0", i);
    if (p.model == GIM_LT && !lt_valid(c)) return set_err(ctx, GIM_ERR_ARG, "instance %u: graph not LT-valid", i);
  }
  return batch_imm(ctxs, n_inst, params, seeds_out, results);
}

gim_status gim_set_option(gim_ctx *ctx, gim_option opt, uint64_t value) {
  if (!ctx) return GIM_ERR_ARG;
  if (opt == GIM_OPT_GROUP_BUDGET && value > 0) {
    ctx->group_budget = (uint32_t)std::min<uint64_t>(value, 0xFFFFFFFEull);
    return GIM_OK;
  }
  if (opt == GIM_OPT_LARGE_PASS_BYTES && value > 0) {
    ctx->big_budget = value;
    return GIM_OK;
  }
  if (opt == GIM_OPT_FRESH_FINAL && value <= 1) {
    ctx->fresh_final = value == 1;
    return GIM_OK;
  }
  if (opt == GIM_OPT_COMPACT_FIRST_PICK && value <= 1) {
    ctx->compact = value == 1;
    return GIM_OK;
  }
  if (opt == GIM_OPT_FRONTIER_BATCH && value >= 32 && value <= 256 && value % 32 == 0) {
    ctx->frontier_batch = (uint32_t)value;
    return GIM_OK;
  }
  if (opt == GIM_OPT_CHUNK_GROUPS && value >= 64 && value <= 4096 && value % 64 == 0) {
    ctx->chunk_groups = (uint32_t)value;
    return GIM_OK;
  }
  if (opt == GIM_OPT_QUEUE_CAP && value >= 256 && value <= kQueueCap && value % 32 == 0) {
    ctx->queue_cap = (uint32_t)value;
    return GIM_OK;
  }
  return set_err(ctx, GIM_ERR_ARG, "unknown option or value out of range");
}

gim_status gim_get_option(gim_ctx *ctx, gim_option opt, uint64_t *value) {
  if (!ctx || !value) return GIM_ERR_ARG;
  if (opt == GIM_OPT_GROUP_BUDGET) {
    *value = ctx->group_budget;
    return GIM_OK;
  }
  if (opt == GIM_OPT_LARGE_PASS_BYTES) {
    *value = ctx->big_budget;
    return GIM_OK;
  }
  if (opt == GIM_OPT_COMPACT_FIRST_PICK) {
    *value = ctx->compact ? 1 : 0;
    return GIM_OK;
  }
  if (opt == GIM_OPT_FRONTIER_BATCH) {
    *value = ctx->frontier_batch;
    return GIM_OK;
  }
  if (opt == GIM_OPT_CHUNK_GROUPS) {
    *value = ctx->chunk_groups;
    return GIM_OK;
  }
  if (opt == GIM_OPT_QUEUE_CAP) {
    *value = ctx->queue_cap;
    return GIM_OK;
  }
  if (opt == GIM_OPT_FRESH_FINAL) {
    *value = ctx->fresh_final ? 1 : 0;
    return GIM_OK;
  }
  return set_err(ctx, GIM_ERR_ARG, "unknown option");
}

gim_status gim_autotune(gim_ctx *const *ctxs, uint32_t n_inst, const gim_imm_params *params, uint64_t sample_sets,
                        uint64_t *budget_out, int *measured_out) {
  if (!ctxs || n_inst == 0 || !ctxs[0] || !params) return GIM_ERR_ARG;
  gim_ctx *ctx = ctxs[0];
  gim_status st = check_ctx(ctx);
  if (st) return st;
  for (uint32_t i = 0; i < n_inst; ++i) {
    if (!ctxs[i] || ctxs[i]->device != ctx->device) return set_err(ctx, GIM_ERR_ARG, "instance %u: bad context", i);
    if (!ctxs[i]->has_graph) return set_err(ctx, GIM_ERR_STATE, "instance %u: no graph loaded", i);
    if (params[i].model == GIM_LT && !lt_valid(ctxs[i])) return set_err(ctx, GIM_ERR_ARG, "instance %u: not LT-valid", i);
  }
  return autotune(ctxs, n_inst, params, sample_sets == 0 ? 2000 : sample_sets, budget_out, measured_out);
}

gim_status gim_rr_count(gim_ctx *ctx, uint64_t *count_out, uint64_t *members_out) {
  gim_status st = check_ctx(ctx);
  if (st) return st;
  if (!count_out) return set_err(ctx, GIM_ERR_ARG, "count_out is null");
  *count_out = ctx->R;
  if (members_out) *members_out = ctx->Z;
  return GIM_OK;
}

gim_status gim_rr_get(gim_ctx *ctx, uint64_t rr_id, uint32_t *members_out, uint32_t cap, uint32_t *len_out) {
  gim_status st = check_ctx(ctx);
  if (st) return st;
  if (!len_out || (cap > 0 && !members_out)) return set_err(ctx, GIM_ERR_ARG, "null output");
  if (rr_id >= ctx->R) return set_err(ctx, GIM_ERR_ARG, "rr_id %llu >= |R|", (unsigned long long)rr_id);
  uint64_t start = 0;
  uint32_t len = 0;
  CU(cudaMemcpyAsync(&start, ctx->st.rr_start + rr_id, 8, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaMemcpyAsync(&len, ctx->st.rr_len + rr_id, 4, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  if (start == kSkipped)
    return set_err(ctx, GIM_ERR_STATE, "RR set %llu holds the compact vertex: only its size is kept (gim_rr_info)",
                   (unsigned long long)rr_id);
  if (start == kNoStart || start + len > ctx->store_used)
    return set_err(ctx, GIM_ERR_STATE, "RR set %llu is not stored", (unsigned long long)rr_id);
  *len_out = len;
  if (len > cap) return set_err(ctx, GIM_ERR_ARG, "RR set of %u members, room for %u", len, cap);
  if (len) {
    CU(cudaMemcpyAsync(members_out, ctx->st.members + start, (uint64_t)len * 4, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    std::sort(members_out, members_out + len);
  }
  return GIM_OK;
}

namespace {
// The collection as a CSR in rr_id order (members ascending within a set). A
// set stored without members (compact) exports none and sets its flag, or
// fails the export when compact_out is null.
gim_status export_impl(gim_ctx *ctx, uint64_t *offsets_out, uint32_t *members_out, uint8_t *compact_out) {
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
    if (start[j] == kSkipped) {
      if (!compact_out)
        return set_err(ctx, GIM_ERR_STATE, "RR set %llu holds the compact vertex: only its size is kept",
                       (unsigned long long)j);
      compact_out[j] = 1;
      offsets_out[j + 1] = o;
      continue;
    }
    if (start[j] == kNoStart || start[j] + len[j] > ctx->store_used)
      return set_err(ctx, GIM_ERR_STATE, "RR set %llu is not stored", (unsigned long long)j);
    if (compact_out) compact_out[j] = 0;
    std::memcpy(members_out + o, store.data() + start[j], (size_t)len[j] * 4);
    std::sort(members_out + o, members_out + o + len[j]);
    offsets_out[j + 1] = o + len[j];
  }
  return GIM_OK;
}
}  // namespace

gim_status gim_rr_export(gim_ctx *ctx, uint64_t *offsets_out, uint32_t *members_out) {
  return export_impl(ctx, offsets_out, members_out, nullptr);
}

gim_status gim_rr_export_compact(gim_ctx *ctx, uint64_t *offsets_out, uint32_t *members_out, uint8_t *compact_out) {
  if (!compact_out) return ctx ? set_err(ctx, GIM_ERR_ARG, "compact_out is null") : GIM_ERR_ARG;
  return export_impl(ctx, offsets_out, members_out, compact_out);
}

gim_status gim_rr_info(gim_ctx *ctx, uint64_t rr_id, uint32_t *len_out, int *stored_out) {
  gim_status st = check_ctx(ctx);
  if (st) return st;
  if (!len_out || !stored_out) return set_err(ctx, GIM_ERR_ARG, "null output");
  if (rr_id >= ctx->R) return set_err(ctx, GIM_ERR_ARG, "rr_id %llu >= |R|", (unsigned long long)rr_id);
  uint64_t start = 0;
  CU(cudaMemcpyAsync(&start, ctx->st.rr_start + rr_id, 8, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaMemcpyAsync(len_out, ctx->st.rr_len + rr_id, 4, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  if (start == kNoStart) return set_err(ctx, GIM_ERR_STATE, "RR set %llu is not stored", (unsigned long long)rr_id);
  *stored_out = start == kSkipped ? 0 : 1;
  return GIM_OK;
}

gim_status gim_coverage_export(gim_ctx *ctx, uint32_t *cnt_out) {
  gim_status st = check_ctx(ctx);
  if (st) return st;
  if (!ctx->has_graph) return set_err(ctx, GIM_ERR_STATE, "no graph loaded");
  if (!cnt_out) return set_err(ctx, GIM_ERR_ARG, "cnt_out is null");
  CU(cudaMemcpyAsync(cnt_out, ctx->st.cnt, (uint64_t)ctx->g.n * ctx->rounds * 4, cudaMemcpyDeviceToHost,
                     ctx->stream));
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
  ctx->sel_kernel_ms = ctx->sel_bytes = ctx->sel_calls = ctx->sel_cov_members = 0;
  return GIM_OK;
}

gim_status gim_selection_stats(gim_ctx *ctx, double out[4]) {
  if (!ctx || !out) return GIM_ERR_ARG;
  out[0] = ctx->sel_kernel_ms;
  out[1] = ctx->sel_bytes;
  out[2] = ctx->sel_calls;
  out[3] = ctx->sel_cov_members;
  return GIM_OK;
}

gim_status gim_diag_barrier_timeout(gim_ctx *ctx, double *waited_ms) {
  gim_status st = check_ctx(ctx);
  if (st) return st;
  // one allocation carved into the tiny instance's buffers (n = 4, k = 1)
  constexpr size_t kBytes = 4096;
  unsigned char *buf = nullptr;
  CU(cudaMalloc(&buf, kBytes));
  CU(cudaMemsetAsync(buf, 0, kBytes, ctx->stream));
  const uint32_t cw_init[4] = {2u, 5u, 3u, 1u};
  CU(cudaMemcpyAsync(buf, cw_init, sizeof cw_init, cudaMemcpyHostToDevice, ctx->stream));
  CU(cudaMemsetAsync(buf + 512, 0xFF, 4, ctx->stream));   // hslot: all light
  GreedyDesc d;
  d.n = 4;
  d.k = 1;
  d.g_begin = 0;
  d.g_blocks = 2;   // declared two, launched one: the barrier is never met
  d.words = 1;
  d.row_words = 1;
  d.R = 0;
  d.cnt_work = reinterpret_cast<uint32_t *>(buf);
  d.inv_off = reinterpret_cast<const uint64_t *>(buf + 64);
  d.inv = reinterpret_cast<const uint32_t *>(buf + 128);
  d.covered = reinterpret_cast<uint32_t *>(buf + 192);
  d.hslot = reinterpret_cast<const uint8_t *>(buf + 512);
  d.hbits = reinterpret_cast<const uint32_t *>(buf + 576);
  d.hmeta = reinterpret_cast<uint32_t *>(buf + 1024);   // hub count 0
  d.members = reinterpret_cast<const uint32_t *>(buf + 640);
  d.rr_start = reinterpret_cast<const uint64_t *>(buf + 704);
  d.rr_len = reinterpret_cast<const uint32_t *>(buf + 768);
  d.best = reinterpret_cast<unsigned long long *>(buf + 832);
  d.seeds = reinterpret_cast<uint32_t *>(buf + 896);
  d.gains = reinterpret_cast<uint32_t *>(buf + 928);
  d.covered_total = reinterpret_cast<unsigned long long *>(buf + 960);
  d.stats = reinterpret_cast<unsigned long long *>(buf + 976);
  d.bar = reinterpret_cast<unsigned int *>(buf + 3072);
  unsigned int *err = reinterpret_cast<unsigned int *>(buf + 3136);
  GreedyDesc *dd = reinterpret_cast<GreedyDesc *>(buf + 3200);
  static_assert(sizeof(GreedyDesc) <= 4096 - 3200, "descriptor fits");
  CU(cudaMemcpyAsync(dd, &d, sizeof d, cudaMemcpyHostToDevice, ctx->stream));
  CU(cudaEventRecord(ctx->ev[6], ctx->stream));
  cudaError_t e = launch_greedy(dd, 1, 1, err, ctx->stream);
  CU(cudaEventRecord(ctx->ev[7], ctx->stream));
  unsigned int flag = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, err, sizeof flag, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  float ms = 0;
  if (e == cudaSuccess) cudaEventElapsedTime(&ms, ctx->ev[6], ctx->ev[7]);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_err(ctx, e, "barrier timeout diagnostic");
  if (waited_ms) *waited_ms = ms;
  ctx->launches++;
  if (flag) return set_err(ctx, GIM_ERR_TIMEOUT, "greedy selection: a block barrier wait gave up (diagnostic)");
  return set_err(ctx, GIM_ERR_STATE, "barrier timeout diagnostic: the wait did not give up");
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
