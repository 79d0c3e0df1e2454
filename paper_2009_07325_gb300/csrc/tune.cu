// Autotuner of the sampling schedule (see gim_autotune in gim.h).
//
// The knobs: the common IC pass's edge budget (how many in-edge groups one
// warp scans for an RR set before a block of the block pass takes it over)
// and its frontier buffer (members a set may reach on one warp), and the
// block pass's work chunk and frontier batch. A small budget or buffer
// sends heavy sets to the block pass early, which bounds the tail of a
// launch with few sets (one large graph); large ones keep them on single
// warps, which is cheaper per coin when many sets are in flight (batches of
// instances). Chunks and batches trade the block's per-step overhead
// against idle warps at its barriers. The best values depend on the degree
// profile of the graphs and on how many instances share a launch, so the
// candidates are timed on a short sampling run shaped like the real
// launches, one knob at a time with the others at their best so far, and
// the winner is cached per profile for the rest of the process.
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "gim_internal.cuh"

namespace gim {

namespace {

using Profile = std::tuple<int, int, int, int, int>;
struct Schedule {
  uint32_t budget, chunk, batch, queue;
};
std::mutex g_tune_mu;
std::map<Profile, Schedule> g_tune_cache;

int lg(double x) { return x <= 1.0 ? 0 : (int)std::floor(std::log2(x)); }

Profile profile_of(gim_ctx *const *ctxs, uint32_t ni, const gim_imm_params *params) {
  double n = 0, m = 0, dmax = 0;
  for (uint32_t i = 0; i < ni; ++i) {
    n += ctxs[i]->g.n;
    m += (double)ctxs[i]->g.m;
    dmax = std::max<double>(dmax, ctxs[i]->max_indeg);
  }
  return Profile{lg(n / ni), lg(m / std::max(n, 1.0)), lg(dmax), (int)params[0].model, lg(ni)};
}

void apply(gim_ctx *const *ctxs, uint32_t ni, const Schedule &x) {
  for (uint32_t i = 0; i < ni; ++i) {
    ctxs[i]->group_budget = x.budget;
    ctxs[i]->chunk_groups = x.chunk;
    ctxs[i]->frontier_batch = x.batch;
    ctxs[i]->queue_cap = x.queue;
  }
}

// Empties every context's collection (the tuning runs leave theirs behind).
gim_status reset_all(gim_ctx *const *ctxs, uint32_t ni, cudaStream_t s) {
  for (uint32_t i = 0; i < ni; ++i) {
    ctxs[i]->R = ctxs[i]->Z = ctxs[i]->store_used = 0;
    ctxs[i]->model = -1;
    ctxs[i]->jhi = ctxs[i]->rhi = 0;
    ctxs[i]->rounds = 1;
    ctxs[i]->skip_vertex = kNoSkip;
    const cudaError_t e = cudaMemsetAsync(ctxs[i]->st.cnt, 0, (uint64_t)ctxs[i]->g.n * 4, s);
    if (e != cudaSuccess) return cuda_err(ctxs[0], e, "autotune reset");
  }
  return GIM_OK;
}

}  // namespace

gim_status autotune(gim_ctx *const *ctxs, uint32_t ni, const gim_imm_params *params, uint64_t sample_sets,
                    uint64_t *budget_out, int *measured_out) {
  gim_ctx *ctx = ctxs[0];
  const Profile key = profile_of(ctxs, ni, params);
  Schedule best{};
  bool cached = false;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      best = it->second;
      cached = true;
    }
  }
  if (!cached) {
    // device time of sampling `sample_sets` sets per instance under schedule x
    // (the first of two runs warms the graph into L2)
    auto time_of = [&](const Schedule &x, double &ms) -> gim_status {
      apply(ctxs, ni, x);
      for (int rep = 0; rep < 2; ++rep) {
        gim_status st = reset_all(ctxs, ni, ctx->stream);
        if (st != GIM_OK) return st;
        std::vector<SampleJobH> jobs;
        for (uint32_t i = 0; i < ni; ++i)
          jobs.push_back(SampleJobH{ctxs[i], (int)params[i].model, params[i].seed, sample_sets});
        const double k0 = ctx->t_kernel_ms[0] + ctx->t_kernel_ms[1];
        st = sample_jobs(jobs, ctx->stream);
        if (st != GIM_OK) return st;
        ms = ctx->t_kernel_ms[0] + ctx->t_kernel_ms[1] - k0;
      }
      return GIM_OK;
    };
    static const uint32_t kBudget[] = {1u << 12, 1u << 14, 1u << 16, 1u << 18, 1u << 30};
    static const uint32_t kChunk[] = {256, 512, 1024, 2048};
    static const uint32_t kBatchC[] = {32, 64, 128};
    static const uint32_t kQueue[] = {1024, 2048, 4096};
    best = Schedule{1u << 14, 512, 128, kQueueCap};
    double best_ms = -1.0;
    auto sweep = [&](uint32_t Schedule::*knob, const uint32_t *cand, size_t nc) -> gim_status {
      for (size_t c = 0; c < nc; ++c) {
        Schedule x = best;
        x.*knob = cand[c];
        double ms = 0;
        const gim_status st = time_of(x, ms);
        if (st != GIM_OK) return st;
        if (best_ms < 0 || ms < best_ms) {
          best = x;
          best_ms = ms;
        }
      }
      return GIM_OK;
    };
    gim_status st;
    if ((st = sweep(&Schedule::budget, kBudget, 5)) != GIM_OK) return st;
    if ((st = sweep(&Schedule::chunk, kChunk, 4)) != GIM_OK) return st;
    if ((st = sweep(&Schedule::batch, kBatchC, 3)) != GIM_OK) return st;
    if ((st = sweep(&Schedule::queue, kQueue, 3)) != GIM_OK) return st;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = best;
  }
  apply(ctxs, ni, best);
  gim_status st = reset_all(ctxs, ni, ctx->stream);
  if (st != GIM_OK) return st;
  const cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_err(ctx, e, "autotune");
  if (budget_out) *budget_out = best.budget;
  if (measured_out) *measured_out = cached ? 0 : 1;
  return GIM_OK;
}

}  // namespace gim
