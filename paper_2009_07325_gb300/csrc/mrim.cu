// Multi-round RR sets (multi-round IM, Sec. IV-H; CR-NAIMM of Sun et al.).
//
// Multi-round RR set j has one root (that of RR set j) and T independent
// reverse traversals from it; round t runs in the live-edge world of rr_id
// t * 2^32 + j, and its vertices v are stored as elements t * n + v. The
// traversals are the plain RR-set kernels: each round is a view of the
// context (same graph, its own small store) whose descriptor fixes the root's
// counter word to round 0's (rhi = 0), the rr_id's high word to t (jhi = t),
// the rr_id's low word to the parent's |R| + position (idoff) and the element
// offset to t * n (moff); the counts go straight to the parent's element
// counts. All T views are sampled in one launch (T instances), then a merge
// writes set j as the concatenation of its rounds, in rr_id order, to the
// parent's store: a length pass with per-tile sums, a scan of the tile sums,
// and a copy pass (one warp per set).
#include <algorithm>
#include <vector>

#include "gim_internal.cuh"

namespace gim {

gim_status cuda_err(gim_ctx *ctx, cudaError_t e, const char *what);
gim_status set_err(gim_ctx *ctx, gim_status st, const char *fmt, ...);
template <typename T>
cudaError_t grow_copy(T *&p, uint64_t &cap, uint64_t need, uint64_t keep, cudaStream_t s);

#define CU(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_err(ctx, e_, #call);   \
  } while (0)

namespace {

constexpr uint32_t kMergeThreads = 256;
constexpr uint32_t kMergeTile = 1024;   // sets per tile: 4 per thread

struct MergeDesc {
  uint32_t T;
  uint32_t count;                       // sets to merge (positions 0 .. count-1 of every view)
  uint64_t R0;                          // the parent's |R| before the merge
  uint64_t base;                        // the parent's first free store entry
  const uint64_t *vstart[kMaxRounds];   // per view: rr_start, rr_len, members
  const uint32_t *vlen[kMaxRounds];
  const uint32_t *vmem[kMaxRounds];
  uint64_t *rr_start;                   // parent
  uint32_t *rr_len;
  uint32_t *members;
  unsigned long long *tiles;            // one sum per tile, then their exclusive prefix
};

// Inclusive block-wide scan of one value per thread (kMergeThreads threads).
__device__ __forceinline__ unsigned long long block_scan(unsigned long long v, unsigned long long *sh) {
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(kFullMask, v, o);
    if (lane >= (uint32_t)o) v += y;
  }
  if (lane == 31) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    unsigned long long s = lane < kMergeThreads / 32 ? sh[lane] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(kFullMask, s, o);
      if (lane >= (uint32_t)o) s += y;
    }
    if (lane < kMergeThreads / 32) sh[lane] = s;
  }
  __syncthreads();
  const unsigned long long r = v + (w ? sh[w - 1] : 0ull);
  __syncthreads();
  return r;
}

// Pass 1: each set's length (sum over rounds) and each tile's total.
__global__ void __launch_bounds__(kMergeThreads) merge_len_kernel(MergeDesc M) {
  __shared__ unsigned long long sh[kMergeThreads / 32];
  const uint64_t t0 = (uint64_t)blockIdx.x * kMergeTile;
  unsigned long long sum = 0;
  for (uint32_t q = 0; q < kMergeTile / kMergeThreads; ++q) {
    const uint64_t i = t0 + q * kMergeThreads + threadIdx.x;
    if (i < M.count) {
      uint32_t len = 0;
      for (uint32_t t = 0; t < M.T; ++t) len += M.vlen[t][i];
      M.rr_len[M.R0 + i] = len;
      sum += len;
    }
  }
  const unsigned long long tot = block_scan(sum, sh);
  if (threadIdx.x == kMergeThreads - 1) M.tiles[blockIdx.x] = tot;
}

// Pass 2 (one block): exclusive prefix of the tile totals, in place.
__global__ void __launch_bounds__(kMergeThreads) merge_scan_kernel(unsigned long long *tiles, uint32_t n_tiles) {
  __shared__ unsigned long long sh[kMergeThreads / 32];
  __shared__ unsigned long long s_total;
  unsigned long long carry = 0;
  for (uint32_t b = 0; b < n_tiles; b += kMergeThreads) {
    const uint32_t i = b + threadIdx.x;
    const unsigned long long v = i < n_tiles ? tiles[i] : 0ull;
    const unsigned long long inc = block_scan(v, sh);
    if (i < n_tiles) tiles[i] = carry + inc - v;
    if (threadIdx.x == kMergeThreads - 1) s_total = inc;
    __syncthreads();
    carry += s_total;
    __syncthreads();
  }
}

// Pass 3: each set's start (tile prefix + prefix inside the tile, four
// consecutive sets per thread), then its rounds copied in order, one warp per set.
__global__ void __launch_bounds__(kMergeThreads) merge_copy_kernel(MergeDesc M) {
  __shared__ unsigned long long sh[kMergeThreads / 32];
  __shared__ unsigned long long s_start[kMergeTile];
  constexpr uint32_t kPer = kMergeTile / kMergeThreads;
  const uint64_t t0 = (uint64_t)blockIdx.x * kMergeTile;
  uint32_t len[kPer];
  unsigned long long sum = 0;
#pragma unroll
  for (uint32_t q = 0; q < kPer; ++q) {
    const uint64_t i = t0 + threadIdx.x * kPer + q;
    len[q] = i < M.count ? M.rr_len[M.R0 + i] : 0u;
    sum += len[q];
  }
  const unsigned long long inc = block_scan(sum, sh);
  unsigned long long at = M.base + M.tiles[blockIdx.x] + (inc - sum);
#pragma unroll
  for (uint32_t q = 0; q < kPer; ++q) {
    const uint64_t i = t0 + threadIdx.x * kPer + q;
    s_start[threadIdx.x * kPer + q] = at;
    if (i < M.count) M.rr_start[M.R0 + i] = at;
    at += len[q];
  }
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  for (uint32_t q = w; q < kMergeTile; q += kMergeThreads / 32) {
    const uint64_t i = t0 + q;
    if (i >= M.count) break;
    unsigned long long dst = s_start[q];
    for (uint32_t t = 0; t < M.T; ++t) {
      const uint64_t src = M.vstart[t][i];
      const uint32_t vl = M.vlen[t][i];
      const uint32_t *vm = M.vmem[t];
      for (uint32_t e = lane; e < vl; e += 32) M.members[dst + e] = vm[src + e];
      dst += vl;
    }
  }
}

// A view of ctx for one round: the same graph and device, its own store.
gim_status make_round_view(gim_ctx *ctx, gim_ctx **out) {
  gim_ctx *v = nullptr;
  const gim_status st = gim_create(&v, ctx->device, ctx->stream);
  if (st != GIM_OK) return set_err(ctx, st, "multi-round: creating a round view failed");
  v->owns_graph = false;
  *out = v;
  return GIM_OK;
}

}  // namespace

void mrim_release(gim_ctx *ctx) {
  for (gim_ctx *v : ctx->round_views) {
    v->st.cnt = nullptr;   // the parent's counts
    gim_destroy(v);
  }
  ctx->round_views.clear();
  if (ctx->mr_tiles) cudaFree(ctx->mr_tiles);
  ctx->mr_tiles = nullptr;
  ctx->mr_tiles_cap = 0;
}

gim_status mrim_sample(gim_ctx *ctx, int model, uint64_t seed, uint64_t count) {
  const uint32_t T = ctx->rounds, n = ctx->g.n;
  cudaStream_t s = ctx->stream;
  if (T < 2 || T > kMaxRounds) return set_err(ctx, GIM_ERR_STATE, "not a multi-round collection");
  if (count == 0) return GIM_OK;
  while (ctx->round_views.size() < T) {
    gim_ctx *v = nullptr;
    const gim_status st = make_round_view(ctx, &v);
    if (st != GIM_OK) return st;
    ctx->round_views.push_back(v);
  }
  std::vector<SampleJobH> jobs;
  for (uint32_t t = 0; t < T; ++t) {
    gim_ctx *v = ctx->round_views[t];
    v->g = ctx->g;
    v->has_graph = true;
    v->lt_ok = ctx->lt_ok;
    v->max_indeg = ctx->max_indeg;
    v->group_budget = ctx->group_budget;
    v->frontier_batch = ctx->frontier_batch;
    v->chunk_groups = ctx->chunk_groups;
    v->queue_cap = ctx->queue_cap;
    v->big_budget = ctx->big_budget;
    v->R = v->Z = v->store_used = 0;
    v->model = -1;
    v->jhi = t;
    v->rhi = 0;
    v->moff = t * n;
    v->idoff = (uint32_t)ctx->R;
    v->st.cnt = ctx->st.cnt;
    v->t_kernel_ms[0] = v->t_kernel_ms[1] = v->n_kernel[0] = v->n_kernel[1] = 0;
    v->launches = 0;
    v->last_error.clear();
    jobs.push_back(SampleJobH{v, model, seed, count});
  }
  gim_status st = sample_jobs(jobs, s);
  gim_ctx *v0 = ctx->round_views[0];
  for (int q = 0; q < 2; ++q) {
    ctx->t_kernel_ms[q] += v0->t_kernel_ms[q];
    ctx->n_kernel[q] += v0->n_kernel[q];
  }
  ctx->launches += v0->launches;
  if (st != GIM_OK) {
    ctx->last_error = "multi-round sampling: " + v0->last_error;
    return st;
  }

  // merge the rounds into the parent's collection
  uint64_t total = 0;
  for (uint32_t t = 0; t < T; ++t) total += ctx->round_views[t]->Z;
  const uint64_t R0 = ctx->R;
  uint64_t cap = ctx->rr_cap, cap2 = ctx->rr_cap;
  CU(grow_copy(ctx->st.rr_start, cap, R0 + count, R0, s));
  CU(grow_copy(ctx->st.rr_len, cap2, R0 + count, R0, s));
  ctx->rr_cap = std::min(cap, cap2);
  if (!ctx->st.members || ctx->store_used + total > ctx->st.cap) {
    uint64_t c = ctx->st.members ? ctx->st.cap : 0;
    CU(grow_copy(ctx->st.members, c, std::max<uint64_t>(ctx->store_used + total, 1), ctx->store_used, s));
    ctx->st.cap = c;
  }
  const uint32_t n_tiles = (uint32_t)((count + kMergeTile - 1) / kMergeTile);
  if (ctx->mr_tiles_cap < n_tiles) {
    if (ctx->mr_tiles) cudaFree(ctx->mr_tiles);
    ctx->mr_tiles = nullptr;
    ctx->mr_tiles_cap = 0;
    CU(cudaMalloc(&ctx->mr_tiles, (uint64_t)n_tiles * sizeof(unsigned long long)));
    ctx->mr_tiles_cap = n_tiles;
  }
  MergeDesc M{};
  M.T = T;
  M.count = (uint32_t)count;
  M.R0 = R0;
  M.base = ctx->store_used;
  for (uint32_t t = 0; t < T; ++t) {
    const gim_ctx *v = ctx->round_views[t];
    M.vstart[t] = v->st.rr_start;
    M.vlen[t] = v->st.rr_len;
    M.vmem[t] = v->st.members;
  }
  M.rr_start = ctx->st.rr_start;
  M.rr_len = ctx->st.rr_len;
  M.members = ctx->st.members;
  M.tiles = ctx->mr_tiles;
  merge_len_kernel<<<n_tiles, kMergeThreads, 0, s>>>(M);
  CU(cudaGetLastError());
  merge_scan_kernel<<<1, kMergeThreads, 0, s>>>(ctx->mr_tiles, n_tiles);
  CU(cudaGetLastError());
  merge_copy_kernel<<<n_tiles, kMergeThreads, 0, s>>>(M);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(s));
  ctx->launches += 3;
  ctx->R += count;
  ctx->Z += total;
  ctx->store_used += total;
  ctx->model = model;
  ctx->seed = seed;
  for (gim_ctx *v : ctx->round_views) v->st.cnt = nullptr;
  return GIM_OK;
}

}  // namespace gim
