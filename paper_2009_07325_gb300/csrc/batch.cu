// Batched IMM: many IMM instances advanced in lockstep on one device.
//
// Each round, every unfinished instance needs the same two steps of Alg. 2 /
// Alg. 1: sample its RR sets up to its current target (theta_i of its
// lower-bound round, or the final theta), then run the greedy selection over
// its collection. The sampling of all instances goes into one launch per
// model whose work items are (instance, rr_id) pairs (sample.cu). The
// selection of all instances runs as multi-instance kernels: every kernel
// covers all instances, each block (or warp) finding its instance from
// fixed block ranges, so a round of the greedy (argmax + cover) is two
// launches for the whole batch. That fixed launch sequence is captured once
// into a CUDA graph and replayed every round; the per-round inputs (set
// counts, buffers) are read from a descriptor table in device memory.
// The host advances each instance's IMM state machine between rounds.
// Every instance's seeds, theta, LB and RR collection are those gim_imm
// computes for it alone.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "gim_internal.cuh"

namespace gim {

namespace {

constexpr int kSelThreads = 256;
constexpr uint32_t kTile = 4096;        // vertices per scan tile (256 threads x 16)
constexpr uint32_t kTileItems = kTile / kSelThreads;

// One instance of a batched selection. Block ranges are fixed for the batch.
struct SelDesc {
  uint32_t n, k, active, count_own;       // count_own: cnt is computed here from sets [0, R)
  unsigned long long R;
  unsigned long long set_begin;           // prefix of R over the batch (fill kernel)
  unsigned long long count_from;          // count_own: sets [0, count_from) are already in cnt
  unsigned long long cnt_begin;           // prefix of the sets counted this round (count kernel)
  const uint32_t *members;
  const uint64_t *rr_start;
  const uint32_t *rr_len;
  uint32_t *cnt;                          // occurrence counts (written by bsel_count when count_own)
  uint32_t *cnt_work;
  uint64_t *inv_off;
  uint32_t *cursor;
  uint32_t *inv;
  uint8_t *covered;
  unsigned long long *best;               // k argmax keys
  uint32_t *seeds;                        // k (into the batch's packed seeds)
  uint32_t *gains;                        // k (packed)
  unsigned long long *covered_total;      // one (packed)
  uint64_t *tile_sum;                     // tiles
  uint32_t tile_begin, tiles;             // scan blocks of this instance
  uint32_t am_begin, am_blocks;           // argmax blocks
  uint32_t cv_begin, cv_blocks;           // cover blocks
};

// Instance of block b: the last i with begin(i) <= b.
template <typename F>
__device__ __forceinline__ uint32_t owner(const SelDesc *d, uint32_t ni, uint64_t b, F begin) {
  uint32_t lo = 0, hi = ni - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (begin(d[mid]) <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long warp_incl_u64(unsigned long long v) {
  const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long t = __shfl_up_sync(kFullMask, v, o);
    if (lane >= (uint32_t)o) v += t;
  }
  return v;
}

// Block-wide exclusive scan (kSelThreads threads); returns the block total.
__device__ __forceinline__ unsigned long long block_excl(unsigned long long v, unsigned long long *excl) {
  __shared__ unsigned long long wt[kSelThreads / 32];
  __shared__ unsigned long long tot;
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  const unsigned long long inc = warp_incl_u64(v);
  if (lane == 31) wt[w] = inc;
  __syncthreads();
  if (w == 0) {
    const unsigned long long x = lane < kSelThreads / 32 ? wt[lane] : 0ull;
    const unsigned long long xi = warp_incl_u64(x);
    if (lane < kSelThreads / 32) wt[lane] = xi - x;
    if (lane == 31) tot = xi;
  }
  __syncthreads();
  *excl = wt[w] + inc - v;
  const unsigned long long t = tot;
  __syncthreads();
  return t;
}

// Clears covered flags, argmax slots and covered counts of active instances.
__global__ void __launch_bounds__(kSelThreads) bsel_clear(const SelDesc *d, uint32_t ni) {
  for (uint32_t i = blockIdx.x; i < ni; i += gridDim.x) {
    const SelDesc &D = d[i];
    if (!D.active) continue;
    for (uint64_t t = threadIdx.x; t < D.R; t += blockDim.x) D.covered[t] = 0;
    for (uint32_t t = threadIdx.x; t < D.k; t += blockDim.x) D.best[t] = 0ull;
    if (threadIdx.x == 0) *D.covered_total = 0ull;
  }
}

// Occurrence counts over the sets [0, R) of instances that count their own
// (a prefix of a shared RR store): zero them ...
__global__ void __launch_bounds__(kSelThreads) bsel_cnt_clear(const SelDesc *d, uint32_t ni) {
  for (uint32_t i = blockIdx.y; i < ni; i += gridDim.y) {
    const SelDesc &D = d[i];
    if (!D.active || !D.count_own || D.count_from != 0) continue;
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < D.n; x += gridDim.x * blockDim.x) D.cnt[x] = 0u;
  }
}

// ... then count every member of every set j in [count_from, R) (one warp per set).
__device__ __forceinline__ unsigned long long counted(const SelDesc &x) {
  return x.active && x.count_own ? x.R - x.count_from : 0ull;
}

__global__ void __launch_bounds__(kSelThreads) bsel_count(const SelDesc *d, uint32_t ni) {
  const unsigned long long total = d[ni - 1].cnt_begin + counted(d[ni - 1]);
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t g = warp; g < total; g += nwarps) {
    const uint32_t i = owner(d, ni, g, [](const SelDesc &x) { return (uint64_t)x.cnt_begin; });
    const SelDesc &D = d[i];
    const uint64_t j = D.count_from + (g - D.cnt_begin);
    const uint64_t b = D.rr_start[j];
    const uint32_t len = D.rr_len[j];
    for (uint32_t t = lane; t < len; t += 32) atomicAdd(&D.cnt[D.members[b + t]], 1u);
  }
}

// Per-tile sums of the occurrence counts.
__global__ void __launch_bounds__(kSelThreads) bsel_tile_sums(const SelDesc *d, uint32_t ni) {
  const uint32_t i = owner(d, ni, blockIdx.x, [](const SelDesc &x) { return (uint64_t)x.tile_begin; });
  const SelDesc &D = d[i];
  if (!D.active) return;
  const uint64_t base = (uint64_t)(blockIdx.x - D.tile_begin) * kTile + (uint64_t)threadIdx.x * kTileItems;
  unsigned long long s = 0;
  for (uint32_t t = 0; t < kTileItems; ++t)
    if (base + t < D.n) s += D.cnt[base + t];
  unsigned long long ex;
  const unsigned long long tot = block_excl(s, &ex);
  if (threadIdx.x == 0) D.tile_sum[blockIdx.x - D.tile_begin] = tot;
}

// Exclusive scan of each instance's tile sums (one block per instance).
__global__ void __launch_bounds__(kSelThreads) bsel_tile_scan(const SelDesc *d, uint32_t ni) {
  for (uint32_t i = blockIdx.x; i < ni; i += gridDim.x) {
    const SelDesc &D = d[i];
    if (!D.active) continue;
    unsigned long long carry = 0;
    for (uint32_t b = 0; b < D.tiles; b += kSelThreads) {
      const uint32_t t = b + threadIdx.x;
      const unsigned long long v = t < D.tiles ? D.tile_sum[t] : 0ull;
      unsigned long long ex;
      const unsigned long long tot = block_excl(v, &ex);
      if (t < D.tiles) D.tile_sum[t] = carry + ex;
      carry += tot;
    }
  }
}

// inv_off = exclusive scan of cnt; cnt_work = cnt + 1 (all unselected); cursor = 0.
__global__ void __launch_bounds__(kSelThreads) bsel_apply(const SelDesc *d, uint32_t ni) {
  const uint32_t i = owner(d, ni, blockIdx.x, [](const SelDesc &x) { return (uint64_t)x.tile_begin; });
  const SelDesc &D = d[i];
  if (!D.active) return;
  const uint32_t tile = blockIdx.x - D.tile_begin;
  const uint64_t base = (uint64_t)tile * kTile + (uint64_t)threadIdx.x * kTileItems;
  uint32_t v[kTileItems];
  unsigned long long s = 0;
  for (uint32_t t = 0; t < kTileItems; ++t) {
    v[t] = base + t < D.n ? D.cnt[base + t] : 0u;
    s += v[t];
  }
  unsigned long long ex;
  block_excl(s, &ex);
  unsigned long long run = D.tile_sum[tile] + ex;
  for (uint32_t t = 0; t < kTileItems; ++t) {
    if (base + t < D.n) {
      D.inv_off[base + t] = run;
      D.cnt_work[base + t] = v[t] + 1u;
      D.cursor[base + t] = 0u;
    }
    run += v[t];
    if (base + t + 1 == D.n) D.inv_off[D.n] = run;
  }
}

// inv: for every set j of every instance, j is appended to the list of each member.
__global__ void __launch_bounds__(kSelThreads) bsel_fill(const SelDesc *d, uint32_t ni) {
  const unsigned long long total = d[ni - 1].set_begin + d[ni - 1].R;   // this round's sets over the batch
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t g = warp; g < total; g += nwarps) {
    const uint32_t i = owner(d, ni, g, [](const SelDesc &x) { return (uint64_t)x.set_begin; });
    const SelDesc &D = d[i];
    const uint64_t j = g - D.set_begin;
    const uint64_t b = D.rr_start[j];
    const uint32_t len = D.rr_len[j];
    for (uint32_t t = lane; t < len; t += 32) {
      const uint32_t x = D.members[b + t];
      const uint32_t c = atomicAdd(&D.cursor[x], 1u);
      D.inv[D.inv_off[x] + c] = (uint32_t)j;
    }
  }
}

__device__ __forceinline__ unsigned long long key_of(uint32_t cw, uint32_t x) {
  return ((unsigned long long)cw << 32) | (unsigned long long)(~x);
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(kFullMask, v, o);
    v = t > v ? t : v;
  }
  return v;
}

// Round t of every instance that still selects: best[t] = max key.
__global__ void __launch_bounds__(kSelThreads) bsel_argmax(const SelDesc *d, uint32_t ni, uint32_t t) {
  __shared__ unsigned long long part[kSelThreads / 32];
  const uint32_t i = owner(d, ni, blockIdx.x, [](const SelDesc &x) { return (uint64_t)x.am_begin; });
  const SelDesc &D = d[i];
  if (!D.active || t >= D.k) return;
  unsigned long long m = 0;
  const uint32_t lb = blockIdx.x - D.am_begin;
  for (uint32_t x = lb * blockDim.x + threadIdx.x; x < D.n; x += D.am_blocks * blockDim.x) {
    const unsigned long long a = key_of(D.cnt_work[x], x);
    m = a > m ? a : m;
  }
  m = warp_max_u64(m);
  if ((threadIdx.x & 31u) == 0) part[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < kSelThreads / 32 ? part[threadIdx.x] : 0ull;
    m = warp_max_u64(m);
    if (threadIdx.x == 0) atomicMax(&D.best[t], m);
  }
}

// Round t: record the chosen seed, mark it selected, cover its uncovered sets.
__global__ void __launch_bounds__(kSelThreads) bsel_cover(const SelDesc *d, uint32_t ni, uint32_t t) {
  __shared__ unsigned long long part[kSelThreads / 32];
  const uint32_t i = owner(d, ni, blockIdx.x, [](const SelDesc &x) { return (uint64_t)x.cv_begin; });
  const SelDesc &D = d[i];
  const uint32_t lb = blockIdx.x - D.cv_begin;
  if (!D.active || t >= D.k) return;
  const unsigned long long key = D.best[t];
  const uint32_t u = ~(uint32_t)(key & 0xFFFFFFFFull);
  const uint32_t cw = (uint32_t)(key >> 32);
  if (lb == 0 && threadIdx.x == 0) {
    D.seeds[t] = u;
    D.gains[t] = cw ? cw - 1u : 0u;
    D.cnt_work[u] = 0u;   // selected; no other thread writes cnt_work[u] in this round
  }
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = (lb * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (D.cv_blocks * blockDim.x) >> 5;
  const uint64_t i0 = D.inv_off[u], i1 = D.inv_off[u + 1];
  unsigned long long newly = 0;
  for (uint64_t p = i0 + warp; p < i1; p += nwarps) {
    const uint32_t j = D.inv[p];
    uint32_t was = 1;
    if (lane == 0) {
      was = D.covered[j];
      if (!was) D.covered[j] = 1;
    }
    was = __shfl_sync(kFullMask, was, 0);
    if (was) continue;
    newly += (lane == 0);
    const uint64_t b = D.rr_start[j];
    const uint32_t len = D.rr_len[j];
    for (uint32_t q = lane; q < len; q += 32) {
      const uint32_t x = D.members[b + q];
      if (x != u) atomicSub(&D.cnt_work[x], 1u);
    }
  }
  const unsigned long long s = warp_sum_u64(newly);
  if (lane == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tot = 0;
    for (uint32_t w = 0; w < kSelThreads / 32; ++w) tot += part[w];
    if (tot) atomicAdd(D.covered_total, tot);
  }
}

#define CU(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_err(ctx, e_, #call);   \
  } while (0)

template <typename T>
cudaError_t ensure_buf(T *&p, uint64_t &cap, uint64_t need) {
  if (need <= cap && p) return cudaSuccess;
  const uint64_t c = std::max<uint64_t>(need, cap * 3 / 2);
  T *q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<uint64_t>(c, 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  if (p) cudaFree(p);
  p = q;
  cap = c;
  return cudaSuccess;
}

// The fixed launch sequence of a batched selection: counts (for instances
// that count a prefix), index build, max_k greedy rounds.
cudaError_t enqueue_selection(SelDesc *d, uint32_t ni, uint32_t scan_blocks, uint32_t am_blocks,
                              uint32_t cv_blocks, uint32_t fill_blocks, uint32_t max_k, uint32_t cnt_blocks,
                              cudaStream_t s) {
  bsel_clear<<<ni, kSelThreads, 0, s>>>(d, ni);
  bsel_cnt_clear<<<dim3(cnt_blocks, std::min<uint32_t>(ni, 65535)), kSelThreads, 0, s>>>(d, ni);
  bsel_count<<<fill_blocks, kSelThreads, 0, s>>>(d, ni);
  bsel_tile_sums<<<scan_blocks, kSelThreads, 0, s>>>(d, ni);
  bsel_tile_scan<<<ni, kSelThreads, 0, s>>>(d, ni);
  bsel_apply<<<scan_blocks, kSelThreads, 0, s>>>(d, ni);
  bsel_fill<<<fill_blocks, kSelThreads, 0, s>>>(d, ni);
  for (uint32_t t = 0; t < max_k; ++t) {
    bsel_argmax<<<am_blocks, kSelThreads, 0, s>>>(d, ni, t);
    bsel_cover<<<cv_blocks, kSelThreads, 0, s>>>(d, ni, t);
  }
  return cudaGetLastError();
}

}  // namespace

// ---------------------------------------------------------------------------
// IMM state machine (Alg. 2, then Alg. 1), advanced by the host.
// ---------------------------------------------------------------------------
void imm_init(ImmState &st, uint32_t n, const gim_imm_params &p) {
  st = ImmState{};
  st.c = imm_constants(n, p.k, p.eps, p.ell);
  if (st.c.i_max < 1) {   // no lower-bound round: LB = 1
    st.phase = 1;
    st.theta = (uint64_t)std::ceil(st.c.lam2 / st.LB);
  }
}

uint64_t imm_target(const ImmState &st, uint32_t n) {
  if (st.phase == 0) {
    const double x = (double)n / std::ldexp(1.0, st.i);
    return (uint64_t)std::ceil(st.c.lam1 / x);
  }
  return st.theta;
}

void imm_advance(ImmState &st, uint32_t n, uint64_t R, uint64_t cov) {
  if (st.phase == 1) {
    st.phase = 2;
    return;
  }
  st.rounds++;
  const double x = (double)n / std::ldexp(1.0, st.i);
  const double est = ((double)n * (double)cov) / (double)R;
  bool stop = false;
  if (est >= (1.0 + st.c.epsp) * x) {
    st.LB = est / (1.0 + st.c.epsp);
    stop = true;
  } else if (++st.i > st.c.i_max) {
    stop = true;
  }
  if (stop) {
    st.phase = 1;
    st.theta = (uint64_t)std::ceil(st.c.lam2 / st.LB);
  }
}

// ---------------------------------------------------------------------------
// MultiSelect: the greedy selection of many instances at once.
// ---------------------------------------------------------------------------
struct MultiSelect::Impl {
  std::vector<SelDesc> h;
  SelDesc *d = nullptr;
  uint32_t *seeds = nullptr;             // packed, sum of k
  uint32_t *gains = nullptr;
  unsigned long long *covered = nullptr; // one per slot
  std::vector<uint64_t> seed_off;
  std::vector<uint32_t> k_cfg;
  uint32_t ni = 0, scan_blocks = 0, am_blocks = 0, cv_blocks = 0, max_k = 0, fill_blocks = 0, cnt_blocks = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~Impl() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (d) cudaFree(d);
    if (seeds) cudaFree(seeds);
    if (gains) cudaFree(gains);
    if (covered) cudaFree(covered);
  }
};

MultiSelect::MultiSelect() : p(new Impl) {}
MultiSelect::~MultiSelect() { delete p; }

gim_status MultiSelect::configure(gim_ctx *ctx, const std::vector<uint32_t> &n, const std::vector<uint32_t> &k) {
  Impl &B = *p;
  B.ni = (uint32_t)n.size();
  B.h.assign(B.ni, SelDesc{});
  B.seed_off.assign(B.ni + 1, 0);
  B.k_cfg = k;
  uint32_t tiles = 0, am = 0, cv = 0, nmax = 0;
  for (uint32_t i = 0; i < B.ni; ++i) {
    SelDesc &D = B.h[i];
    D.n = n[i];
    D.k = k[i];
    D.tile_begin = tiles;
    D.tiles = (D.n + kTile - 1) / kTile;
    tiles += D.tiles;
    D.am_begin = am;
    D.am_blocks = std::max<uint32_t>(1, std::min<uint32_t>((D.n + 4095) / 4096, 64));
    am += D.am_blocks;
    // cover parallelism grows with the graph: a hub seed covers a large share of the sets
    D.cv_begin = cv;
    D.cv_blocks = std::max<uint32_t>(8, std::min<uint32_t>((D.n + 65535) / 65536, 256));
    cv += D.cv_blocks;
    B.seed_off[i + 1] = B.seed_off[i] + D.k;
    B.max_k = std::max(B.max_k, D.k);
    nmax = std::max(nmax, D.n);
  }
  B.scan_blocks = tiles;
  B.am_blocks = am;
  B.cv_blocks = cv;
  B.fill_blocks = (uint32_t)ctx->sm_count * 8;
  B.cnt_blocks = std::max<uint32_t>(1, std::min<uint32_t>((nmax + 4095) / 4096, 256));
  CU(cudaMalloc(&B.d, std::max<uint32_t>(B.ni, 1) * sizeof(SelDesc)));
  CU(cudaMalloc(&B.seeds, std::max<uint64_t>(B.seed_off[B.ni], 1) * 4));
  CU(cudaMalloc(&B.gains, std::max<uint64_t>(B.seed_off[B.ni], 1) * 4));
  CU(cudaMalloc(&B.covered, std::max<uint32_t>(B.ni, 1) * 8ull));
  return GIM_OK;
}

uint64_t MultiSelect::seed_offset(uint32_t i) const { return p->seed_off[i]; }

gim_status MultiSelect::run(gim_ctx *ctx, const std::vector<SelInput> &in, cudaStream_t s,
                            std::vector<unsigned long long> &cov, std::vector<uint32_t> &seeds) {
  Impl &B = *p;
  unsigned long long total_sets = 0, total_counted = 0;
  for (uint32_t i = 0; i < B.ni; ++i) {
    SelDesc &D = B.h[i];
    const SelInput &x = in[i];
    D.active = x.active ? 1u : 0u;
    D.k = x.k && x.k <= B.k_cfg[i] ? x.k : B.k_cfg[i];
    D.set_begin = total_sets;
    D.cnt_begin = total_counted;
    D.R = D.active ? x.R : 0;
    D.count_own = 0;
    D.count_from = 0;
    if (!D.active) continue;
    total_sets += x.R;
    SelectBuffers &b = *x.buf;
    const uint32_t *own_before = b.cnt_own;
    if (b.n_cap < (uint64_t)D.n + 4 || !b.cnt_work || !b.inv_off || !b.cursor || (!x.cnt && !b.cnt_own)) {
      uint64_t c0 = b.n_cap, c1 = b.n_cap, c2 = b.n_cap, c3 = b.n_cap;
      CU(ensure_buf(b.cnt_work, c0, (uint64_t)D.n + 4));
      CU(ensure_buf(b.inv_off, c1, (uint64_t)D.n + 4));
      CU(ensure_buf(b.cursor, c2, (uint64_t)D.n + 4));
      if (!x.cnt) CU(ensure_buf(b.cnt_own, c3, (uint64_t)D.n + 4));
      b.n_cap = std::min(c0, std::min(c1, c2));
      if (!x.cnt) b.n_cap = std::min(b.n_cap, c3);
    }
    CU(ensure_buf(b.inv, b.z_cap, std::max<uint64_t>(x.Z, 1)));
    CU(ensure_buf(b.covered, b.r_cap, std::max<uint64_t>(x.R, 1)));
    if (b.k_cap < D.k || !b.best || !b.seeds || !b.gains) {   // the three k-sized buffers share k_cap
      uint64_t k0 = b.k_cap, k1 = b.k_cap, k2 = b.k_cap;
      CU(ensure_buf(b.best, k0, D.k));
      CU(ensure_buf(b.seeds, k1, D.k));
      CU(ensure_buf(b.gains, k2, D.k));
      b.k_cap = std::min(k0, std::min(k1, k2));
    }
    CU(ensure_buf(b.scan_tmp, b.scan_cap, (uint64_t)D.tiles + 1));
    D.members = x.members;
    D.rr_start = x.rr_start;
    D.rr_len = x.rr_len;
    D.count_own = x.cnt ? 0u : 1u;
    D.cnt = x.cnt ? const_cast<uint32_t *>(x.cnt) : b.cnt_own;
    if (!x.cnt) {
      // counts carried over from the slot's previous round survive only in the same buffer
      const bool keep = b.cnt_own == own_before && x.count_from <= x.R;
      D.count_from = keep ? x.count_from : 0;
      total_counted += x.R - D.count_from;
    }
    D.cnt_work = b.cnt_work;
    D.inv_off = b.inv_off;
    D.cursor = b.cursor;
    D.inv = b.inv;
    D.covered = b.covered;
    D.best = b.best;
    D.seeds = B.seeds + B.seed_off[i];
    D.gains = B.gains + B.seed_off[i];
    D.covered_total = B.covered + i;
    D.tile_sum = b.scan_tmp;
  }
  CU(cudaMemcpyAsync(B.d, B.h.data(), B.ni * sizeof(SelDesc), cudaMemcpyHostToDevice, s));
  if (!B.exec) {
    // the launch sequence is fixed for these slots; the round's inputs live in B.d
    CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const cudaError_t ce =
        enqueue_selection(B.d, B.ni, B.scan_blocks, B.am_blocks, B.cv_blocks, B.fill_blocks, B.max_k, B.cnt_blocks,
                          s);
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(s, &g);
    if (ce != cudaSuccess) return cuda_err(ctx, ce, "selection capture");
    if (ee != cudaSuccess) return cuda_err(ctx, ee, "selection capture");
    B.graph = g;
    CU(cudaGraphInstantiate(&B.exec, B.graph, 0));
  }
  CU(cudaGraphLaunch(B.exec, s));
  ctx->launches += 7 + 2ull * B.max_k;
  cov.resize(B.ni);
  seeds.resize(B.seed_off[B.ni]);
  CU(cudaMemcpyAsync(cov.data(), B.covered, B.ni * 8ull, cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(seeds.data(), B.seeds, B.seed_off[B.ni] * 4, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  return GIM_OK;
}

// Runs IMM on every context of the batch (see gim_batch_imm in gim.h).
gim_status batch_imm(gim_ctx *const *ctxs, uint32_t ni, const gim_imm_params *params, uint32_t *const *seeds_out,
                     gim_imm_result *results) {
  gim_ctx *ctx = ctxs[0];
  cudaStream_t s = ctx->stream;
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<ImmState> S(ni);
  std::vector<uint32_t> ns(ni), ks(ni);
  for (uint32_t i = 0; i < ni; ++i) {
    gim_ctx *c = ctxs[i];
    c->R = c->Z = c->store_used = 0;
    c->model = -1;
    CU(cudaMemsetAsync(c->st.cnt, 0, (uint64_t)c->g.n * 4, s));
    imm_init(S[i], c->g.n, params[i]);
    ns[i] = c->g.n;
    ks[i] = params[i].k;
  }
  MultiSelect ms;
  gim_status st = ms.configure(ctx, ns, ks);
  if (st != GIM_OK) return st;
  std::vector<SelInput> in(ni);
  std::vector<unsigned long long> cov;
  std::vector<uint32_t> seeds;
  double t_sample = 0, t_select = 0;
  for (;;) {
    // 1. sampling up to every unfinished instance's target
    std::vector<SampleJobH> jobs;
    bool any = false;
    for (uint32_t i = 0; i < ni; ++i) {
      if (S[i].phase == 2) continue;
      any = true;
      gim_ctx *c = ctxs[i];
      const uint64_t target = imm_target(S[i], c->g.n);
      if (target >= 0xFFFFFFFFull) return set_err(ctx, GIM_ERR_ARG, "instance %u: theta above 2^32-2 RR sets", i);
      if (target > c->R) jobs.push_back(SampleJobH{c, (int)params[i].model, params[i].seed, target - c->R});
    }
    if (!any) break;
    auto ts = std::chrono::steady_clock::now();
    if ((st = sample_jobs(jobs, s)) != GIM_OK) return st;
    t_sample += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ts).count();
    // 2. selection over every unfinished instance's collection
    ts = std::chrono::steady_clock::now();
    for (uint32_t i = 0; i < ni; ++i) {
      gim_ctx *c = ctxs[i];
      SelInput &x = in[i];
      x.active = S[i].phase != 2;
      x.R = c->R;
      x.Z = c->Z;
      x.members = c->st.members;
      x.rr_start = c->st.rr_start;
      x.rr_len = c->st.rr_len;
      x.cnt = c->st.cnt;
      x.buf = &c->sel;
    }
    if ((st = ms.run(ctx, in, s, cov, seeds)) != GIM_OK) return st;
    t_select += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ts).count();
    // 3. advance every instance's state machine
    for (uint32_t i = 0; i < ni; ++i) {
      if (S[i].phase == 2) continue;
      const bool final_round = S[i].phase == 1;
      imm_advance(S[i], ctxs[i]->g.n, ctxs[i]->R, cov[i]);
      if (final_round)
        std::copy(seeds.begin() + ms.seed_offset(i), seeds.begin() + ms.seed_offset(i + 1), seeds_out[i]);
    }
  }
  for (uint32_t i = 0; i < ni; ++i) {
    results[i].theta = S[i].theta;
    results[i].lb = S[i].LB;
    results[i].rr_count = ctxs[i]->R;
    results[i].lb_rounds = S[i].rounds;
    results[i].status = GIM_OK;
  }
  ctx->t_sample_ms = t_sample;
  ctx->t_select_ms = t_select;
  ctx->t_wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  ctx->lb_rounds = 0;
  return GIM_OK;
}

}  // namespace gim
