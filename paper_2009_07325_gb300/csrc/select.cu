// Greedy maximum coverage over the RR collection (the maximum-coverage step of Alg. 1;
// Sec. III-H, Alg. 7), on the device.
//
// Instead of Alg. 7's scan of the whole RR store for every seed, a
// vertex -> RR-set inverted index is built once per call (exclusive scan of
// the occurrence counts, then a fill), so a round only touches the RR sets
// that contain the new seed. Each round is two kernels:
//   argmax: the unselected vertex with the largest count, lowest id on ties
//           (the max-reduction of Sec. III-H), as a max over 64-bit keys
//           (count+1) << 32 | ~id; a selected vertex has key ~id < 2^32;
//   cover:  every RR set containing the seed that is not yet covered is
//           flagged covered and the counts of its members are lowered.
// Counts are kept as count + 1 for unselected vertices and 0 once selected.
#include <algorithm>

#include "gim_internal.cuh"

namespace gim {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr uint64_t kScanTile = (uint64_t)kScanThreads * kScanItems;

__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t v) {
  const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t o = __shfl_up_sync(kFullMask, v, d);
    if (lane >= (uint32_t)d) v += o;
  }
  return v;
}

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ __forceinline__ uint64_t block_excl_scan(uint64_t v, uint64_t *out_excl) {
  __shared__ uint64_t warp_tot[32];
  __shared__ uint64_t block_tot;
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  const uint64_t inc = warp_incl_scan(v);
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const uint32_t nw = blockDim.x >> 5;
    const uint64_t t = lane < nw ? warp_tot[lane] : 0;
    const uint64_t ti = warp_incl_scan(t);
    if (lane < nw) warp_tot[lane] = ti - t;
    if (lane == 31) block_tot = ti;   // lane 31's inclusive value is the block total
  }
  __syncthreads();
  const uint64_t total = block_tot;
  *out_excl = warp_tot[wid] + inc - v;
  __syncthreads();
  return total;
}

// Pass 1: per-tile sums of cnt.
__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(const uint32_t *__restrict__ cnt, uint32_t n,
                                                                   uint64_t *__restrict__ tile_sum) {
  const uint64_t base = blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) s += cnt[base + i];
  uint64_t ex;
  const uint64_t tot = block_excl_scan(s, &ex);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

// Pass 2: exclusive scan of the tile sums in one block (loops over chunks).
__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(uint64_t *__restrict__ tile_sum, uint64_t tiles) {
  uint64_t carry = 0;
  for (uint64_t b = 0; b < tiles; b += kScanThreads) {
    const uint64_t i = b + threadIdx.x;
    const uint64_t v = i < tiles ? tile_sum[i] : 0;
    uint64_t ex;
    const uint64_t tot = block_excl_scan(v, &ex);
    if (i < tiles) tile_sum[i] = carry + ex;
    carry += tot;
  }
}

// Pass 3: inv_off = exclusive scan of cnt; also cnt_work = cnt + 1 (all
// unselected) and cursor = 0.
__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const uint32_t *__restrict__ cnt, uint32_t n,
                                                                   const uint64_t *__restrict__ tile_off,
                                                                   uint64_t *__restrict__ inv_off,
                                                                   uint32_t *__restrict__ cnt_work,
                                                                   uint32_t *__restrict__ cursor) {
  const uint64_t base = blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < n ? cnt[base + i] : 0u;
    s += v[i];
  }
  uint64_t ex;
  block_excl_scan(s, &ex);
  uint64_t run = tile_off[blockIdx.x] + ex;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) {
      inv_off[base + i] = run;
      cnt_work[base + i] = v[i] + 1u;
      cursor[base + i] = 0u;
    }
    run += v[i];
    if (base + i + 1 == n) inv_off[n] = run;
  }
}

// inv[inv_off[x] + c] = j for every member x of every RR set j.
__global__ void __launch_bounds__(256) fill_inv_kernel(DevStore st, uint64_t R, const uint64_t *__restrict__ inv_off,
                                                       uint32_t *__restrict__ cursor, uint32_t *__restrict__ inv) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t j = warp; j < R; j += nwarps) {
    const uint64_t b = st.rr_start[j];
    const uint32_t len = st.rr_len[j];
    for (uint32_t t = lane; t < len; t += 32) {
      const uint32_t x = st.members[b + t];
      const uint32_t c = atomicAdd(&cursor[x], 1u);
      inv[inv_off[x] + c] = (uint32_t)j;
    }
  }
}

__device__ __forceinline__ unsigned long long key_of(uint32_t cw, uint32_t x) {
  return ((unsigned long long)cw << 32) | (unsigned long long)(~x);
}

__device__ __forceinline__ unsigned long long warp_max(unsigned long long v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const unsigned long long o = __shfl_xor_sync(kFullMask, v, d);
    v = o > v ? o : v;
  }
  return v;
}

// best[t] = max over x of key_of(cnt_work[x], x); best[t] must be 0 on entry.
__global__ void __launch_bounds__(256) argmax_kernel(const uint32_t *__restrict__ cnt_work, uint32_t n,
                                                     unsigned long long *__restrict__ best) {
  __shared__ unsigned long long part[8];
  unsigned long long m = 0;
  const uint32_t n4 = n / 4;
  const uint4 *c4 = reinterpret_cast<const uint4 *>(cnt_work);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += gridDim.x * blockDim.x) {
    const uint4 c = c4[i];
    const uint32_t x = i * 4;
    unsigned long long a = key_of(c.x, x), b = key_of(c.y, x + 1), d = key_of(c.z, x + 2), f = key_of(c.w, x + 3);
    a = a > b ? a : b;
    d = d > f ? d : f;
    a = a > d ? a : d;
    m = a > m ? a : m;
  }
  if (blockIdx.x == 0 && threadIdx.x < (n & 3u)) {
    const uint32_t x = n4 * 4 + threadIdx.x;
    const unsigned long long a = key_of(cnt_work[x], x);
    m = a > m ? a : m;
  }
  m = warp_max(m);
  if ((threadIdx.x & 31u) == 0) part[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0ull;
    m = warp_max(m);
    if (threadIdx.x == 0) atomicMax(best, m);
  }
}

// Round t: record the seed chosen by argmax, mark it selected and cover
// every not-yet-covered RR set that contains it (one warp per set).
__global__ void __launch_bounds__(256) cover_kernel(uint32_t t, DevStore st, const unsigned long long *__restrict__ best,
                                                    uint32_t *__restrict__ cnt_work,
                                                    const uint64_t *__restrict__ inv_off,
                                                    const uint32_t *__restrict__ inv, uint8_t *__restrict__ covered,
                                                    uint32_t *__restrict__ seeds, uint32_t *__restrict__ gains,
                                                    unsigned long long *__restrict__ covered_total) {
  __shared__ unsigned long long part[8];
  const unsigned long long key = best[t];
  const uint32_t u = ~(uint32_t)(key & 0xFFFFFFFFull);
  const uint32_t cw = (uint32_t)(key >> 32);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    seeds[t] = u;
    gains[t] = cw ? cw - 1u : 0u;
    cnt_work[u] = 0u;   // selected; no other thread writes cnt_work[u] in this round
  }
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t i0 = inv_off[u], i1 = inv_off[u + 1];
  unsigned long long newly = 0;
  for (uint64_t i = i0 + warp; i < i1; i += nwarps) {
    const uint32_t j = inv[i];
    uint32_t was = 1;
    if (lane == 0) {
      was = covered[j];
      if (!was) covered[j] = 1;
    }
    was = __shfl_sync(kFullMask, was, 0);
    if (was) continue;
    newly += (lane == 0);
    const uint64_t b = st.rr_start[j];
    const uint32_t len = st.rr_len[j];
    for (uint32_t q = lane; q < len; q += 32) {
      const uint32_t x = st.members[b + q];
      if (x != u) atomicSub(&cnt_work[x], 1u);
    }
  }
  unsigned long long s = newly;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(kFullMask, s, d);
  if (lane == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tot = 0;
    for (uint32_t w = 0; w < (blockDim.x >> 5); ++w) tot += part[w];
    if (tot) atomicAdd(covered_total, tot);
  }
}

template <typename T>
cudaError_t ensure(T *&p, uint64_t &cap, uint64_t need) {
  if (need <= cap && p) return cudaSuccess;
  uint64_t c = std::max<uint64_t>(need, cap * 3 / 2);
  if (c == 0) c = 1;
  T *q = nullptr;
  cudaError_t e = cudaMalloc(&q, c * sizeof(T));
  if (e != cudaSuccess) return e;
  if (p) cudaFree(p);
  p = q;
  cap = c;
  return cudaSuccess;
}

}  // namespace

cudaError_t run_select(const DevGraph &g, const DevStore &st, uint64_t R, uint64_t Z, uint32_t k, SelectBuffers &b,
                       int sm_count, cudaStream_t s, uint64_t *launches) {
  const uint32_t n = g.n;
  cudaError_t e;
  // buffers (n-sized ones share one capacity)
  if (b.n_cap < (uint64_t)n + 1 || !b.cnt_work) {
    uint64_t c0 = b.n_cap, c1 = b.n_cap, c2 = b.n_cap;
    if ((e = ensure(b.cnt_work, c0, (uint64_t)n + 4)) != cudaSuccess) return e;
    if ((e = ensure(b.inv_off, c1, (uint64_t)n + 4)) != cudaSuccess) return e;
    if ((e = ensure(b.cursor, c2, (uint64_t)n + 4)) != cudaSuccess) return e;
    b.n_cap = std::min(c0, std::min(c1, c2));
  }
  if ((e = ensure(b.inv, b.z_cap, std::max<uint64_t>(Z, 1))) != cudaSuccess) return e;
  if ((e = ensure(b.covered, b.r_cap, std::max<uint64_t>(R, 1))) != cudaSuccess) return e;
  if (b.k_cap < k || !b.best) {
    uint64_t c0 = b.k_cap, c1 = b.k_cap, c2 = b.k_cap;
    if ((e = ensure(b.best, c0, k)) != cudaSuccess) return e;
    if ((e = ensure(b.seeds, c1, k)) != cudaSuccess) return e;
    if ((e = ensure(b.gains, c2, k)) != cudaSuccess) return e;
    b.k_cap = std::min(c0, std::min(c1, c2));
  }
  const uint64_t tiles = ((uint64_t)n + kScanTile - 1) / kScanTile;
  if ((e = ensure(b.scan_tmp, b.scan_cap, tiles + 1)) != cudaSuccess) return e;
  if (!b.covered_total) {
    if ((e = cudaMalloc(&b.covered_total, sizeof(unsigned long long))) != cudaSuccess) return e;
  }

  // inverted index
  scan_tiles_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(st.cnt, n, b.scan_tmp);
  scan_sums_kernel<<<1, kScanThreads, 0, s>>>(b.scan_tmp, tiles);
  scan_apply_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(st.cnt, n, b.scan_tmp, b.inv_off, b.cnt_work, b.cursor);
  *launches += 3;
  if (R > 0) {
    const uint64_t want = (R + 7) / 8;
    const unsigned blocks = (unsigned)std::min<uint64_t>(want, (uint64_t)sm_count * 16);
    fill_inv_kernel<<<blocks, 256, 0, s>>>(st, R, b.inv_off, b.cursor, b.inv);
    *launches += 1;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(b.covered, 0, std::max<uint64_t>(R, 1), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(b.best, 0, k * sizeof(unsigned long long), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(b.covered_total, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;

  const unsigned am_blocks =
      (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(((uint64_t)n / 4 + 255) / 256, (uint64_t)sm_count * 4));
  const unsigned cv_blocks = (unsigned)sm_count * 8;
  for (uint32_t t = 0; t < k; ++t) {
    argmax_kernel<<<am_blocks, 256, 0, s>>>(b.cnt_work, n, b.best + t);
    cover_kernel<<<cv_blocks, 256, 0, s>>>(t, st, b.best, b.cnt_work, b.inv_off, b.inv, b.covered, b.seeds, b.gains,
                                           b.covered_total);
    *launches += 2;
  }
  return cudaGetLastError();
}

}  // namespace gim
