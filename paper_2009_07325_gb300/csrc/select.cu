// Greedy maximum coverage over the RR collection (the maximum-coverage step of Alg. 1;
// Sec. III-H, Alg. 7), on the device.
//
// Instead of Alg. 7's scan of the whole RR store for every seed, a
// vertex -> RR-set inverted index is built once per call (exclusive scan of
// the occurrence counts, then a fill), so a round only touches the RR sets
// that contain the new seed. Each round has two steps:
//   argmax: the unselected vertex with the largest count, lowest id on ties
//           (the max-reduction of Sec. III-H), as a max over 64-bit keys
//           (count+1) << 32 | ~id; a selected vertex has key ~id < 2^32;
//   cover:  every RR set containing the seed that is not yet covered is
//           flagged covered and the counts of its members are lowered.
// Counts are kept as count + 1 for unselected vertices and 0 once selected.
// gim_select_seeds runs all k rounds in the persistent greedy kernel
// (greedy.cu); the allocation-free entry point at the end of this file runs
// them as two launches per round (argmax_kernel, cover_kernel).
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>

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

// Checks a caller-given RR collection in CSR form: offsets non-decreasing,
// offsets[0] = 0 and offsets[R] = Z. Sets bit 1 of *flags otherwise.
__global__ void __launch_bounds__(256) na_check_offsets_kernel(const uint64_t *__restrict__ off, uint64_t R,
                                                               uint64_t Z, unsigned int *__restrict__ flags) {
  bool bad = false;
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j <= R; j += (uint64_t)gridDim.x * blockDim.x) {
    if (j == 0 && off[0] != 0) bad = true;
    if (j == R && off[R] != Z) bad = true;
    if (j < R && off[j + 1] < off[j]) bad = true;
  }
  if (bad) atomicOr(flags, 1u);
}

// Set lengths and occurrence counts of a caller-given collection (counts must
// be zero on entry). A member id >= n sets bit 2 of *flags and is skipped.
__global__ void __launch_bounds__(256) na_lengths_counts_kernel(const uint64_t *__restrict__ off,
                                                                const uint32_t *__restrict__ members, uint64_t R,
                                                                uint32_t n, uint32_t *__restrict__ len,
                                                                uint32_t *__restrict__ cnt,
                                                                unsigned int *__restrict__ flags) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  bool bad = false;
  for (uint64_t j = warp; j < R; j += nwarps) {
    const uint64_t b = off[j], e = off[j + 1];
    if (lane == 0) len[j] = (uint32_t)(e - b);
    for (uint64_t t = b + lane; t < e; t += 32) {
      const uint32_t x = members[t];
      if (x < n)
        atomicAdd(&cnt[x], 1u);
      else
        bad = true;
    }
  }
  if (bad) atomicOr(flags, 2u);
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

}  // namespace gim

// ===========================================================================
// Allocation-free greedy selection (gim_select_seeds_noalloc in gim.h).
//
// Some callers cannot let a library call cudaMalloc/cudaFree: processes whose
// device memory is fully reserved up front by their own pool or arena (so a
// foreign allocation would fail or break their budget), and latency-critical
// paths that cannot afford the synchronisation an allocation may imply. For
// them this entry point returns what gim_select_seeds returns (the same
// seeds, gains and covered count), running the k rounds as argmax_kernel /
// cover_kernel pairs, with every scratch buffer carved out of one fixed-size
// array that lives in the library's device image. Callers pass their inputs
// and outputs in device memory they own.
// ===========================================================================
namespace {

constexpr uint64_t na_align(uint64_t x) { return (x + 255) / 256 * 256; }

constexpr uint32_t kNaMaxN = 1u << 16;            // vertices
constexpr uint64_t kNaMaxSets = 1ull << 18;       // RR sets
constexpr uint64_t kNaMaxMembers = 1ull << 20;    // members over all sets
constexpr uint32_t kNaMaxK = 1024;                // seeds
constexpr uint64_t kNaTiles = (kNaMaxN + gim::kScanTile - 1) / gim::kScanTile;

constexpr uint64_t kNaCnt = 0;
constexpr uint64_t kNaCntWork = kNaCnt + na_align(4ull * (kNaMaxN + 4));
constexpr uint64_t kNaInvOff = kNaCntWork + na_align(4ull * (kNaMaxN + 4));
constexpr uint64_t kNaCursor = kNaInvOff + na_align(8ull * (kNaMaxN + 4));
constexpr uint64_t kNaInv = kNaCursor + na_align(4ull * (kNaMaxN + 4));
constexpr uint64_t kNaCovered = kNaInv + na_align(4ull * kNaMaxMembers);
constexpr uint64_t kNaLen = kNaCovered + na_align(kNaMaxSets);
constexpr uint64_t kNaBest = kNaLen + na_align(4ull * kNaMaxSets);
constexpr uint64_t kNaGains = kNaBest + na_align(8ull * kNaMaxK);
constexpr uint64_t kNaTotal = kNaGains + na_align(4ull * kNaMaxK);
constexpr uint64_t kNaScan = kNaTotal + 256;
constexpr uint64_t kNaFlags = kNaScan + na_align(8ull * (kNaTiles + 1));
constexpr uint64_t kNaBytes = kNaFlags + 256;     // about 6.6 MB

}  // namespace

// The scratch of gim_select_seeds_noalloc: loaded with the library on every
// device that uses it and kept until the process exits.
static __device__ __align__(256) unsigned char gim_noalloc_scratch[kNaBytes];

namespace {

std::mutex g_na_mutex;
unsigned char *g_na_ptr[256] = {};   // device address of the scratch, per device ordinal

void na_msg(char *msg, size_t msg_len, const char *text) {
  if (msg && msg_len) {
    std::strncpy(msg, text, msg_len - 1);
    msg[msg_len - 1] = '\0';
  }
}

}  // namespace

extern "C" gim_status gim_select_seeds_noalloc(uint32_t n, uint64_t num_sets, uint64_t num_members,
                                               const uint64_t *d_rr_offsets, const uint32_t *d_rr_members,
                                               uint32_t k, uint32_t *d_seeds_out, uint32_t *d_gains_out,
                                               uint64_t *d_covered_out, void *stream, char *msg, size_t msg_len) {
  using namespace gim;
  na_msg(msg, msg_len, "");
  if (n < 1 || n > kNaMaxN || num_sets > kNaMaxSets || num_members > kNaMaxMembers || k < 1 || k > kNaMaxK ||
      k > n) {
    char buf[256];
    std::snprintf(buf, sizeof buf,
                  "size above the limit: need 1 <= n <= %u, sets <= %llu, members <= %llu, 1 <= k <= min(n, %u)",
                  kNaMaxN, (unsigned long long)kNaMaxSets, (unsigned long long)kNaMaxMembers, kNaMaxK);
    na_msg(msg, msg_len, buf);
    return GIM_ERR_ARG;
  }
  if (!d_rr_offsets || (num_members && !d_rr_members) || !d_seeds_out) {
    na_msg(msg, msg_len, "null input or output pointer");
    return GIM_ERR_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    cudaGetLastError();
    na_msg(msg, msg_len, "no usable current CUDA device");
    return GIM_ERR_CUDA;
  }
  unsigned char *base = nullptr;
  {
    // set-up, once per device, with that device current: the host-side name
    // of the array is not a device address, so ask the runtime for it
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
      void *p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, gim_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        na_msg(msg, msg_len, "cudaGetSymbolAddress of the selection scratch failed");
        return GIM_ERR_CUDA;
      }
      g_na_ptr[dev] = static_cast<unsigned char *>(p);
    }
    base = g_na_ptr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t *cnt = reinterpret_cast<uint32_t *>(base + kNaCnt);
  uint32_t *cnt_work = reinterpret_cast<uint32_t *>(base + kNaCntWork);
  uint64_t *inv_off = reinterpret_cast<uint64_t *>(base + kNaInvOff);
  uint32_t *cursor = reinterpret_cast<uint32_t *>(base + kNaCursor);
  uint32_t *inv = reinterpret_cast<uint32_t *>(base + kNaInv);
  uint8_t *covered = base + kNaCovered;
  uint32_t *len = reinterpret_cast<uint32_t *>(base + kNaLen);
  unsigned long long *best = reinterpret_cast<unsigned long long *>(base + kNaBest);
  uint32_t *gains = d_gains_out ? d_gains_out : reinterpret_cast<uint32_t *>(base + kNaGains);
  unsigned long long *total = reinterpret_cast<unsigned long long *>(base + kNaTotal);
  uint64_t *scan_tmp = reinterpret_cast<uint64_t *>(base + kNaScan);
  unsigned int *flags = reinterpret_cast<unsigned int *>(base + kNaFlags);

  auto fail = [&](cudaError_t e, const char *what) {
    cudaGetLastError();
    char buf[256];
    std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    na_msg(msg, msg_len, buf);
    return e == cudaErrorMemoryAllocation ? GIM_ERR_OOM : GIM_ERR_CUDA;
  };
  cudaError_t e;
  unsigned int hflags = 0;
  // everything that must start at zero is cleared here: the array keeps the
  // previous call's contents
  if ((e = cudaMemsetAsync(flags, 0, 4, s)) != cudaSuccess) return fail(e, "clear flags");
  if ((e = cudaMemsetAsync(cnt, 0, 4ull * n, s)) != cudaSuccess) return fail(e, "clear counts");
  const unsigned ob = (unsigned)std::min<uint64_t>((num_sets + 256) / 256, 1024);
  na_check_offsets_kernel<<<ob, 256, 0, s>>>(d_rr_offsets, num_sets, num_members, flags);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "offset check");
  if ((e = cudaMemcpyAsync(&hflags, flags, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return fail(e, "flags");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(e, "offset check");
  if (hflags) {
    na_msg(msg, msg_len, "rr offsets must start at 0, not decrease and end at num_members");
    return GIM_ERR_ARG;
  }
  if (num_sets) {
    const unsigned lb = (unsigned)std::min<uint64_t>((num_sets + 7) / 8, 2048);
    na_lengths_counts_kernel<<<lb, 256, 0, s>>>(d_rr_offsets, d_rr_members, num_sets, n, len, cnt, flags);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "counts");
    if ((e = cudaMemcpyAsync(&hflags, flags, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return fail(e, "flags");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(e, "counts");
    if (hflags) {
      na_msg(msg, msg_len, "a member id is >= n");
      return GIM_ERR_ARG;
    }
  }
  DevStore st;
  st.members = const_cast<uint32_t *>(d_rr_members);
  st.rr_start = const_cast<uint64_t *>(d_rr_offsets);   // set j starts at offsets[j]
  st.rr_len = len;
  st.cnt = cnt;
  st.cap = num_members;
  const uint64_t tiles = ((uint64_t)n + kScanTile - 1) / kScanTile;
  scan_tiles_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(cnt, n, scan_tmp);
  scan_sums_kernel<<<1, kScanThreads, 0, s>>>(scan_tmp, tiles);
  scan_apply_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(cnt, n, scan_tmp, inv_off, cnt_work, cursor);
  if (num_sets) {
    const unsigned fb = (unsigned)std::min<uint64_t>((num_sets + 7) / 8, 2048);
    fill_inv_kernel<<<fb, 256, 0, s>>>(st, num_sets, inv_off, cursor, inv);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "inverted index");
  if ((e = cudaMemsetAsync(covered, 0, std::max<uint64_t>(num_sets, 1), s)) != cudaSuccess) return fail(e, "clear");
  if ((e = cudaMemsetAsync(best, 0, 8ull * k, s)) != cudaSuccess) return fail(e, "clear");
  if ((e = cudaMemsetAsync(total, 0, 8, s)) != cudaSuccess) return fail(e, "clear");
  int sm = 0;
  if ((e = cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return fail(e, "sm count");
  const unsigned am = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(((uint64_t)n / 4 + 255) / 256, 4ull * sm));
  for (uint32_t t = 0; t < k; ++t) {
    argmax_kernel<<<am, 256, 0, s>>>(cnt_work, n, best + t);
    cover_kernel<<<(unsigned)sm * 8, 256, 0, s>>>(t, st, best, cnt_work, inv_off, inv, covered, d_seeds_out, gains,
                                                   total);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "greedy rounds");
  if (d_covered_out &&
      (e = cudaMemcpyAsync(d_covered_out, total, 8, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
    return fail(e, "covered count");
  return GIM_OK;
}
