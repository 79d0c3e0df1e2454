// Batched IMM: many IMM instances advanced in lockstep on one device.
//
// Each round, every unfinished instance needs the same two steps of Alg. 2 /
// Alg. 1: sample its RR sets up to its current target (theta_i of its
// lower-bound round, or the final theta), then run the greedy selection over
// its collection. The sampling of all instances goes into one launch per
// model whose work items are (instance, rr_id) pairs (sample.cu). The
// selection of all instances runs as multi-instance kernels: every kernel
// covers all instances, each block (or warp) finding its instance from
// fixed block ranges. The preparation (counts, inverted index) is a fixed
// launch sequence, captured once into a CUDA graph and replayed every round;
// the per-round inputs (set counts, buffers) are read from a descriptor
// table in device memory. The k greedy rounds of every instance then run in
// one cooperative launch of the persistent greedy kernel (greedy.cu), each
// instance in its own block group, so instances with small k or small
// graphs finish without waiting for the others.
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
  unsigned long long fill_R;              // sets this instance adds to the index (0 when ext)
  unsigned long long grp_begin;           // prefix of ceil(fill_R / 32) over the batch (fill kernel)
  unsigned long long count_from;          // count_own: sets [0, count_from) are already in cnt
  unsigned long long cnt_begin;           // prefix of the sets counted this round (count kernel)
  const uint32_t *members;
  const uint64_t *rr_start;
  const uint32_t *rr_len;
  uint32_t *cnt;                          // occurrence counts (written by bsel_count when count_own)
  uint32_t *cnt_work;
  uint64_t *inv_off;
  unsigned long long *cursor;
  uint32_t *inv;
  uint32_t *covered;                      // words of the covered bitmap
  uint32_t words;                         // ceil(R/32)
  uint32_t hub_min;                       // a vertex in at least this many sets is a hub
  uint8_t *hslot;                         // n: hub slot or 0xFF
  uint32_t *hbits;                        // hub rows of `words` words
  uint32_t *hmeta;                        // hub count, ids, counts + 1
  unsigned int *err;                      // bit 2: more hubs than kHeavyCap (cannot happen: see hub_min);
                                          // bit 4: a set stored without members where its members are needed
  uint32_t ext;                           // 1: lists, hub split and rows come from another instance's index
  const uint32_t *ext_hmeta;              // that index's hub count and ids
  unsigned long long *best;               // k argmax keys
  uint32_t *seeds;                        // k (into the batch's packed seeds)
  uint32_t *gains;                        // k (packed)
  unsigned long long *covered_total;      // one (packed)
  unsigned long long *stats;              // two (packed): see GreedyDesc::stats
  uint64_t *tile_sum;                     // tiles
  unsigned int *bar;                      // greedy group barrier
  uint32_t tile_begin, tiles;             // scan blocks of this instance
  // 1: the first greedy pick is taken from the occurrence counts before the
  // index exists (best[0], from bsel_tile_sums); the sets holding it are
  // marked covered by the fill and left out of the index, and the light
  // counts are the lengths of the lists filled (bsel_first_*)
  uint32_t fuse;
  // a compact collection's vertex: its sets are stored without members
  // (rr_start = kSkipped); they are covered by a first pick equal to it, and
  // any other use of them is an error (bit 4 of err)
  uint32_t skip;
  // 1 (a fused instance whose collection holds such sets): the first pick is
  // taken from cnt before anything else (bsel_pick), its sets are marked
  // covered (bsel_detect), and the inverted lists are laid out by `lay`, the
  // counts over the uncovered stored sets only (bsel_count_open), since cnt
  // also counts members that are not stored
  uint32_t compact;
  uint32_t *lay;                          // layout counts: cnt, or the slot's own counts when compact
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

// Clears covered flags, argmax slots, covered counts and the greedy group
// barrier of active instances (blockIdx.y: instance, blockIdx.x: chunk).
__global__ void __launch_bounds__(kSelThreads) bsel_clear(const SelDesc *d, uint32_t ni) {
  for (uint32_t i = blockIdx.y; i < ni; i += gridDim.y) {
    const SelDesc &D = d[i];
    if (!D.active) continue;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < D.words; t += stride) D.covered[t] = 0u;
    if (blockIdx.x == 0) {
      for (uint32_t t = threadIdx.x; t < D.k; t += blockDim.x) D.best[t] = 0ull;
      if (threadIdx.x == 0) {
        *D.covered_total = 0ull;
        D.stats[0] = D.stats[1] = 0ull;
        *D.bar = 0u;
        D.hmeta[0] = 0u;
      }
    }
  }
}

// Occurrence counts over the sets [0, R) of instances that count their own
// (a prefix of a shared RR store): zero them ...
__global__ void __launch_bounds__(kSelThreads) bsel_cnt_clear(const SelDesc *d, uint32_t ni) {
  for (uint32_t i = blockIdx.y; i < ni; i += gridDim.y) {
    const SelDesc &D = d[i];
    if (!D.active) continue;
    uint32_t *c = D.compact ? D.lay : (D.count_own && D.count_from == 0) ? D.cnt : nullptr;
    if (!c) continue;
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < D.n; x += gridDim.x * blockDim.x) c[x] = 0u;
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
    if (b == kSkipped) {
      if (lane == 0) atomicOr(D.err, 4u);
      continue;
    }
    const uint32_t len = D.rr_len[j];
    for (uint32_t t = lane; t < len; t += 32) atomicAdd(&D.cnt[D.members[b + t]], 1u);
  }
}

// Per-tile sums of the occurrence counts. A tile is kTile consecutive
// vertices read as kTileItems rows of kSelThreads (coalesced).
__global__ void __launch_bounds__(kSelThreads) bsel_tile_sums(const SelDesc *d, uint32_t ni) {
  const uint32_t i = owner(d, ni, blockIdx.x, [](const SelDesc &x) { return (uint64_t)x.tile_begin; });
  const SelDesc &D = d[i];
  if (!D.active || D.ext) return;
  const uint64_t base = (uint64_t)(blockIdx.x - D.tile_begin) * kTile + threadIdx.x;
  unsigned long long s = 0, key = 0;
#pragma unroll 4
  for (uint32_t t = 0; t < kTileItems; ++t) {
    const uint64_t x = base + (uint64_t)t * kSelThreads;
    if (x < D.n) {
      const uint32_t c = D.cnt[x], l = D.lay[x];
      s += l < D.hub_min ? l : 0u;        // hubs have no inverted list
      // the greedy's key (count + 1) << 32 | ~id: the largest is the first pick (lowest id on ties)
      const unsigned long long kx = ((unsigned long long)(c + 1u) << 32) | (uint32_t)~(uint32_t)x;
      key = kx > key ? kx : key;
    }
  }
  unsigned long long ex;
  const unsigned long long tot = block_excl(s, &ex);
  if (threadIdx.x == 0) D.tile_sum[blockIdx.x - D.tile_begin] = tot;
  if (D.fuse && !D.compact) {   // one atomic per block (a compact instance took it in bsel_pick)
    __shared__ unsigned long long wk[kSelThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long y = __shfl_xor_sync(kFullMask, key, o);
      key = y > key ? y : key;
    }
    if ((threadIdx.x & 31u) == 0) wk[threadIdx.x >> 5] = key;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < kSelThreads / 32; ++w) key = wk[w] > key ? wk[w] : key;
      atomicMax(D.best, key);
    }
  }
}

// Exclusive scan of each instance's tile sums (one block per instance).
__global__ void __launch_bounds__(kSelThreads) bsel_tile_scan(const SelDesc *d, uint32_t ni) {
  for (uint32_t i = blockIdx.x; i < ni; i += gridDim.x) {
    const SelDesc &D = d[i];
    if (!D.active || D.ext) continue;
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

// Splits the vertices: a hub (count >= hub_min) takes the next hub slot,
// with its id and count + 1 in hmeta; a light vertex keeps count + 1 in
// cnt_work and gets its inverted list's offset (exclusive scan of the light
// counts) and a cursor at that offset. The tile is scanned row by row
// (kSelThreads consecutive vertices per row), so every access is coalesced.
__global__ void __launch_bounds__(kSelThreads) bsel_apply(const SelDesc *d, uint32_t ni) {
  const uint32_t i = owner(d, ni, blockIdx.x, [](const SelDesc &x) { return (uint64_t)x.tile_begin; });
  const SelDesc &D = d[i];
  if (!D.active || D.ext) return;
  const uint32_t tile = blockIdx.x - D.tile_begin;
  unsigned long long run = D.tile_sum[tile];
  for (uint32_t r = 0; r < kTileItems; ++r) {
    const uint64_t row0 = (uint64_t)tile * kTile + (uint64_t)r * kSelThreads;
    if (row0 >= D.n) break;                  // block-uniform
    const uint64_t x = row0 + threadIdx.x;
    const uint32_t v = x < D.n ? D.lay[x] : 0u;
    const bool hub = v >= D.hub_min;
    const uint32_t light = hub ? 0u : v;
    unsigned long long ex;
    const unsigned long long tot = block_excl(light, &ex);
    const unsigned long long pos = run + ex;
    if (x < D.n) {
      D.inv_off[x] = pos;
      D.cursor[x] = pos;
      uint8_t hs = 0xFFu;
      uint32_t cw = v + 1u;
      if (hub) {
        const uint32_t slot = atomicAdd(D.hmeta, 1u);
        if (slot < kHeavyCap) {
          D.hmeta[1 + slot] = (uint32_t)x;
          D.hmeta[1 + kHeavyCap + slot] = D.fuse ? 1u : v + 1u;
          hs = (uint8_t)slot;
        } else {
          atomicOr(D.err, 2u);
        }
        cw = 0u;
      }
      D.hslot[x] = hs;
      D.cnt_work[x] = cw;
      if (x + 1 == D.n) D.inv_off[D.n] = pos + light;
    }
    run += tot;
  }
}

// An instance on another instance's index: the light counts from its own
// counts with that index's hub split, its hub counts for that index's hubs
// (blockIdx.y: instance).
__global__ void __launch_bounds__(kSelThreads) bsel_ext_apply(const SelDesc *d, uint32_t ni) {
  for (uint32_t i = blockIdx.y; i < ni; i += gridDim.y) {
    const SelDesc &D = d[i];
    if (!D.active || !D.ext) continue;
    const uint32_t H = D.ext_hmeta[0] < kHeavyCap ? D.ext_hmeta[0] : kHeavyCap;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < D.n; x += stride)
      D.cnt_work[x] = D.hslot[x] == 0xFFu ? D.cnt[x] + 1u : 0u;
    if (blockIdx.x == 0) {
      for (uint32_t t = threadIdx.x; t < H; t += blockDim.x) {
        const uint32_t v = D.ext_hmeta[1 + t];
        D.hmeta[1 + t] = v;
        D.hmeta[1 + kHeavyCap + t] = D.cnt[v] + 1u;
      }
      if (threadIdx.x == 0) D.hmeta[0] = H;
    }
  }
}

// Zeroes the bitmap rows of the hubs found (blockIdx.y: instance).
__global__ void __launch_bounds__(kSelThreads) bsel_hub_clear(const SelDesc *d, uint32_t ni) {
  for (uint32_t i = blockIdx.y; i < ni; i += gridDim.y) {
    const SelDesc &D = d[i];
    if (!D.active || D.ext) continue;
    const uint32_t H = D.hmeta[0] < kHeavyCap ? D.hmeta[0] : kHeavyCap;
    const uint64_t total = (uint64_t)H * D.words;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total; t += stride) D.hbits[t] = 0u;
  }
}

// Finds, for a position p of the concatenated member lists of a warp's 32
// sets, the set that holds it: the last lane s with pre(s) <= p (pre: the
// exclusive prefix of the set sizes, one per lane; warp-wide).
__device__ __forceinline__ uint32_t set_of(uint32_t pre, uint32_t p) {
  uint32_t s = 0;
#pragma unroll
  for (uint32_t step = 16; step; step >>= 1) {
    const uint32_t t = s + step;
    if (__shfl_sync(kFullMask, pre, t) <= p) s = t;
  }
  return s;
}

// For every set j of every instance: j is appended to the inverted list of
// each light member and set in the bitmap row of each hub member. A warp
// takes 32 consecutive sets at a time and walks their members as one list
// (lane s holds set j0 + s), so small sets fill the lanes; four members per
// lane are in flight, since the cursor atomics return a value and the loop
// is bound by their latency. With the fused first pick, a first pass finds
// the sets that hold the pick: they are marked covered (round 0 covers
// them), counted for the statistics, and left out of the index.
__global__ void __launch_bounds__(kSelThreads) bsel_fill(const SelDesc *d, uint32_t ni) {
  const unsigned long long total = d[ni - 1].grp_begin + (d[ni - 1].fill_R + 31) / 32;   // groups over the batch
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t g = warp; g < total; g += nwarps) {
    const uint32_t i = owner(d, ni, g, [](const SelDesc &x) { return (uint64_t)x.grp_begin; });
    const SelDesc &D = d[i];
    const uint64_t j0 = (g - D.grp_begin) * 32;
    const uint64_t jl = j0 + lane;
    const bool valid = jl < D.fill_R;
    const uint64_t b = valid ? D.rr_start[jl] : 0ull;
    const uint32_t len = valid ? D.rr_len[jl] : 0u;
    const bool compact = valid && b == kSkipped;   // stored without members: holds D.skip
    // a compact instance's sets that hold the first pick are marked already (bsel_detect)
    const bool covd = D.compact && valid && ((__ldcg(D.covered + (jl >> 5)) >> (jl & 31u)) & 1u);
    const uint32_t walk = (compact || covd) ? 0u : len;   // members this set contributes to the walk
    uint32_t incl = walk;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(kFullMask, incl, o);
      if (lane >= (uint32_t)o) incl += t;
    }
    const uint32_t T = __shfl_sync(kFullMask, incl, 31);   // members of the 32 sets
    const uint32_t pre = incl - walk;
    const bool hubs = D.hmeta[0] != 0u;
    uint32_t skip = 0;   // bit s: set j0 + s is covered by the first pick
    const uint32_t cmask = __ballot_sync(kFullMask, compact);
    if (cmask && !D.compact && (!D.fuse || ~(uint32_t)*D.best != D.skip)) {
      // a compact set's members are needed (a selection without the fused first
      // pick, or a first pick other than the compact vertex): the selection fails
      if (lane == 0) atomicOr(D.err, 4u);
    }
    if (D.fuse && !D.compact) {
      const uint32_t u1 = ~(uint32_t)*D.best;
      uint32_t hit = cmask;   // a compact set holds D.skip, which is the first pick here
      for (uint32_t p0 = 0; p0 < T; p0 += 128) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t p = p0 + 32 * q + lane;
          const uint32_t s = set_of(pre, p);
          const uint64_t bs = ((uint64_t)__shfl_sync(kFullMask, (uint32_t)(b >> 32), s) << 32) |
                              __shfl_sync(kFullMask, (uint32_t)b, s);
          const uint32_t ps = __shfl_sync(kFullMask, pre, s);
          if (p < T && D.members[bs + (p - ps)] == u1) hit |= 1u << s;
        }
      }
      skip = __reduce_or_sync(kFullMask, hit);
      if ((skip >> lane) & 1u) {
        atomicOr(D.covered + (jl >> 5), 1u << (jl & 31u));
        atomicAdd(D.stats, (unsigned long long)len);
      }
    }
    for (uint32_t p0 = 0; p0 < T; p0 += 128) {
      uint32_t x[4], hs[4], jq[4];
      unsigned long long pos[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t p = p0 + 32 * q + lane;
        const uint32_t s = set_of(pre, p);
        const uint64_t bs = ((uint64_t)__shfl_sync(kFullMask, (uint32_t)(b >> 32), s) << 32) |
                            __shfl_sync(kFullMask, (uint32_t)b, s);
        const uint32_t ps = __shfl_sync(kFullMask, pre, s);
        jq[q] = (uint32_t)j0 + s;
        x[q] = (p < T && !((skip >> s) & 1u)) ? D.members[bs + (p - ps)] : 0xFFFFFFFFu;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) hs[q] = (hubs && x[q] != 0xFFFFFFFFu) ? D.hslot[x[q]] : 0xFFu;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (x[q] == 0xFFFFFFFFu) continue;
        if (hs[q] != 0xFFu)
          atomicOr(D.hbits + (uint64_t)hs[q] * D.words + (jq[q] >> 5), 1u << (jq[q] & 31u));
        else
          pos[q] = atomicAdd(&D.cursor[x[q]], 1ull);   // the entry's place in inv, in one round trip
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (x[q] != 0xFFFFFFFFu && hs[q] == 0xFFu) D.inv[pos[q]] = jq[q];
    }
  }
}

// Compact collections, step 1 (before the tile sums): the first pick, the
// largest key (count + 1) << 32 | ~id over the occurrence counts, into
// best[0] (one block per tile, like bsel_tile_sums).
__global__ void __launch_bounds__(kSelThreads) bsel_pick(const SelDesc *d, uint32_t ni) {
  const uint32_t i = owner(d, ni, blockIdx.x, [](const SelDesc &x) { return (uint64_t)x.tile_begin; });
  const SelDesc &D = d[i];
  if (!D.active || !D.compact) return;
  const uint64_t base = (uint64_t)(blockIdx.x - D.tile_begin) * kTile + threadIdx.x;
  unsigned long long key = 0;
#pragma unroll 4
  for (uint32_t t = 0; t < kTileItems; ++t) {
    const uint64_t x = base + (uint64_t)t * kSelThreads;
    if (x < D.n) {
      const unsigned long long kx = ((unsigned long long)(D.cnt[x] + 1u) << 32) | (uint32_t)~(uint32_t)x;
      key = kx > key ? kx : key;
    }
  }
  __shared__ unsigned long long wk[kSelThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(kFullMask, key, o);
    key = y > key ? y : key;
  }
  if ((threadIdx.x & 31u) == 0) wk[threadIdx.x >> 5] = key;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kSelThreads / 32; ++w) key = wk[w] > key ? wk[w] : key;
    atomicMax(D.best, key);
  }
}

// A warp's group of 32 consecutive sets [j0, j0 + 32) of a compact
// instance, walked as one list of the members that are stored (lane s holds
// set j0 + s): sizes, starts, exclusive prefix of the stored sizes.
struct Group32 {
  uint64_t jl, b;
  uint32_t len, walk, pre, T;
  bool valid, compact;
};

__device__ __forceinline__ Group32 group32(const SelDesc &D, uint64_t j0, bool skip_covered) {
  const uint32_t lane = threadIdx.x & 31u;
  Group32 G;
  G.jl = j0 + lane;
  G.valid = G.jl < D.fill_R;
  G.b = G.valid ? D.rr_start[G.jl] : 0ull;
  G.len = G.valid ? D.rr_len[G.jl] : 0u;
  G.compact = G.valid && G.b == kSkipped;
  const bool covd = skip_covered && G.valid && ((__ldcg(D.covered + (G.jl >> 5)) >> (G.jl & 31u)) & 1u);
  G.walk = (G.compact || covd) ? 0u : G.len;
  uint32_t incl = G.walk;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(kFullMask, incl, o);
    if (lane >= (uint32_t)o) incl += t;
  }
  G.T = __shfl_sync(kFullMask, incl, 31);
  G.pre = incl - G.walk;
  return G;
}

// The stored member at walk position p (< G.T) of a group: warp-wide.
__device__ __forceinline__ uint32_t group_member(const SelDesc &D, const Group32 &G, uint32_t p, uint32_t &s) {
  s = set_of(G.pre, p);
  const uint64_t bs = ((uint64_t)__shfl_sync(kFullMask, (uint32_t)(G.b >> 32), s) << 32) |
                      __shfl_sync(kFullMask, (uint32_t)G.b, s);
  const uint32_t ps = __shfl_sync(kFullMask, G.pre, s);
  return p < G.T ? D.members[bs + (p - ps)] : 0xFFFFFFFFu;
}

// Compact collections, step 2: every set that holds the first pick is
// covered in round 0 - a set kept without members holds the compact vertex,
// which must be the first pick (else bit 4 of err), a stored set is scanned.
// Marks them covered and counts their members for the statistics.
__global__ void __launch_bounds__(kSelThreads) bsel_detect(const SelDesc *d, uint32_t ni) {
  const unsigned long long total = d[ni - 1].grp_begin + (d[ni - 1].fill_R + 31) / 32;
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t g = warp; g < total; g += nwarps) {
    const uint32_t i = owner(d, ni, g, [](const SelDesc &x) { return (uint64_t)x.grp_begin; });
    const SelDesc &D = d[i];
    if (!D.compact) continue;
    const Group32 G = group32(D, (g - D.grp_begin) * 32, false);
    const uint32_t u1 = ~(uint32_t)*D.best;
    const uint32_t cmask = __ballot_sync(kFullMask, G.compact);
    if (cmask && u1 != D.skip && lane == 0) atomicOr(D.err, 4u);
    uint32_t hit = cmask;
    for (uint32_t p0 = 0; p0 < G.T; p0 += 128) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t s;
        const uint32_t x = group_member(D, G, p0 + 32 * q + lane, s);
        if (x == u1) hit |= 1u << s;
      }
    }
    hit = __reduce_or_sync(kFullMask, hit);
    if ((hit >> lane) & 1u) {
      atomicOr(D.covered + (G.jl >> 5), 1u << (G.jl & 31u));
      atomicAdd(D.stats, (unsigned long long)G.len);
    }
  }
}

// Compact collections, step 3: the layout counts, over the stored sets left
// uncovered.
__global__ void __launch_bounds__(kSelThreads) bsel_count_open(const SelDesc *d, uint32_t ni) {
  const unsigned long long total = d[ni - 1].grp_begin + (d[ni - 1].fill_R + 31) / 32;
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t g = warp; g < total; g += nwarps) {
    const uint32_t i = owner(d, ni, g, [](const SelDesc &x) { return (uint64_t)x.grp_begin; });
    const SelDesc &D = d[i];
    if (!D.compact) continue;
    const Group32 G = group32(D, (g - D.grp_begin) * 32, true);
    for (uint32_t p0 = 0; p0 < G.T; p0 += 128) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t s;
        const uint32_t x = group_member(D, G, p0 + 32 * q + lane, s);
        if (x != 0xFFFFFFFFu) atomicAdd(D.lay + x, 1u);
      }
    }
  }
}

// Fused first pick, light side (one block per tile, like bsel_apply): a
// light vertex's count is the length of its filled list (the uncovered sets
// holding it), plus one while unselected; the first pick's is 0.
__global__ void __launch_bounds__(kSelThreads) bsel_first_light(const SelDesc *d, uint32_t ni) {
  const uint32_t i = owner(d, ni, blockIdx.x, [](const SelDesc &x) { return (uint64_t)x.tile_begin; });
  const SelDesc &D = d[i];
  if (!D.active || !D.fuse) return;
  const uint32_t u1 = ~(uint32_t)*D.best;
  const uint32_t tile = blockIdx.x - D.tile_begin;
  const uint64_t base = (uint64_t)tile * kTile + threadIdx.x;
#pragma unroll 4
  for (uint32_t t = 0; t < kTileItems; ++t) {
    const uint64_t x = base + (uint64_t)t * kSelThreads;
    if (x < D.n && D.hslot[x] == 0xFFu)
      D.cnt_work[x] = x == u1 ? 0u : (uint32_t)(D.cursor[x] - D.inv_off[x]) + 1u;
  }
  if (tile == 0 && threadIdx.x == 0) {
    // round 0's record: the pick covers every set that holds it
    const uint32_t c = D.cnt[u1];
    D.seeds[0] = u1;
    D.gains[0] = c;
    *D.covered_total = c;
    D.stats[1] = D.hslot[u1] == 0xFFu ? c : D.words;   // the pick's list or row, read by a plain round 0
  }
}

// Fused first pick, hub side (blockIdx.y: instance): a hub's count is the
// population of its row (the fill set bits for uncovered sets only), plus
// one while unselected; the first pick's is 0.
__global__ void __launch_bounds__(kSelThreads) bsel_first_hubs(const SelDesc *d, uint32_t ni) {
  for (uint32_t i = blockIdx.y; i < ni; i += gridDim.y) {
    const SelDesc &D = d[i];
    if (!D.active || !D.fuse) continue;
    const uint32_t H = D.hmeta[0] < kHeavyCap ? D.hmeta[0] : kHeavyCap;
    const uint32_t u1 = ~(uint32_t)*D.best;
    for (uint32_t h = 0; h < H; ++h) {
      const uint32_t *row = D.hbits + (uint64_t)h * D.words;
      uint32_t c = 0;
      for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < D.words; w += gridDim.x * blockDim.x)
        c += __popc(row[w]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFullMask, c, o);
      uint32_t *hc = D.hmeta + 1 + kHeavyCap + h;
      if ((threadIdx.x & 31u) == 0 && c) atomicAdd(hc, c);
      if (D.hmeta[1 + h] == u1 && blockIdx.x == 0 && threadIdx.x == 0) *hc = 0u;   // no bits: the pick's sets are covered
    }
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

// The fixed launch sequence that prepares a batched selection: counts (for
// instances that count a prefix) and the inverted index. The greedy rounds
// follow as cooperative launches of the greedy kernel (greedy.cu).
// compact: some instance holds a compact collection (the sequence then
// includes its three steps; they do nothing for the other instances).
cudaError_t enqueue_selection(SelDesc *d, uint32_t ni, uint32_t scan_blocks, uint32_t fill_blocks,
                              uint32_t cnt_blocks, bool compact, cudaStream_t s) {
  const uint32_t ny = std::min<uint32_t>(ni, 65535);
  bsel_clear<<<dim3(64, ny), kSelThreads, 0, s>>>(d, ni);
  bsel_cnt_clear<<<dim3(cnt_blocks, ny), kSelThreads, 0, s>>>(d, ni);
  bsel_count<<<fill_blocks, kSelThreads, 0, s>>>(d, ni);
  if (compact) {
    bsel_pick<<<scan_blocks, kSelThreads, 0, s>>>(d, ni);
    bsel_detect<<<fill_blocks, kSelThreads, 0, s>>>(d, ni);
    bsel_count_open<<<fill_blocks, kSelThreads, 0, s>>>(d, ni);
  }
  bsel_tile_sums<<<scan_blocks, kSelThreads, 0, s>>>(d, ni);
  bsel_tile_scan<<<ni, kSelThreads, 0, s>>>(d, ni);
  bsel_apply<<<scan_blocks, kSelThreads, 0, s>>>(d, ni);
  bsel_ext_apply<<<dim3(64, ny), kSelThreads, 0, s>>>(d, ni);
  bsel_hub_clear<<<dim3(128, ny), kSelThreads, 0, s>>>(d, ni);
  bsel_fill<<<fill_blocks, kSelThreads, 0, s>>>(d, ni);
  bsel_first_light<<<scan_blocks, kSelThreads, 0, s>>>(d, ni);
  bsel_first_hubs<<<dim3(16, ny), kSelThreads, 0, s>>>(d, ni);
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
  unsigned long long *stats = nullptr;   // two per slot
  std::vector<unsigned long long> h_stats;
  std::vector<uint64_t> seed_off;
  std::vector<uint32_t> k_cfg;
  uint32_t ni = 0, scan_blocks = 0, fill_blocks = 0, cnt_blocks = 0;
  cudaGraph_t graph[2] = {nullptr, nullptr};   // without and with the compact-collection steps
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  // greedy rounds: block groups, and the waves of instances that share one cooperative launch
  std::vector<GreedyDesc> gh;
  GreedyDesc *gd = nullptr;
  unsigned int *sync = nullptr;          // ni group barriers, then the error flag
  std::vector<uint32_t> wave_first, wave_grid;
  ~Impl() {
    for (int v = 0; v < 2; ++v) {
      if (exec[v]) cudaGraphExecDestroy(exec[v]);
      if (graph[v]) cudaGraphDestroy(graph[v]);
    }
    if (gd) cudaFree(gd);
    if (sync) cudaFree(sync);
    if (d) cudaFree(d);
    if (seeds) cudaFree(seeds);
    if (gains) cudaFree(gains);
    if (covered) cudaFree(covered);
    if (stats) cudaFree(stats);
  }
};

MultiSelect::MultiSelect() : p(new Impl) {}
MultiSelect::~MultiSelect() { delete p; }

gim_status MultiSelect::configure(gim_ctx *ctx, const std::vector<uint32_t> &n, const std::vector<uint32_t> &k,
                                  const std::vector<bool> *index_only) {
  Impl &B = *p;
  B.ni = (uint32_t)n.size();
  B.h.assign(B.ni, SelDesc{});
  B.seed_off.assign(B.ni + 1, 0);
  B.k_cfg = k;
  uint32_t tiles = 0, nmax = 0;
  double nsum = 0;
  for (uint32_t i = 0; i < B.ni; ++i) {
    SelDesc &D = B.h[i];
    D.n = n[i];
    D.k = k[i];
    D.tile_begin = tiles;
    D.tiles = (D.n + kTile - 1) / kTile;
    tiles += D.tiles;
    B.seed_off[i + 1] = B.seed_off[i] + D.k;
    nmax = std::max(nmax, D.n);
    if (!(index_only && (*index_only)[i])) nsum += D.n;
  }
  B.scan_blocks = tiles;
  B.fill_blocks = (uint32_t)ctx->sm_count * 8;
  B.cnt_blocks = std::max<uint32_t>(1, std::min<uint32_t>((nmax + 4095) / 4096, 256));

  // greedy block groups: in proportion to n (the argmax reads all n counts
  // every round), at least one block and about 8K vertices per block at
  // least; instances are packed into waves of at most G blocks
  const uint32_t G = greedy_max_blocks(ctx->sm_count);
  B.gh.assign(B.ni, GreedyDesc{});
  B.wave_first.clear();
  B.wave_grid.clear();
  uint32_t cur = 0;
  for (uint32_t i = 0; i < B.ni; ++i) {
    GreedyDesc &g = B.gh[i];
    const bool only = index_only && (*index_only)[i];
    const double share = (nsum > 0 && !only) ? (double)G * n[i] / nsum : 1.0;
    uint32_t nb = (uint32_t)std::max(1.0, std::floor(share));
    nb = std::min<uint32_t>(nb, std::max<uint32_t>(1, (n[i] + 8191) / 8192));
    nb = std::min(nb, G);
    if (B.wave_first.empty() || cur + nb > G) {
      B.wave_first.push_back(i);
      B.wave_grid.push_back(0);
      cur = 0;
    }
    g.n = n[i];
    g.g_begin = cur;
    g.g_blocks = nb;
    cur += nb;
    B.wave_grid.back() = cur;
  }
  CU(cudaMalloc(&B.gd, std::max<uint32_t>(B.ni, 1) * sizeof(GreedyDesc)));
  CU(cudaMalloc(&B.sync, (B.ni + 1) * sizeof(unsigned int)));
  CU(cudaMalloc(&B.d, std::max<uint32_t>(B.ni, 1) * sizeof(SelDesc)));
  CU(cudaMalloc(&B.seeds, std::max<uint64_t>(B.seed_off[B.ni], 1) * 4));
  CU(cudaMalloc(&B.gains, std::max<uint64_t>(B.seed_off[B.ni], 1) * 4));
  CU(cudaMalloc(&B.covered, std::max<uint32_t>(B.ni, 1) * 8ull));
  CU(cudaMalloc(&B.stats, std::max<uint32_t>(B.ni, 1) * 16ull));
  B.h_stats.assign(2 * (size_t)std::max<uint32_t>(B.ni, 1), 0ull);
  return GIM_OK;
}

uint64_t MultiSelect::seed_offset(uint32_t i) const { return p->seed_off[i]; }
uint32_t MultiSelect::slots() const { return p->ni; }
uint32_t MultiSelect::k_of(uint32_t i) const { return p->k_cfg[i]; }

gim_status MultiSelect::run(gim_ctx *ctx, const std::vector<SelInput> &in, cudaStream_t s,
                            std::vector<unsigned long long> &cov, std::vector<uint32_t> &seeds,
                            std::vector<uint32_t> *gains) {
  Impl &B = *p;
  unsigned long long total_sets = 0, total_counted = 0;
  for (uint32_t i = 0; i < B.ni; ++i) {
    SelDesc &D = B.h[i];
    const SelInput &x = in[i];
    D.active = x.active ? 1u : 0u;
    D.k = x.k && x.k <= B.k_cfg[i] ? x.k : B.k_cfg[i];
    D.grp_begin = total_sets;
    D.cnt_begin = total_counted;
    D.R = D.active ? x.R : 0;
    D.ext = (D.active && x.index) ? 1u : 0u;
    D.fill_R = D.ext ? 0 : D.R;
    D.count_own = 0;
    D.count_from = 0;
    // the first pick rides on the fill for an instance that indexes its own
    // collection for itself (not a shared index, not multi-round)
    D.fuse = (D.active && !D.ext && !x.index_only && x.part_n == 0 && D.k >= 1) ? 1u : 0u;
    D.skip = x.skip;
    D.compact = (D.fuse && x.skip != kNoSkip && x.cnt) ? 1u : 0u;
    if (!D.active) continue;
    total_sets += (D.fill_R + 31) / 32;
    SelectBuffers &b = *x.buf;
    const uint32_t *own_before = b.cnt_own;
    const bool need_own = !x.cnt || D.compact;   // own counts, or a compact instance's layout counts
    if (b.n_cap < (uint64_t)D.n + 4 || !b.cnt_work || !b.inv_off || !b.cursor || !b.hslot ||
        (need_own && !b.cnt_own)) {   // the n-sized buffers share n_cap
      uint64_t c0 = b.n_cap, c1 = b.n_cap, c2 = b.n_cap, c3 = b.n_cap, c4 = b.n_cap;
      CU(ensure_buf(b.cnt_work, c0, (uint64_t)D.n + 4));
      CU(ensure_buf(b.inv_off, c1, (uint64_t)D.n + 4));
      CU(ensure_buf(b.cursor, c2, (uint64_t)D.n + 4));
      CU(ensure_buf(b.hslot, c4, (uint64_t)D.n + 4));
      if (need_own) CU(ensure_buf(b.cnt_own, c3, (uint64_t)D.n + 4));
      b.n_cap = std::min(std::min(c0, c4), std::min(c1, c2));
      if (need_own) b.n_cap = std::min(b.n_cap, c3);
    }
    // A hub is a vertex in at least hub_min sets: at least R/32 (its bitmap
    // row is no longer than its inverted list would be) and at least
    // Z/kHeavyCap, so that the counts (summing to at most Z) admit at most
    // kHeavyCap hubs.
    D.words = (uint32_t)((x.R + 31) / 32);
    const uint64_t hm = std::max<uint64_t>(std::max<uint64_t>((x.R + 31) / 32, (x.Z + kHeavyCap - 1) / kHeavyCap), 1);
    D.hub_min = (uint32_t)std::min<uint64_t>(hm, 0xFFFFFFFFull);
    if (!D.ext) {
      CU(ensure_buf(b.inv, b.z_cap, std::max<uint64_t>(x.Z, 1)));
      CU(ensure_buf(b.hbits, b.hb_cap, (uint64_t)kHeavyCap * std::max<uint32_t>(D.words, 1)));
    }
    CU(ensure_buf(b.covered, b.r_cap, std::max<uint64_t>(D.words, 1)));
    if (!b.hmeta) CU(cudaMalloc(&b.hmeta, (1 + 2 * kHeavyCap) * sizeof(uint32_t)));
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
    D.lay = D.compact ? b.cnt_own : D.cnt;
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
    D.stats = B.stats + 2 * i;
    D.tile_sum = b.scan_tmp;
    D.bar = B.sync + i;
    D.hslot = b.hslot;
    D.hbits = b.hbits;
    D.hmeta = b.hmeta;
    D.err = B.sync + B.ni;
    D.ext_hmeta = nullptr;
  }
  // lists, hub split and rows of the shared indexes: taken only now, once
  // every instance (the index builders among them) has its buffers
  for (uint32_t i = 0; i < B.ni; ++i) {
    SelDesc &D = B.h[i];
    if (!D.ext) continue;
    const SelectBuffers &ix = *in[i].index;
    if (!ix.inv_off || !ix.inv || !ix.hslot || !ix.hbits || !ix.hmeta || ix.n_cap < (uint64_t)D.n + 4)
      return set_err(ctx, GIM_ERR_STATE, "selection: a shared index without its buffers");
    D.inv_off = ix.inv_off;
    D.inv = ix.inv;
    D.hslot = ix.hslot;
    D.hbits = ix.hbits;
    D.ext_hmeta = ix.hmeta;
  }
  for (uint32_t i = 0; i < B.ni; ++i) {
    const SelDesc &D = B.h[i];
    GreedyDesc &g = B.gh[i];
    g.k = D.active && !in[i].index_only ? D.k : 0u;
    if (!D.active) continue;
    g.words = D.words;
    g.row_words = D.ext ? (uint32_t)((in[i].index_R + 31) / 32) : D.words;
    g.R = (uint32_t)D.R;
    g.cnt_work = D.cnt_work;
    g.inv_off = D.inv_off;
    g.inv = D.inv;
    g.covered = D.covered;
    g.hslot = D.hslot;
    g.hbits = D.hbits;
    g.hmeta = D.hmeta;
    g.members = D.members;
    g.rr_start = D.rr_start;
    g.rr_len = D.rr_len;
    g.best = D.best;
    g.seeds = D.seeds;
    g.gains = D.gains;
    g.covered_total = D.covered_total;
    g.stats = D.stats;
    g.bar = D.bar;
    g.part_n = in[i].part_n;
    g.part_k = in[i].part_k;
    g.fuse = D.fuse;
    g.inv_end = D.fuse ? D.cursor : nullptr;
  }
  CU(cudaMemcpyAsync(B.d, B.h.data(), B.ni * sizeof(SelDesc), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(B.gd, B.gh.data(), B.ni * sizeof(GreedyDesc), cudaMemcpyHostToDevice, s));
  CU(cudaMemsetAsync(B.sync + B.ni, 0, sizeof(unsigned int), s));
  bool any_compact = false;
  for (uint32_t i = 0; i < B.ni; ++i) any_compact = any_compact || B.h[i].compact;
  const int gv = any_compact ? 1 : 0;
  if (!B.exec[gv]) {
    // the launch sequence is fixed for these slots; the round's inputs live in B.d
    CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const cudaError_t ce = enqueue_selection(B.d, B.ni, B.scan_blocks, B.fill_blocks, B.cnt_blocks, any_compact, s);
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(s, &g);
    if (ce != cudaSuccess) return cuda_err(ctx, ce, "selection capture");
    if (ee != cudaSuccess) return cuda_err(ctx, ee, "selection capture");
    B.graph[gv] = g;
    CU(cudaGraphInstantiate(&B.exec[gv], B.graph[gv], 0));
  }
  CU(cudaEventRecord(ctx->ev[8], s));
  CU(cudaGraphLaunch(B.exec[gv], s));
  ctx->launches += any_compact ? 14 : 11;
  for (size_t w = 0; w < B.wave_first.size(); ++w) {
    const uint32_t first = B.wave_first[w];
    const uint32_t count = (w + 1 < B.wave_first.size() ? B.wave_first[w + 1] : B.ni) - first;
    bool part = false;
    for (uint32_t i = first; i < first + count; ++i) part = part || B.gh[i].part_n != 0;
    CU(launch_greedy(B.gd + first, count, B.wave_grid[w], B.sync + B.ni, s, part));
    ctx->launches += 1;
  }
  CU(cudaEventRecord(ctx->ev[9], s));
  cov.resize(B.ni);
  seeds.resize(B.seed_off[B.ni]);
  if (gains) gains->resize(B.seed_off[B.ni]);
  unsigned int flags = 0;
  CU(cudaMemcpyAsync(B.h_stats.data(), B.stats, B.ni * 16ull, cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(cov.data(), B.covered, B.ni * 8ull, cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(seeds.data(), B.seeds, B.seed_off[B.ni] * 4, cudaMemcpyDeviceToHost, s));
  if (gains) CU(cudaMemcpyAsync(gains->data(), B.gains, B.seed_off[B.ni] * 4, cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(&flags, B.sync + B.ni, sizeof flags, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (flags & 2u) return set_err(ctx, GIM_ERR_STATE, "greedy selection: more hubs than slots");
  if (flags & 4u)
    return set_err(ctx, GIM_ERR_STATE,
                   "selection: the collection keeps some sets without members (compact), and this selection "
                   "needs them: its first pick is not the compact vertex");
  if (flags) return set_err(ctx, GIM_ERR_TIMEOUT, "greedy selection: a block barrier wait gave up");
  // device time and algorithmic bytes: reading the store and writing the
  // index (8 per member) and scanning the counts (4 per vertex); then per
  // round reading all counts (4 per vertex), the seed's list or row (4 per
  // word) and, per member of a newly covered set, its id (4) and a count
  // read-modify-write (8); plus the covered bitmap
  float ms = 0;
  cudaEventElapsedTime(&ms, ctx->ev[8], ctx->ev[9]);
  ctx->sel_kernel_ms += ms;
  ctx->sel_calls += 1;
  for (uint32_t i = 0; i < B.ni; ++i) {
    const SelDesc &D = B.h[i];
    if (!D.active) continue;
    const double n = D.n, Z = (double)in[i].Z;
    ctx->sel_bytes += (D.ext ? 0.0 : 8.0 * Z) + 4.0 * n + (double)D.k * 4.0 * n +
                      4.0 * (double)B.h_stats[2 * i + 1] + 12.0 * (double)B.h_stats[2 * i] + 4.0 * D.words;
    ctx->sel_cov_members += (double)B.h_stats[2 * i];
  }
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
    c->jhi = c->rhi = 0;
    c->rounds = 1;
    c->skip_vertex = kNoSkip;   // the batch keeps every set
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
      if (S[i].phase == 1 && c->fresh_final && c->jhi == 0) {   // fresh final phase: rr_ids 2^63 + j
        c->R = c->Z = c->store_used = 0;
        c->jhi = c->rhi = 1u << 31;
        CU(cudaMemsetAsync(c->st.cnt, 0, (uint64_t)c->g.n * 4, s));
      }
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
