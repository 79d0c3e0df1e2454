// The k rounds of greedy maximum coverage (the maximum-coverage step of
// Alg. 1; Sec. III-H) as one persistent kernel.
//
// Every round needs the argmax over all counts before any set can be
// covered, and all covers done before the next argmax, so a round is two
// global steps. Launched as two kernels per round, a selection of k seeds
// costs 2k launches whose work, after the first few rounds, is far smaller
// than a launch. Here one cooperative launch runs all rounds: the blocks of
// an instance (a block group) meet at a group barrier between the steps.
//
//   argmax: each block takes the max of the 64-bit keys (count+1) << 32 | ~id
//           over its contiguous slice of the light counts (read at L2, 16
//           bytes per load), the group's first block also over the hub
//           counts, and merges it into best[t] with one atomicMax;
//   cover:  every block reads best[t] (lowest id wins ties) and the group
//           covers the RR sets that hold the seed: through its inverted
//           list (light seed, one set per warp) or its row of the hub
//           bitmap (hub seed, one bitmap word per thread). A newly covered
//           set is claimed with an atomicOr on the covered bitmap, and its
//           members' counts are lowered: a light member's in place, a hub's
//           in the block's shared-memory histogram, flushed once per round.
//           So the hottest counters (hubs sit in a large share of the
//           sets) see one global atomic per block and round, not one per set.
//
// Multi-round IM (part_n > 0): the elements are (vertex, round) pairs in
// rounds of part_n ids, and a round takes at most part_k seeds. Every block
// counts the seeds per round as it reads them (best[t] is the same for all
// blocks) and leaves the elements of full rounds out of its argmax.
//
// A group barrier is a counter that every block of the group bumps; a block
// waits until it reaches the round's target. Every wait is bounded: past the
// limit the block sets the error flag and the whole group returns, so the
// host sees an error instead of a hung kernel. A cooperative launch
// guarantees that all blocks are resident, so the barrier can always be
// met. Independent instances (a batch) run in disjoint block groups.
#include <algorithm>

#include "gim_internal.cuh"

namespace gim {

namespace {

constexpr long long kWaitCycles = 4ll << 30;   // about 2 s at 2 GHz: a barrier wait that never ends

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(unsigned int *p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// All blocks of the group have arrived `target` times in total. False if
// the wait gave up (here or in another block). The arrival is a release
// (after the block barrier, it publishes every write of the block) and the
// wait an acquire; the block barrier after it passes that on to the block.
__device__ __forceinline__ bool group_sync(unsigned int *bar, unsigned int target, unsigned int *err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    red_release_add(bar, 1u);
    const long long t0 = clock64();
    for (uint32_t polls = 0; ld_acquire(bar) < target; ++polls) {
      if ((polls & 15u) == 15u) {   // the error flag and the clock: every 16 polls
        if (ld_acquire(err)) {
          ok = 0;
          break;
        }
        if (clock64() - t0 > kWaitCycles) {
          atomicOr(err, 1u);
          ok = 0;
          break;
        }
      }
      if (polls > 64) __nanosleep(64);   // a barrier is usually met within a few polls
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ unsigned long long key_of(uint32_t cw, uint32_t x) {
  return ((unsigned long long)cw << 32) | (unsigned long long)(~x);
}

__device__ __forceinline__ unsigned long long umax(unsigned long long a, unsigned long long b) { return a > b ? a : b; }

__device__ __forceinline__ unsigned long long warp_max(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = umax(v, __shfl_xor_sync(kFullMask, v, o));
  return v;
}

// Covers the RR set stored at [b, b + len) (claimed by this warp): lowers
// the counts of its members other than the seed u. Each lane keeps four members in flight
// (their loads, then their hub lookups, then their decrements), since a
// set's members are scattered over the count array and the loop is bound by
// load latency. With no hubs (H = 0) the lookup is skipped. A light
// member's decrement is a fire-and-forget reduction at L2; a hub's goes to
// the block's shared-memory histogram.
__device__ __forceinline__ uint32_t cover_members(const GreedyDesc &D, uint64_t b, uint32_t len, uint32_t u,
                                                  uint32_t H, int *s_delta, uint32_t lane) {
  for (uint32_t q0 = 0; q0 < len; q0 += 128) {
    uint32_t x[4], hs[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t q = q0 + 32 * i + lane;
      x[i] = q < len ? D.members[b + q] : u;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) hs[i] = (H && x[i] != u) ? D.hslot[x[i]] : 0xFFu;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (x[i] == u) continue;
      if (hs[i] != 0xFFu)
        atomicAdd(s_delta + hs[i], -1);
      else
        atomicSub(D.cnt_work + x[i], 1u);
    }
  }
  return len;
}

__device__ __forceinline__ uint32_t cover_set(const GreedyDesc &D, uint32_t j, uint32_t u, uint32_t H,
                                              int *s_delta, uint32_t lane) {
  return cover_members(D, D.rr_start[j], D.rr_len[j], u, H, s_delta, lane);
}

// Adds the block's pending hub count changes to the hub counts.
__device__ __forceinline__ void flush_hubs(int *s_delta, uint32_t *hc, uint32_t H) {
  __syncthreads();
  for (uint32_t s = threadIdx.x; s < H; s += kGreedyThreads) {
    const int v = s_delta[s];
    if (v) {
      atomicAdd(hc + s, (uint32_t)v);
      s_delta[s] = 0;
    }
  }
}

// Largest key over the light counts [x0, x1) and (block 0 of the group) the
// hub counts, leaving out the elements of rounds whose bit is set in
// `closed` (round = x / pn; pn = 0: no rounds).
__device__ __forceinline__ unsigned long long argmax_part(const GreedyDesc &D, uint32_t x0, uint32_t x1, uint32_t H,
                                                          const uint32_t *hid, const uint32_t *hc, uint32_t lb,
                                                          uint32_t pn, uint32_t closed) {
  unsigned long long m = 0;
#pragma unroll 1
  for (uint32_t x = x0 + threadIdx.x; x < x1; x += kGreedyThreads)
    if (!((closed >> (x / pn)) & 1u)) m = umax(m, key_of(__ldcg(D.cnt_work + x), x));
  if (lb == 0)
#pragma unroll 1
    for (uint32_t s = threadIdx.x; s < H; s += kGreedyThreads)
      if (!((closed >> (hid[s] / pn)) & 1u)) m = umax(m, key_of(__ldcg(hc + s), hid[s]));
  return m;
}

// kPart: some instance of the launch is multi-round (part_n > 0). A separate
// kernel keeps the plain one's code and registers (two blocks per SM).
template <bool kPart>
__device__ __forceinline__ void greedy_body(const GreedyDesc *d, uint32_t ni, unsigned int *err) {
  __shared__ unsigned long long part[kGreedyThreads / 32];
  __shared__ int s_delta[kHeavyCap];
  __shared__ uint32_t s_picks[kMaxRounds];
  __shared__ uint32_t s_closed;
  uint32_t lo = 0, hi = ni - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (d[mid].g_begin <= blockIdx.x)
      lo = mid;
    else
      hi = mid - 1;
  }
  const GreedyDesc D = d[lo];
  const uint32_t lb = blockIdx.x - D.g_begin;
  if (D.k == 0 || lb >= D.g_blocks) return;
  const uint32_t nb = D.g_blocks, n = D.n;
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
  for (uint32_t s = threadIdx.x; s < kHeavyCap; s += kGreedyThreads) s_delta[s] = 0;
  if (threadIdx.x < kMaxRounds) s_picks[threadIdx.x] = 0;
  if (threadIdx.x == 0) s_closed = 0;
  const uint32_t pn = kPart ? D.part_n : 0u;
  __syncthreads();
  const uint32_t H = D.hmeta[0] < kHeavyCap ? D.hmeta[0] : kHeavyCap;   // written before this launch
  const uint32_t *hid = D.hmeta + 1;
  uint32_t *hc = D.hmeta + 1 + kHeavyCap;

  // this block's slice of the light counts, 4-aligned so it can be read as uint4
  const uint32_t per = (uint32_t)((((uint64_t)n + nb - 1) / nb + 3) & ~3ull);
  const uint64_t lo64 = (uint64_t)lb * per, hi64 = lo64 + per;
  const uint32_t x0 = lo64 < n ? (uint32_t)lo64 : n;
  const uint32_t x1 = hi64 < n ? (uint32_t)hi64 : n;
  const uint32_t x1v = x0 + ((x1 - x0) & ~3u);
  const uint4 *cw4 = reinterpret_cast<const uint4 *>(D.cnt_work);

  const uint32_t gwarp = lb * (kGreedyThreads / 32) + wib;
  const uint32_t nwarps = nb * (kGreedyThreads / 32);
  unsigned int target = 0;
  unsigned long long newly = 0, cov_members = 0, list_words = 0;   // per thread; summed at the end
  // The largest key of this block's light slice in the last round it was
  // scanned (0: none yet). Counts never rise during a selection, so while
  // its vertex keeps its count the slice's maximum is unchanged and the
  // slice need not be read again (exact, ties included: the key is unique).
  __shared__ unsigned long long s_light;
  __shared__ int s_rescan;
  if (threadIdx.x == 0) s_light = 0ull;

  for (uint32_t t = D.fuse; t < D.k; ++t) {
    // argmax (counts change between rounds: read them at L2)
    unsigned long long m = 0;
    if (pn) {
      m = argmax_part(D, x0, x1, H, hid, hc, lb, pn, s_closed);
      m = warp_max(m);
      if (lane == 0) part[wib] = m;
      __syncthreads();
      if (wib == 0) {
        m = warp_max(lane < kGreedyThreads / 32 ? part[lane] : 0ull);
        if (lane == 0) atomicMax(D.best + t, m);
      }
    } else {
      if (threadIdx.x == 0) {
        const unsigned long long c = s_light;
        s_rescan = c == 0ull || __ldcg(D.cnt_work + ~(uint32_t)c) != (uint32_t)(c >> 32);
      }
      __syncthreads();
      if (s_rescan) {
#pragma unroll 4
        for (uint32_t x = x0 + 4 * threadIdx.x; x < x1v; x += 4 * kGreedyThreads) {
          const uint4 c = __ldcg(cw4 + (x >> 2));
          m = umax(m, umax(umax(key_of(c.x, x), key_of(c.y, x + 1)), umax(key_of(c.z, x + 2), key_of(c.w, x + 3))));
        }
        for (uint32_t x = x1v + threadIdx.x; x < x1; x += kGreedyThreads)
          m = umax(m, key_of(__ldcg(D.cnt_work + x), x));
        m = warp_max(m);
        if (lane == 0) part[wib] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
          unsigned long long b = 0;
#pragma unroll
          for (int w = 0; w < kGreedyThreads / 32; ++w) b = umax(b, part[w]);
          s_light = b;
        }
      }
      // the group's first block also takes the hub counts (few; read every round)
      if (lb == 0 && H) {
        unsigned long long h = 0;
        for (uint32_t s = threadIdx.x; s < H; s += kGreedyThreads) h = umax(h, key_of(__ldcg(hc + s), hid[s]));
        h = warp_max(h);
        __syncthreads();
        if (lane == 0) part[wib] = h;
        __syncthreads();
        if (threadIdx.x == 0) {
          unsigned long long b = s_light;
#pragma unroll
          for (int w = 0; w < kGreedyThreads / 32; ++w) b = umax(b, part[w]);
          atomicMax(D.best + t, b);
        }
      } else if (threadIdx.x == 0) {
        atomicMax(D.best + t, s_light);
      }
    }
    target += nb;
    if (!group_sync(D.bar, target, err)) return;

    // cover (the seed's slot and list bounds are loaded together)
    const unsigned long long key = __ldcg(D.best + t);
    const uint32_t u = ~(uint32_t)(key & 0xFFFFFFFFull);
    const uint32_t cw = (uint32_t)(key >> 32);
    const uint32_t us = D.hslot[u];
    const uint64_t i0 = D.inv_off[u], i1 = D.inv_end ? D.inv_end[u] : D.inv_off[u + 1];
    if constexpr (kPart) {
      if (pn && threadIdx.x == 0) {   // this round's seed counts toward its round (read by the next argmax)
        const uint32_t r = u / pn;
        if (r < kMaxRounds && ++s_picks[r] == D.part_k) s_closed |= 1u << r;
      }
    }
    if (lb == 0 && threadIdx.x == 0) {
      D.seeds[t] = u;
      D.gains[t] = cw ? cw - 1u : 0u;
      if (us == 0xFFu)
        D.cnt_work[u] = 0u;   // selected; no thread lowers the seed's count in this round
      else
        hc[us] = 0u;
    }
    if (us == 0xFFu) {
      // light seed: its inverted list, one set per warp. Lane 0 claims the
      // set on the covered bitmap and the warp follows its answer (lanes that
      // read the bitmap themselves could see a bit lane 0 has just set); the
      // set's place is loaded in the same round trip as the claim.
      for (uint64_t p = i0 + gwarp; p < i1; p += nwarps) {
        const uint32_t j = D.inv[p];
        if (j >= D.R) continue;   // beyond this instance's prefix of a shared index
        const uint64_t sb = D.rr_start[j];
        const uint32_t sl = D.rr_len[j];
        uint32_t fresh = 0;
        if (lane == 0) {
          const uint32_t bit = 1u << (j & 31u);
          fresh = (atomicOr(D.covered + (j >> 5), bit) & bit) ? 0u : 1u;
        }
        fresh = __shfl_sync(kFullMask, fresh, 0);
        if (!fresh) continue;
        const uint32_t len = cover_members(D, sb, sl, u, H, s_delta, lane);
        if (lane == 0) {
          newly += 1;
          cov_members += len;
        }
      }
      if (lb == 0 && threadIdx.x == 0) list_words += i1 - i0;
    } else {
      // hub seed: its bitmap row, 32 words per warp; the warp then covers the
      // new sets of those words one at a time
      const uint32_t *row = D.hbits + (uint64_t)us * D.row_words;
      const uint32_t last_mask = (D.R & 31u) ? (1u << (D.R & 31u)) - 1u : 0xFFFFFFFFu;
      for (uint32_t w0 = gwarp * 32u; w0 < D.words; w0 += nwarps * 32u) {
        const uint32_t w = w0 + lane;
        uint32_t mine = 0;
        if (w < D.words) {
          const uint32_t bits = row[w] & ~__ldcg(D.covered + w) & (w + 1 == D.words ? last_mask : 0xFFFFFFFFu);
          if (bits) mine = bits & ~atomicOr(D.covered + w, bits);
        }
        newly += __popc(mine);
        uint32_t pend = __ballot_sync(kFullMask, mine != 0u);
        while (pend) {
          const uint32_t src = __ffs(pend) - 1;
          pend &= pend - 1;
          uint32_t bits = __shfl_sync(kFullMask, mine, src);
          const uint32_t base = (w0 + src) << 5;
          while (bits) {
            const uint32_t b = __ffs(bits) - 1;
            bits &= bits - 1;
            const uint32_t len = cover_set(D, base + b, u, H, s_delta, lane);
            if (lane == 0) cov_members += len;
          }
        }
      }
      if (lb == 0 && threadIdx.x == 0) list_words += D.words;
    }
    flush_hubs(s_delta, hc, H);
    target += nb;
    if (!group_sync(D.bar, target, err)) return;
  }

  // block sums of the per-thread counters
  unsigned long long v[3] = {newly, cov_members, list_words};
  __shared__ unsigned long long acc[3];
  if (threadIdx.x < 3) acc[threadIdx.x] = 0ull;
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    unsigned long long x = v[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFullMask, x, o);
    if (lane == 0 && x) atomicAdd(acc + c, x);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (acc[0]) atomicAdd(D.covered_total, acc[0]);
    if (acc[1]) atomicAdd(D.stats, acc[1]);
    if (acc[2]) atomicAdd(D.stats + 1, acc[2]);
  }
}

__global__ void __launch_bounds__(kGreedyThreads) greedy_kernel(const GreedyDesc *d, uint32_t ni, unsigned int *err) {
  greedy_body<false>(d, ni, err);
}

// at most 64 registers, so that it fits the grid sized for greedy_kernel
__global__ void __launch_bounds__(kGreedyThreads, 2) greedy_part_kernel(const GreedyDesc *d, uint32_t ni,
                                                                          unsigned int *err) {
  greedy_body<true>(d, ni, err);
}

}  // namespace

uint32_t greedy_max_blocks(int sm_count) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, greedy_kernel, kGreedyThreads, 0) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  // two blocks per SM at most: the barrier's cost grows with the group
  return (uint32_t)std::max(1, std::min(per_sm, 2) * sm_count);
}

cudaError_t launch_greedy(const GreedyDesc *d, uint32_t ni, uint32_t grid, unsigned int *err, cudaStream_t s,
                          bool part) {
  if (grid == 0 || ni == 0) return cudaSuccess;
  void *args[] = {(void *)&d, (void *)&ni, (void *)&err};
  const void *fn = part ? (const void *)greedy_part_kernel : (const void *)greedy_kernel;
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kGreedyThreads), args, 0, s);
}

}  // namespace gim
