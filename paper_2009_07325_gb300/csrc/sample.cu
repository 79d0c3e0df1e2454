// RR-set sampling kernels (Sec. III-B to III-G; Alg. 3 and Alg. 6).
//
// A persistent grid of warps; each warp is one worker that takes RR-set ids
// from a device work counter (the role of Alg. 6's N_RR) and builds one RR
// set at a time:
//   IC: reverse BFS over in-edges. Frontier vertices are taken in batches of
//       up to 32, whose queue entries, offsets and row thresholds are loaded
//       in one round trip; the rows are then scanned one after another by the
//       whole warp, two groups of four consecutive edges per lane per step
//       (one Philox call gives a group's four coin words). When all in-edges
//       of a row share one probability (weighted cascade, uniform p) the
//       row's threshold is used and the scan reads no edge data; otherwise
//       one 16-byte load fetches the group's four thresholds. Live edges are
//       buffered in shared memory; the buffer is resolved 32 edges at a time
//       (read the source, test-and-set its bit in the worker's visited bitmap,
//       append the newly visited to the worker's queue, which doubles as the
//       member list: Sec. III-A, each vertex is expanded once).
//   LT: the reverse walk of Sec. III-G: one draw per step, the chosen in-edge
//       found by a 33-way warp search over the row's sorted cumulative
//       thresholds, stop at no edge or at a vertex already on the path.
// A finished set reserves its place in the store with one atomic (Alg. 6's
// tail_RR) and is copied there; the occurrence counts (Occur) are bumped.
// Sets that outgrow the worker's queue, or find the store full, are listed
// as deferred and redone by the large-set pass (queue of n entries) after
// the host has grown the store. RR set j depends only on (seed, j), so the
// redo yields the same set.
#include "gim_internal.cuh"

namespace gim {

namespace {

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t comp(const uint4 &v, int q) {
  return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
}

__device__ __forceinline__ void defer(const SampleJob &job, SampleCtl *ctl, uint64_t j) {
  const unsigned long long d = atomicAdd(&ctl->n_deferred, 1ull);
  if (d < job.deferred_cap)
    job.deferred[d] = j;
  else
    atomicOr(&ctl->err, kErrDeferredFull);
}

// Copies the finished set q[0..size) to the store, bumps the occurrence
// counts and clears the visited bits (bm may be null). Lane-uniform control.
__device__ __forceinline__ void commit_set(const DevStore &st, const SampleJob &job, SampleCtl *ctl, uint64_t j,
                                           const uint32_t *q, uint32_t size, uint32_t *bm) {
  const uint32_t lane = lane_id();
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(&ctl->store_tail, (unsigned long long)size);
  base = __shfl_sync(kFullMask, base, 0);
  const bool fits = base + size <= st.cap;
  for (uint32_t i = lane; i < size; i += 32) {
    const uint32_t x = q[i];
    if (fits) {
      st.members[base + i] = x;
      atomicAdd(&st.cnt[x], 1u);
    }
    if (bm) bm[x >> 5] = 0u;   // every set bit of the bitmap belongs to this set
  }
  __syncwarp();
  if (lane == 0) {
    if (fits) {
      st.rr_start[j] = base;
      st.rr_len[j] = size;
      atomicAdd(&ctl->members, (unsigned long long)size);
    } else {
      defer(job, ctl, j);
    }
  }
}

// Coins of group grp (in-edges 4grp .. 4grp+3) for the row [s, e): bit qi is
// set iff edge 4grp+qi lies in the row and is live. One Philox call yields
// the four coin words. The threshold is the row's common one when it has
// one (rt != kPerEdge), so the scan of such a row touches no memory.
__device__ __forceinline__ uint32_t group_live(const uint32_t *__restrict__ thr, uint32_t grp, uint32_t s, uint32_t e,
                                               uint32_t rt, uint32_t jlo, uint32_t jhi, PhiloxKey key) {
  const uint4 r = philox10(grp, kTagEdge, jlo, jhi, key);
  uint4 tv;
  if (rt != kPerEdge)
    tv = make_uint4(rt, rt, rt, rt);
  else
    tv = reinterpret_cast<const uint4 *>(thr)[grp];
  uint32_t live = ((r.x >> 8) < tv.x ? 1u : 0u) | ((r.y >> 8) < tv.y ? 2u : 0u) | ((r.z >> 8) < tv.z ? 4u : 0u) |
                  ((r.w >> 8) < tv.w ? 8u : 0u);
  const uint32_t e0 = grp << 2;            // s - 3 <= e0 <= e - 1
  if (e0 < s || e0 + 4 > e) {
    const uint32_t lo = s > e0 ? s - e0 : 0u;
    const uint32_t hi = e - e0 < 4u ? e - e0 : 4u;
    live &= ((1u << hi) - 1u) & ~((1u << lo) - 1u);
  }
  return live;
}

constexpr uint32_t kCandCap = 512;   // per-warp buffer of live edges awaiting their visited test

// Resolves the buffered live edges cand[0..ncand): reads each one's source,
// test-and-sets its visited bit and appends the newly visited sources to the
// queue (32 edges per round trip). Lane-uniform control.
__device__ __forceinline__ void ic_flush(const uint32_t *__restrict__ src, const uint32_t *cand, uint32_t ncand,
                                         uint32_t *bm, uint32_t *q, uint32_t qcap, uint32_t &tail, bool &overflow) {
  const uint32_t lane = lane_id();
  const uint32_t below = (1u << lane) - 1u;
  __syncwarp();
  for (uint32_t i0 = 0; i0 < ncand; i0 += 32) {
    const uint32_t i = i0 + lane;
    uint32_t u = 0;
    bool fresh = false;
    if (i < ncand) {
      u = src[cand[i]];
      const uint32_t bit = 1u << (u & 31u);
      fresh = (atomicOr(&bm[u >> 5], bit) & bit) == 0u;
    }
    const uint32_t fm = __ballot_sync(kFullMask, fresh);
    if (fm) {
      const uint32_t pos = tail + __popc(fm & below);
      if (fresh) {
        if (pos < qcap)
          q[pos] = u;
        else
          atomicAnd(&bm[u >> 5], ~(1u << (u & 31u)));   // not queued: leave no trace
      }
      tail += __popc(fm);
      if (tail > qcap) {
        tail = qcap;
        overflow = true;
      }
    }
  }
  __syncwarp();
}

template <bool kLarge>
__global__ void __launch_bounds__(256) sample_ic_kernel(DevGraph g, DevStore st, WorkerScratch ws, SampleJob job,
                                                        SampleCtl *ctl) {
  __shared__ uint32_t cand_all[8][kCandCap];
  const uint32_t lane = lane_id();
  const uint32_t worker = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (worker >= ws.workers) return;
  uint32_t *cand = cand_all[threadIdx.x >> 5];
  uint32_t *bm = ws.bitmap + (uint64_t)worker * ws.words_per_worker;
  uint32_t *q = ws.queue + (uint64_t)worker * ws.qcap;
  const uint32_t qcap = ws.qcap;

  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(&ctl->next, 1ull);
    item = __shfl_sync(kFullMask, item, 0);
    if (item >= job.count) break;
    const uint64_t j = job.j_list ? job.j_list[item] : job.j_begin + item;
    const uint32_t jlo = (uint32_t)j, jhi = (uint32_t)(j >> 32);
    const uint32_t root = draw_root(job.key, j, g.n);
    if (lane == 0) {
      q[0] = root;
      bm[root >> 5] = 1u << (root & 31u);   // the worker's bitmap is all zero here
    }
    uint32_t head = 0, tail = 1;
    bool overflow = false;
    while (head < tail && !overflow) {
      __syncwarp();
      // a batch of up to 32 frontier vertices: their rows are fetched at once
      const uint32_t nb = tail - head < 32u ? tail - head : 32u;
      uint32_t rs = 0, re = 0, rr = 0;
      if (lane < nb) {
        const uint32_t v = q[head + lane];
        rs = g.off[v];
        re = g.off[v + 1];
        rr = g.rthr[v];
      }
      head += nb;
      uint32_t ncand = 0;
      for (uint32_t b = 0; b < nb && !overflow; ++b) {
        const uint32_t s = __shfl_sync(kFullMask, rs, b), e = __shfl_sync(kFullMask, re, b);
        const uint32_t rt = __shfl_sync(kFullMask, rr, b);
        if (e <= s || rt == 0u) continue;      // a row whose coins are all 0 adds nothing
        const uint32_t g0 = s >> 2, g1 = (e - 1) >> 2;
        for (uint32_t base = g0; base <= g1; base += 64) {
          const uint32_t ga = base + lane, gb = base + 32 + lane;
          uint32_t la = 0, lb = 0;
          if (ga <= g1) la = group_live(g.thr, ga, s, e, rt, jlo, jhi, job.key);
          if (gb <= g1) lb = group_live(g.thr, gb, s, e, rt, jlo, jhi, job.key);
          const uint32_t mine = __popc(la) + __popc(lb);
          if (__ballot_sync(kFullMask, mine != 0u) == 0u) continue;
          uint32_t incl = mine;
#pragma unroll
          for (int d = 1; d < 32; d <<= 1) {
            const uint32_t o = __shfl_up_sync(kFullMask, incl, d);
            if (lane >= (uint32_t)d) incl += o;
          }
          const uint32_t total = __shfl_sync(kFullMask, incl, 31);
          if (ncand + total > kCandCap) {
            ic_flush(g.src, cand, ncand, bm, q, qcap, tail, overflow);
            ncand = 0;
          }
          uint32_t pos = ncand + incl - mine;
#pragma unroll
          for (int qi = 0; qi < 4; ++qi)
            if ((la >> qi) & 1u) cand[pos++] = (ga << 2) + qi;
#pragma unroll
          for (int qi = 0; qi < 4; ++qi)
            if ((lb >> qi) & 1u) cand[pos++] = (gb << 2) + qi;
          ncand += total;
        }
      }
      ic_flush(g.src, cand, ncand, bm, q, qcap, tail, overflow);
    }
    if (overflow) {
      for (uint32_t i = lane; i < tail; i += 32) bm[q[i] >> 5] = 0u;
      __syncwarp();
      if (lane == 0) defer(job, ctl, j);
      continue;
    }
    commit_set(st, job, ctl, j, q, tail, bm);
  }
}

// Finds the first index a in [s, e) with U < cum[a], or e if there is none.
// cum is non-decreasing within the row. Warp-uniform result.
__device__ __forceinline__ uint32_t lt_pick(const uint64_t *__restrict__ cum, uint32_t s, uint32_t e, uint32_t U) {
  const uint32_t lane = lane_id();
  uint32_t lo = s, hi = e;   // invariant: the answer lies in [lo, hi]
  while (hi - lo > 32) {
    const uint32_t len = hi - lo;
    const uint32_t p = lo + (uint32_t)(((uint64_t)len * (lane + 1)) / 33u);
    const uint32_t b = __ballot_sync(kFullMask, (uint64_t)U < cum[p]);
    if (b == 0) {
      lo = __shfl_sync(kFullMask, p, 31) + 1;
    } else {
      const int f = __ffs(b) - 1;
      const uint32_t pf = __shfl_sync(kFullMask, p, f);
      const uint32_t pb = __shfl_sync(kFullMask, p, f > 0 ? f - 1 : 0);
      hi = pf;
      if (f > 0) lo = pb + 1;
    }
  }
  const uint32_t len = hi - lo;
  const bool gt = lane < len && (uint64_t)U < cum[lo + lane];
  const uint32_t b = __ballot_sync(kFullMask, gt);
  return b ? lo + (uint32_t)(__ffs(b) - 1) : hi;
}

// LT walk. kLarge = false keeps the path in shared memory (capacity qcap per
// warp) and tests "already visited" by a warp-wide compare against the path;
// kLarge = true keeps it in the worker's global queue with the visited bitmap.
template <bool kLarge>
__global__ void __launch_bounds__(256) sample_lt_kernel(DevGraph g, DevStore st, WorkerScratch ws, SampleJob job,
                                                        SampleCtl *ctl) {
  extern __shared__ uint32_t smem[];
  const uint32_t lane = lane_id();
  const uint32_t worker = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (worker >= ws.workers) return;
  const uint32_t qcap = ws.qcap;
  uint32_t *bm = kLarge ? ws.bitmap + (uint64_t)worker * ws.words_per_worker : nullptr;
  uint32_t *path = kLarge ? ws.queue + (uint64_t)worker * qcap : smem + (threadIdx.x >> 5) * qcap;

  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(&ctl->next, 1ull);
    item = __shfl_sync(kFullMask, item, 0);
    if (item >= job.count) break;
    const uint64_t j = job.j_list ? job.j_list[item] : job.j_begin + item;
    const uint32_t jlo = (uint32_t)j, jhi = (uint32_t)(j >> 32);
    uint32_t x = draw_root(job.key, j, g.n);
    if (lane == 0) {
      path[0] = x;
      if (kLarge) bm[x >> 5] = 1u << (x & 31u);
    }
    __syncwarp();
    uint32_t L = 1;
    bool overflow = false;
    for (;;) {
      const uint32_t U = philox10(x, kTagStep, jlo, jhi, job.key).x;
      const uint32_t s = g.off[x], e = g.off[x + 1];
      if (e == s) break;
      const uint32_t a = lt_pick(g.cum, s, e, U);
      if (a >= e) break;
      const uint32_t u = g.src[a];
      bool seen;
      if (kLarge) {
        uint32_t old = 0;
        if (lane == 0) old = atomicOr(&bm[u >> 5], 1u << (u & 31u));
        seen = (__shfl_sync(kFullMask, old, 0) >> (u & 31u)) & 1u;
      } else {
        bool hit = false;
        for (uint32_t i = lane; i < L; i += 32) hit |= (path[i] == u);
        seen = __any_sync(kFullMask, hit);
      }
      if (seen) break;
      if (L == qcap) {
        overflow = true;
        if (kLarge && lane == 0) atomicAnd(&bm[u >> 5], ~(1u << (u & 31u)));
        break;
      }
      if (lane == 0) path[L] = u;
      ++L;
      __syncwarp();
      x = u;
    }
    if (overflow) {
      if (kLarge) {
        for (uint32_t i = lane; i < L; i += 32) bm[path[i] >> 5] = 0u;
        __syncwarp();
      }
      if (lane == 0) defer(job, ctl, j);
      continue;
    }
    commit_set(st, job, ctl, j, path, L, bm);
    __syncwarp();
  }
}

// Rollback helper: lowers the occurrence counts of the sets among
// [j_begin, j_begin + count) that were stored (rr_start != kNoStart).
__global__ void uncount_kernel(DevStore st, uint64_t j_begin, uint64_t count) {
  const uint32_t lane = lane_id();
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t i = warp; i < count; i += nwarps) {
    const uint64_t j = j_begin + i;
    const uint64_t b = st.rr_start[j];
    if (b == kNoStart) continue;
    const uint32_t len = st.rr_len[j];
    for (uint32_t t = lane; t < len; t += 32) atomicSub(&st.cnt[st.members[b + t]], 1u);
  }
}

// Pure Philox4x32-10 throughput: each thread draws `per_thread` blocks on
// consecutive counters (the IC coin counter layout) and folds the words so
// that nothing is optimised away. Measures the ALU ceiling of the coin work.
__global__ void __launch_bounds__(256) philox_rate_kernel(PhiloxKey key, uint32_t per_thread, uint32_t *sink) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t acc = 0;
  for (uint32_t i = 0; i < per_thread; i += 2) {
    const uint32_t c = t * per_thread + i;
    const uint4 a = philox10(c, kTagEdge, 0x1234u, 0u, key);
    const uint4 b = philox10(c + 1, kTagEdge, 0x1234u, 0u, key);
    acc += (a.x ^ a.y ^ a.z ^ a.w) + (b.x ^ b.y ^ b.z ^ b.w);
  }
  if (acc == 0x9E3779B9u) sink[t & 1023] = acc;   // practically never stored
}

}  // namespace

cudaError_t launch_philox_rate(int blocks, uint32_t per_thread, uint32_t *sink, cudaStream_t s) {
  philox_rate_kernel<<<blocks, 256, 0, s>>>(PhiloxKey{0x01234567u, 0x89ABCDEFu}, per_thread, sink);
  return cudaGetLastError();
}

cudaError_t launch_sample(int model, const DevGraph &g, const DevStore &st, const WorkerScratch &ws, const SampleJob &job,
                          SampleCtl *ctl, bool large, int grid, int block, cudaStream_t s) {
  if (model == GIM_IC) {
    if (large)
      sample_ic_kernel<true><<<grid, block, 0, s>>>(g, st, ws, job, ctl);
    else
      sample_ic_kernel<false><<<grid, block, 0, s>>>(g, st, ws, job, ctl);
  } else {
    if (large) {
      sample_lt_kernel<true><<<grid, block, 0, s>>>(g, st, ws, job, ctl);
    } else {
      const size_t sm = (size_t)(block / 32) * ws.qcap * sizeof(uint32_t);
      sample_lt_kernel<false><<<grid, block, sm, s>>>(g, st, ws, job, ctl);
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_uncount(const DevStore &st, uint64_t j_begin, uint64_t count, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  uint64_t blocks = (count + 7) / 8;
  if (blocks > 4096) blocks = 4096;
  uncount_kernel<<<(unsigned)blocks, 256, 0, s>>>(st, j_begin, count);
  return cudaGetLastError();
}

}  // namespace gim
