// RR-set sampling kernels (Sec. III-B to III-G; Alg. 3 and Alg. 6).
//
// Every launch serves a table of instances (graph + RR collection + ids to
// draw); a device work counter hands out global items, and item i belongs to
// the instance whose item range contains it (or names its instance
// explicitly in the large-set passes). RR set j depends only on
// (graph, seed, j), so which worker draws it, in which pass and in which
// order never changes the set.
//
// IC, common pass: a persistent grid of warps, one RR set per warp at a time
//   (the role of Alg. 6's N_RR counter is the work counter). Reverse BFS over
//   in-edges: frontier vertices are taken in batches of up to 32 (queue
//   entries, offsets and row thresholds fetched in one round trip); each row
//   is scanned by the whole warp, two groups of four consecutive in-edges per
//   lane per step, one Philox call giving a group's four coin words. A row
//   whose in-edges share one probability (weighted cascade, uniform p) uses
//   its common threshold, so the scan reads no edge data; otherwise one
//   16-byte load fetches a group's four thresholds. A row whose common
//   probability is at most 2^-8 (the hub rows of weighted cascade, where
//   almost all coin work lies) is scanned in super-groups of 16 in-edges:
//   one Philox call gives the top bytes of 16 coin uniforms, and only an
//   edge whose byte is zero (1 in 256) draws its low 16 bits, 32 such edges
//   at a time from a per-warp pending list (sgroup_zero, resolve_pending).
//   Live edges are buffered
//   in shared memory and resolved 32 per round trip: read the source,
//   insert it into the worker's visited hash set, append the newly visited
//   to the worker's queue (which doubles as the member list: Sec. III-A,
//   each vertex is expanded once). The hash set is stamped with a per-set
//   epoch, so it is never cleared. A set that outgrows the queue or scans
//   more than its edge budget is abandoned and deferred.
// IC, large-set pass: one 128-thread block per deferred set (16 per SM),
//   with an n-bit visited bitmap and a queue. Each batch of up to 128
//   frontier vertices is cut into chunks of at most 2048 in-edges (512
//   Philox calls), or 4096 in a super-group row (256 calls), that the
//   block's warps take from a shared counter, longest first, so the heavy
//   tail of huge RR sets is spread over 4 warps. Only __syncthreads
//   barriers are used.
// LT: the reverse walk of Sec. III-G (four walks per warp in the common pass, see
//   lt_multi_kernel; one warp per walk in the large pass): one draw per step,
//   the chosen in-edge found by a 33-way warp search over the row's sorted
//   cumulative thresholds, stop at no edge or at a vertex already on the
//   path (common pass: path in shared memory; large pass: queue + bitmap).
// A finished set reserves its place in its instance's store with one atomic
// (Alg. 6's tail_RR) and is copied there; the occurrence counts (Occur) are
// bumped. A set that finds its store full is deferred too; the host grows the
// store and runs the large-set pass on the deferred list.
#include "gim_internal.cuh"

namespace gim {

namespace {

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// Instance of global item `item`: the last one whose item_begin <= item.
__device__ __forceinline__ uint32_t find_inst(const InstDesc *inst, uint32_t n_inst, unsigned long long item) {
  uint32_t lo = 0, hi = n_inst - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (inst[mid].item_begin <= item)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Decodes work item `item` of launch L into (instance, rr_id).
__device__ __forceinline__ void decode_item(const SampleLaunch &L, unsigned long long item, uint32_t &ii, uint64_t &j) {
  if (L.items) {
    const unsigned long long p = L.items[item];
    ii = (uint32_t)(p >> 32);
    j = (uint32_t)p;
  } else {
    ii = find_inst(L.inst, L.n_inst, item);
    j = L.inst[ii].j_begin + (item - L.inst[ii].item_begin);
  }
}

// The fields of an instance a kernel reads. Single-instance launches build it
// from a kernel parameter, so every field is warp-uniform (uniform registers);
// batched launches read the instance's row of the descriptor table.
struct InstView {
  uint32_t n;
  const uint32_t *off, *src, *thr, *rthr, *rw;
  const uint64_t *cum;
  uint32_t *members;
  unsigned long long store_cap;
  uint64_t *rr_start;
  uint32_t *rr_len;
  uint32_t *cnt;
  PhiloxKey key;
  unsigned long long j_begin;
  uint32_t jhi;    // the rr_id of the set at position j is (jhi : j + idoff); positions stay below 2^32
  uint32_t rhi;    // high word of the root draw
  uint32_t moff;   // stored member = moff + vertex
  uint32_t idoff;
  uint32_t skip;   // sets holding this vertex keep only their size (kNoSkip: none)
};

__device__ __forceinline__ InstView view_of(const InstDesc &d) {
  return InstView{d.n, d.off, d.src, d.thr, d.rthr, d.rw, d.cum, d.members, d.store_cap, d.rr_start, d.rr_len, d.cnt,
                  d.key, d.j_begin, d.jhi, d.rhi, d.moff, d.idoff, d.skip};
}

// Low word of the rr_id of the set at position j.
__device__ __forceinline__ uint32_t id_lo(const InstView &V, uint64_t j) { return (uint32_t)j + V.idoff; }

// Instance and rr_id of work item `item`, and the instance's view.
template <bool kOne>
__device__ __forceinline__ InstView item_view(const SampleLaunch &L, const InstDesc &one, unsigned long long item,
                                              uint32_t &ii, uint64_t &j) {
  if (kOne) {
    ii = 0;
    j = L.items ? (uint64_t)(uint32_t)L.items[item] : one.j_begin + item;
    return view_of(one);
  }
  decode_item(L, item, ii, j);
  return view_of(L.inst[ii]);
}

__device__ __forceinline__ void defer(const SampleLaunch &L, uint32_t ii, uint64_t j, uint32_t slot = kNoSlot) {
  const unsigned long long d = atomicAdd(&L.ctl->n_deferred, 1ull);
  if (d < L.deferred_cap) {
    L.deferred[d] = ((unsigned long long)ii << 32) | (uint32_t)j;
    if (L.deferred_slots) L.deferred_slots[d] = slot;
  } else {
    atomicOr(&L.ctl->err, kErrDeferredFull);
  }
}

// Warp-wide: copies the finished set q[0..size) to instance ii's store and
// bumps its occurrence counts; clears the set's bitmap bits when bm != null.
// Defers the set if the store is full. A set that holds the instance's
// skipped vertex is counted but not copied (rr_start = kSkipped).
__device__ __forceinline__ void commit_warp(const SampleLaunch &L, const InstView &V, uint32_t ii, uint64_t j,
                                            const uint32_t *q, uint32_t size, uint32_t *bm) {
  InstDesc &D = L.inst[ii];
  const uint32_t lane = lane_id();
  bool skipped = false;
  if (V.skip != kNoSkip) {
    if (bm) {
      skipped = (bm[V.skip >> 5] >> (V.skip & 31u)) & 1u;
    } else {
      bool has = false;
      for (uint32_t i = lane; i < size; i += 32) has |= q[i] == V.skip;
      skipped = __any_sync(kFullMask, has);
    }
    __syncwarp();
  }
  unsigned long long base = 0;
  if (lane == 0 && !skipped) base = atomicAdd(&D.store_tail, (unsigned long long)size);
  base = __shfl_sync(kFullMask, base, 0);
  const bool fits = skipped || base + size <= V.store_cap;
  const bool copy = fits && !skipped;
  uint32_t *members = V.members;
  uint32_t *cnt = V.cnt;
  for (uint32_t i = lane; i < size; i += 32) {
    const uint32_t x = q[i];
    if (copy) members[base + i] = V.moff + x;
    if (fits) atomicAdd(&cnt[V.moff + x], 1u);
    if (bm) bm[x >> 5] = 0u;   // every set bit of the bitmap belongs to this set
  }
  __syncwarp();
  if (lane == 0) {
    if (fits) {
      V.rr_start[j] = skipped ? kSkipped : base;
      V.rr_len[j] = size;
      if (!skipped) atomicAdd(&D.members_added, (unsigned long long)size);
    } else {
      defer(L, ii, j);
    }
  }
}

// The coin test (word >> 8) < t for a threshold t in [1, 2^24] is
// word <= t * 256 - 1; lim() gives that bound (t = 0 rows are never scanned).
__device__ __forceinline__ uint32_t lim(uint32_t t) { return (t << 8) - 1u; }

// Coins of in-edges with threshold t <= 2^16 (p <= 2^-8): the edge's 24-bit
// uniform is drawn as its top byte, byte e mod 16 of the words of group
// kScreenIdx + e/16 (almost always nonzero: dead), and, only when that byte
// is zero, its low 16 bits, half-word e mod 8 of group kResidIdx + e/8; then
// live iff those bits < t. The coin probability is t / 2^24 as for the
// one-word coin, and one Philox call settles 16 edges instead of 4.
constexpr uint32_t kScreenMax = 1u << 16;
constexpr uint32_t kScreenIdx = 0x80000000u;   // group indices of the top bytes
constexpr uint32_t kResidIdx = 0x40000000u;    // group indices of the residuals (one-word groups stay below 2^30)
__device__ __forceinline__ bool screened(uint32_t t) { return t - 1u < kScreenMax; }   // 1 <= t <= 2^16

// Bit i of the result is set iff byte i of x is zero (exact per byte). The
// marks at bits 0, 8, 16, 24 of t >> 7 are gathered to bits 24..27 by one
// multiply (shifts 24, 17, 10, 3; the other partial products land on
// distinct lower bits, so nothing carries into 24..27).
__device__ __forceinline__ uint32_t zero_bytes(uint32_t x) {
  const uint32_t t = ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x | 0x7F7F7F7Fu);   // 0x80 in each zero byte
  return ((t >> 7) * 0x01020408u) >> 24;
}

__device__ __forceinline__ uint32_t word_of(const uint4 &r, uint32_t i) {
  return i == 0 ? r.x : i == 1 ? r.y : i == 2 ? r.z : r.w;
}

// Second part of a screened coin: the 16-bit residual of in-edge x against t.
__device__ __forceinline__ bool resid_live(uint32_t x, uint32_t t, const CoinKey &ck) {
  const uint4 h = coin_words(kResidIdx | (x >> 3), ck);
  return ((word_of(h, (x >> 1) & 3u) >> ((x & 1u) << 4)) & 0xFFFFu) < t;
}

// 0x80 in each zero byte of x, 0 elsewhere (exact per byte).
__device__ __forceinline__ uint32_t zero_marks(uint32_t x) {
  return ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x | 0x7F7F7F7Fu);
}

// Spreads bits 0..3 of a nibble to bits 0, 8, 16, 24 (one multiply; the
// other partial products land on distinct bits outside the mask).
__device__ __forceinline__ uint32_t spread4(uint32_t nib) { return (nib * 0x00204081u) & 0x01010101u; }

// First part of the coins of super-group sg (in-edges 16sg .. 16sg+15) of
// the row [s, e), in a transposed layout: bit 8b + w is set iff edge
// 16sg + 4w + b (byte b of word w of the draw) lies in the row and its top
// byte is zero, i.e. its coin depends on its residual (resid_live).
__device__ __forceinline__ uint32_t sgroup_zero(uint32_t sg, uint32_t s, uint32_t e, const CoinKey &ck) {
  const uint4 r = coin_words(kScreenIdx | sg, ck);
  uint32_t z = (zero_marks(r.x) >> 7) | (zero_marks(r.y) >> 6) | (zero_marks(r.z) >> 5) | (zero_marks(r.w) >> 4);
  const uint32_t e0 = sg << 4;                // s - 15 <= e0 <= e - 1
  if (e0 < s || e0 + 16 > e) {
    const uint32_t lo = s > e0 ? s - e0 : 0u;
    const uint32_t hi = e - e0 < 16u ? e - e0 : 16u;
    const uint32_t m = ((1u << hi) - 1u) & ~((1u << lo) - 1u);   // bit 4w + b: edge in the row
    z &= spread4(m & 0xFu) | (spread4((m >> 4) & 0xFu) << 1) | (spread4((m >> 8) & 0xFu) << 2) |
         (spread4(m >> 12) << 3);
  }
  return z;
}

// In-super-group index 4w + b of bit p = 8b + w of a transposed mask.
__device__ __forceinline__ uint32_t zero_edge(uint32_t p) { return ((p & 7u) << 2) + (p >> 3); }

// Coins of group grp (in-edges 4grp .. 4grp+3) for the row [s, e): bit qi is
// set iff edge 4grp+qi lies in the row and is live. One Philox call yields
// the four coin words. The threshold is the row's common one when it has
// one (rt != kPerEdge; rl = lim(rt); never a screened one: such rows go
// through sgroup_zero), so the scan of such a row touches no memory; there
// the usual answer (no live edge: all four words above the bound) is
// settled by their minimum. With per-edge thresholds, screened edges take
// their top byte from word grp mod 4 of their super-group's draw.
__device__ __forceinline__ uint32_t group_live(const uint32_t *__restrict__ thr, uint32_t grp, uint32_t s, uint32_t e,
                                               uint32_t rt, uint32_t rl, const CoinKey &ck) {
  uint32_t live;
  if (rt != kPerEdge) {
    const uint4 r = coin_words(grp, ck);
    if (min(min(r.x, r.y), min(r.z, r.w)) > rl) return 0u;
    live = (r.x <= rl ? 1u : 0u) | (r.y <= rl ? 2u : 0u) | (r.z <= rl ? 4u : 0u) | (r.w <= rl ? 8u : 0u);
  } else {
    const uint4 tv = reinterpret_cast<const uint4 *>(thr)[grp];
    // a zero threshold never fires; lim(0) wraps, so such edges are masked out
    const uint32_t nz = (tv.x ? 1u : 0u) | (tv.y ? 2u : 0u) | (tv.z ? 4u : 0u) | (tv.w ? 8u : 0u);
    const uint32_t sc = (screened(tv.x) ? 1u : 0u) | (screened(tv.y) ? 2u : 0u) | (screened(tv.z) ? 4u : 0u) |
                        (screened(tv.w) ? 8u : 0u);
    live = 0u;
    if ((nz & ~sc) != 0u) {
      const uint4 r = coin_words(grp, ck);
      live = ((r.x <= lim(tv.x) ? 1u : 0u) | (r.y <= lim(tv.y) ? 2u : 0u) | (r.z <= lim(tv.z) ? 4u : 0u) |
              (r.w <= lim(tv.w) ? 8u : 0u)) & nz & ~sc;
    }
    if (sc) {
      uint32_t z = zero_bytes(word_of(coin_words(kScreenIdx | (grp >> 2), ck), grp & 3u)) & sc;
      while (z) {
        const uint32_t qi = __ffs(z) - 1;
        z &= z - 1;
        if (resid_live((grp << 2) + qi, word_of(tv, qi), ck)) live |= 1u << qi;
      }
    }
  }
  const uint32_t e0 = grp << 2;            // s - 3 <= e0 <= e - 1
  if (e0 < s || e0 + 4 > e) {
    const uint32_t lo = s > e0 ? s - e0 : 0u;
    const uint32_t hi = e - e0 < 4u ? e - e0 : 4u;
    live &= ((1u << hi) - 1u) & ~((1u << lo) - 1u);
  }
  return live;
}

// Exclusive prefix of a per-lane count across the warp; total = the sum.
__device__ __forceinline__ uint32_t warp_excl(uint32_t mine, uint32_t &total) {
  const uint32_t lane = lane_id();
  uint32_t incl = mine;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(kFullMask, incl, d);
    if (lane >= (uint32_t)d) incl += o;
  }
  total = __shfl_sync(kFullMask, incl, 31);
  return incl - mine;
}

// Groups (of four in-edges) each lane scans per warp step: that many
// independent Philox chains are in flight per lane.
constexpr uint32_t kGPL = 2;
constexpr uint32_t kStepGroups = 32 * kGPL;
// Super-groups (of 16 in-edges) each lane scans per warp step in a screened
// row: four in the block-per-set pass, two in the warp-per-set pass (whose
// per-warp state is larger).
constexpr uint32_t kSGPL = 4;
constexpr uint32_t kStepSG = 32 * kSGPL;
constexpr uint32_t kSGPLCommon = 2;
constexpr uint32_t kStepSGCommon = 32 * kSGPLCommon;

// Coins of one warp step over groups [base, base + kStepGroups) of the row
// [s, e) whose last group is glast; lv[q] holds lane group base + 32q + lane.
// Returns the lane's number of live edges.
__device__ __forceinline__ uint32_t step_live(const uint32_t *__restrict__ thr, uint32_t base, uint32_t glast,
                                              uint32_t s, uint32_t e, uint32_t rt, uint32_t rl, const CoinKey &ck,
                                              uint32_t (&lv)[kGPL]) {
  const uint32_t lane = lane_id();
  uint32_t n = 0;
#pragma unroll
  for (uint32_t q = 0; q < kGPL; ++q) {
    const uint32_t g = base + 32 * q + lane;
    lv[q] = g <= glast ? group_live(thr, g, s, e, rt, rl, ck) : 0u;
    n += __popc(lv[q]);
  }
  return n;
}

// Edges whose top byte was zero wait in a per-warp list with their
// thresholds until 32 or more can be settled together: one converged round
// of residual draws per 32 edges, instead of a round (with one or two active
// lanes) in almost every warp step.
constexpr uint32_t kPend = 64;

// Settles the pending edges pe/pt[0 .. npend): the live ones go to cand
// (flush() empties cand when it is full; ncand is its fill).
template <typename Flush>
__device__ __forceinline__ void resolve_pending(const uint32_t *pe, const uint32_t *pt, uint32_t &npend, uint32_t *cand,
                                                uint32_t &ncand, uint32_t cap, const CoinKey &ck, Flush &&flush) {
  const uint32_t lane = lane_id();
  __syncwarp();
  for (uint32_t i0 = 0; i0 < npend; i0 += 32) {
    const uint32_t i = i0 + lane;
    uint32_t x = 0;
    bool live = false;
    if (i < npend) {
      x = pe[i];
      live = resid_live(x, pt[i], ck);
    }
    const uint32_t lm = __ballot_sync(kFullMask, live);
    if (!lm) continue;
    const uint32_t n = __popc(lm);
    if (ncand + n > cap) {
      flush();
      ncand = 0;
    }
    if (live) cand[ncand + __popc(lm & ((1u << lane) - 1u))] = x;
    ncand += n;
  }
  npend = 0;
  __syncwarp();
}

// One warp step over super-groups [base, base + 32 SG) of a screened
// row [s, e) (threshold rt, last super-group glast): the top bytes of 16
// coins per call; edges with a zero byte join the pending list.
template <uint32_t SG, typename Flush>
__device__ __forceinline__ void step_screened(uint32_t base, uint32_t glast, uint32_t s, uint32_t e, uint32_t rt,
                                              const CoinKey &ck, uint32_t *pe, uint32_t *pt, uint32_t &npend,
                                              uint32_t *cand, uint32_t &ncand, uint32_t cap, Flush &&flush) {
  const uint32_t lane = lane_id();
  uint32_t z[SG];
  uint32_t cnt = 0;
#pragma unroll
  for (uint32_t q = 0; q < SG; ++q) {
    const uint32_t g = base + 32 * q + lane;
    z[q] = g <= glast ? sgroup_zero(g, s, e, ck) : 0u;
    cnt += __popc(z[q]);
  }
  if (__ballot_sync(kFullMask, cnt != 0u) == 0u) return;
  uint32_t total;
  const uint32_t excl = warp_excl(cnt, total);
  if (npend + total > kPend) resolve_pending(pe, pt, npend, cand, ncand, cap, ck, flush);
  if (total <= kPend) {
    uint32_t pos = npend + excl;
#pragma unroll
    for (uint32_t q = 0; q < SG; ++q) {
      uint32_t m = z[q];
      const uint32_t g = base + 32 * q + lane;
      while (m) {
        const uint32_t p = __ffs(m) - 1;
        m &= m - 1;
        pe[pos] = (g << 4) + zero_edge(p);
        pt[pos] = rt;
        ++pos;
      }
    }
    npend += total;
    __syncwarp();
    return;
  }
  // more zero bytes in one step than the list holds (never seen in practice):
  // settle them here, one per lane at a time
  for (;;) {
    uint32_t x = 0;
    bool has = false;
#pragma unroll
    for (uint32_t q = 0; q < SG; ++q)
      if (!has && z[q]) {
        const uint32_t p = __ffs(z[q]) - 1;
        z[q] &= z[q] - 1;
        x = ((base + 32 * q + lane) << 4) + zero_edge(p);
        has = true;
      }
    if (__ballot_sync(kFullMask, has) == 0u) break;
    const bool live = has && resid_live(x, rt, ck);
    const uint32_t lm = __ballot_sync(kFullMask, live);
    if (!lm) continue;
    const uint32_t n = __popc(lm);
    if (ncand + n > cap) {
      flush();
      ncand = 0;
    }
    if (live) cand[ncand + __popc(lm & ((1u << lane) - 1u))] = x;
    ncand += n;
  }
}

// Appends the live edges of one warp step to cand, starting at pos.
__device__ __forceinline__ void push_live(uint32_t *cand, uint32_t pos, uint32_t base, const uint32_t (&lv)[kGPL]) {
  const uint32_t lane = lane_id();
#pragma unroll
  for (uint32_t q = 0; q < kGPL; ++q)
#pragma unroll
    for (int qi = 0; qi < 4; ++qi)
      if ((lv[q] >> qi) & 1u) cand[pos++] = ((base + 32 * q + lane) << 2) + qi;
}

constexpr uint32_t kCandCap = 512;   // per-warp buffer of live edges awaiting their visited test
static_assert(kCandCap >= 128 * kGPL, "one warp step's live edges fit the buffer");


// Visited set of the common pass: open addressing over kHashSlots 64-bit
// slots holding epoch << 32 | vertex; a slot whose epoch is not the current
// set's is free. Returns true iff u was not in the set and is now.
__device__ __forceinline__ bool hash_insert(unsigned long long *ht, uint32_t epoch, uint32_t u) {
  const unsigned long long want = ((unsigned long long)epoch << 32) | u;
  uint32_t h = (u * 0x9E3779B1u) >> (32 - kHashBits);
  for (uint32_t probe = 0; probe < kHashSlots; ++probe) {
    unsigned long long cur = ht[h];
    for (int tries = 0; tries < 64; ++tries) {       // a slot changes at most once per set
      if ((uint32_t)(cur >> 32) == epoch) {
        if ((uint32_t)cur == u) return false;
        break;
      }
      const unsigned long long prev = atomicCAS(&ht[h], cur, want);
      if (prev == cur) return true;
      cur = prev;
    }
    h = (h + 1) & (kHashSlots - 1);
  }
  return false;   // unreachable: at most kQueueCap + kCandCap < kHashSlots vertices per set
}

// Resolves the buffered live edges cand[0..ncand) of the common pass (a
// set that reaches qcap members is abandoned).
__device__ __forceinline__ void common_flush(const uint32_t *__restrict__ src, const uint32_t *cand, uint32_t ncand,
                                             unsigned long long *ht, uint32_t epoch, uint32_t *q, uint32_t &tail,
                                             bool &overflow, uint32_t qcap) {
  const uint32_t lane = lane_id();
  const uint32_t below = (1u << lane) - 1u;
  __syncwarp();
  for (uint32_t i0 = 0; i0 < ncand; i0 += 32) {
    const uint32_t i = i0 + lane;
    uint32_t u = 0;
    bool fresh = false;
    if (i < ncand) {
      u = src[cand[i]];
      fresh = hash_insert(ht, epoch, u);
    }
    const uint32_t fm = __ballot_sync(kFullMask, fresh);
    if (fm) {
      const uint32_t pos = tail + __popc(fm & below);
      if (fresh && pos < qcap) q[pos] = u;
      tail += __popc(fm);
      if (tail > qcap) {
        tail = qcap;
        overflow = true;   // the set is abandoned; its hash entries expire with the epoch
      }
    }
  }
  __syncwarp();
}

template <bool kOne>
__global__ void __launch_bounds__(256, 4) ic_common_kernel(SampleLaunch L, CommonScratch cs, InstDesc one) {
  __shared__ uint32_t cand_all[8][kCandCap];
  __shared__ uint32_t pe_all[8][kPend], pt_all[8][kPend];
  const uint32_t lane = lane_id();
  const uint32_t worker = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (worker >= cs.workers) return;
  uint32_t *cand = cand_all[threadIdx.x >> 5];
  uint32_t *pe = pe_all[threadIdx.x >> 5], *pt = pt_all[threadIdx.x >> 5];
  uint32_t *q = cs.queue + (uint64_t)worker * kQueueCap;
  const uint32_t qcap = L.queue_cap >= 32u && L.queue_cap <= kQueueCap ? L.queue_cap : kQueueCap;
  unsigned long long *ht = cs.hash + (uint64_t)worker * kHashSlots;
  uint32_t epoch = cs.epoch[worker];

  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(&L.ctl->next, 1ull);
    item = __shfl_sync(kFullMask, item, 0);
    if (item >= L.total_items) break;
    uint32_t ii = 0;
    uint64_t j = 0;
    const InstView V = item_view<kOne>(L, one, item, ii, j);
    const uint32_t *__restrict__ off = V.off;
    const uint32_t *__restrict__ rthr = V.rthr;
    const uint32_t *__restrict__ thr = V.thr;
    const uint32_t *__restrict__ src = V.src;
    const PhiloxKey key = V.key;
    const CoinKey ck = coin_key(id_lo(V, j), V.jhi, key);

    if (++epoch == 0xFFFFFFFFu) {              // epochs ran out: wipe the table once
      for (uint32_t h = lane; h < kHashSlots; h += 32) ht[h] = 0ull;
      __syncwarp();
      epoch = 1;
    }
    const uint32_t root = draw_root(key, id_lo(V, j), V.rhi, V.n);
    if (lane == 0) {
      q[0] = root;
      ht[(root * 0x9E3779B1u) >> (32 - kHashBits)] = ((unsigned long long)epoch << 32) | root;
    }
    uint32_t head = 0, tail = 1, scanned = 0;
    bool overflow = false, budget_stop = false;
    while (head < tail && !overflow) {
      __syncwarp();
      if (scanned > L.group_budget) {          // a heavy set: hand it to the large-set pass
        overflow = true;
        budget_stop = true;
        break;
      }
      const uint32_t nb = tail - head < 32u ? tail - head : 32u;
      uint32_t rs = 0, re = 0, rr = 0;
      if (lane < nb) {
        const uint32_t v = q[head + lane];
        rs = off[v];
        re = off[v + 1];
        rr = rthr[v];
      }
      head += nb;
      uint32_t ncand = 0, npend = 0;
      auto flush = [&]() { common_flush(src, cand, ncand, ht, epoch, q, tail, overflow, qcap); };
      for (uint32_t b = 0; b < nb && !overflow; ++b) {
        const uint32_t s = __shfl_sync(kFullMask, rs, b), e = __shfl_sync(kFullMask, re, b);
        const uint32_t rt = __shfl_sync(kFullMask, rr, b);
        if (e <= s || rt == 0u) continue;      // a row whose coins are all 0 adds nothing
        if (screened(rt)) {                    // 16 coins per Philox call
          const uint32_t g0 = s >> 4, g1 = (e - 1) >> 4;
          scanned += 4 * (g1 - g0 + 1);
          for (uint32_t base = g0; base <= g1 && !overflow; base += kStepSGCommon)
            step_screened<kSGPLCommon>(base, g1, s, e, rt, ck, pe, pt, npend, cand, ncand, kCandCap, flush);
          continue;
        }
        const uint32_t rl = lim(rt);
        const uint32_t g0 = s >> 2, g1 = (e - 1) >> 2;
        scanned += g1 - g0 + 1;
        for (uint32_t base = g0; base <= g1 && !overflow; base += kStepGroups) {
          uint32_t lv[kGPL];
          const uint32_t mine = step_live(thr, base, g1, s, e, rt, rl, ck, lv);
          if (__ballot_sync(kFullMask, mine != 0u) == 0u) continue;
          uint32_t total;
          const uint32_t excl = warp_excl(mine, total);
          if (ncand + total > kCandCap) {
            common_flush(src, cand, ncand, ht, epoch, q, tail, overflow, qcap);
            ncand = 0;
          }
          push_live(cand, ncand + excl, base, lv);
          ncand += total;
        }
      }
      if (npend) resolve_pending(pe, pt, npend, cand, ncand, kCandCap, ck, flush);
      common_flush(src, cand, ncand, ht, epoch, q, tail, overflow, qcap);
    }
    if (overflow) {
      // Past the budget the set stops between frontier batches: q[0, tail) is
      // its visited set and the rows of q[0, head) are expanded with every live
      // edge resolved, so it is saved for the block pass to continue (RR set j
      // does not depend on who expands which row when). A set that outgrew
      // the queue lost vertices and starts over.
      uint32_t slot = kNoSlot;
      if (budget_stop && L.ic_ovf) {
        if (lane == 0) slot = atomicAdd(L.lt_ovf_next, 1u);
        slot = __shfl_sync(kFullMask, slot, 0);
        if (slot < L.ic_ovf_cap) {
          uint32_t *sv = L.ic_ovf + (uint64_t)slot * kIcOvfStride;
          for (uint32_t i = lane; i < tail; i += 32) sv[2 + i] = q[i];
          if (lane == 0) {
            sv[0] = tail;
            sv[1] = head;
          }
        } else {
          slot = kNoSlot;
        }
      }
      if (lane == 0) defer(L, ii, j, slot);
      continue;
    }
    commit_warp(L, V, ii, j, q, tail, nullptr);
  }
  if (lane == 0) cs.epoch[worker] = epoch;
}

// ---------------------------------------------------------------------------
// IC large-set pass: one block of kBigBlock threads per RR set.
// ---------------------------------------------------------------------------
constexpr uint32_t kBatch = kBigBlock;        // frontier vertices per block step, at most (one row per thread)
constexpr uint32_t kBigWarps = kBigBlock / 32;
constexpr uint32_t kBigCand = 128 * kGPL;    // per-warp candidate buffer: one warp step's live edges at most
// A chunk is L.chunk_groups groups of 4 in-edges, or half as many
// super-groups of 16 in a screened row; a chunk's last warp step may be
// partial (its groups past the chunk are masked off). The chunks of a batch
// are handed out longest first: every chunk of the rows that need several
// (found by a search over their few prefix entries), then the one-chunk rows
// in queue order (found by a direct index), so the short ones fill the gaps
// at the end of a batch.

// Resolves a warp's buffered live edges: a source not yet in the set joins
// the queue. Past the queue's capacity the vertex is not kept (its bit is
// cleared again) and the set will be abandoned.
__device__ __forceinline__ void block_flush(const uint32_t *__restrict__ src, const uint32_t *cand, uint32_t ncand,
                                            uint32_t *bm, uint32_t *q, uint32_t qcap, uint32_t *s_tail) {
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
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(s_tail, (uint32_t)__popc(fm));
      base = __shfl_sync(kFullMask, base, 0);
      if (fresh) {
        const uint32_t pos = base + __popc(fm & below);
        if (pos < qcap)
          q[pos] = u;
        else
          atomicAnd(&bm[u >> 5], ~(1u << (u & 31u)));
      }
    }
  }
  __syncwarp();
}

template <bool kOne>
__global__ void __launch_bounds__(kBigBlock, kBigBlocksPerSM) ic_block_kernel(SampleLaunch L, BigScratch bs, InstDesc one) {
  __shared__ uint32_t cand_all[kBigWarps][kBigCand];
  __shared__ uint32_t pe_all[kBigWarps][kPend], pt_all[kBigWarps][kPend];
  __shared__ uint32_t b_s[kBatch], b_e[kBatch], b_rt[kBatch];
  __shared__ uint32_t m_row[kBatch], m_pre[kBatch + 1], s_row[kBatch];   // multi-chunk rows, one-chunk rows
  __shared__ uint32_t w_tot[kBigWarps][2];
  __shared__ unsigned long long s_item, s_base;
  __shared__ uint32_t s_tail, s_next, s_head, s_slot;
  const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
  uint32_t *cand = cand_all[warp];
  uint32_t *pe = pe_all[warp], *pt = pt_all[warp];
  uint32_t *bm = bs.bitmap + (uint64_t)blockIdx.x * bs.words_per_slot;
  const uint32_t qcap = bs.q_cap;
  uint32_t *q = bs.queue + (uint64_t)blockIdx.x * qcap;
  // the schedule's knobs (the host keeps L.batch in [32, kBatch] and L.chunk_groups >= 64)
  const uint32_t batch = L.batch, cgroups = L.chunk_groups;

  for (;;) {
    // thread 0 takes the next set and plants its root (the previous set ended
    // with a barrier, so the queue and bitmap are free); one barrier publishes both
    if (tid == 0) {
      const unsigned long long it = atomicAdd(&L.ctl->next, 1ull);
      s_item = it;
      if (it < L.total_items) {
        const uint32_t slot = L.item_slots && L.ic_ovf ? L.item_slots[it] : kNoSlot;
        if (slot < L.ic_ovf_cap) {   // a set the warp pass saved: continue it
          const uint32_t *sv = L.ic_ovf + (uint64_t)slot * kIcOvfStride;
          s_slot = slot;
          s_tail = sv[0];
          s_head = sv[1];
        } else {
          uint32_t i0;
          uint64_t j0;
          const InstView V0 = item_view<kOne>(L, one, it, i0, j0);
          const uint32_t root = draw_root(V0.key, id_lo(V0, j0), V0.rhi, V0.n);
          q[0] = root;
          bm[root >> 5] = 1u << (root & 31u);   // the slot's bitmap is all zero here
          s_slot = kNoSlot;
          s_tail = 1;
          s_head = 0;
        }
      }
    }
    __syncthreads();
    const unsigned long long item = s_item;
    if (item >= L.total_items) break;
    if (s_slot != kNoSlot) {   // the saved visited set: queue entries and bitmap bits
      const uint32_t *sv = L.ic_ovf + (uint64_t)s_slot * kIcOvfStride + 2;
      const uint32_t t = s_tail;
      for (uint32_t i = tid; i < t; i += kBigBlock) {
        const uint32_t v = sv[i];
        q[i] = v;
        atomicOr(&bm[v >> 5], 1u << (v & 31u));
      }
      __syncthreads();
    }
    uint32_t ii;
    uint64_t j;
    const InstView V = item_view<kOne>(L, one, item, ii, j);
    const uint32_t *__restrict__ off = V.off;
    const uint32_t *__restrict__ rthr = V.rthr;
    const uint32_t *__restrict__ thr = V.thr;
    const uint32_t *__restrict__ src = V.src;
    const PhiloxKey key = V.key;
    const CoinKey ck = coin_key(id_lo(V, j), V.jhi, key);
    uint32_t ncand = 0, npend = 0;             // this warp's buffered live edges, pending screened edges
    auto flush = [&]() { block_flush(src, cand, ncand, bm, q, qcap, &s_tail); };
    uint32_t head = s_head;                    // frontier vertices expanded (the same in every thread)
    for (;;) {
      const uint32_t tail = s_tail;
      if (head >= tail || tail > qcap) break;   // done, or the queue overflowed
      const uint32_t nb = tail - head < batch ? tail - head : batch;
      uint32_t nch = 0;                        // chunks of this thread's frontier row
      if (tid < nb) {
        const uint32_t v = q[head + tid];
        const uint32_t s = off[v], e = off[v + 1], rt = rthr[v];
        b_s[tid] = s;
        b_e[tid] = e;
        b_rt[tid] = rt;
        // a chunk is cgroups groups of 4 in-edges, or cgroups / 2 super-groups of 16
        const bool sc = screened(rt);
        const uint32_t sh = sc ? 4u : 2u, cg = sc ? cgroups >> 1 : cgroups;
        nch = (e > s && rt != 0u) ? (((e - 1) >> sh) - (s >> sh) + cg) / cg : 0u;
      }
      // block-wide exclusive prefixes: one-chunk rows and multi-chunk rows
      // (packed, 16 bits each: at most kBatch of either), chunks of the latter
      uint32_t wsum_r, wsum_c;
      const uint32_t wex_r = warp_excl((nch == 1u ? 1u : 0u) | (nch > 1u ? 0x10000u : 0u), wsum_r);
      const uint32_t wex_c = warp_excl(nch > 1u ? nch : 0u, wsum_c);
      if (lane == 0) {
        w_tot[warp][0] = wsum_r;
        w_tot[warp][1] = wsum_c;
      }
      if (tid == 0) s_next = 0;
      __syncthreads();
      uint32_t before_r = 0, before_c = 0, all_r = 0, all_c = 0;
      for (uint32_t w = 0; w < kBigWarps; ++w) {
        if (w < warp) {
          before_r += w_tot[w][0];
          before_c += w_tot[w][1];
        }
        all_r += w_tot[w][0];
        all_c += w_tot[w][1];
      }
      const uint32_t n_multi = all_r >> 16, n_one = all_r & 0xFFFFu;
      if (nch == 1u) {
        s_row[(before_r + wex_r) & 0xFFFFu] = tid;
      } else if (nch > 1u) {
        const uint32_t m = (before_r + wex_r) >> 16;
        m_row[m] = tid;
        m_pre[m] = before_c + wex_c;
      }
      if (tid == 0) m_pre[n_multi] = all_c;
      __syncthreads();
      const uint32_t nchunks = all_c + n_one;
      for (;;) {
        uint32_t c = 0;
        if (lane == 0) c = atomicAdd(&s_next, 1u);
        c = __shfl_sync(kFullMask, c, 0);
        if (c >= nchunks) break;
        uint32_t row, k;                       // the chunk's row and its index within the row
        if (c < all_c) {
          uint32_t lo = 0, hi = n_multi - 1;   // multi-chunk row m with m_pre[m] <= c < m_pre[m + 1]
          while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (m_pre[mid] <= c)
              lo = mid;
            else
              hi = mid - 1;
          }
          row = m_row[lo];
          k = c - m_pre[lo];
        } else {
          row = s_row[c - all_c];
          k = 0;
        }
        const uint32_t s = b_s[row], e = b_e[row], rt = b_rt[row], rl = lim(rt);
        if (screened(rt)) {
          const uint32_t g0 = s >> 4, g1 = (e - 1) >> 4;
          const uint32_t csg = cgroups >> 1;
          const uint32_t c0 = g0 + k * csg;
          const uint32_t c1 = c0 + csg - 1 < g1 ? c0 + csg - 1 : g1;
          for (uint32_t base = c0; base <= c1; base += kStepSG)
            step_screened<kSGPL>(base, c1, s, e, rt, ck, pe, pt, npend, cand, ncand, kBigCand, flush);
          continue;
        }
        const uint32_t g0 = s >> 2, g1 = (e - 1) >> 2;
        const uint32_t c0 = g0 + k * cgroups;
        const uint32_t c1 = c0 + cgroups - 1 < g1 ? c0 + cgroups - 1 : g1;
        for (uint32_t base = c0; base <= c1; base += kStepGroups) {
          uint32_t lv[kGPL];
          const uint32_t mine = step_live(thr, base, c1, s, e, rt, rl, ck, lv);
          if (__ballot_sync(kFullMask, mine != 0u) == 0u) continue;
          uint32_t total;
          const uint32_t excl = warp_excl(mine, total);
          if (ncand + total > kBigCand) {
            block_flush(src, cand, ncand, bm, q, qcap, &s_tail);
            ncand = 0;
          }
          push_live(cand, ncand + excl, base, lv);
          ncand += total;
        }
      }
      // Resolve the buffered live edges only when the frontier runs low: while
      // at least a batch of queued vertices is still unexpanded, the next
      // batch does not need them, and the warps keep them buffered.
      if (tail - (head + nb) < batch) {
        if (npend) resolve_pending(pe, pt, npend, cand, ncand, kBigCand, ck, flush);
        block_flush(src, cand, ncand, bm, q, qcap, &s_tail);
        ncand = 0;
      }
      __syncthreads();                         // appended vertices visible; batch done
      head += nb;
    }
    // commit the set: q[0 .. s_tail); a set that outgrew the queue is
    // abandoned (its bits cleared) and handed to a pass with n-entry queues
    const uint32_t size = s_tail;
    if (size > qcap) {
      for (uint32_t i = tid; i < qcap; i += kBigBlock) bm[q[i] >> 5] = 0u;
      if (tid == 0) defer(L, ii, j);
      __syncthreads();
      continue;
    }
    // a set holding the skipped vertex is counted but not copied (its bit,
    // read before the bitmap is cleared)
    if (tid == 0) {
      const bool sk = V.skip != kNoSkip && ((bm[V.skip >> 5] >> (V.skip & 31u)) & 1u);
      s_base = sk ? kSkipped : atomicAdd(&L.inst[ii].store_tail, (unsigned long long)size);
    }
    __syncthreads();
    const unsigned long long base = s_base;
    const bool skipped = base == kSkipped;
    const bool fits = skipped || base + size <= V.store_cap;
    for (uint32_t i = tid; i < size; i += kBigBlock) {
      const uint32_t x = q[i];
      if (fits) {
        if (!skipped) V.members[base + i] = V.moff + x;
        atomicAdd(&V.cnt[V.moff + x], 1u);
      }
      bm[x >> 5] = 0u;
    }
    if (tid == 0) {
      if (fits) {
        V.rr_start[j] = base;
        V.rr_len[j] = size;
        if (!skipped) atomicAdd(&L.inst[ii].members_added, (unsigned long long)size);
      } else {
        defer(L, ii, j);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// LT walk.
// ---------------------------------------------------------------------------

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

// The in-edge an equal-weight row [s, e) (d = e - s in-edges, common fp32
// weight wbits) chooses for the draw U: the first i with U < T(i), or d for
// none. For such a row the LT preparation stores the exact integer
// thresholds T(i) = round_half_up((i+1)·M·2^(E+32)), clamped to 2^32 (weight
// M·2^E), except that the last becomes 2^32 when the row's total is within
// 1e-6 of 1. So the walk computes them from the weight instead of loading
// them: it starts from the fp32 guess floor(U / (w·2^32)), moves to the
// first threshold above U, and reads the stored last threshold only when it
// reaches the row's end. Returns ~0u when the guess does not settle within a
// few steps, or when the prefix sums would leave the exact range (rows of
// 2^29 in-edges or more); the caller then searches the stored thresholds.
__device__ __forceinline__ uint32_t lt_equal_pick(uint32_t wbits, uint32_t s, uint32_t e, uint32_t U,
                                                  const uint64_t *__restrict__ cum) {
  const uint32_t d = e - s;
  uint32_t mant;
  const int ex = ulp_exponent(__uint_as_float(wbits), &mant);
  if (mant == 0u) return d;                       // zero weights: no in-edge is ever chosen
  if ((unsigned long long)d * mant >= (1ull << 53)) return ~0u;
  const int k = ex + 32;
  const float w = __uint_as_float(wbits);
  float gf = floorf(__uint2float_rn(U) * __frcp_rn(w * 4294967296.0f));
  if (!(gf < (float)(d - 1))) gf = (float)(d - 1);
  uint32_t g = gf > 0.0f ? (uint32_t)gf : 0u;
  const unsigned long long u64 = U;
  // T(g - 1) = lt_round_int(g·M, k), T(g) = lt_round_int((g+1)·M, k)
  for (int it = 0; it < 8 && g > 0 && u64 < lt_round_int((unsigned long long)g * mant, k); ++it) --g;
  for (int it = 0; it < 8 && g + 1 < d && u64 >= lt_round_int((unsigned long long)(g + 1) * mant, k); ++it) ++g;
  if ((g > 0 && u64 < lt_round_int((unsigned long long)g * mant, k)) ||
      (g + 1 < d && u64 >= lt_round_int((unsigned long long)(g + 1) * mant, k)))
    return ~0u;
  if (g + 1 < d) return g;                        // T(g - 1) <= U < T(g)
  return u64 < cum[e - 1] ? g : d;                // the last threshold may be raised to 2^32
}

// The in-edge LT chooses at row [s, e) for the draw U: its index, or e for
// none (the first a with U < cum[a]; Sec. III-G), and in u its source.
// When every in-edge of the row has the same weight w (rw != kPerEdge) the
// prefix sums are i·w exactly, so the answer lies within one index of
// floor(U / (w·2^32)): the warp loads the 32 thresholds and sources around
// that guess in one round trip and takes the first threshold above U. The
// window settles the answer unless it starts past s with its first
// threshold already above U, or ends before e with none above U; then (and
// for rows of unequal weights) the 33-way search of lt_pick decides.
__device__ __forceinline__ uint32_t lt_choose(const uint64_t *__restrict__ cum, const uint32_t *__restrict__ src,
                                              uint32_t s, uint32_t e, uint32_t wbits, uint32_t U, uint32_t &u) {
  if (wbits != kPerEdge) {
    const uint32_t i = lt_equal_pick(wbits, s, e, U, cum);   // warp-uniform
    if (i != ~0u) {
      if (i < e - s) u = src[s + i];
      return s + i;
    }
  }
  const uint32_t a = lt_pick(cum, s, e, U);
  if (a < e) u = src[a];
  return a;
}

// LT large pass: one warp per block and walk, with the slot's bitmap as the
// visited set and its queue as the path (walks the common pass deferred).
__global__ void __launch_bounds__(32) lt_large_kernel(SampleLaunch L, BigScratch bs) {
  const uint32_t lane = lane_id();
  const uint32_t cap = bs.q_cap;
  uint32_t *bm = bs.bitmap + (uint64_t)blockIdx.x * bs.words_per_slot;
  uint32_t *path = bs.queue + (uint64_t)blockIdx.x * bs.q_cap;

  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(&L.ctl->next, 1ull);
    item = __shfl_sync(kFullMask, item, 0);
    if (item >= L.total_items) break;
    uint32_t ii = 0;
    uint64_t j = 0;
    if (lane == 0) decode_item(L, item, ii, j);
    ii = __shfl_sync(kFullMask, ii, 0);
    j = __shfl_sync(kFullMask, j, 0);
    const InstView V = view_of(L.inst[ii]);
    const uint32_t *__restrict__ off = V.off;
    const uint64_t *__restrict__ cum = V.cum;
    const uint32_t *__restrict__ src = V.src;
    const uint32_t *__restrict__ rw = V.rw;
    const PhiloxKey key = V.key;
    const uint32_t jlo = id_lo(V, j), jhi = V.jhi;
    uint32_t x = draw_root(key, id_lo(V, j), V.rhi, V.n);
    uint32_t len = 1;
    const uint32_t slot = L.item_slots ? L.item_slots[item] : kNoSlot;
    if (slot < L.lt_ovf_cap && cap >= kLtGroupPath) {
      // continue a walk from the kLtGroupPath vertices it had reached (the
      // walk is a function of the vertex sequence, so it resumes exactly)
      const uint32_t *saved = L.lt_ovf + (uint64_t)slot * kLtGroupPath;
      for (uint32_t i = lane; i < kLtGroupPath; i += 32) {
        const uint32_t p = saved[i];
        path[i] = p;
        atomicOr(&bm[p >> 5], 1u << (p & 31u));
      }
      len = kLtGroupPath;
      x = saved[kLtGroupPath - 1];
    } else if (lane == 0) {
      path[0] = x;
      bm[x >> 5] = 1u << (x & 31u);
    }
    __syncwarp();
    bool overflow = false;
    for (;;) {
      const uint32_t s = off[x], e = off[x + 1], wb = rw[x];
      const uint32_t U = philox10(x, kTagStep, jlo, jhi, key).x;
      if (e == s) break;
      uint32_t u = 0;
      const uint32_t a = lt_choose(cum, src, s, e, wb, U, u);
      if (a >= e) break;
      uint32_t old = 0;
      if (lane == 0) old = atomicOr(&bm[u >> 5], 1u << (u & 31u));
      const bool seen = (__shfl_sync(kFullMask, old, 0) >> (u & 31u)) & 1u;
      if (seen) break;
      if (len == cap) {
        overflow = true;
        if (lane == 0) atomicAnd(&bm[u >> 5], ~(1u << (u & 31u)));
        break;
      }
      if (lane == 0) path[len] = u;
      ++len;
      __syncwarp();
      x = u;
    }
    if (overflow) {
      for (uint32_t i = lane; i < len; i += 32) bm[path[i] >> 5] = 0u;
      __syncwarp();
      if (lane == 0) defer(L, ii, j);
      continue;
    }
    commit_warp(L, V, ii, j, path, len, bm);
    __syncwarp();
  }
}

// LT common pass: four walks per warp, eight lanes each. A walk's step is
// a chain of dependent loads (the row, then the thresholds around the
// draw, then the source), so a warp keeps four chains in flight. Each group
// of eight lanes owns one walk and its path (kLtGroupPath entries in shared
// memory): the row's window of eight thresholds and sources (or an 9-way
// search for rows of unequal weights), the visited test against the path
// eight entries at a time, the commit of the finished path. Every warp-wide
// primitive runs in code all 32 lanes reach, each group using its own byte of
// a ballot; a group whose walk ended takes the next work item. Walks longer
// than the path buffer are handed to the large pass.
constexpr uint32_t kLtLanes = 8;
constexpr uint32_t kLtWalks = 32 / kLtLanes;
constexpr uint32_t kLtMultiWarps = 8;   // warps per block

__global__ void __launch_bounds__(32 * kLtMultiWarps) lt_multi_kernel(SampleLaunch L) {
  extern __shared__ uint32_t smem[];
  const uint32_t lane = lane_id();
  const uint32_t grp = lane / kLtLanes, gl = lane % kLtLanes, lead = grp * kLtLanes;
  uint32_t *path = smem + ((threadIdx.x >> 5) * kLtWalks + grp) * kLtGroupPath;

  // this group's walk (the same values in all eight lanes)
  bool active = false, done = false;
  uint32_t ii = 0, x = 0, len = 0;
  uint64_t j = 0;
  InstView V{};
  for (;;) {
    // groups without a walk take the next item
    unsigned long long item = ~0ull;
    if (!active && !done && gl == 0) item = atomicAdd(&L.ctl->next, 1ull);
    item = __shfl_sync(kFullMask, item, lead);
    if (!active && !done) {
      if (item >= L.total_items) {
        done = true;
      } else {
        decode_item(L, item, ii, j);
        V = view_of(L.inst[ii]);
        x = draw_root(V.key, id_lo(V, j), V.rhi, V.n);
        if (gl == 0) path[0] = x;
        len = 1;
        active = true;
      }
    }
    __syncwarp();
    if (__ballot_sync(kFullMask, active) == 0u) break;   // every group is done

    // one step of every active walk
    bool ended = false, overflow = false;
    uint32_t u = 0, s = 0, e = 0, wb = kPerEdge, U = 0;
    if (active) {
      s = V.off[x];
      e = V.off[x + 1];
      wb = V.rw[x];
      U = philox10(x, kTagStep, id_lo(V, j), V.jhi, V.key).x;
      if (e == s) ended = true;
    }
    // rows of equal weights: the chosen in-edge from the computed thresholds,
    // then only its source is read (all eight lanes load the same word)
    bool need = active && !ended;          // still looking for the chosen edge
    if (need && wb != kPerEdge) {
      const uint32_t i = lt_equal_pick(wb, s, e, U, V.cum);
      if (i != ~0u) {
        need = false;
        if (i < e - s)
          u = V.src[s + i];
        else
          ended = true;                     // no edge chosen
      }
    }
    // otherwise a 9-way search: the answer lies in [lo, hi], hi = e meaning
    // no edge; narrowing stops at eight candidates lo..hi, all probed
    uint32_t lo = s, hi = e;
    while (__ballot_sync(kFullMask, need) != 0u) {
      uint32_t p = 0;
      bool probe = false;
      if (need) {
        if (hi - lo >= kLtLanes) {
          p = lo + (uint32_t)(((uint64_t)(hi - lo) * (gl + 1)) / (kLtLanes + 1));   // < hi
          probe = true;
        } else {
          p = lo + gl;
          probe = p <= hi && p < e;
        }
      }
      const bool hit = probe && (uint64_t)U < V.cum[p];
      const uint32_t sp = probe ? V.src[p] : 0u;
      const uint32_t b = (__ballot_sync(kFullMask, hit) >> lead) & 0xFFu;
      const uint32_t f = b ? (uint32_t)(__ffs(b) - 1) : 0u;
      const uint32_t pf = __shfl_sync(kFullMask, p, lead + f);
      const uint32_t pb = __shfl_sync(kFullMask, p, lead + (f > 0 ? f - 1 : 0));
      const uint32_t plast = __shfl_sync(kFullMask, p, lead + kLtLanes - 1);
      const uint32_t us = __shfl_sync(kFullMask, sp, lead + f);
      if (need) {
        if (hi - lo >= kLtLanes) {
          if (b == 0u) {
            lo = plast + 1;
          } else {
            hi = pf;
            if (f > 0) lo = pb + 1;
          }
        } else {
          // hi < e has a threshold above U, so no hit among lo..hi means hi = e
          if (b != 0u)
            u = us;
          else
            ended = true;                   // U above every threshold of the row
          need = false;
        }
      }
    }
    // visited test against the path, eight entries at a time
    bool seen = false;
    {
      const uint32_t mine = (active && !ended) ? len : 0u;
      uint32_t top = mine;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) top = max(top, __shfl_xor_sync(kFullMask, top, o));
      for (uint32_t i0 = 0; i0 < top; i0 += kLtLanes) {
        const uint32_t i = i0 + gl;
        const bool hit = i < mine && path[i] == u;
        seen |= ((__ballot_sync(kFullMask, hit) >> lead) & 0xFFu) != 0u;
      }
    }
    if (active && !ended) {
      if (seen) {
        ended = true;
      } else if (len == kLtGroupPath) {
        ended = true;
        overflow = true;
      } else {
        if (gl == 0) path[len] = u;
        ++len;
        x = u;
      }
    }
    __syncwarp();
    // commit the walks that ended
    const bool commit = active && ended && !overflow;
    // a walk through the skipped vertex is counted but not copied
    bool sk = false;
    {
      const uint32_t mine = (commit && V.skip != kNoSkip) ? len : 0u;
      uint32_t top = mine;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) top = max(top, __shfl_xor_sync(kFullMask, top, o));
      for (uint32_t i0 = 0; i0 < top; i0 += kLtLanes) {
        const uint32_t i = i0 + gl;
        const bool hit = i < mine && path[i] == V.skip;
        sk |= ((__ballot_sync(kFullMask, hit) >> lead) & 0xFFu) != 0u;
      }
    }
    unsigned long long base = 0;
    if (commit && gl == 0) base = sk ? kSkipped : atomicAdd(&L.inst[ii].store_tail, (unsigned long long)len);
    base = __shfl_sync(kFullMask, base, lead);
    if (commit) {
      const bool fits = sk || base + len <= V.store_cap;
      if (fits)
        for (uint32_t i = gl; i < len; i += kLtLanes) {
          const uint32_t m = V.moff + path[i];
          if (!sk) V.members[base + i] = m;
          atomicAdd(&V.cnt[m], 1u);
        }
      if (gl == 0) {
        if (fits) {
          V.rr_start[j] = base;
          V.rr_len[j] = len;
          if (!sk) atomicAdd(&L.inst[ii].members_added, (unsigned long long)len);
        } else {
          defer(L, ii, j);
        }
      }
    }
    if (active && overflow) {
      // save the path so that the large pass continues the walk
      uint32_t slot = kNoSlot;
      if (gl == 0 && L.lt_ovf) {
        slot = atomicAdd(L.lt_ovf_next, 1u);
        if (slot >= L.lt_ovf_cap) slot = kNoSlot;
      }
      slot = __shfl_sync(0xFFu << lead, slot, lead);
      if (slot != kNoSlot)
        for (uint32_t i = gl; i < kLtGroupPath; i += kLtLanes) L.lt_ovf[(uint64_t)slot * kLtGroupPath + i] = path[i];
      if (gl == 0) defer(L, ii, j, slot);
    }
    if (active && ended) active = false;
    __syncwarp();
  }
}

// Rollback helper: lowers the occurrence counts of the sets of a launch's
// items that were stored (rr_start != kNoStart).
__global__ void uncount_kernel(SampleLaunch L) {
  const uint32_t lane = lane_id();
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t item = warp; item < L.total_items; item += nwarps) {
    uint32_t ii;
    uint64_t j;
    decode_item(L, item, ii, j);
    const InstDesc &D = L.inst[ii];
    const uint64_t b = D.rr_start[j];
    if (b == kNoStart) continue;
    if (b == kSkipped) {   // its members are not kept: the host empties the collection instead
      if (lane == 0) atomicOr(&L.ctl->err, kErrUncountSkipped);
      continue;
    }
    const uint32_t len = D.rr_len[j];
    for (uint32_t t = lane; t < len; t += 32) atomicSub(&D.cnt[D.members[b + t]], 1u);
  }
}

// Pure Philox4x32-10 throughput: each thread draws `per_thread` blocks on
// consecutive counters of one RR set (the IC coin counter layout, computed
// as the sampler does: coin_key once, coin_words per group) and folds the
// words so that nothing is optimised away. Measures the ALU ceiling of the
// coin work.
__global__ void __launch_bounds__(256) philox_rate_kernel(PhiloxKey key, uint32_t per_thread, uint32_t *sink) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  const CoinKey ck = coin_key(0x1234u, 0u, key);
  uint32_t acc = 0;
  for (uint32_t i = 0; i < per_thread; i += 2) {
    const uint32_t c = t * per_thread + i;
    const uint4 a = coin_words(c, ck);
    const uint4 b = coin_words(c + 1, ck);
    acc += (a.x ^ a.y ^ a.z ^ a.w) + (b.x ^ b.y ^ b.z ^ b.w);
  }
  if (acc == 0x9E3779B9u) sink[t & 1023] = acc;   // practically never stored
}

}  // namespace

int ic_common_blocks_per_sm() {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ic_common_kernel<false>, 256, 0) != cudaSuccess) b = 4;
  return b > 0 ? b : 1;
}

int lt_common_blocks_per_sm() {
  int b = 0;
  const size_t sm = kLtMultiWarps * kLtWalks * kLtGroupPath * sizeof(uint32_t);
  // more than 48 KB of dynamic shared memory must be allowed (per device)
  if (cudaFuncSetAttribute(lt_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
    cudaGetLastError();
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, lt_multi_kernel, 32 * kLtMultiWarps, sm) != cudaSuccess) {
    cudaGetLastError();
    b = 2;
  }
  return b > 0 ? b : 1;
}

cudaError_t launch_ic_common(const SampleLaunch &L, const CommonScratch &cs, const InstDesc *one, cudaStream_t s) {
  if (one)
    ic_common_kernel<true><<<(cs.workers + 7) / 8, 256, 0, s>>>(L, cs, *one);
  else
    ic_common_kernel<false><<<(cs.workers + 7) / 8, 256, 0, s>>>(L, cs, InstDesc{});
  return cudaGetLastError();
}

cudaError_t launch_ic_block(const SampleLaunch &L, const BigScratch &bs, uint32_t grid, const InstDesc *one,
                            cudaStream_t s) {
  if (one)
    ic_block_kernel<true><<<grid, kBigBlock, 0, s>>>(L, bs, *one);
  else
    ic_block_kernel<false><<<grid, kBigBlock, 0, s>>>(L, bs, InstDesc{});
  return cudaGetLastError();
}

cudaError_t launch_lt_common(const SampleLaunch &L, uint32_t grid, cudaStream_t s) {
  lt_multi_kernel<<<grid, 32 * kLtMultiWarps, kLtMultiWarps * kLtWalks * kLtGroupPath * sizeof(uint32_t), s>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_lt_large(const SampleLaunch &L, const BigScratch &bs, uint32_t grid, cudaStream_t s) {
  lt_large_kernel<<<grid, 32, 0, s>>>(L, bs);
  return cudaGetLastError();
}

cudaError_t launch_uncount(const SampleLaunch &L, cudaStream_t s) {
  if (L.total_items == 0) return cudaSuccess;
  uint64_t blocks = (L.total_items + 7) / 8;
  if (blocks > 4096) blocks = 4096;
  uncount_kernel<<<(unsigned)blocks, 256, 0, s>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_philox_rate(int blocks, uint32_t per_thread, uint32_t *sink, cudaStream_t s) {
  philox_rate_kernel<<<blocks, 256, 0, s>>>(PhiloxKey{0x01234567u, 0x89ABCDEFu}, per_thread, sink);
  return cudaGetLastError();
}

}  // namespace gim
