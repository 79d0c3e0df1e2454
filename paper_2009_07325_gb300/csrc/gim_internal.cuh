// Internal declarations of libgim: context layout, device-side Philox, and
// the kernels' host launchers. Nothing here is part of the public C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "gim.h"

namespace gim {

constexpr uint32_t kFullMask = 0xFFFFFFFFu;
constexpr uint64_t kNoStart = ~0ull;          // rr_start of a set not (yet) stored
constexpr uint64_t kSkipped = ~0ull - 1;      // rr_start of a set holding the skipped vertex: counted, members not kept
constexpr uint32_t kNoSkip = 0xFFFFFFFFu;     // no skipped vertex

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). Counter words are
// (idx, tag, j_lo, j_hi); the key is the 64-bit seed split into two words.
// ---------------------------------------------------------------------------
struct PhiloxKey {
  uint32_t k0, k1;
};

__host__ __device__ __forceinline__ uint4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, PhiloxKey key) {
  uint32_t k0 = key.k0, k1 = key.k1;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    // one 32x32 -> 64-bit product per multiplier gives both halves
    const unsigned long long a = (unsigned long long)0xD2511F53u * c0;
    const unsigned long long b = (unsigned long long)0xCD9E8D57u * c2;
    const uint32_t y0 = (uint32_t)(b >> 32) ^ c1 ^ k0;
    const uint32_t y2 = (uint32_t)(a >> 32) ^ c3 ^ k1;
    c0 = y0;
    c1 = (uint32_t)b;
    c2 = y2;
    c3 = (uint32_t)a;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return make_uint4(c0, c1, c2, c3);
}

enum : uint32_t { kTagRoot = 0, kTagEdge = 1, kTagStep = 2 };

// The IC coin words of in-edge group g in RR set j are
// philox10(g, kTagEdge, j_lo, j_hi, key). Three of the four counter words
// are fixed for the whole set, so everything of rounds 1 and 2 that does not
// depend on g is computed once per set (coin_key) and a group costs one
// 32x32 multiply in each of those rounds instead of two. coin_words(g, ck)
// equals philox10(g, kTagEdge, j_lo, j_hi, key) bit for bit.
struct CoinKey {
  uint32_t c, d, e, f;   // round-1 c2 mask, round-2 c0 mask, round-2 c2 mask, round-2 c3
  PhiloxKey k2;          // the key after two rounds
};

__host__ __device__ __forceinline__ CoinKey coin_key(uint32_t jlo, uint32_t jhi, PhiloxKey key) {
  const unsigned long long b1 = (unsigned long long)0xCD9E8D57u * jlo;
  const uint32_t c0r1 = (uint32_t)(b1 >> 32) ^ kTagEdge ^ key.k0;   // c0 after round 1
  const uint32_t c1r1 = (uint32_t)b1;                               // c1 after round 1
  const uint32_t k0b = key.k0 + 0x9E3779B9u, k1b = key.k1 + 0xBB67AE85u;
  const unsigned long long a2 = (unsigned long long)0xD2511F53u * c0r1;
  CoinKey ck;
  ck.c = jhi ^ key.k1;
  ck.d = c1r1 ^ k0b;
  ck.e = (uint32_t)(a2 >> 32) ^ k1b;
  ck.f = (uint32_t)a2;
  ck.k2.k0 = k0b + 0x9E3779B9u;
  ck.k2.k1 = k1b + 0xBB67AE85u;
  return ck;
}

__host__ __device__ __forceinline__ uint4 coin_words(uint32_t g, const CoinKey &ck) {
  const unsigned long long a1 = (unsigned long long)0xD2511F53u * g;   // round 1: only c0 varies
  const uint32_t c2r1 = (uint32_t)(a1 >> 32) ^ ck.c;
  const unsigned long long b2 = (unsigned long long)0xCD9E8D57u * c2r1;   // round 2: only c2 varies
  uint32_t c0 = (uint32_t)(b2 >> 32) ^ ck.d;
  uint32_t c1 = (uint32_t)b2;
  uint32_t c2 = (uint32_t)a1 ^ ck.e;
  uint32_t c3 = ck.f;
  uint32_t k0 = ck.k2.k0, k1 = ck.k2.k1;
#pragma unroll
  for (int r = 2; r < 10; ++r) {
    const unsigned long long a = (unsigned long long)0xD2511F53u * c0;
    const unsigned long long b = (unsigned long long)0xCD9E8D57u * c2;
    const uint32_t y0 = (uint32_t)(b >> 32) ^ c1 ^ k0;
    const uint32_t y2 = (uint32_t)(a >> 32) ^ c3 ^ k1;
    c0 = y0;
    c1 = (uint32_t)b;
    c2 = y2;
    c3 = (uint32_t)a;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return make_uint4(c0, c1, c2, c3);
}

// randSelect(V) of Alg. 3: the root of the RR set with rr_id (jhi:jlo), high
// word of a 64-bit draw times n.
__device__ __forceinline__ uint32_t draw_root(PhiloxKey key, uint32_t jlo, uint32_t jhi, uint32_t n) {
  const uint4 r = philox10(0u, kTagRoot, jlo, jhi, key);
  const uint64_t w = ((uint64_t)r.y << 32) | r.x;
  return (uint32_t)__umul64hi(w, (uint64_t)n);
}

// ---------------------------------------------------------------------------
// LT thresholds in exact integer arithmetic (graph preparation and the walk).
// ---------------------------------------------------------------------------
// fp32 weight w = M * 2^E exactly (M < 2^24); returns E, or INT_MAX for w = 0.
__device__ __forceinline__ int ulp_exponent(float w, uint32_t *mant) {
  const uint32_t b = __float_as_uint(w);
  const uint32_t ef = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
  if (ef == 0 && m == 0) {
    *mant = 0;
    return 0x7FFFFFFF;
  }
  *mant = ef ? (m | 0x800000u) : m;
  return ef ? (int)ef - 150 : -149;
}

// round_half_up(Q * 2^k), clamped to 2^32, for Q < 2^53.
__device__ __forceinline__ unsigned long long lt_round_int(unsigned long long Q, int k) {
  unsigned long long c;
  if (k >= 0)
    c = Q << k;                                   // k <= 9 for weights <= 1: no overflow
  else if (k < -60)
    c = 0ull;                                     // Q * 2^k < 2^-7
  else
    c = (Q + (1ull << (-k - 1))) >> (-k);
  return c > 4294967296ull ? 4294967296ull : c;
}

// ---------------------------------------------------------------------------
// Device-resident graph (in-edge CSR by target).
// ---------------------------------------------------------------------------
struct DevGraph {
  uint32_t n = 0;
  uint64_t m = 0;
  uint32_t *off = nullptr;   // n+1
  uint32_t *src = nullptr;   // m rounded up to a multiple of 4, zero padded
  uint32_t *thr = nullptr;   // same length: IC coin threshold ceil(w * 2^24)
  uint32_t *rthr = nullptr;  // n: the row's common threshold when all its in-edges share one, else kPerEdge
  uint64_t *cum = nullptr;   // m: LT cumulative thresholds in 2^-32 units (built on the first LT use)
  float *w = nullptr;        // m: the fp32 weights as loaded (the LT thresholds are built from them)
  uint32_t *rw = nullptr;    // n: fp32 bits of the row's common weight when all its in-edges share one, else kPerEdge
  uint64_t *off64 = nullptr; // n+1: the offsets as uploaded (validated and narrowed on the device)
  uint32_t n_cap = 0;        // the arrays hold graphs of up to n_cap vertices and m_cap (padded) edges
  uint64_t m_cap = 0;
};

constexpr uint32_t kPerEdge = 0xFFFFFFFFu;   // rthr value of a row whose thresholds differ

// Output side of a sampling launch.
struct DevStore {
  uint32_t *members = nullptr;   // store_cap entries
  uint64_t cap = 0;
  uint64_t *rr_start = nullptr;  // by rr_id
  uint32_t *rr_len = nullptr;    // by rr_id
  uint32_t *cnt = nullptr;       // n occurrence counts (Occur)
};

// One instance of a sampling launch: a graph, an RR collection and the ids
// to draw. The kernels read these from a device array, so one launch can
// serve many IMM instances (a single-instance call is a batch of one).
struct InstDesc {
  // graph
  uint32_t n;
  uint32_t jhi;   // high word of every rr_id of this job: 0, or 2^31 for a fresh final phase (rr_ids 2^63 + j)
  const uint32_t *off, *src, *thr, *rthr, *rw;
  const uint64_t *cum;
  // RR collection
  uint32_t *members;
  unsigned long long store_cap;
  uint64_t *rr_start;
  uint32_t *rr_len;
  uint32_t *cnt;
  // job: global items [item_begin, item_begin + count) are positions j_begin ...
  // The set at position j has rr_id (jhi : j + idoff); its root is drawn with
  // the high word rhi (= jhi except for a multi-round set's later rounds,
  // which share round 0's root), and its members are stored as moff + v.
  PhiloxKey key;
  unsigned long long j_begin;
  unsigned long long item_begin;
  uint32_t rhi;
  uint32_t moff;
  uint32_t idoff;
  uint32_t skip;   // a set holding this vertex keeps only its size (rr_start = kSkipped); kNoSkip: none
  // written by the kernels
  unsigned long long store_tail;     // store entries reserved (starts at the entries already used)
  unsigned long long members_added;  // members of the sets stored by this launch
};

// Device counters of one sampling launch.
struct SampleCtl {
  unsigned long long next;        // next work item
  unsigned long long n_deferred;  // sets handed to the next pass
  unsigned int err;               // error bits (kErr*)
  unsigned int pad;
};

enum : unsigned int { kErrDeferredFull = 1u, kErrUncountSkipped = 2u };

// A sampling launch: the instances, the work items and where to defer.
struct SampleLaunch {
  InstDesc *inst;
  uint32_t n_inst;
  unsigned long long total_items;
  const unsigned long long *items;   // nullable: item i is (instance << 32 | rr_id) = items[i]
  unsigned long long *deferred;      // deferred sets, packed like items
  unsigned long long deferred_cap;
  SampleCtl *ctl;
  uint32_t group_budget;             // common pass: edge groups (4 in-edges) a set may scan
  uint32_t queue_cap;                // common pass: members a set may reach (<= kQueueCap)
  uint32_t batch;                    // block pass: frontier vertices per block step (<= kBigBlock)
  uint32_t chunk_groups;             // block pass: groups per chunk (a multiple of 64)
  // LT walks that outgrow the common pass's path keep it in an overflow slot
  // (kLtGroupPath entries) so that the large pass continues them instead of
  // starting over: items[i] / deferred[d] have slot item_slots[i] /
  // deferred_slots[d] (kNoSlot: none)
  const uint32_t *item_slots;        // nullable
  uint32_t *deferred_slots;          // nullable
  uint32_t *lt_ovf;                  // lt_ovf_cap slots of kLtGroupPath vertices
  unsigned int *lt_ovf_next;         // slots handed out in this sampling call (LT or IC: one model per launch)
  uint32_t lt_ovf_cap;
  // IC sets the warp-per-set pass hands on past their budget keep their
  // state in a slot of kIcOvfStride words (members so far, rows expanded,
  // then the members), so the block-per-set pass continues them
  uint32_t *ic_ovf;                  // ic_ovf_cap slots
  uint32_t ic_ovf_cap;
};
constexpr uint32_t kNoSlot = 0xFFFFFFFFu;
constexpr uint32_t kLtGroupPath = 384;     // LT common pass: path entries per walk (shared memory)
constexpr uint32_t kLtOvfSlots = 16384;     // LT walks continued from a saved path per sampling call

constexpr uint32_t kQueueCap = 4096;        // common pass: members per set before it is deferred
constexpr uint32_t kIcOvfStride = kQueueCap + 2;   // an IC overflow slot: tail, head, then the queue
constexpr uint32_t kIcOvfSlots = 65536;       // IC sets continued from a saved state per sampling pass
constexpr uint32_t kHashBits = 13;
constexpr uint32_t kHashSlots = 1u << kHashBits;   // common pass: visited hash slots per worker

// Scratch of the common (warp per set) IC pass; independent of n.
struct CommonScratch {
  uint32_t *queue = nullptr;              // kQueueCap per worker
  unsigned long long *hash = nullptr;     // kHashSlots per worker: epoch << 32 | vertex
  uint32_t *epoch = nullptr;              // per worker
  uint32_t workers = 0;
};

// Scratch of the large-set passes: per slot an n-bit visited bitmap (all zero
// between sets) and a queue: min(n, kSlotQueue) entries in the first pass,
// n entries in later ones. IC uses one kBigBlock-thread block per slot,
// LT one warp per slot.
struct BigScratch {
  uint32_t *bitmap = nullptr;
  uint32_t *queue = nullptr;
  uint64_t words_per_slot = 0;
  uint32_t n_cap = 0;                  // vertices the bitmaps cover
  uint32_t q_cap = 0;                  // queue entries per slot (a set outgrowing them is handed on)
  uint32_t slots = 0;
};
constexpr uint32_t kSlotQueue = 1u << 20;   // queue entries per slot in the first large-set pass

// Four warps per heavy set and 16 sets per SM: a heavy set's levels are short
// (critical branching), so fewer warps per set wait less at its barriers
// (128 threads: 36.8-37.0 ms per headline IMM; 192 x 10: 37.0; 256 x 8: 38.0-38.3;
// 96 x 21: 37.8; 64 x 32: 40.5-40.6)
constexpr int kBigBlock = 128;
constexpr int kBigBlocksPerSM = 16;   // block-per-set pass: blocks (slots) per SM, 32 registers per thread

// Host launchers (sample.cu).
// `one` (nullable): the launch's only instance, passed by value so that the
// kernel reads its fields from kernel parameters.
cudaError_t launch_ic_common(const SampleLaunch &L, const CommonScratch &cs, const InstDesc *one, cudaStream_t s);
cudaError_t launch_ic_block(const SampleLaunch &L, const BigScratch &bs, uint32_t grid, const InstDesc *one,
                            cudaStream_t s);
cudaError_t launch_lt_common(const SampleLaunch &L, uint32_t grid, cudaStream_t s);
cudaError_t launch_lt_large(const SampleLaunch &L, const BigScratch &bs, uint32_t grid, cudaStream_t s);
cudaError_t launch_uncount(const SampleLaunch &L, cudaStream_t s);
cudaError_t launch_philox_rate(int blocks, uint32_t per_thread, uint32_t *sink, cudaStream_t s);
int ic_common_blocks_per_sm();
int lt_common_blocks_per_sm();

// Graph preprocessing (graph.cu).
// Offsets: info[0] |= kGraphBadOffsets and info[1] = the first row whose
// offsets decrease (info[1] must start at ~0u), info[2] = the largest
// in-degree; g.off gets the offsets narrowed to 32 bits.
cudaError_t launch_offsets_prep(DevGraph &g, unsigned int *info, cudaStream_t s);
// IC thresholds and row checks; d_flags[0] collects kGraph* flags and
// d_flags[3] (zero on entry) counts the rows listed for the warp pass.
cudaError_t launch_graph_prep(DevGraph &g, unsigned int *d_flags, cudaStream_t s);
// The LT thresholds g.cum (allocated by the caller) from g.w; kGraphNotLT in *d_flags if a row sums above 1.
cudaError_t launch_lt_prep(DevGraph &g, unsigned int *d_flags, cudaStream_t s);
enum : unsigned int {
  kGraphBadSource = 1u, kGraphNotAscending = 2u, kGraphBadWeight = 4u, kGraphNotLT = 8u, kGraphBadOffsets = 16u
};

// Selection buffers of one instance (grown on demand, kept between calls).
// Vertices that lie in many RR sets ("hubs": count >= a threshold chosen per
// selection) get a bitmap over the sets instead of an inverted list, and
// their counts live in a short array; the others ("light" vertices) get
// inverted lists (batch.cu, greedy.cu).
constexpr uint32_t kHeavyCap = 255;     // hubs per selection at most (slot ids fit a byte; 0xFF = light)
struct SelectBuffers {
  uint32_t *cnt_work = nullptr;  // n: light count + 1 while unselected, 0 once selected or a hub
  uint64_t *inv_off = nullptr;   // n+1
  unsigned long long *cursor = nullptr;   // n: the next free position of each light vertex's list in inv
  uint32_t *inv = nullptr;       // Z rr ids
  uint32_t *covered = nullptr;   // ceil(R/32) words: bit j set once RR set j is covered
  unsigned long long *best = nullptr;   // k argmax keys
  uint32_t *seeds = nullptr;     // k
  uint32_t *gains = nullptr;     // k
  unsigned long long *covered_total = nullptr;
  uint64_t *scan_tmp = nullptr;  // block partial sums
  uint32_t *cnt_own = nullptr;   // n: counts over a prefix of a shared store (serving)
  uint8_t *hslot = nullptr;      // n: hub slot of a vertex, 0xFF if light
  uint32_t *hbits = nullptr;     // kHeavyCap rows of ceil(R/32) words: bit j of row s = set j holds hub s
  uint32_t *hmeta = nullptr;     // 1 + 2 kHeavyCap: hub count, hub ids, hub counts + 1 (0 once selected)
  uint64_t n_cap = 0, z_cap = 0, r_cap = 0, k_cap = 0, scan_cap = 0, hb_cap = 0;
};

// Frees every buffer of b and resets it (api.cu).
void free_select_buffers(SelectBuffers &b);

// The k greedy rounds of one instance in the persistent greedy kernel
// (greedy.cu). Blocks [g_begin, g_begin + g_blocks) of the launch serve it.
struct GreedyDesc {
  uint32_t n = 0, k = 0;                 // k = 0: nothing to select
  uint32_t g_begin = 0, g_blocks = 0;
  uint32_t words = 0;                    // ceil(R/32): covered bitmap words, hub row words read
  uint32_t row_words = 0;                // hub row stride (the index's own ceil(R/32))
  uint32_t R = 0;                        // sets selected over: list entries >= R are skipped
  uint32_t *cnt_work = nullptr;          // n: light count + 1 while unselected, else 0
  const uint64_t *inv_off = nullptr;     // n + 1 (hubs have empty lists)
  const uint32_t *inv = nullptr;         // rr ids per light vertex
  uint32_t *covered = nullptr;           // words, zero on entry
  const uint8_t *hslot = nullptr;        // n: hub slot or 0xFF
  const uint32_t *hbits = nullptr;       // hub rows
  uint32_t *hmeta = nullptr;             // hub count, ids, counts + 1
  const uint32_t *members = nullptr;
  const uint64_t *rr_start = nullptr;
  const uint32_t *rr_len = nullptr;
  unsigned long long *best = nullptr;    // k argmax keys, zero on entry
  uint32_t *seeds = nullptr;             // k
  uint32_t *gains = nullptr;             // k
  unsigned long long *covered_total = nullptr;   // zero on entry
  unsigned long long *stats = nullptr;   // 2, zero on entry: members of newly covered sets, seed list/row words
  unsigned int *bar = nullptr;           // group barrier counter, zero on entry
  // first pick taken by the index fill (fuse = 1): round 0's seed, gain and
  // covered sets are already recorded, light lists hold only the sets left
  // uncovered and end at inv_end[x]; the launch starts at round 1
  uint32_t fuse = 0;
  const unsigned long long *inv_end = nullptr;   // n: end of each light list (null: inv_off[x + 1])
  // multi-round IM: elements x in [r * part_n, (r + 1) * part_n) belong to
  // round r, and at most part_k seeds are taken per round (part_n = 0: no
  // partition). k is then part_k times the number of rounds.
  uint32_t part_n = 0, part_k = 0;
};
constexpr int kGreedyThreads = 512;
constexpr uint32_t kMaxRounds = 32;      // rounds of a multi-round collection (one bit each in the greedy)
// Blocks one cooperative launch of the greedy kernel may use on this device.
uint32_t greedy_max_blocks(int sm_count);
// Runs the greedy rounds of d[0..ni) (device array) as one cooperative
// launch of `grid` blocks. *err (device, zero on entry) becomes nonzero if a
// group barrier gave up waiting.
// part: some instance has part_n > 0 (multi-round); it must then fit the
// grid that greedy_max_blocks gives (the multi-round kernel has the same
// occupancy or better).
cudaError_t launch_greedy(const GreedyDesc *d, uint32_t ni, uint32_t grid, unsigned int *err, cudaStream_t s,
                          bool part = false);

// Per-device state shared by every context of the device: sampling scratch
// and launch tables. Its mutex serialises the sampling of all contexts that
// use the device.
constexpr int kMaxDevices = 64;
struct DeviceShared {
  std::mutex mu;
  int refs = 0;
  int sm_count = 0;
  uint32_t lt_grid = 0;
  CommonScratch cs;
  BigScratch big;
  uint64_t big_budget = 0;             // the budget `big` was sized for
  InstDesc *d_desc = nullptr;
  uint64_t desc_cap = 0;
  InstDesc *h_desc = nullptr;          // pinned
  uint64_t h_desc_cap = 0;
  unsigned long long *d_def = nullptr; // two deferred-set lists
  uint32_t *d_defslot = nullptr;       // their overflow slots (same layout)
  uint64_t def_cap = 0;
  uint32_t *lt_ovf = nullptr;          // kLtOvfSlots saved LT paths
  uint32_t *ic_ovf = nullptr;          // kIcOvfSlots saved IC states
  unsigned int *d_ovf_next = nullptr;
  SampleCtl *d_ctl = nullptr;
  SampleCtl *h_ctl = nullptr;          // pinned
};

// A sampling job: RR sets [ctx->R, ctx->R + count) of ctx under (model, seed).
struct SampleJobH {
  gim_ctx *ctx;
  int model;
  uint64_t seed;
  uint64_t count;
};

// Multi-round RR sets |R| .. |R|+count-1 of ctx's multi-round collection
// (ctx->rounds > 1): every round sampled through its view in one launch, then
// merged into the collection in rr_id order.
gim_status mrim_sample(gim_ctx *ctx, int model, uint64_t seed, uint64_t count);
// Frees ctx's per-round views and the merge scratch.
void mrim_release(gim_ctx *ctx);
// Builds the LT thresholds of ctx's graph on its first LT use and sets
// ctx->lt_ok (a graph shared from another context must have them already).
gim_status ensure_lt(gim_ctx *ctx);
bool lt_valid(gim_ctx *ctx);

// IMM constants (Tang, Shi, Xiao 2015): ell', eps', lambda', lambda*, and
// the number of lower-bound rounds floor(log2 n) - 1.
struct ImmConst {
  double ellp, epsp, lam1, lam2;
  int i_max;
};

// engine.cu
ImmConst imm_constants(uint32_t n, uint32_t k, double eps, double ell);
// The same for multi-round IM with T rounds of k seeds (T = 1: imm_constants).
ImmConst mrim_constants(uint32_t n, uint32_t k, uint32_t T, double eps, double ell);
gim_status set_err(gim_ctx *ctx, gim_status st, const char *fmt, ...);
gim_status cuda_err(gim_ctx *ctx, cudaError_t e, const char *what);
gim_status shared_acquire(gim_ctx *ctx);
void shared_release(int device);
DeviceShared &device_shared(int device);
gim_status sample_jobs(std::vector<SampleJobH> &jobs, cudaStream_t s);

// IMM state machine (batch.cu): the lower-bound search of Alg. 2, then the
// final sampling and selection, advanced by the host one round at a time.
struct ImmState {
  ImmConst c;
  int i = 1;             // lower-bound round (1-based)
  int phase = 0;         // 0 lower-bound search, 1 final selection, 2 done
  double LB = 1.0;
  uint64_t theta = 0;
  uint32_t rounds = 0;
};
void imm_init(ImmState &st, uint32_t n, const gim_imm_params &p);
uint64_t imm_target(const ImmState &st, uint32_t n);                  // RR sets the next selection needs
void imm_advance(ImmState &st, uint32_t n, uint64_t R, uint64_t cov);  // after a selection over R sets

// One instance of a batched selection round.
struct SelInput {
  bool active = false;
  uint64_t R = 0, Z = 0;                 // sets [0, R) with Z members in all (Z bounds the index)
  const uint32_t *members = nullptr;
  const uint64_t *rr_start = nullptr;
  const uint32_t *rr_len = nullptr;
  const uint32_t *cnt = nullptr;         // occurrence counts over [0, R); null: counted into buf->cnt_own
  uint64_t count_from = 0;               // cnt == null: buf->cnt_own already counts sets [0, count_from)
  SelectBuffers *buf = nullptr;          // the instance's selection buffers (grown on demand)
  uint32_t k = 0;                        // rounds this time (<= the configured k); 0: the configured k
  // Optional: use the index (inverted lists, hub split, hub rows) that
  // another instance of the same run builds or built over a collection this
  // one is a prefix of (the server's pools); its lists and rows are read up
  // to set R only. index_R = the sets that index covers.
  const SelectBuffers *index = nullptr;
  uint64_t index_R = 0;
  bool index_only = false;               // build this instance's index only (no greedy rounds)
  uint32_t part_n = 0, part_k = 0;       // multi-round partition (see GreedyDesc)
  uint32_t skip = kNoSkip;               // sets [0, R) holding this vertex may be stored without members
};

// Greedy selection of a fixed set of slots (n, k fixed), one CUDA graph per
// configuration replayed for every round.
class MultiSelect {
 public:
  MultiSelect();
  ~MultiSelect();
  // index_only (optional): instances that only ever build an index get one greedy block
  gim_status configure(gim_ctx *ctx, const std::vector<uint32_t> &n, const std::vector<uint32_t> &k,
                       const std::vector<bool> *index_only = nullptr);
  // Runs one selection round of every active slot; cov, seeds (and gains)
  // come back packed by slot (seed_offset).
  gim_status run(gim_ctx *ctx, const std::vector<SelInput> &in, cudaStream_t s, std::vector<unsigned long long> &cov,
                 std::vector<uint32_t> &seeds, std::vector<uint32_t> *gains = nullptr);
  uint32_t slots() const;
  uint32_t k_of(uint32_t i) const;
  uint64_t seed_offset(uint32_t i) const;

 private:
  struct Impl;
  Impl *p;
};

// tune.cu
gim_status autotune(gim_ctx *const *ctxs, uint32_t ni, const gim_imm_params *params, uint64_t sample_sets,
                    uint64_t *budget_out, int *measured_out);

// batch.cu
gim_status batch_imm(gim_ctx *const *ctxs, uint32_t ni, const gim_imm_params *params, uint32_t *const *seeds_out,
                     gim_imm_result *results);
template <typename T>
cudaError_t grow_copy(T *&p, uint64_t &cap, uint64_t need, uint64_t keep, cudaStream_t s);

}  // namespace gim

// Public context (opaque to callers).
struct gim_ctx {
  int device = 0;
  int sm_count = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string last_error;
  uint64_t launches = 0;

  bool has_graph = false;
  bool owns_graph = true;         // false for a server pool that shares another context's graph
  int lt_ok = -1;                 // 1 / 0: LT-valid or not; -1: not known yet (LT thresholds not built)
  uint32_t max_indeg = 0;         // of the loaded graph (degree profile of the autotuner)
  gim::DevGraph g;
  gim::DevGraph g_spare;          // the arrays of the previous graph, reused by the next load that fits
  unsigned int *d_info = nullptr;  // 4 device words for the graph checks (kept across loads)

  // RR collection
  int model = -1;
  uint64_t seed = 0;
  uint32_t jhi = 0;   // rr_id of the set at position j is (jhi:j): 2^31 after a fresh final phase, else 0
  uint32_t rhi = 0;   // high word of the root draw (= jhi; 0 in a multi-round view)
  uint32_t moff = 0;  // stored member = moff + vertex (t * n in round t's view)
  uint32_t idoff = 0; // rr_id low word = position + idoff (a view's chunk starts at the parent's |R|)
  uint32_t rounds = 1;            // T of a multi-round collection; elements t * n + v (1: plain RR sets)
  uint64_t cnt_cap = 0;           // entries of st.cnt (n * rounds at most)
  std::vector<gim_ctx *> round_views;   // per-round sampling views of a multi-round collection
  unsigned long long *mr_tiles = nullptr;   // multi-round merge scratch
  uint64_t mr_tiles_cap = 0;
  uint64_t R = 0;                 // |R|
  uint64_t Z = 0;                 // members over all stored sets
  uint64_t store_used = 0;        // store entries reserved (>= Z: holes after a store overflow)
  uint64_t rr_cap = 0;
  gim::DevStore st;

  bool shared_held = false;       // holds a reference on the device's shared scratch
  uint32_t group_budget = 1u << 14;   // GIM_OPT_GROUP_BUDGET
  uint32_t frontier_batch = 128;      // GIM_OPT_FRONTIER_BATCH
  uint32_t chunk_groups = 512;        // GIM_OPT_CHUNK_GROUPS
  uint32_t queue_cap = 4096;          // GIM_OPT_QUEUE_CAP
  uint64_t big_budget = 16ull << 30;  // GIM_OPT_LARGE_PASS_BYTES
  bool fresh_final = false;           // GIM_OPT_FRESH_FINAL
  bool compact = false;               // GIM_OPT_COMPACT_FIRST_PICK
  // Sets holding this vertex keep only their size and counts (compact
  // collections: gim_imm sets it to its first selection's first pick).
  uint32_t skip_vertex = gim::kNoSkip;

  gim::SelectBuffers sel;
  gim::MultiSelect *msel = nullptr;   // gim_select_seeds / gim_imm: a one-slot batched selection
  uint32_t msel_n = 0, msel_k = 0;

  cudaEvent_t ev[10] = {};
  double t_sample_ms = 0, t_select_ms = 0, t_wall_ms = 0, lb_rounds = 0;
  // sampling-kernel launches since the last reset of these counters
  double t_kernel_ms[2] = {0, 0};       // common-case pass, large-set pass
  double n_kernel[2] = {0, 0};
  // selections since the last reset: device time, algorithmic bytes, calls, members of covered sets
  double sel_kernel_ms = 0, sel_bytes = 0, sel_calls = 0, sel_cov_members = 0;
};
