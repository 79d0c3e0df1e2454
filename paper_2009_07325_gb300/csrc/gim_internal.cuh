// Internal declarations of libgim: context layout, device-side Philox, and
// the kernels' host launchers. Nothing here is part of the public C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "gim.h"

namespace gim {

constexpr uint32_t kFullMask = 0xFFFFFFFFu;
constexpr uint64_t kNoStart = ~0ull;          // rr_start of a set not (yet) stored

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). Counter words are
// (idx, tag, j_lo, j_hi); the key is the 64-bit seed split into two words.
// ---------------------------------------------------------------------------
struct PhiloxKey {
  uint32_t k0, k1;
};

__device__ __forceinline__ uint4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, PhiloxKey key) {
  uint32_t k0 = key.k0, k1 = key.k1;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t a_lo = 0xD2511F53u * c0, a_hi = __umulhi(0xD2511F53u, c0);
    const uint32_t b_lo = 0xCD9E8D57u * c2, b_hi = __umulhi(0xCD9E8D57u, c2);
    const uint32_t y0 = b_hi ^ c1 ^ k0;
    const uint32_t y2 = a_hi ^ c3 ^ k1;
    c0 = y0;
    c1 = b_lo;
    c2 = y2;
    c3 = a_lo;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return make_uint4(c0, c1, c2, c3);
}

enum : uint32_t { kTagRoot = 0, kTagEdge = 1, kTagStep = 2 };

// randSelect(V) of Alg. 3: the root of RR set j, high word of a 64-bit draw times n.
__device__ __forceinline__ uint32_t draw_root(PhiloxKey key, uint64_t j, uint32_t n) {
  const uint4 r = philox10(0u, kTagRoot, (uint32_t)j, (uint32_t)(j >> 32), key);
  const uint64_t w = ((uint64_t)r.y << 32) | r.x;
  return (uint32_t)__umul64hi(w, (uint64_t)n);
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
  uint64_t *cum = nullptr;   // m: LT cumulative thresholds in 2^-32 units
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

// Device counters of one sampling launch.
struct SampleCtl {
  unsigned long long next;        // next work item
  unsigned long long store_tail;  // store entries reserved
  unsigned long long members;     // store entries of stored sets
  unsigned long long n_deferred;  // sets handed to the large-set pass
  unsigned int err;               // error bits (kErr*)
  unsigned int pad;
};

enum : unsigned int { kErrDeferredFull = 1u };

// Per-worker scratch for the sampling kernels.
struct WorkerScratch {
  uint32_t *bitmap = nullptr;    // words_per_worker per worker, all zero between sets
  uint32_t *queue = nullptr;     // qcap per worker
  uint64_t words_per_worker = 0;
  uint32_t qcap = 0;
  uint32_t workers = 0;
};

struct SampleJob {
  PhiloxKey key;
  uint64_t j_begin;              // first rr_id when items are a contiguous range
  uint64_t count;                // number of work items
  const uint64_t *j_list;        // nullable: item i is rr_id j_list[i]
  uint64_t *deferred;            // where too-large (or unstorable) sets are listed
  uint64_t deferred_cap;
};

// Host launchers (sample.cu).
cudaError_t launch_sample(int model, const DevGraph &g, const DevStore &st, const WorkerScratch &ws, const SampleJob &job,
                          SampleCtl *ctl, bool large, int grid, int block, cudaStream_t s);
cudaError_t launch_uncount(const DevStore &st, uint64_t j_begin, uint64_t count, cudaStream_t s);
cudaError_t launch_philox_rate(int blocks, uint32_t per_thread, uint32_t *sink, cudaStream_t s);

// Graph preprocessing (graph.cu).
cudaError_t launch_graph_prep(DevGraph &g, const float *d_w, unsigned int *d_flags, cudaStream_t s);
enum : unsigned int { kGraphBadSource = 1u, kGraphNotAscending = 2u, kGraphBadWeight = 4u, kGraphNotLT = 8u };

// Selection (select.cu).
struct SelectBuffers {
  uint32_t *cnt_work = nullptr;  // n (count + 1 while unselected, 0 once selected)
  uint64_t *inv_off = nullptr;   // n+1
  uint32_t *cursor = nullptr;    // n
  uint32_t *inv = nullptr;       // Z rr ids
  uint8_t *covered = nullptr;    // R flags
  unsigned long long *best = nullptr;   // k argmax keys
  uint32_t *seeds = nullptr;     // k
  uint32_t *gains = nullptr;     // k
  unsigned long long *covered_total = nullptr;
  uint64_t *scan_tmp = nullptr;  // block partial sums
  uint64_t n_cap = 0, z_cap = 0, r_cap = 0, k_cap = 0, scan_cap = 0;
};

cudaError_t run_select(const DevGraph &g, const DevStore &st, uint64_t R, uint64_t Z, uint32_t k, SelectBuffers &b,
                       int sm_count, cudaStream_t s, uint64_t *launches);

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
  int lt_ok = 0;
  gim::DevGraph g;

  // RR collection
  int model = -1;
  uint64_t seed = 0;
  uint64_t R = 0;                 // |R|
  uint64_t Z = 0;                 // members over all stored sets
  uint64_t store_used = 0;        // store entries reserved (>= Z: holes after a store overflow)
  uint64_t rr_cap = 0;
  gim::DevStore st;

  // sampling scratch
  gim::WorkerScratch ws_small, ws_lt, ws_large;   // IC common case, LT common case, large-set pass
  gim::SampleCtl *ctl = nullptr;      // device
  gim::SampleCtl *ctl_host = nullptr; // pinned mirror
  uint64_t *deferred = nullptr;
  uint64_t deferred_cap = 0;
  int small_grid = 0, small_block = 0;

  gim::SelectBuffers sel;

  cudaEvent_t ev[8] = {};
  double t_sample_ms = 0, t_select_ms = 0, t_wall_ms = 0, lb_rounds = 0;
  // sampling-kernel launches since the last reset of these counters
  double t_kernel_ms[2] = {0, 0};       // common-case pass, large-set pass
  double n_kernel[2] = {0, 0};
};
