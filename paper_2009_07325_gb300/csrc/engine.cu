// Host-side sampling engine: per-device shared scratch and the orchestration
// of sampling jobs (one or many contexts per launch), including the
// large-set passes and on-demand growth of the RR stores.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <vector>

#include "gim_internal.cuh"

namespace gim {

gim_status set_err(gim_ctx *ctx, gim_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->last_error = buf;
  return st;
}

gim_status cuda_err(gim_ctx *ctx, cudaError_t e, const char *what) {
  cudaGetLastError();   // clear a non-sticky error so the context stays usable
  if (e == cudaErrorMemoryAllocation) return set_err(ctx, GIM_ERR_OOM, "%s: out of device memory", what);
  return set_err(ctx, GIM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CU(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_err(ctx, e_, #call);   \
  } while (0)

namespace {

constexpr uint64_t kInitialStore = 1ull << 24;  // store entries at first use

DeviceShared g_shared[kMaxDevices];

template <typename T>
void dfree(T *&p) {
  if (p) cudaFree(p);
  p = nullptr;
}

}  // namespace

// Grows the device array p (capacity cap elements) to hold at least need
// elements, keeping the first keep elements.
template <typename T>
cudaError_t grow_copy(T *&p, uint64_t &cap, uint64_t need, uint64_t keep, cudaStream_t s) {
  if (need <= cap && p) return cudaSuccess;
  const uint64_t c = std::max<uint64_t>(need, cap * 2);
  T *q = nullptr;
  cudaError_t e = cudaMalloc(&q, c * sizeof(T));
  if (e != cudaSuccess) return e;
  if (p && keep) {
    e = cudaMemcpyAsync(q, p, keep * sizeof(T), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
      cudaFree(q);
      return e;
    }
  }
  if (p) {
    cudaStreamSynchronize(s);
    cudaFree(p);
  }
  p = q;
  cap = c;
  return cudaSuccess;
}
template cudaError_t grow_copy<uint32_t>(uint32_t *&, uint64_t &, uint64_t, uint64_t, cudaStream_t);
template cudaError_t grow_copy<uint64_t>(uint64_t *&, uint64_t &, uint64_t, uint64_t, cudaStream_t);
template cudaError_t grow_copy<unsigned long long>(unsigned long long *&, uint64_t &, uint64_t, uint64_t,
                                                   cudaStream_t);

// IMM constants (Tang, Shi, Xiao 2015) in a fixed evaluation order. With T
// rounds of k seeds (multi-round IM) the count of feasible seed sets is
// C(n, k)^T, so ln C(n, k) becomes T ln C(n, k), and the greedy's guarantee
// over that partition matroid, 1/2, replaces 1 - 1/e; T = 1 is IMM.
ImmConst mrim_constants(uint32_t n, uint32_t k, uint32_t T, double eps, double ell) {
  ImmConst c;
  const double logn = std::log((double)n);
  c.ellp = ell * (1.0 + std::log(2.0) / logn);
  c.epsp = std::sqrt(2.0) * eps;
  double lnc = 0.0;
  for (uint32_t i = 0; i < k; ++i) lnc += std::log((double)(n - i)) - std::log((double)(i + 1));
  lnc *= (double)T;
  c.lam1 = (2.0 + 2.0 * c.epsp / 3.0) * (lnc + c.ellp * logn + std::log(std::log2((double)n))) * (double)n /
           (c.epsp * c.epsp);
  const double g = T == 1 ? 1.0 - std::exp(-1.0) : 0.5;
  const double alpha = std::sqrt(c.ellp * logn + std::log(2.0));
  const double beta = std::sqrt(g * (lnc + c.ellp * logn + std::log(2.0)));
  const double t = g * alpha + beta;
  c.lam2 = 2.0 * (double)n * t * t / (eps * eps);
  c.i_max = (31 - __builtin_clz(n)) - 1;
  return c;
}

ImmConst imm_constants(uint32_t n, uint32_t k, double eps, double ell) { return mrim_constants(n, k, 1, eps, ell); }


DeviceShared &device_shared(int device) { return g_shared[device]; }

gim_status ensure_lt(gim_ctx *ctx) {
  if (!ctx->has_graph) return set_err(ctx, GIM_ERR_STATE, "no graph loaded");
  if (ctx->lt_ok >= 0) return GIM_OK;
  if (!ctx->owns_graph) return set_err(ctx, GIM_ERR_STATE, "the LT thresholds of a shared graph are not built");
  DevGraph &g = ctx->g;
  cudaStream_t s = ctx->stream;
  if (!g.cum) CU(cudaMalloc(&g.cum, std::max<uint64_t>(g.m_cap, 1) * 8));
  if (!ctx->d_info) CU(cudaMalloc(&ctx->d_info, 4 * sizeof(unsigned int)));
  unsigned int *d_flags = ctx->d_info;
  unsigned int flags = 0;
  cudaError_t e = cudaMemsetAsync(d_flags, 0, 4, s);
  if (e == cudaSuccess) e = launch_lt_prep(g, d_flags, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, d_flags, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_err(ctx, e, "LT thresholds");
  ctx->launches++;
  ctx->lt_ok = (flags & kGraphNotLT) ? 0 : 1;
  return GIM_OK;
}

// True iff the graph is LT-valid, building its LT thresholds first if needed
// (a failure to build them leaves the error on ctx and reads as not valid).
bool lt_valid(gim_ctx *ctx) { return ensure_lt(ctx) == GIM_OK && ctx->lt_ok == 1; }

namespace {

// Frees every buffer of D (the caller holds D.mu).
void shared_free(DeviceShared &D) {
  dfree(D.cs.queue);
  dfree(D.cs.hash);
  dfree(D.cs.epoch);
  D.cs = CommonScratch{};
  dfree(D.big.bitmap);
  dfree(D.big.queue);
  D.big = BigScratch{};
  dfree(D.d_desc);
  D.desc_cap = 0;
  if (D.h_desc) cudaFreeHost(D.h_desc);
  D.h_desc = nullptr;
  D.h_desc_cap = 0;
  dfree(D.d_def);
  dfree(D.d_defslot);
  D.def_cap = 0;
  dfree(D.lt_ovf);
  dfree(D.ic_ovf);
  dfree(D.d_ovf_next);
  dfree(D.d_ctl);
  if (D.h_ctl) cudaFreeHost(D.h_ctl);
  D.h_ctl = nullptr;
  D.refs = 0;
}

}  // namespace

gim_status shared_acquire(gim_ctx *ctx) {
  DeviceShared &D = g_shared[ctx->device];
  std::lock_guard<std::mutex> lock(D.mu);
  if (D.refs == 0) {
    D.sm_count = ctx->sm_count;
    const uint32_t workers = (uint32_t)ctx->sm_count * (uint32_t)ic_common_blocks_per_sm() * 8u;
    D.cs.workers = workers;
    cudaError_t e = cudaMalloc(&D.cs.queue, (uint64_t)workers * kQueueCap * 4);
    if (e == cudaSuccess) e = cudaMalloc(&D.cs.hash, (uint64_t)workers * kHashSlots * 8);
    if (e == cudaSuccess) e = cudaMalloc(&D.cs.epoch, (uint64_t)workers * 4);
    if (e == cudaSuccess) e = cudaMemset(D.cs.hash, 0, (uint64_t)workers * kHashSlots * 8);
    if (e == cudaSuccess) e = cudaMemset(D.cs.epoch, 0, (uint64_t)workers * 4);
    if (e == cudaSuccess) e = cudaMalloc(&D.d_ctl, sizeof(SampleCtl));
    if (e == cudaSuccess) e = cudaMalloc(&D.lt_ovf, (uint64_t)kLtOvfSlots * kLtGroupPath * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&D.ic_ovf, (uint64_t)kIcOvfSlots * kIcOvfStride * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&D.d_ovf_next, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMallocHost(&D.h_ctl, sizeof(SampleCtl));
    if (e != cudaSuccess) {
      shared_free(D);   // nothing is kept from a failed set-up, so a retry starts clean
      return cuda_err(ctx, e, "per-device sampling scratch");
    }
    D.lt_grid = (uint32_t)ctx->sm_count * (uint32_t)lt_common_blocks_per_sm();
  }
  D.refs++;
  return GIM_OK;
}

void shared_release(int device) {
  DeviceShared &D = g_shared[device];
  std::lock_guard<std::mutex> lock(D.mu);
  if (--D.refs > 0) return;
  shared_free(D);
}

namespace {

// Large-pass scratch for graphs of up to n vertices (bitmap + n-entry queue per slot).
gim_status ensure_big(gim_ctx *ctx, DeviceShared &D, uint32_t n, bool full_queue) {
  const uint64_t budget = ctx->big_budget;
  const uint32_t qc = full_queue ? n : std::min(n, kSlotQueue);
  if (D.big.slots && D.big.n_cap >= n && D.big.q_cap >= qc && D.big_budget == budget &&
      (full_queue || D.big.q_cap <= std::max(qc, kSlotQueue)))
    return GIM_OK;
  dfree(D.big.bitmap);
  dfree(D.big.queue);
  D.big = BigScratch{};
  const uint64_t words = ((uint64_t)n + 31) / 32;
  const uint64_t wps = (words + 31) / 32 * 32;
  const uint64_t per = wps * 4 + (uint64_t)qc * 4;
  uint64_t slots = std::min<uint64_t>(budget / std::max<uint64_t>(per, 1), (uint64_t)D.sm_count * kBigBlocksPerSM);
  slots = std::max<uint64_t>(slots, 1);
  CU(cudaMalloc(&D.big.bitmap, wps * 4 * slots));
  CU(cudaMalloc(&D.big.queue, (uint64_t)qc * 4 * slots));
  CU(cudaMemset(D.big.bitmap, 0, wps * 4 * slots));
  D.big.words_per_slot = wps;
  D.big.n_cap = n;
  D.big.q_cap = qc;
  D.big.slots = (uint32_t)slots;
  D.big_budget = budget;
  return GIM_OK;
}

gim_status ensure_lists(gim_ctx *ctx, DeviceShared &D, uint64_t n_inst, uint64_t items) {
  if (D.desc_cap < n_inst) {
    dfree(D.d_desc);
    D.desc_cap = 0;
    CU(cudaMalloc(&D.d_desc, n_inst * sizeof(InstDesc)));
    D.desc_cap = n_inst;
  }
  if (D.h_desc_cap < n_inst) {
    if (D.h_desc) cudaFreeHost(D.h_desc);
    D.h_desc = nullptr;
    D.h_desc_cap = 0;
    CU(cudaMallocHost(&D.h_desc, n_inst * sizeof(InstDesc)));
    D.h_desc_cap = n_inst;
  }
  if (D.def_cap < 2 * items) {
    dfree(D.d_def);
    dfree(D.d_defslot);
    D.def_cap = 0;
    CU(cudaMalloc(&D.d_def, 2 * items * sizeof(unsigned long long)));
    CU(cudaMalloc(&D.d_defslot, 2 * items * sizeof(uint32_t)));
    D.def_cap = 2 * items;
  }
  return GIM_OK;
}

// Room for `count` more RR sets in ctx's collection; new ids marked unstored.
gim_status ensure_collection(gim_ctx *ctx, uint64_t count, cudaStream_t s) {
  const uint64_t R0 = ctx->R;
  uint64_t cap = ctx->rr_cap, cap2 = ctx->rr_cap;
  CU(grow_copy(ctx->st.rr_start, cap, R0 + count, R0, s));
  CU(grow_copy(ctx->st.rr_len, cap2, R0 + count, R0, s));
  ctx->rr_cap = std::min(cap, cap2);
  CU(cudaMemsetAsync(ctx->st.rr_start + R0, 0xFF, count * sizeof(uint64_t), s));
  if (!ctx->st.members) {
    uint64_t c = 0;
    CU(grow_copy(ctx->st.members, c, std::max<uint64_t>(kInitialStore, count * 4), 0, s));
    ctx->st.cap = c;
  }
  return GIM_OK;
}

void fill_desc(InstDesc &d, gim_ctx *c, uint64_t seed, uint64_t item_begin) {
  d = InstDesc{};
  d.n = c->g.n;
  d.off = c->g.off;
  d.src = c->g.src;
  d.thr = c->g.thr;
  d.rthr = c->g.rthr;
  d.rw = c->g.rw;
  d.cum = c->g.cum;
  d.members = c->st.members;
  d.store_cap = c->st.cap;
  d.rr_start = c->st.rr_start;
  d.rr_len = c->st.rr_len;
  d.cnt = c->st.cnt;
  d.key = PhiloxKey{(uint32_t)seed, (uint32_t)(seed >> 32)};
  d.j_begin = c->R;
  d.jhi = c->jhi;
  d.rhi = c->rhi;
  d.moff = c->moff;
  d.idoff = c->idoff;
  d.skip = c->skip_vertex;
  d.item_begin = item_begin;
  d.store_tail = c->store_used;
  d.members_added = 0;
}

struct Pass {
  bool large;
  uint64_t items;
  const unsigned long long *list;
  unsigned long long *out;
  const uint32_t *list_slots;   // overflow slots of list (nullable)
  uint32_t *out_slots;          // overflow slots of out
};

// Runs one launch over the group's descriptors and settles every store.
gim_status run_one(gim_ctx *ctx, DeviceShared &D, int model, std::vector<SampleJobH *> &grp, const Pass &P,
                   cudaStream_t s, SampleLaunch *used) {
  const uint32_t ni = (uint32_t)grp.size();
  // the host descriptors carry each instance's current store (it may have grown)
  for (uint32_t i = 0; i < ni; ++i) {
    gim_ctx *c = grp[i]->ctx;
    D.h_desc[i].members = c->st.members;
    D.h_desc[i].store_cap = c->st.cap;
    D.h_desc[i].store_tail = c->store_used;
    D.h_desc[i].members_added = 0;
  }
  CU(cudaMemcpyAsync(D.d_desc, D.h_desc, ni * sizeof(InstDesc), cudaMemcpyHostToDevice, s));
  SampleCtl init{};
  CU(cudaMemcpyAsync(D.d_ctl, &init, sizeof init, cudaMemcpyHostToDevice, s));
  SampleLaunch L{};
  L.inst = D.d_desc;
  L.n_inst = ni;
  L.total_items = P.items;
  L.items = P.list;
  L.deferred = P.out;
  L.deferred_cap = D.def_cap / 2;
  L.ctl = D.d_ctl;
  L.group_budget = P.large ? 0xFFFFFFFFu : ctx->group_budget;   // the first context's knobs serve the launch
  // the knobs as gim_set_option admits them (kernels index shared arrays by the batch)
  L.queue_cap = std::min<uint32_t>(std::max<uint32_t>(ctx->queue_cap, 256u), kQueueCap);
  L.batch = std::min<uint32_t>(std::max<uint32_t>(ctx->frontier_batch, 32u), (uint32_t)kBigBlock);
  L.chunk_groups = std::max<uint32_t>(ctx->chunk_groups, 64u);
  L.item_slots = P.list_slots;
  L.deferred_slots = P.out_slots;
  L.lt_ovf = D.lt_ovf;
  L.lt_ovf_next = D.d_ovf_next;
  L.lt_ovf_cap = kLtOvfSlots;
  L.ic_ovf = D.ic_ovf;
  L.ic_ovf_cap = kIcOvfSlots;
  if (used) *used = L;
  CU(cudaEventRecord(ctx->ev[6], s));
  cudaError_t e;
  if (model == GIM_IC) {
    const InstDesc *one = ni == 1 ? &D.h_desc[0] : nullptr;
    e = P.large ? launch_ic_block(L, D.big, (uint32_t)std::min<uint64_t>(P.items, D.big.slots), one, s)
                : launch_ic_common(L, D.cs, one, s);
  } else {
    e = P.large ? launch_lt_large(L, D.big, (uint32_t)std::min<uint64_t>(P.items, D.big.slots), s)
                : launch_lt_common(L, D.lt_grid, s);
  }
  if (e != cudaSuccess) return cuda_err(ctx, e, "sampling kernel launch");
  CU(cudaEventRecord(ctx->ev[7], s));
  ctx->launches++;
  CU(cudaMemcpyAsync(D.h_desc, D.d_desc, ni * sizeof(InstDesc), cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(D.h_ctl, D.d_ctl, sizeof(SampleCtl), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  float ms = 0;
  cudaEventElapsedTime(&ms, ctx->ev[6], ctx->ev[7]);
  ctx->t_kernel_ms[P.large ? 1 : 0] += ms;
  ctx->n_kernel[P.large ? 1 : 0] += 1;
  if (D.h_ctl->err & kErrDeferredFull) return set_err(ctx, GIM_ERR_OOM, "deferred-set list overflow");
  // settle: account members, grow stores whose reservations ran past the end
  for (uint32_t i = 0; i < ni; ++i) {
    gim_ctx *c = grp[i]->ctx;
    const InstDesc &d = D.h_desc[i];
    c->Z += d.members_added;
    if (d.store_tail > c->st.cap) {
      const uint64_t old = c->st.cap;
      uint64_t cap = c->st.cap;
      CU(grow_copy(c->st.members, cap, std::max<uint64_t>(old * 2, d.store_tail * 2), old, s));
      c->st.cap = cap;
      c->store_used = old;   // the last partial reservation leaves a hole below the old end
    } else {
      c->store_used = d.store_tail;
    }
  }
  return GIM_OK;
}

}  // namespace

// Samples every job's RR sets [ctx->R, ctx->R + count) under its (model,
// seed): one common-pass launch per model over all jobs of that model, then
// large-set passes over the deferred sets until none is left. On failure the
// occurrence counts of the failed group are rolled back.
gim_status sample_jobs(std::vector<SampleJobH> &jobs, cudaStream_t s) {
  if (jobs.empty()) return GIM_OK;
  gim_ctx *ctx = jobs[0].ctx;   // errors and timings are reported on the first context
  DeviceShared &D = g_shared[ctx->device];
  std::lock_guard<std::mutex> lock(D.mu);
  gim_status st;
  for (auto &jb : jobs)
    if (jb.count && (st = ensure_collection(jb.ctx, jb.count, s)) != GIM_OK) {
      if (jb.ctx != ctx) ctx->last_error = jb.ctx->last_error;
      return st;
    }
  for (int model = GIM_IC; model <= GIM_LT; ++model) {
    std::vector<SampleJobH *> grp;
    uint64_t total = 0;
    uint32_t nmax = 0;
    for (auto &jb : jobs)
      if (jb.model == model && jb.count) {
        grp.push_back(&jb);
        total += jb.count;
        nmax = std::max(nmax, jb.ctx->g.n);
      }
    if (grp.empty()) continue;
    if ((st = ensure_lists(ctx, D, grp.size(), total)) != GIM_OK) return st;
    uint64_t item = 0;
    std::vector<uint64_t> Z0, used0;
    for (uint32_t i = 0; i < grp.size(); ++i) {
      fill_desc(D.h_desc[i], grp[i]->ctx, grp[i]->seed, item);
      item += grp[i]->count;
      Z0.push_back(grp[i]->ctx->Z);
      used0.push_back(grp[i]->ctx->store_used);
    }
    std::vector<InstDesc> first(D.h_desc, D.h_desc + grp.size());
    SampleLaunch L0{};
    auto rollback = [&]() {
      for (uint32_t i = 0; i < grp.size(); ++i) {   // stores may have been reallocated since
        first[i].members = grp[i]->ctx->st.members;
        first[i].store_cap = grp[i]->ctx->st.cap;
      }
      cudaMemcpyAsync(D.d_desc, first.data(), first.size() * sizeof(InstDesc), cudaMemcpyHostToDevice, s);
      SampleLaunch u = L0;
      u.items = nullptr;
      u.total_items = total;
      launch_uncount(u, s);
      cudaStreamSynchronize(s);
      for (uint32_t i = 0; i < grp.size(); ++i) {
        gim_ctx *c = grp[i]->ctx;
        c->Z = Z0[i];
        c->store_used = used0[i];
        if (c->skip_vertex != kNoSkip) {
          // the counts of sets stored without members cannot be lowered again:
          // a compact collection is emptied instead of rolled back
          c->R = c->Z = c->store_used = 0;
          c->model = -1;
          c->skip_vertex = kNoSkip;
          cudaMemsetAsync(c->st.cnt, 0, (uint64_t)c->g.n * c->rounds * 4, s);
          cudaStreamSynchronize(s);
        }
      }
    };
    unsigned long long *list_a = D.d_def, *list_b = D.d_def + D.def_cap / 2;
    uint32_t *slot_a = D.d_defslot, *slot_b = D.d_defslot + D.def_cap / 2;
    CU(cudaMemsetAsync(D.d_ovf_next, 0, sizeof(unsigned int), s));   // saved LT paths / IC states of this call
    Pass P{false, total, nullptr, list_a, nullptr, slot_a};
    if ((st = run_one(ctx, D, model, grp, P, s, &L0)) != GIM_OK) return rollback(), st;
    uint64_t pending = D.h_ctl->n_deferred;
    int rounds = 0;
    while (pending > 0) {
      if (++rounds > 40) {
        rollback();
        return set_err(ctx, GIM_ERR_OOM, "large-set pass did not converge");
      }
      // first with capped queues (more sets in flight); what is still pending
      // after that (a set beyond kSlotQueue members, or a full store) gets n
      if ((st = ensure_big(ctx, D, nmax, rounds > 1)) != GIM_OK) return rollback(), st;
      Pass Q{true, pending, list_a, list_b, slot_a, slot_b};
      if ((st = run_one(ctx, D, model, grp, Q, s, nullptr)) != GIM_OK) return rollback(), st;
      pending = D.h_ctl->n_deferred;
      std::swap(list_a, list_b);
      std::swap(slot_a, slot_b);
    }
    for (auto *jb : grp) {
      jb->ctx->R += jb->count;
      jb->ctx->model = jb->model;
      jb->ctx->seed = jb->seed;
    }
  }
  return GIM_OK;
}

}  // namespace gim
