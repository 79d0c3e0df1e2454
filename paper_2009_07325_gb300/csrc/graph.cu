// Graph preprocessing on the device: validation of the in-edge CSR and the IC
// coin thresholds at load, the LT cumulative thresholds on the first LT use
// (Sec. III-B CSR layout; Sec. III-G LT edge choice).
#include <algorithm>

#include "gim_internal.cuh"

namespace gim {

// Edge-parallel: IC threshold thr[e] = ceil(w[e] * 2^24), so that the coin
// "U < p" of Alg. 3 with U = (word >> 8) * 2^-24 becomes (word >> 8) < thr[e].
// Also checks source range and weight range. Padding entries get thr = 0.
__global__ void prep_edges_kernel(uint32_t n, uint64_t m, uint64_t m_pad, const uint32_t *__restrict__ src,
                                  const float *__restrict__ w, uint32_t *__restrict__ thr,
                                  unsigned int *__restrict__ flags) {
  unsigned int bad = 0;
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m_pad;
       e += (uint64_t)gridDim.x * blockDim.x) {
    if (e < m) {
      const float p = w[e];
      if (!(p >= 0.0f && p <= 1.0f)) bad |= kGraphBadWeight;
      if (src[e] >= n) bad |= kGraphBadSource;
      // exact: scaling by a power of two, then an integral ceiling
      thr[e] = (p >= 0.0f && p <= 1.0f) ? (uint32_t)ceilf(p * 16777216.0f) : 0u;
    } else {
      thr[e] = 0u;
    }
  }
  if (bad) atomicOr(flags, bad);
}

__device__ __forceinline__ unsigned long long warp_incl_scan_u64(unsigned long long v) {
  const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long o = __shfl_up_sync(kFullMask, v, d);
    if (lane >= (uint32_t)d) v += o;
  }
  return v;
}

__device__ __forceinline__ unsigned long long lt_round(double P) {
  const double x = __dmul_rn(P, 4294967296.0);
  const double f = floor(x);
  unsigned long long c = (unsigned long long)f;
  if (__dsub_rn(x, f) >= 0.5) c += 1ull;
  return c > 4294967296ull ? 4294967296ull : c;
}

// At graph load, per row: ascending sources within the row, the row's
// common IC threshold (rthr) and the row's common weight (rw: the fp32 bits
// when every in-edge of the row carries the same weight, else kPerEdge).
// Rows of at most kSmallRow in-edges take one thread each; the others are
// listed (big, count in *nbig) for a block each (prep_big_rows_kernel).
constexpr uint32_t kSmallRow = 64;

__global__ void __launch_bounds__(256) prep_rows_kernel(uint32_t n, const uint32_t *__restrict__ off,
                                                        const uint32_t *__restrict__ src,
                                                        const float *__restrict__ w,
                                                        const uint32_t *__restrict__ thr,
                                                        uint32_t *__restrict__ rthr, uint32_t *__restrict__ rw,
                                                        uint32_t *__restrict__ big, unsigned int *__restrict__ nbig,
                                                        unsigned int *__restrict__ flags) {
  unsigned int bad = 0;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const uint32_t s = off[v], e = off[v + 1];
    if (e - s > kSmallRow) {
      big[atomicAdd(nbig, 1u)] = v;
      continue;
    }
    const uint32_t common0 = e > s ? thr[s] : 0u;
    const uint32_t w0 = e > s ? __float_as_uint(w[s]) : kPerEdge;
    bool differs = false, wdiffers = false;
    uint32_t prev = 0;
    for (uint32_t i = s; i < e; ++i) {
      const uint32_t si = src[i];
      if (thr[i] != common0) differs = true;
      if (__float_as_uint(w[i]) != w0) wdiffers = true;
      if (i > s && !(prev < si)) bad |= kGraphNotAscending;
      prev = si;
    }
    rthr[v] = differs ? kPerEdge : common0;
    rw[v] = wdiffers ? kPerEdge : w0;
  }
  if (bad) atomicOr(flags, bad);
}

// Block per listed row (more than kSmallRow in-edges): the same checks, 256
// edges per step, so a hub row of 10^5 in-edges is not left to one warp.
__global__ void __launch_bounds__(256) prep_big_rows_kernel(const uint32_t *__restrict__ off,
                                                            const uint32_t *__restrict__ src,
                                                            const float *__restrict__ w,
                                                            const uint32_t *__restrict__ thr,
                                                            uint32_t *__restrict__ rthr, uint32_t *__restrict__ rw,
                                                            const uint32_t *__restrict__ big,
                                                            const unsigned int *__restrict__ nbig,
                                                            unsigned int *__restrict__ flags) {
  const uint32_t nb = *nbig;
  unsigned int bad = 0;
  for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x) {
    const uint32_t v = big[b];
    const uint32_t s = off[v], e = off[v + 1];   // e - s > kSmallRow
    const uint32_t common0 = thr[s];
    const uint32_t w0 = __float_as_uint(w[s]);
    bool differs = false, wdiffers = false;
    for (uint32_t i = s + threadIdx.x; i < e; i += blockDim.x) {
      const uint32_t si = src[i];
      if (thr[i] != common0) differs = true;
      if (__float_as_uint(w[i]) != w0) wdiffers = true;
      if (i > s && !(src[i - 1] < si)) bad |= kGraphNotAscending;
    }
    const int any_diff = __syncthreads_or(differs);
    const int any_wdiff = __syncthreads_or(wdiffers);
    if (threadIdx.x == 0) {
      rthr[v] = any_diff ? kPerEdge : common0;
      rw[v] = any_wdiff ? kPerEdge : w0;
    }
  }
  if (bad) atomicOr(flags, bad);
}

// On the first LT use of the graph, per row: the LT thresholds
//   cum[e_i] = min(2^32, round_half_up(P_i * 2^32)),
// P_i the fp64 running sum of the row's weights in CSR order; a row summing
// to within 1e-6 of 1 gets cum[last] = 2^32 so that it always selects an
// edge, and a row summing above 1 + 1e-6 marks the graph as not valid for LT.
// The running sum is computed exactly: with E the smallest ulp exponent of
// the row's non-zero weights, every weight is an integer q_t times 2^E; when
// all prefix sums of the q_t stay below 2^53, every fp64 partial sum is
// representable, so the sequential fp64 additions never round and P_i equals
// the integer prefix sum Q_i times 2^E. Then P_i * 2^32 = Q_i * 2^(E+32) is
// rounded half up in integer arithmetic (lt_round_int). Other rows (weights
// spanning more than 2^29 ulps, or huge sums) take the strictly sequential
// fp64 loop (lt_round). Both give the same thresholds. Rows of at most
// kSmallRow in-edges take one thread each (prep_lt_kernel); the others are
// listed for a block each (prep_lt_big_kernel), which scans 256 in-edges
// at a time.

// The row fix-ups and the LT-validity flag from the row total P.
__device__ __forceinline__ void lt_row_end(double P, uint32_t s, uint32_t e, uint64_t *cum, unsigned int &bad) {
  if (e > s && fabs(__dsub_rn(P, 1.0)) <= 1e-6) cum[e - 1] = 4294967296ull;
  if (P > 1.0 + 1e-6) bad |= kGraphNotLT;
}

// Sequential fp64 prefix sums of the row (the fallback): returns P.
__device__ __forceinline__ double lt_row_sequential(const float *__restrict__ w, uint64_t *cum, uint32_t s, uint32_t e) {
  double P = 0.0;
  for (uint32_t i = s; i < e; ++i) {
    P = __dadd_rn(P, (double)w[i]);
    cum[i] = lt_round(P);
  }
  return P;
}

__global__ void __launch_bounds__(256) prep_lt_kernel(uint32_t n, const uint32_t *__restrict__ off,
                                                      const float *__restrict__ w, uint64_t *__restrict__ cum,
                                                      uint32_t *__restrict__ big, unsigned int *__restrict__ nbig,
                                                      unsigned int *__restrict__ flags) {
  unsigned int bad = 0;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const uint32_t s = off[v], e = off[v + 1];
    if (e - s > kSmallRow) {
      big[atomicAdd(nbig, 1u)] = v;
      continue;
    }
    int emin = 0x7FFFFFFF;
    uint32_t mant;
    for (uint32_t i = s; i < e; ++i) emin = min(emin, ulp_exponent(w[i], &mant));
    double P = 0.0;
    if (emin == 0x7FFFFFFF) {
      for (uint32_t i = s; i < e; ++i) cum[i] = 0ull;   // all weights zero
    } else {
      bool exact = true;
      unsigned long long Q = 0;
      for (uint32_t i = s; i < e && exact; ++i) {
        const int ex = ulp_exponent(w[i], &mant);
        if (ex != 0x7FFFFFFF) {
          const int sh = ex - emin;
          if (sh > 29) {
            exact = false;                               // q would reach 2^53
            break;
          }
          Q += (unsigned long long)mant << sh;
          if (Q >= (1ull << 53)) {
            exact = false;
            break;
          }
        }
        cum[i] = lt_round_int(Q, emin + 32);
      }
      P = exact ? __dmul_rn(__ull2double_rn(Q), __longlong_as_double((long long)(emin + 1023) << 52))
                : lt_row_sequential(w, cum, s, e);
    }
    lt_row_end(P, s, e, cum, bad);
  }
  if (bad) atomicOr(flags, bad);
}

__global__ void __launch_bounds__(256) prep_lt_big_kernel(const uint32_t *__restrict__ off,
                                                          const float *__restrict__ w, uint64_t *__restrict__ cum,
                                                          const uint32_t *__restrict__ big,
                                                          const unsigned int *__restrict__ nbig,
                                                          unsigned int *__restrict__ flags) {
  __shared__ int s_min[8];
  __shared__ unsigned long long s_tot[8];
  __shared__ double s_P;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, wid = tid >> 5;
  const uint32_t nb = *nbig;
  unsigned int bad = 0;
  for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x) {
    const uint32_t v = big[b];
    const uint32_t s = off[v], e = off[v + 1];
    uint32_t mant;
    int emin = 0x7FFFFFFF;
    for (uint32_t i = s + tid; i < e; i += 256) emin = min(emin, ulp_exponent(w[i], &mant));
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) emin = min(emin, __shfl_xor_sync(kFullMask, emin, d));
    if (lane == 0) s_min[wid] = emin;
    __syncthreads();
    emin = s_min[0];
#pragma unroll
    for (int t = 1; t < 8; ++t) emin = min(emin, s_min[t]);
    bool exact = true;
    unsigned long long carry = 0;
    if (emin == 0x7FFFFFFF) {
      for (uint32_t i = s + tid; i < e; i += 256) cum[i] = 0ull;
    } else {
      for (uint32_t base = s; base < e; base += 256) {
        const uint32_t i = base + tid;
        unsigned long long q = 0;
        bool ok = true;
        if (i < e) {
          const int ex = ulp_exponent(w[i], &mant);
          if (ex != 0x7FFFFFFF) {
            const int sh = ex - emin;
            if (sh > 29) ok = false;
            else q = (unsigned long long)mant << sh;
          }
        }
        if (!__syncthreads_and(ok)) {
          exact = false;
          break;
        }
        const unsigned long long wincl = warp_incl_scan_u64(q);
        if (lane == 31) s_tot[wid] = wincl;
        __syncthreads();
        unsigned long long before = carry, total = carry;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          if ((uint32_t)t < wid) before += s_tot[t];
          total += s_tot[t];
        }
        __syncthreads();                              // s_tot is rewritten by the next chunk
        if (total >= (1ull << 53)) {                  // the same decision in every thread
          exact = false;
          break;
        }
        if (i < e) cum[i] = lt_round_int(before + wincl, emin + 32);
        carry = total;
      }
    }
    double P = 0.0;
    if (emin == 0x7FFFFFFF) {
      P = 0.0;
    } else if (exact) {
      P = __dmul_rn(__ull2double_rn(carry), __longlong_as_double((long long)(emin + 1023) << 52));
    } else {
      if (tid == 0) s_P = lt_row_sequential(w, cum, s, e);
      __syncthreads();
      P = s_P;
    }
    if (tid == 0) lt_row_end(P, s, e, cum, bad);
    __syncthreads();                                  // shared words are reused by the next row
  }
  if (bad) atomicOr(flags, bad);
}

// Row-parallel check of the uploaded 64-bit offsets (non-decreasing), their
// narrowing to 32 bits, and the largest in-degree.
__global__ void prep_offsets_kernel(uint32_t n, const uint64_t *__restrict__ off64, uint32_t *__restrict__ off32,
                                    unsigned int *__restrict__ info) {
  uint32_t maxd = 0;
  for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v <= n; v += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t o = off64[v];
    off32[v] = (uint32_t)o;
    if (v > 0) {
      const uint64_t p = off64[v - 1];
      if (o < p) {
        atomicOr(info, kGraphBadOffsets);
        atomicMin(info + 1, (unsigned int)(v - 1));
      } else {
        const uint64_t d = o - p;
        maxd = max(maxd, d > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)d);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) maxd = max(maxd, __shfl_xor_sync(kFullMask, maxd, o));
  if ((threadIdx.x & 31u) == 0 && maxd) atomicMax(info + 2, maxd);
}

cudaError_t launch_offsets_prep(DevGraph &g, unsigned int *info, cudaStream_t s) {
  int blocks = (int)std::min<uint64_t>(((uint64_t)g.n + 256) / 256, 152ull * 8);
  if (blocks < 1) blocks = 1;
  prep_offsets_kernel<<<blocks, 256, 0, s>>>(g.n, g.off64, g.off, info);
  return cudaGetLastError();
}

cudaError_t launch_graph_prep(DevGraph &g, unsigned int *d_flags, cudaStream_t s) {
  const uint64_t m_pad = (g.m + 3) / 4 * 4 + 4;
  int blocks = (int)std::min<uint64_t>((m_pad + 255) / 256, 152ull * 16);
  if (blocks < 1) blocks = 1;
  prep_edges_kernel<<<blocks, 256, 0, s>>>(g.n, g.m, m_pad, g.src, g.w, g.thr, d_flags);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // the uploaded 64-bit offsets are no longer needed: their space holds the big-row list
  uint32_t *big = reinterpret_cast<uint32_t *>(g.off64);
  unsigned int *nbig = d_flags + 3;
  int rb = (int)std::min<uint64_t>(((uint64_t)g.n + 255) / 256, 152ull * 16);
  if (rb < 1) rb = 1;
  prep_rows_kernel<<<rb, 256, 0, s>>>(g.n, g.off, g.src, g.w, g.thr, g.rthr, g.rw, big, nbig, d_flags);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  prep_big_rows_kernel<<<152 * 8, 256, 0, s>>>(g.off, g.src, g.w, g.thr, g.rthr, g.rw, big, nbig, d_flags);
  return cudaGetLastError();
}

cudaError_t launch_lt_prep(DevGraph &g, unsigned int *d_flags, cudaStream_t s) {
  // the uploaded 64-bit offsets are no longer needed: their space holds the big-row list
  uint32_t *big = reinterpret_cast<uint32_t *>(g.off64);
  unsigned int *nbig = d_flags + 3;
  cudaError_t e = cudaMemsetAsync(nbig, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  int rb = (int)std::min<uint64_t>(((uint64_t)g.n + 255) / 256, 152ull * 16);
  if (rb < 1) rb = 1;
  prep_lt_kernel<<<rb, 256, 0, s>>>(g.n, g.off, g.w, g.cum, big, nbig, d_flags);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  prep_lt_big_kernel<<<152 * 8, 256, 0, s>>>(g.off, g.w, g.cum, big, nbig, d_flags);
  return cudaGetLastError();
}

}  // namespace gim
