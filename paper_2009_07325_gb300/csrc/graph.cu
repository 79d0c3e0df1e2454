// Graph preprocessing on the device: validation of the in-edge CSR, the IC
// coin thresholds and the LT cumulative thresholds (Sec. III-B CSR layout;
// Sec. III-G LT edge choice).
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

// Row-parallel: ascending sources within a row, and the LT thresholds.
// cum[e_i] = min(2^32, round_half_up(P_i * 2^32)), P_i the fp64 running sum of
// the row's weights in CSR order; a row summing to within 1e-6 of 1 gets
// cum[last] = 2^32 so that it always selects an edge. A row summing above
// 1 + 1e-6 marks the graph as not valid for LT.
__global__ void prep_rows_kernel(uint32_t n, const uint32_t *__restrict__ off, const uint32_t *__restrict__ src,
                                 const float *__restrict__ w, uint64_t *__restrict__ cum,
                                 unsigned int *__restrict__ flags) {
  unsigned int bad = 0;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const uint32_t s = off[v], e = off[v + 1];
    double P = 0.0;
    for (uint32_t i = s; i < e; ++i) {
      if (i > s && !(src[i - 1] < src[i])) bad |= kGraphNotAscending;
      P = __dadd_rn(P, (double)w[i]);
      const double x = __dmul_rn(P, 4294967296.0);
      const double f = floor(x);
      unsigned long long c = (unsigned long long)f;
      if (__dsub_rn(x, f) >= 0.5) c += 1ull;
      if (c > 4294967296ull) c = 4294967296ull;
      cum[i] = c;
    }
    if (e > s && fabs(__dsub_rn(P, 1.0)) <= 1e-6) cum[e - 1] = 4294967296ull;
    if (P > 1.0 + 1e-6) bad |= kGraphNotLT;
  }
  if (bad) atomicOr(flags, bad);
}

cudaError_t launch_graph_prep(DevGraph &g, const float *d_w, unsigned int *d_flags, cudaStream_t s) {
  const uint64_t m_pad = (g.m + 3) / 4 * 4 + 4;
  int blocks = (int)std::min<uint64_t>((m_pad + 255) / 256, 152ull * 16);
  if (blocks < 1) blocks = 1;
  prep_edges_kernel<<<blocks, 256, 0, s>>>(g.n, g.m, m_pad, g.src, d_w, g.thr, d_flags);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int rb = (int)std::min<uint64_t>((g.n + 127) / 128, 152ull * 32);
  if (rb < 1) rb = 1;
  prep_rows_kernel<<<rb, 128, 0, s>>>(g.n, g.off, g.src, d_w, g.cum, d_flags);
  return cudaGetLastError();
}

}  // namespace gim
