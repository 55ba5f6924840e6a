// K1: cost table C(z) and energy-manifold histogram h[c] (Eq. 1, Appendix B/C).
//
// A clause is violated exactly when each of its three literals is false:
// literal x_v is false when bit v of z is 0, literal NOT x_v when it is 1.
// With M = the clause's variable mask and F = the bits that falsify its
// literals, clause i is violated by z  <=>  ((z ^ F_i) & M_i) == 0, and
// C(z) = number of violated clauses.
//
// Bit-sliced evaluation. A thread owns 32-assignment words z = 32w + l
// (l = 0..31). Variables 0..4 vary inside a word with the fixed lane
// patterns 0xAAAAAAAA, 0xCCCCCCCC, 0xF0F0F0F0, 0xFF00FF00, 0xFFFF0000;
// variables >= 5 are constant inside it (bit v-5 of w). So clause i violates
// the lanes  V_i(w) = L_i  if ((w ^ Fh_i) & Mh_i) == 0, else 0,
// with L_i the AND of the low literals' falsifying patterns. The 1-bit lane
// vectors V_i are summed into bit-planes with a Harley-Seal carry-save tree
// (eight clauses -> ones/twos/fours planes + a ripple counter of eights),
// and the planes are transposed into one byte per assignment with three
// 8x8 bit-matrix delta swaps. The histogram is counted in per-warp shared
// bins and merged with one 64-bit atomic per bin per CTA (integer, exact).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "common.cuh"

namespace gq {

struct SlicedClauses {
  int m8;          // clause count padded to a multiple of 8 (padding: L = 0)
  int m;           // real clause count (histogram size m + 1)
  uint32_t L[256];
  uint32_t Mh[256];
  uint32_t Fh[256];
};

struct MaskClauses {
  int m;
  uint64_t M[255];
  uint64_t F[255];
};

constexpr int kCostWordsPerThread = 4;
constexpr int kCostThreads = 256;

__device__ __forceinline__ uint32_t lop_xor3(uint32_t a, uint32_t b, uint32_t c) { return a ^ b ^ c; }
__device__ __forceinline__ uint32_t lop_maj(uint32_t a, uint32_t b, uint32_t c) {
  return (a & b) | (c & (a | b));
}
// carry-save adder: (h, l) = a + b + c in two bit-planes
#define GQ_CSA(h, l, a, b, c)            \
  do {                                   \
    uint32_t _a = (a), _b = (b), _c = (c); \
    l = lop_xor3(_a, _b, _c);            \
    h = lop_maj(_a, _b, _c);             \
  } while (0)

// 8x8 bit-matrix transpose of a 64-bit word (row r = byte r): three delta swaps.
__device__ __forceinline__ uint64_t transpose8x8(uint64_t x) {
  uint64_t t;
  t = (x ^ (x >> 7)) & 0x00AA00AA00AA00AAull;
  x = x ^ t ^ (t << 7);
  t = (x ^ (x >> 14)) & 0x0000CCCC0000CCCCull;
  x = x ^ t ^ (t << 14);
  t = (x ^ (x >> 28)) & 0x00000000F0F0F0F0ull;
  x = x ^ t ^ (t << 28);
  return x;
}

template <bool kHist>
__global__ void __launch_bounds__(kCostThreads)
build_cost_sliced_kernel(const __grid_constant__ SlicedClauses cl, uint64_t nwords,
                         uint8_t *__restrict__ cost, unsigned long long *__restrict__ hist) {
  __shared__ uint4 s_cl[256];                 // (L, Mh, Fh, 0)
  __shared__ uint32_t s_hist[kCostThreads / 32][256];
  const int warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < cl.m8; i += blockDim.x)
    s_cl[i] = make_uint4(cl.L[i], cl.Mh[i], cl.Fh[i], 0u);
  for (int i = threadIdx.x; i < (kCostThreads / 32) * 256; i += blockDim.x)
    (&s_hist[0][0])[i] = 0u;
  __syncthreads();

  // words of this thread: base + threadIdx.x + j * blockDim.x
  const uint64_t base = (uint64_t)blockIdx.x * (kCostThreads * kCostWordsPerThread);
  uint32_t w[kCostWordsPerThread];
  bool valid[kCostWordsPerThread];
#pragma unroll
  for (int j = 0; j < kCostWordsPerThread; ++j) {
    uint64_t ww = base + threadIdx.x + (uint64_t)j * kCostThreads;
    valid[j] = ww < nwords;
    w[j] = (uint32_t)ww;
  }

  uint32_t ones[kCostWordsPerThread], twos[kCostWordsPerThread], fours[kCostWordsPerThread];
  uint32_t e[5][kCostWordsPerThread];  // ripple counter of eights (planes 3..7)
#pragma unroll
  for (int j = 0; j < kCostWordsPerThread; ++j) {
    ones[j] = twos[j] = fours[j] = 0u;
#pragma unroll
    for (int b = 0; b < 5; ++b) e[b][j] = 0u;
  }

  for (int i = 0; i < cl.m8; i += 8) {
    uint4 c[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) c[q] = s_cl[i + q];
#pragma unroll
    for (int j = 0; j < kCostWordsPerThread; ++j) {
      uint32_t v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = (((w[j] ^ c[q].z) & c[q].y) == 0u) ? c[q].x : 0u;
      uint32_t twosA, twosB, foursA, foursB, eights;
      GQ_CSA(twosA, ones[j], ones[j], v[0], v[1]);
      GQ_CSA(twosB, ones[j], ones[j], v[2], v[3]);
      GQ_CSA(foursA, twos[j], twos[j], twosA, twosB);
      GQ_CSA(twosA, ones[j], ones[j], v[4], v[5]);
      GQ_CSA(twosB, ones[j], ones[j], v[6], v[7]);
      GQ_CSA(foursB, twos[j], twos[j], twosA, twosB);
      GQ_CSA(eights, fours[j], fours[j], foursA, foursB);
      // ripple-add the eights plane into the counter of planes 3..7
      uint32_t carry = eights;
#pragma unroll
      for (int b = 0; b < 5; ++b) {
        uint32_t t = e[b][j] & carry;
        e[b][j] ^= carry;
        carry = t;
      }
    }
  }

  // transpose bit-planes -> bytes, store, and count
#pragma unroll
  for (int j = 0; j < kCostWordsPerThread; ++j) {
    if (!valid[j]) continue;
    const uint32_t pl[8] = {ones[j], twos[j], fours[j], e[0][j], e[1][j], e[2][j], e[3][j], e[4][j]};
    uint32_t outw[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      // row b of the 8x8 matrix = byte k of plane b
      uint32_t lo = 0u, hi = 0u;
#pragma unroll
      for (int b = 0; b < 4; ++b) lo |= ((pl[b] >> (8 * k)) & 0xFFu) << (8 * b);
#pragma unroll
      for (int b = 0; b < 4; ++b) hi |= ((pl[b + 4] >> (8 * k)) & 0xFFu) << (8 * b);
      uint64_t x = transpose8x8(((uint64_t)hi << 32) | lo);
      outw[2 * k] = (uint32_t)x;
      outw[2 * k + 1] = (uint32_t)(x >> 32);
    }
    uint4 *dst = reinterpret_cast<uint4 *>(cost + (uint64_t)w[j] * 32u);
    dst[0] = make_uint4(outw[0], outw[1], outw[2], outw[3]);
    dst[1] = make_uint4(outw[4], outw[5], outw[6], outw[7]);
    if (kHist) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
#pragma unroll
        for (int s = 0; s < 4; ++s) atomicAdd(&s_hist[warp][(outw[q] >> (8 * s)) & 0xFFu], 1u);
      }
    }
  }
  if (!kHist) return;
  __syncthreads();
  for (int c = threadIdx.x; c <= cl.m; c += blockDim.x) {
    unsigned long long t = 0;
#pragma unroll
    for (int wv = 0; wv < kCostThreads / 32; ++wv) t += s_hist[wv][c];
    if (t) atomicAdd(&hist[c], t);
  }
}

// Plain per-assignment evaluation for small tables (N < 2^12).
template <bool kHist>
__global__ void __launch_bounds__(kCostThreads)
build_cost_small_kernel(const __grid_constant__ MaskClauses cl, uint64_t N,
                        uint8_t *__restrict__ cost, unsigned long long *__restrict__ hist) {
  __shared__ uint32_t s_hist[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) s_hist[i] = 0u;
  __syncthreads();
  for (uint64_t z = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; z < N;
       z += (uint64_t)gridDim.x * blockDim.x) {
    int c = 0;
    for (int i = 0; i < cl.m; ++i) c += ((z ^ cl.F[i]) & cl.M[i]) == 0ull;
    cost[z] = (uint8_t)c;
    if (kHist) atomicAdd(&s_hist[c], 1u);
  }
  if (!kHist) return;
  __syncthreads();
  for (int c = threadIdx.x; c <= cl.m; c += blockDim.x)
    if (s_hist[c]) atomicAdd(&hist[c], (unsigned long long)s_hist[c]);
}

}  // namespace gq

using namespace gq;

static const uint32_t kLanePattern[5] = {0xAAAAAAAAu, 0xCCCCCCCCu, 0xF0F0F0F0u, 0xFF00FF00u,
                                         0xFFFF0000u};

extern "C" int gqaoa_build_cost(const int32_t *lits, int n, int m, uint8_t *cost, uint64_t *hist,
                                void *stream) {
  gq::NvtxRange nvtx_range("gqaoa_build_cost");
  if (n < 1 || n > GQAOA_MAX_N || m < 0 || m > GQAOA_MAX_M) return GQAOA_ERANGE;
  if (!cost || (m > 0 && !lits)) return GQAOA_EINVAL;
  for (int i = 0; i < 3 * m; ++i) {
    int32_t l = lits[i];
    if (l == 0 || l > n || l < -n) return GQAOA_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint64_t N = 1ull << n;
  unsigned long long *h = reinterpret_cast<unsigned long long *>(hist);
  if (h) GQ_CUDA(cudaMemsetAsync(h, 0, sizeof(uint64_t) * (size_t)(m + 1), st));

  if (n >= 12) {
    if (!aligned16(cost)) return GQAOA_EINVAL;
    SlicedClauses sc;
    memset(&sc, 0, sizeof(sc));
    sc.m = m;
    sc.m8 = (m + 7) / 8 * 8;
    for (int i = 0; i < m; ++i) {
      uint32_t L = 0xFFFFFFFFu, Mh = 0u, Fh = 0u;
      for (int j = 0; j < 3; ++j) {
        int32_t l = lits[3 * i + j];
        int v = (l > 0 ? l : -l) - 1;
        bool falsify_one = l < 0;  // NOT x_v is false when x_v = 1
        if (v < 5) {
          L &= falsify_one ? kLanePattern[v] : ~kLanePattern[v];
        } else {
          Mh |= 1u << (v - 5);
          if (falsify_one) Fh |= 1u << (v - 5);
        }
      }
      sc.L[i] = L;
      sc.Mh[i] = Mh;
      sc.Fh[i] = Fh;
    }
    // padding clauses: L = 0 -> never violated
    const uint64_t nwords = N / 32;
    const uint64_t per_cta = (uint64_t)kCostThreads * kCostWordsPerThread;
    const uint64_t grid = (nwords + per_cta - 1) / per_cta;
    if (h)
      build_cost_sliced_kernel<true><<<(unsigned)grid, kCostThreads, 0, st>>>(sc, nwords, cost, h);
    else
      build_cost_sliced_kernel<false><<<(unsigned)grid, kCostThreads, 0, st>>>(sc, nwords, cost, h);
  } else {
    MaskClauses mc;
    memset(&mc, 0, sizeof(mc));
    mc.m = m;
    for (int i = 0; i < m; ++i) {
      uint64_t M = 0, F = 0;
      for (int j = 0; j < 3; ++j) {
        int32_t l = lits[3 * i + j];
        int v = (l > 0 ? l : -l) - 1;
        M |= 1ull << v;
        if (l < 0) F |= 1ull << v;
      }
      mc.M[i] = M;
      mc.F[i] = F;
    }
    unsigned grid = (unsigned)((N + kCostThreads - 1) / kCostThreads);
    if (h)
      build_cost_small_kernel<true><<<grid, kCostThreads, 0, st>>>(mc, N, cost, h);
    else
      build_cost_small_kernel<false><<<grid, kCostThreads, 0, st>>>(mc, N, cost, h);
  }
  GQ_CHECK_LAUNCH();
  return GQAOA_OK;
}
