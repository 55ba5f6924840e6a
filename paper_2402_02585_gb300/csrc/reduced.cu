// Cost-class (reduced) model of single-angle-pair G-QAOA on the GPU.
//
// Appendix C: G-QAOA does not distinguish the assignments inside one energy
// manifold, so from |+> the state stays a function of the cost value,
// psi_k(z) = f_k(C(z)), and a round (Eq. 3) acts on the m + 1 class
// amplitudes, weighted by the manifold sizes h[c]:
//     g_k(c) = e^{-i gamma c} f_{k-1}(c),  f_k(c) = g_k(c) + alpha S_k / N,
//     S_k = sum_c h[c] g_k(c),  alpha = e^{-i beta} - 1.
// This is the paper's own fast path (the O(2^n) cost table is built once,
// then every evolution costs O(p m)); it serves the angle grid searches of
// the paper's protocol (Appendix C: a pi/180 grid, or 4000 random points
// above n = 20), while the statevector kernels remain the evolution itself.
//
// One group of 1..16 lanes per (instance, angle point) item, each lane
// holding 8, 12 or 16 classes of a window that starts at the row's lowest
// non-empty class c_min (classes below it are empty and stay out of every
// sum), so P(C = 0) and the Max-SAT weight D both sit in the group's first
// slot. Amplitudes are scaled by sqrt(N) (u = sqrt(N) f, u_0 = 1) and the
// weights are w[c] = h[c] / N, so S / N = sum_c w[c] g(c) and
// P = w[0] |u(0)|^2 do not depend on N. Complex64 amplitudes with phase tables
// rounded to complex64 (as the statevector path); the sums over classes are
// FP32, per lane and across the lane group.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.cuh"

namespace gq {

int phase_tables(const double *gammas, const double *betas, int64_t count, int entries,
                 float2 *phase, double2 *alpha, cudaStream_t st);
int sm_count();

namespace {

struct ReducedArgs {
  const float *wt;             // [B][tstride]: w of class c_min(b) + s, s < tstride
  const float *cwt;            // [B][tstride]: c w of the same classes
  const int32_t *cmin;         // [B]: lowest non-empty class
  const float2 *phase;         // [A][tstride]
  const double2 *alpha;        // [A]
  float *out;                  // [B][p][3][A]
  unsigned long long *keys;    // [B][p] minima of warps spanning instances, or null
  unsigned long long *part;    // [p][nblocks] minima of the other warps
  uint64_t nitems;             // B * A
  uint64_t nblocks;            // warp item blocks, ceil(nitems / (32 / kG))
  int tstride;                 // entries per phase table and weight row (>= hist_stride)
  int A;
  int p;
};

constexpr int kRedThreads = 64;  // two warps per CTA: fine-grained placement over the SMs

// Per instance (one warp per row): the lowest non-empty class and the FP32
// weight rows, shifted to start there; and the running minima set to "none".
__global__ void reduced_prep_kernel(const uint64_t *__restrict__ hist, int stride, int tstride,
                                    int n, int B, float *__restrict__ wt, float *__restrict__ cwt,
                                    int32_t *__restrict__ cmin, unsigned long long *keys,
                                    uint64_t nkeys) {
  const int lane = threadIdx.x & 31;
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const double inv_n = ldexp(1.0, -n);
  for (uint64_t b = gw; b < (uint64_t)B; b += nw) {
    const uint64_t *h = hist + b * (uint64_t)stride;
    int cs = 256;
    for (int c0 = 0; c0 < stride && cs == 256; c0 += 32) {
      const unsigned nz =
          __ballot_sync(0xffffffffu, c0 + lane < stride && h[c0 + lane] != 0ull);
      if (nz) cs = c0 + __ffs(nz) - 1;
    }
    if (lane == 0) cmin[b] = cs;
    for (int s = lane; s < tstride; s += 32) {
      const int c = cs + s;
      const uint64_t hc = c < stride ? h[c] : 0ull;
      wt[b * (uint64_t)tstride + s] = (float)((double)hc * inv_n);
      cwt[b * (uint64_t)tstride + s] = (float)((double)c * (double)hc * inv_n);
    }
  }
  if (keys)
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nkeys;
         i += (uint64_t)gridDim.x * blockDim.x)
      keys[i] = ~0ull;
}

// FP32 butterfly over the kG lanes of an aligned lane group: every lane ends
// with the same sum (each step adds the same two values in either order).
template <int kG>
__device__ __forceinline__ float group_fsum(float v) {
#pragma unroll
  for (int o = kG / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Order-preserving image of a float's bits (negative values below positive
// ones, -0 equal to +0, NaN above everything), so the unsigned minimum is the
// smallest value.
__device__ __forceinline__ uint32_t order_key(float v) {
  uint32_t b = __float_as_uint(v);
  if (b == 0x80000000u) b = 0u;
  uint32_t k = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
  if ((b & 0x7fffffffu) > 0x7f800000u) k = 0xffffffffu;
  return k;
}

// Packed minimum key: order_key of <H_P> in the high word, the angle point in
// the low word, so the unsigned 64-bit minimum is the smallest value and,
// among equal values, the first point.
__device__ __forceinline__ unsigned long long pack_key(uint32_t k, int ai) {
  return ((unsigned long long)k << 32) | (uint32_t)ai;
}

// Whether the warp item block [wb ipw, (wb + 1) ipw) (cut at nitems) lies in
// one instance, and which.
__device__ __forceinline__ bool block_instance(uint64_t wb, int ipw, uint64_t nitems, int A,
                                               uint64_t *b) {
  const uint64_t first = wb * (uint64_t)ipw;
  const uint64_t last = (first + ipw < nitems ? first + ipw : nitems) - 1;
  *b = first / (uint64_t)A;
  return *b == last / (uint64_t)A;
}

// One item = (instance, angle point) per group of kG lanes (a power of two up
// to 16; 32 / kG items per warp, consecutive angle points); lane l of a group
// holds the classes c = c_min + l + kG j, j < kJ, so kG kJ >= hist_stride
// covers every non-empty class. A round costs per slot a complex multiply and
// the S sum (6 FP32 instructions), the mixer add and the <H_P> term (5), plus
// log2(kG) butterfly steps for each of the three group sums. The readouts
// (FP32, as computed) are stored round-major ([B][p][3][A]), so a warp's
// stores of one round cover contiguous angle points; the per-round minimum of a warp whose items lie in
// one instance goes to its own slot of `part` (no atomics), that of a warp
// spanning instances to `keys` by atomic minimum.
template <int kG, int kJ>
__global__ void __launch_bounds__(kRedThreads, 8) reduced_sweep_kernel(const __grid_constant__ ReducedArgs a) {
  constexpr int kPerWarp = 32 / kG;
  const int lane = threadIdx.x & 31, gl = lane % kG;
  const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x / 32);
  for (uint64_t base = ((uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5)) * kPerWarp;
       base < a.nitems; base += nwarps * kPerWarp) {
    // a group past the last item repeats it (the shuffles need every lane)
    // and writes nothing
    const uint64_t want = base + (uint64_t)(lane / kG);
    const bool valid = want < a.nitems;
    const uint64_t item = valid ? want : a.nitems - 1;
    const uint64_t b = item / (uint64_t)a.A;
    const int ai = (int)(item % (uint64_t)a.A);
    const int cs = a.cmin[b];
    const float *wr = a.wt + b * (uint64_t)a.tstride, *cwr = a.cwt + b * (uint64_t)a.tstride;
    const float2 *tab = a.phase + (size_t)ai * a.tstride;
    float w[kJ], cw[kJ];
    float2 T[kJ], u[kJ];
#pragma unroll
    for (int j = 0; j < kJ; ++j) {
      const int s = gl + kG * j, c = cs + s;  // s < kG kJ <= tstride
      w[j] = wr[s];
      cw[j] = cwr[s];
      T[j] = tab[c < a.tstride ? c : a.tstride - 1];  // any finite entry for an empty slot
      u[j] = make_float2(1.f, 0.f);
    }
    const double2 al = a.alpha[ai];
    const float alr = (float)al.x, ali = (float)al.y;
    // round k's readout f of this item at o[(3 k + f) A]
    float *o = a.out + b * (uint64_t)a.p * 3 * (uint64_t)a.A + (uint64_t)ai;
    const uint64_t stride_f = (uint64_t)a.A;
    const uint64_t wb = base / kPerWarp;
    uint64_t b_block;
    const bool pure = block_instance(wb, kPerWarp, a.nitems, a.A, &b_block);
    unsigned long long *key = a.keys ? a.keys + b * (uint64_t)a.p : nullptr;
    unsigned long long *part = a.part + wb;
    for (int k = 0; k < a.p; ++k) {
      // phase, then S / N
      float sr = 0.f, si = 0.f;
#pragma unroll
      for (int j = 0; j < kJ; ++j) {
        const float2 x = cmul(T[j], u[j]);
        u[j] = x;
        sr = fmaf(w[j], x.x, sr);
        si = fmaf(w[j], x.y, si);
      }
      sr = group_fsum<kG>(sr);
      si = group_fsum<kG>(si);
      const float2 am = make_float2(alr * sr - ali * si, alr * si + ali * sr);
      // mixer add, f_k = g_k + a_k, and <H_P> = sum_c c w_c |f_k(c)|^2
      float e = 0.f;
#pragma unroll
      for (int j = 0; j < kJ; ++j) {
        u[j].x += am.x;
        u[j].y += am.y;
        e = fmaf(cw[j], fmaf(u[j].x, u[j].x, u[j].y * u[j].y), e);
      }
      e = group_fsum<kG>(e);
      // D = w |f(c_min)|^2 from the group's first slot; P = D when c_min = 0,
      // else class 0 is empty and P = 0
      const float d = w[0] * fmaf(u[0].x, u[0].x, u[0].y * u[0].y);
      if (gl == 0 && valid) {
        o[0] = cs == 0 ? d : 0.f;
        o[stride_f] = e;
        o[2 * stride_f] = d;
      }
      o += 3 * stride_f;
      if (key) {
        const uint32_t kv = valid ? order_key(e) : 0xffffffffu;
        if (pure) {
          // the warp's smallest key and the first lane holding it (items
          // ascend with the lane, so that is the smallest angle point)
          const uint32_t kmin = __reduce_min_sync(0xffffffffu, kv);
          const int first = __ffs(__ballot_sync(0xffffffffu, kv == kmin)) - 1;
          const int a_first = __shfl_sync(0xffffffffu, ai, first);
          if (lane == 0) part[(uint64_t)k * a.nblocks] = pack_key(kmin, a_first);
        } else if (gl == 0 && valid) {
          atomicMin(key + k, pack_key(kv, ai));
        }
      }
    }
  }
}

// best[b][k] = the angle point of the minimum over the warps of instance b
// (their `part` slots) and the atomics of the warps spanning instances
// (`keys`); -1 where every value was NaN. One CTA per (b, k), its threads
// reading that round's row of `part` side by side.
constexpr int kBestThreads = 256;

__global__ void __launch_bounds__(kBestThreads)
reduced_best_kernel(const unsigned long long *__restrict__ keys,
                    const unsigned long long *__restrict__ part, uint64_t nblocks, int ipw,
                    uint64_t nitems, int A, int B, int p, int32_t *__restrict__ best) {
  __shared__ unsigned long long s_min[kBestThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint64_t i = blockIdx.x; i < (uint64_t)B * (uint64_t)p; i += gridDim.x) {
    const uint64_t b = i / (uint64_t)p, k = i % (uint64_t)p;
    // the blocks that lie in instance b (block_instance's test): first item
    // at or after b A, last item (cut at nitems) before (b + 1) A
    const uint64_t lo = (b * (uint64_t)A + ipw - 1) / (uint64_t)ipw;
    const uint64_t hi = (b + 1) * (uint64_t)A == nitems
                            ? nblocks
                            : (b + 1) * (uint64_t)A / (uint64_t)ipw;
    unsigned long long m = ~0ull;
    const unsigned long long *row = part + k * nblocks;
#pragma unroll 4
    for (uint64_t wb = lo + threadIdx.x; wb < hi; wb += kBestThreads) {
      const unsigned long long v = row[wb];
      m = v < m ? v : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
      m = v < m ? v : m;
    }
    if (lane == 0) s_min[warp] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 0; w < kBestThreads / 32; ++w) m = s_min[w] < m ? s_min[w] : m;
      const unsigned long long v = keys[i];
      m = v < m ? v : m;
      best[i] = (uint32_t)(m >> 32) == 0xffffffffu ? -1 : (int32_t)(uint32_t)m;
    }
    __syncthreads();  // s_min is rewritten for the next (b, k)
  }
}

template <int kG, int kJ>
int launch_reduced(const ReducedArgs &args, cudaStream_t st) {
  auto kernel = reduced_sweep_kernel<kG, kJ>;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kRedThreads, 0) !=
          cudaSuccess ||
      per_sm < 1)
    return GQAOA_ECUDA;
  uint64_t blocks = (uint64_t)per_sm * (uint64_t)sm_count();
  const uint64_t per_block = (kRedThreads / 32) * (32 / kG);  // items per CTA pass
  const uint64_t need = (args.nitems + per_block - 1) / per_block;
  if (need < blocks) blocks = need;
  kernel<<<(unsigned)blocks, kRedThreads, 0, st>>>(args);
  GQ_CHECK_LAUNCH();
  return GQAOA_OK;
}

struct ReducedWs {
  float2 *phase;                // [A][tstride]
  double2 *alpha;               // [A]
  unsigned long long *keys;     // [B][p]
  unsigned long long *part;     // [p][nblocks]
  float *wt, *cwt;              // [B][tstride]
  int32_t *cmin;                // [B]
};

int table_entries(int hist_stride) { return (int)round_up((size_t)hist_stride, 32); }

// lanes per item of the kernel shape chosen for hist_stride (below)
int group_lanes(int hist_stride) {
  if (hist_stride <= 16) return 1;
  if (hist_stride <= 32) return 2;
  if (hist_stride <= 64) return 4;
  if (hist_stride <= 128) return 8;
  return 16;
}

uint64_t item_blocks(int hist_stride, int B, int A) {
  const uint64_t ipw = 32 / group_lanes(hist_stride);
  return ((uint64_t)B * (uint64_t)A + ipw - 1) / ipw;
}

size_t reduced_ws_layout(int hist_stride, int B, int A, int p, char *base, ReducedWs *w) {
  const size_t ts = (size_t)table_entries(hist_stride);
  const size_t o_alpha = round_up(sizeof(float2) * ts * (size_t)A, 256);
  const size_t o_keys = o_alpha + round_up(sizeof(double2) * (size_t)A, 256);
  const size_t o_part = o_keys + round_up(sizeof(unsigned long long) * (size_t)B * (size_t)p, 256);
  const size_t o_wt = o_part + round_up(sizeof(unsigned long long) * (size_t)p *
                                            (size_t)item_blocks(hist_stride, B, A), 256);
  const size_t o_cwt = o_wt + round_up(sizeof(float) * ts * (size_t)B, 256);
  const size_t o_cmin = o_cwt + round_up(sizeof(float) * ts * (size_t)B, 256);
  if (base) {
    w->phase = reinterpret_cast<float2 *>(base);
    w->alpha = reinterpret_cast<double2 *>(base + o_alpha);
    w->keys = reinterpret_cast<unsigned long long *>(base + o_keys);
    w->part = reinterpret_cast<unsigned long long *>(base + o_part);
    w->wt = reinterpret_cast<float *>(base + o_wt);
    w->cwt = reinterpret_cast<float *>(base + o_cwt);
    w->cmin = reinterpret_cast<int32_t *>(base + o_cmin);
  }
  return o_cmin + round_up(sizeof(int32_t) * (size_t)B, 256);
}

int check_shape(int hist_stride, int batch, int angles, int p) {
  if (hist_stride < 1 || hist_stride > 256 || batch < 1 || angles < 1 || angles > (1 << 24) ||
      p < 1 || p > (1 << 20))
    return GQAOA_ERANGE;
  if ((uint64_t)batch * (uint64_t)angles > (1ull << 40)) return GQAOA_ERANGE;
  if ((uint64_t)batch * (uint64_t)p > 0x7fffffffull) return GQAOA_ERANGE;
  return GQAOA_OK;
}

}  // namespace
}  // namespace gq

using namespace gq;

extern "C" int gqaoa_reduced_sweep_workspace_size(int hist_stride, int batch, int angles, int p,
                                                  size_t *bytes) {
  if (!bytes) return GQAOA_EINVAL;
  const int rc = check_shape(hist_stride, batch, angles, p);
  if (rc) return rc;
  *bytes = reduced_ws_layout(hist_stride, batch, angles, p, nullptr, nullptr);
  return GQAOA_OK;
}

extern "C" int gqaoa_reduced_sweep(const uint64_t *hist, int hist_stride, int n, int batch,
                                   const double *gammas, const double *betas, int angles, int p,
                                   float *out, int32_t *best, void *ws, size_t ws_bytes,
                                   void *stream) {
  gq::NvtxRange nvtx_range("gqaoa_reduced_sweep");
  if (n < 1 || n > GQAOA_MAX_N) return GQAOA_ERANGE;
  int rc = check_shape(hist_stride, batch, angles, p);
  if (rc) return rc;
  if (!hist || !gammas || !betas || !out || !ws) return GQAOA_EINVAL;
  if (!aligned8(hist) || !aligned8(gammas) || !aligned8(betas) ||
      (reinterpret_cast<uintptr_t>(out) & 3u) != 0 || !aligned16(ws) ||
      (best && (reinterpret_cast<uintptr_t>(best) & 3u) != 0))
    return GQAOA_EINVAL;
  if (ws_bytes < reduced_ws_layout(hist_stride, batch, angles, p, nullptr, nullptr))
    return GQAOA_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ReducedWs w = {};
  reduced_ws_layout(hist_stride, batch, angles, p, static_cast<char *>(ws), &w);
  const int entries = table_entries(hist_stride);
  rc = phase_tables(gammas, betas, angles, entries, w.phase, w.alpha, st);
  if (rc) return rc;
  const uint64_t nkeys = (uint64_t)batch * (uint64_t)p;
  const uint64_t prep_warps = (uint64_t)batch > nkeys / 32 ? (uint64_t)batch : nkeys / 32;
  const unsigned prep_grid = (unsigned)(prep_warps < 8ull * 1024 ? (prep_warps + 7) / 8 : 1024);
  reduced_prep_kernel<<<prep_grid, 256, 0, st>>>(hist, hist_stride, entries, n, batch, w.wt,
                                                 w.cwt, w.cmin, best ? w.keys : nullptr, nkeys);
  GQ_CHECK_LAUNCH();
  ReducedArgs args = {};
  args.wt = w.wt;
  args.cwt = w.cwt;
  args.cmin = w.cmin;
  args.phase = w.phase;
  args.alpha = w.alpha;
  args.out = out;
  args.keys = best ? w.keys : nullptr;
  args.part = w.part;
  args.nitems = (uint64_t)batch * (uint64_t)angles;
  args.nblocks = item_blocks(hist_stride, batch, angles);
  args.tstride = entries;
  args.A = angles;
  args.p = p;
  // the smallest lane group whose 8, 12 or 16 classes per lane hold the row
  // (group_lanes above gives the same lane counts)
  if (hist_stride <= 8) rc = launch_reduced<1, 8>(args, st);
  else if (hist_stride <= 12) rc = launch_reduced<1, 12>(args, st);
  else if (hist_stride <= 16) rc = launch_reduced<1, 16>(args, st);
  else if (hist_stride <= 24) rc = launch_reduced<2, 12>(args, st);
  else if (hist_stride <= 32) rc = launch_reduced<2, 16>(args, st);
  else if (hist_stride <= 48) rc = launch_reduced<4, 12>(args, st);
  else if (hist_stride <= 64) rc = launch_reduced<4, 16>(args, st);
  else if (hist_stride <= 96) rc = launch_reduced<8, 12>(args, st);
  else if (hist_stride <= 128) rc = launch_reduced<8, 16>(args, st);
  else if (hist_stride <= 192) rc = launch_reduced<16, 12>(args, st);
  else rc = launch_reduced<16, 16>(args, st);
  if (rc || !best) return rc;
  const unsigned best_grid = (unsigned)(nkeys < 4096ull ? nkeys : 4096ull);
  reduced_best_kernel<<<best_grid, kBestThreads, 0, st>>>(w.keys, w.part, args.nblocks,
                                                 32 / group_lanes(hist_stride), args.nitems,
                                                 angles, batch, p, best);
  GQ_CHECK_LAUNCH();
  return GQAOA_OK;
}
