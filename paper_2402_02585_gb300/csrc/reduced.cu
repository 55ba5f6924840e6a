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
// holding 12 or 16 classes. Amplitudes are scaled by sqrt(N)
// (u = sqrt(N) f, u_0 = 1) and the weights are w[c] = h[c] / N, so
// S / N = sum_c w[c] g(c) and P = w[0] |u(0)|^2 do not depend on N.
// Complex64 amplitudes with phase tables rounded to complex64 (as the
// statevector path); the sums over classes are FP32 per lane and
// double-float across the lane group.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.cuh"

namespace gq {

int phase_tables(const double *gammas, const double *betas, int64_t count, float2 *phase,
                 double2 *alpha, cudaStream_t st);
int sm_count();

namespace {

struct ReducedArgs {
  const uint64_t *hist;  // [B][stride]
  const float2 *phase;   // [A][256]
  const double2 *alpha;  // [A]
  double *out;           // [B][A][p][3]
  uint64_t nitems;       // B * A
  int stride;
  int n;
  int A;
  int p;
};

// Double-float butterfly over the kG lanes of an aligned lane group (every
// lane of the group ends with the same sum, in the same order for all groups).
template <int kG>
__device__ __forceinline__ void df_group(float &hi, float &lo) {
#pragma unroll
  for (int o = kG / 2; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    float s, e;
    two_sum(hi, h2, s, e);
    hi = s;
    lo = __fadd_rn(__fadd_rn(lo, l2), e);
  }
}

// One item = (instance, angle point) per group of kG lanes (a power of two up
// to 16; 32 / kG items per warp); lane l of a group holds the classes
// c = l + kG j, j < kJ, so kG kJ >= hist_stride. Small groups keep the
// per-round butterflies short: a round costs kJ classes of arithmetic per
// lane and log2(kG) butterfly steps for each of its three sums.
template <int kG, int kJ>
__global__ void __launch_bounds__(256) reduced_sweep_kernel(const __grid_constant__ ReducedArgs a) {
  constexpr int kPerWarp = 32 / kG;
  const int lane = threadIdx.x & 31, gl = lane % kG, g0 = lane - gl;
  const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x / 32);
  const double inv_n = ldexp(1.0, -a.n);
  for (uint64_t base = ((uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5)) * kPerWarp;
       base < a.nitems; base += nwarps * kPerWarp) {
    // a group past the last item repeats it (the shuffles need every lane)
    // and writes nothing
    const uint64_t want = base + (uint64_t)(lane / kG);
    const bool valid = want < a.nitems;
    const uint64_t item = valid ? want : a.nitems - 1;
    const uint64_t b = item / (uint64_t)a.A;
    const int ai = (int)(item % (uint64_t)a.A);
    const uint64_t *h = a.hist + b * (uint64_t)a.stride;
    float w[kJ];
    float2 T[kJ], u[kJ];
    int cs = 256;  // lowest non-empty class
#pragma unroll
    for (int j = 0; j < kJ; ++j) {
      const int c = gl + kG * j;
      const uint64_t hc = c < a.stride ? h[c] : 0ull;
      w[j] = (float)((double)hc * inv_n);
      T[j] = a.phase[(size_t)ai * 256 + c];
      u[j] = make_float2(1.f, 0.f);
      if (hc != 0ull && c < cs) cs = c;
    }
#pragma unroll
    for (int o = kG / 2; o > 0; o >>= 1) cs = min(cs, __shfl_xor_sync(0xffffffffu, cs, o));
    const int cs_lane = g0 + (cs & (kG - 1));
    const double2 al = a.alpha[ai];
    const float alr = (float)al.x, ali = (float)al.y;
    float2 ad = make_float2(0.f, 0.f);  // pending mixer add
    double *o = a.out + item * (uint64_t)a.p * 3;
    // round k's readouts are group-uniform; lane k mod kG of the group keeps
    // them and the group converts them to FP64 and stores them every kG
    // rounds, so every lane of a warp does the (slow) FP64 conversions at once
    float kp = 0.f, ke = 0.f, kel = 0.f, kd = 0.f;
    for (int k = 0; k < a.p; ++k) {
      // phase (with the previous round's mixer add), then S / N
      float sr = 0.f, si = 0.f;
#pragma unroll
      for (int j = 0; j < kJ; ++j) {
        const float2 x = cmul(T[j], make_float2(u[j].x + ad.x, u[j].y + ad.y));
        u[j] = x;
        sr = fmaf(w[j], x.x, sr);
        si = fmaf(w[j], x.y, si);
      }
      float lr = 0.f, li = 0.f;
      df_group<kG>(sr, lr);
      df_group<kG>(si, li);
      const float Sr = sr + lr, Si = si + li;
      const float2 am = make_float2(alr * Sr - ali * Si, alr * Si + ali * Sr);
      // readouts of f_k = g_k + a_k
      float e = 0.f, pz = 0.f, dm = 0.f;
#pragma unroll
      for (int j = 0; j < kJ; ++j) {
        const int c = gl + kG * j;
        const float yr = u[j].x + am.x, yi = u[j].y + am.y;
        const float q = w[j] * fmaf(yr, yr, yi * yi);
        e = fmaf((float)c, q, e);
        if (c == 0) pz = q;
        if (c == cs) dm = q;
      }
      float el = 0.f;
      df_group<kG>(e, el);
      pz = __shfl_sync(0xffffffffu, pz, g0);
      dm = __shfl_sync(0xffffffffu, dm, cs_lane);
      const int kr = k & (kG - 1);
      if (kr == gl) { kp = pz; ke = e; kel = el; kd = dm; }
      if (kr == kG - 1 || k + 1 == a.p) {
        const int kk = k - kr + gl;  // this lane's pending round
        if (valid && kk <= k) {
          o[3 * kk] = (double)kp;
          o[3 * kk + 1] = (double)ke + (double)kel;
          o[3 * kk + 2] = (double)kd;
        }
      }
      ad = am;
    }
  }
}

// best[b][k] = the angle point with the smallest <H_P> after round k + 1
// (the smallest index among equal values). One CTA of kArgThreads per (b, k);
// the reads of one (b, k) are p * 24 bytes apart, so each thread keeps
// several in flight.
constexpr int kArgThreads = 1024;

__global__ void __launch_bounds__(kArgThreads) reduced_argmin_kernel(const double *__restrict__ out,
                                                                     int A, int p,
                                                                     int32_t *__restrict__ best) {
  __shared__ double s_v[kArgThreads / 32];
  __shared__ int s_i[kArgThreads / 32];
  const int b = blockIdx.x / p, k = blockIdx.x % p;
  const double *col = out + ((size_t)b * A * p + k) * 3 + 1;
  double bv = INFINITY;
  int bi = 0x7fffffff;
#pragma unroll 8
  for (int ai = threadIdx.x; ai < A; ai += kArgThreads) {
    const double v = col[(size_t)ai * p * 3];
    if (v < bv) { bv = v; bi = ai; }  // ascending ai: the first minimum stays
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
    if (v2 < bv || (v2 == bv && i2 < bi)) { bv = v2; bi = i2; }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { s_v[warp] = bv; s_i[warp] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kArgThreads / 32; ++w)
      if (s_v[w] < bv || (s_v[w] == bv && s_i[w] < bi)) { bv = s_v[w]; bi = s_i[w]; }
    best[(size_t)b * p + k] = bi == 0x7fffffff ? -1 : bi;
  }
}

template <int kG, int kJ>
int launch_reduced(const ReducedArgs &args, cudaStream_t st) {
  auto kernel = reduced_sweep_kernel<kG, kJ>;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess ||
      per_sm < 1)
    return GQAOA_ECUDA;
  uint64_t blocks = (uint64_t)per_sm * (uint64_t)sm_count();
  const uint64_t per_block = 8ull * (32 / kG);  // items per CTA pass
  const uint64_t need = (args.nitems + per_block - 1) / per_block;
  if (need < blocks) blocks = need;
  kernel<<<(unsigned)blocks, 256, 0, st>>>(args);
  GQ_CHECK_LAUNCH();
  return GQAOA_OK;
}

size_t reduced_ws_layout(int A, char *base, float2 **phase, double2 **alpha) {
  const size_t o_alpha = round_up(sizeof(float2) * 256 * (size_t)A, 256);
  if (base) {
    *phase = reinterpret_cast<float2 *>(base);
    *alpha = reinterpret_cast<double2 *>(base + o_alpha);
  }
  return o_alpha + round_up(sizeof(double2) * (size_t)A, 256);
}

}  // namespace
}  // namespace gq

using namespace gq;

extern "C" int gqaoa_reduced_sweep_workspace_size(int angles, size_t *bytes) {
  if (!bytes) return GQAOA_EINVAL;
  if (angles < 1 || angles > (1 << 24)) return GQAOA_ERANGE;
  *bytes = reduced_ws_layout(angles, nullptr, nullptr, nullptr);
  return GQAOA_OK;
}

extern "C" int gqaoa_reduced_sweep(const uint64_t *hist, int hist_stride, int n, int batch,
                                   const double *gammas, const double *betas, int angles, int p,
                                   double *out, int32_t *best, void *ws, size_t ws_bytes,
                                   void *stream) {
  gq::NvtxRange nvtx_range("gqaoa_reduced_sweep");
  if (n < 1 || n > GQAOA_MAX_N || hist_stride < 1 || hist_stride > 256 || batch < 1 ||
      angles < 1 || angles > (1 << 24) || p < 1 || p > (1 << 20))
    return GQAOA_ERANGE;
  if ((uint64_t)batch * (uint64_t)angles > (1ull << 40)) return GQAOA_ERANGE;
  if (!hist || !gammas || !betas || !out || !ws) return GQAOA_EINVAL;
  if (!aligned8(hist) || !aligned8(gammas) || !aligned8(betas) || !aligned8(out) ||
      !aligned16(ws) || (best && (reinterpret_cast<uintptr_t>(best) & 3u) != 0))
    return GQAOA_EINVAL;
  if (ws_bytes < reduced_ws_layout(angles, nullptr, nullptr, nullptr)) return GQAOA_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float2 *phase = nullptr;
  double2 *alpha = nullptr;
  reduced_ws_layout(angles, static_cast<char *>(ws), &phase, &alpha);
  int rc = phase_tables(gammas, betas, angles, phase, alpha, st);
  if (rc) return rc;
  ReducedArgs args = {};
  args.hist = hist;
  args.phase = phase;
  args.alpha = alpha;
  args.out = out;
  args.nitems = (uint64_t)batch * (uint64_t)angles;
  args.stride = hist_stride;
  args.n = n;
  args.A = angles;
  args.p = p;
  // lane groups as small as 12 or 16 classes per lane allow: per item-round
  // a group issues about kG (14 kJ + 30 log2 kG) / 32 warp instructions
  if (hist_stride <= 16) rc = launch_reduced<1, 16>(args, st);
  else if (hist_stride <= 32) rc = launch_reduced<2, 16>(args, st);
  else if (hist_stride <= 48) rc = launch_reduced<4, 12>(args, st);
  else if (hist_stride <= 64) rc = launch_reduced<4, 16>(args, st);
  else if (hist_stride <= 96) rc = launch_reduced<8, 12>(args, st);
  else if (hist_stride <= 128) rc = launch_reduced<8, 16>(args, st);
  else if (hist_stride <= 192) rc = launch_reduced<16, 12>(args, st);
  else rc = launch_reduced<16, 16>(args, st);
  if (rc || !best) return rc;
  if ((uint64_t)batch * (uint64_t)p > 0x7fffffffull) return GQAOA_ERANGE;
  reduced_argmin_kernel<<<(unsigned)((uint64_t)batch * p), kArgThreads, 0, st>>>(out, angles, p,
                                                                          best);
  GQ_CHECK_LAUNCH();
  return GQAOA_OK;
}
