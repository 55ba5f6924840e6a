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
// One warp per (instance, angle point) item; lane l holds the classes
// c = l + 32 j. Amplitudes are scaled by sqrt(N) (u = sqrt(N) f, u_0 = 1) and
// the weights are w[c] = h[c] / N, so S / N = sum_c w[c] g(c) and
// P = w[0] |u(0)|^2 do not depend on N. Complex64 amplitudes with FP64 phase
// tables rounded to complex64 (as the statevector path); the sums over
// classes are FP32 per lane and double-float across the warp.
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

__device__ __forceinline__ void df_warp32(float &hi, float &lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    float s, e;
    two_sum(hi, h2, s, e);
    hi = s;
    lo = __fadd_rn(__fadd_rn(lo, l2), e);
  }
}

template <int kJ>
__global__ void __launch_bounds__(256) reduced_sweep_kernel(const __grid_constant__ ReducedArgs a) {
  const int lane = threadIdx.x & 31;
  const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x / 32);
  const double inv_n = ldexp(1.0, -a.n);
  for (uint64_t item = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
       item < a.nitems; item += nwarps) {
    const uint64_t b = item / (uint64_t)a.A;
    const int ai = (int)(item % (uint64_t)a.A);
    const uint64_t *h = a.hist + b * (uint64_t)a.stride;
    float w[kJ];
    float2 T[kJ], u[kJ];
    int cs = 256;  // lowest non-empty class
#pragma unroll
    for (int j = 0; j < kJ; ++j) {
      const int c = lane + 32 * j;
      const uint64_t hc = c < a.stride ? h[c] : 0ull;
      w[j] = (float)((double)hc * inv_n);
      T[j] = a.phase[(size_t)ai * 256 + c];
      u[j] = make_float2(1.f, 0.f);
      const unsigned bal = __ballot_sync(0xffffffffu, hc != 0ull);
      if (bal != 0u && cs == 256) cs = 32 * j + __ffs(bal) - 1;
    }
    const double2 al = a.alpha[ai];
    const float alr = (float)al.x, ali = (float)al.y;
    float2 ad = make_float2(0.f, 0.f);  // pending mixer add
    double *o = a.out + item * (uint64_t)a.p * 3;
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
      df_warp32(sr, lr);
      df_warp32(si, li);
      const float Sr = sr + lr, Si = si + li;
      const float2 am = make_float2(alr * Sr - ali * Si, alr * Si + ali * Sr);
      // readouts of f_k = g_k + a_k
      float e = 0.f, pz = 0.f, dm = 0.f;
#pragma unroll
      for (int j = 0; j < kJ; ++j) {
        const int c = lane + 32 * j;
        const float yr = u[j].x + am.x, yi = u[j].y + am.y;
        const float q = w[j] * fmaf(yr, yr, yi * yi);
        e = fmaf((float)c, q, e);
        if (c == 0) pz = q;
        if (c == cs) dm = q;
      }
      float el = 0.f;
      df_warp32(e, el);
      pz = __shfl_sync(0xffffffffu, pz, 0);
      dm = __shfl_sync(0xffffffffu, dm, cs & 31);
      if (lane == 0) {
        o[3 * k] = (double)pz;
        o[3 * k + 1] = (double)e + (double)el;
        o[3 * k + 2] = (double)dm;
      }
      ad = am;
    }
  }
}

// best[b][k] = the angle point with the smallest <H_P> after round k + 1
// (the smallest index among equal values). One CTA per (b, k).
__global__ void __launch_bounds__(256) reduced_argmin_kernel(const double *__restrict__ out,
                                                             int A, int p,
                                                             int32_t *__restrict__ best) {
  __shared__ double s_v[8];
  __shared__ int s_i[8];
  const int b = blockIdx.x / p, k = blockIdx.x % p;
  double bv = INFINITY;
  int bi = 0x7fffffff;
  for (int ai = threadIdx.x; ai < A; ai += blockDim.x) {
    const double v = out[(((size_t)b * A + ai) * p + k) * 3 + 1];
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
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (s_v[w] < bv || (s_v[w] == bv && s_i[w] < bi)) { bv = s_v[w]; bi = s_i[w]; }
    best[(size_t)b * p + k] = bi == 0x7fffffff ? -1 : bi;
  }
}

template <int kJ>
int launch_reduced(const ReducedArgs &args, cudaStream_t st) {
  auto kernel = reduced_sweep_kernel<kJ>;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess ||
      per_sm < 1)
    return GQAOA_ECUDA;
  uint64_t blocks = (uint64_t)per_sm * (uint64_t)sm_count();
  const uint64_t need = (args.nitems + 7) / 8;
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
  switch ((hist_stride + 31) / 32) {
    case 1: rc = launch_reduced<1>(args, st); break;
    case 2: rc = launch_reduced<2>(args, st); break;
    case 3: rc = launch_reduced<3>(args, st); break;
    case 4: rc = launch_reduced<4>(args, st); break;
    case 5: rc = launch_reduced<5>(args, st); break;
    case 6: rc = launch_reduced<6>(args, st); break;
    case 7: rc = launch_reduced<7>(args, st); break;
    default: rc = launch_reduced<8>(args, st); break;
  }
  if (rc || !best) return rc;
  if ((uint64_t)batch * (uint64_t)p > 0x7fffffffull) return GQAOA_ERANGE;
  reduced_argmin_kernel<<<(unsigned)((uint64_t)batch * p), 256, 0, st>>>(out, angles, p, best);
  GQ_CHECK_LAUNCH();
  return GQAOA_OK;
}
