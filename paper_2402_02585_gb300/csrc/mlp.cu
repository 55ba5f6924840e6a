// K9: the learned angle proposer (forward, backward, Adam) and the feature
// builder.
//
// The paper finds that optimal single-angle-pair angles cluster as a function
// of the instance size and clause count (Section III.B, Fig. 2, Appendix D)
// and suggests determining angles from statistical characteristics of the
// density of states (Section V). The proposer maps an instance's normalised
// cost histogram h[c] / 2^n (its density of states), n and m to p angle pairs:
//
//   z1 = W1 x + b1, h1 = GELU(z1); z2 = W2 h1 + b2, h2 = GELU(z2);
//   o = W3 h2 + b3;  angles = 2 pi sigmoid(o);
//   loss = mean 2 (1 - cos(angles - labels))   (angles are 2 pi periodic)
//
// GELU uses the exact normal CDF (erff). The layers are small dense
// contractions (d_in = 130, d_h = 256, d_out = 32 at the bench shape): they run
// as a shared-memory tiled FP32 GEMM (64x64 tiles, 4x4 outputs per thread)
// with the bias, GELU and GELU-backward fused into the epilogue. Column sums
// for bias gradients are two-level and deterministic. Parameters are one flat
// FP32 vector [W1 (d_h x d_in), b1, W2 (d_h x d_h), b2, W3 (d_out x d_h), b3].
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.cuh"

namespace gq {

constexpr int kBM = 64, kBN = 64, kBK = 16;
constexpr float kTwoPi = 6.283185307179586f;

enum Epi { kEpiStore = 0, kEpiBiasGelu = 1, kEpiBias = 2, kEpiGeluBwd = 3 };

struct GemmArgs {
  int M, N, K;
  const float *A; int lda;   // op(A) is M x K
  const float *B; int ldb;   // op(B) is K x N
  float *C; int ldc;
  const float *bias;         // [N] (kEpiBiasGelu, kEpiBias)
  float *Zout;               // pre-activation out (kEpiBiasGelu), ld = ldc
  const float *Zin;          // pre-activation in (kEpiGeluBwd), ld = ldc
};

__device__ __forceinline__ float gelu_f(float x) {
  return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) +
         x * expf(-0.5f * x * x) * 0.3989422804014327f;
}

// C = op(A) op(B) with a fused epilogue. TA: A is stored K x M (lda >= M);
// TB: B is stored N x K (ldb >= K).
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256) gemm_kernel(const GemmArgs g) {
  __shared__ float As[kBK][kBM + 4];
  __shared__ float Bs[kBK][kBN + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

  for (int k0 = 0; k0 < g.K; k0 += kBK) {
#pragma unroll
    for (int r = 0; r < (kBM * kBK) / 256; ++r) {
      const int i = threadIdx.x + r * 256;
      int mm, kk;
      if (TA) { mm = i % kBM; kk = i / kBM; } else { kk = i % kBK; mm = i / kBK; }
      const int gm = m0 + mm, gk = k0 + kk;
      float v = 0.f;
      if (gm < g.M && gk < g.K) v = TA ? g.A[(size_t)gk * g.lda + gm] : g.A[(size_t)gm * g.lda + gk];
      As[kk][mm] = v;
    }
#pragma unroll
    for (int r = 0; r < (kBN * kBK) / 256; ++r) {
      const int i = threadIdx.x + r * 256;
      int nn, kk;
      if (TB) { kk = i % kBK; nn = i / kBK; } else { nn = i % kBN; kk = i / kBN; }
      const int gn = n0 + nn, gk = k0 + kk;
      float v = 0.f;
      if (gn < g.N && gk < g.K) v = TB ? g.B[(size_t)gn * g.ldb + gk] : g.B[(size_t)gk * g.ldb + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= g.N) continue;
      const size_t o = (size_t)m * g.ldc + n;
      float v = acc[i][j];
      if (EPI == kEpiBiasGelu) {
        v += g.bias[n];
        g.Zout[o] = v;
        v = gelu_f(v);
      } else if (EPI == kEpiBias) {
        v += g.bias[n];
      } else if (EPI == kEpiGeluBwd) {
        v *= gelu_grad_f(g.Zin[o]);
      }
      g.C[o] = v;
    }
  }
}

template <bool TA, bool TB, int EPI>
static cudaError_t gemm(const GemmArgs &g, cudaStream_t st) {
  dim3 grid((g.N + kBN - 1) / kBN, (g.M + kBM - 1) / kBM);
  gemm_kernel<TA, TB, EPI><<<grid, 256, 0, st>>>(g);
  return cudaPeekAtLastError();
}

// angles = 2 pi sigmoid(o); with labels: the periodic loss 2 (1 - cos(d)),
// d = angle - label, its gradient 2 sin(d) / count, and per-block loss partials.
__global__ void head_kernel(const float *__restrict__ o, const float *__restrict__ labels,
                            int64_t total, float inv_count, float *__restrict__ angles,
                            float *__restrict__ dO, double *__restrict__ loss_parts) {
  __shared__ double s_scr[kWarps];
  double l = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float s = 1.0f / (1.0f + expf(-o[i]));
    const float a = kTwoPi * s;
    if (angles) angles[i] = a;
    if (labels) {
      // 2 (1 - cos d) = 4 sin^2(d/2) and 2 sin d = 4 sin(d/2) cos(d/2): no
      // cancellation for small d
      float sh, ch;
      sincosf(0.5f * (a - labels[i]), &sh, &ch);
      l += 4.0 * (double)sh * (double)sh;
      dO[i] = 4.0f * sh * ch * inv_count * kTwoPi * s * (1.0f - s);
    }
  }
  if (labels) {
    const double t = block_sum(l, s_scr);
    if (threadIdx.x == 0) loss_parts[blockIdx.x] = t;
  }
}

__global__ void loss_final_kernel(const double *__restrict__ parts, int nparts, double inv_count,
                                  double *__restrict__ loss) {
  if (threadIdx.x != 0) return;
  double t = 0.0;
  for (int i = 0; i < nparts; ++i) t += parts[i];
  *loss = t * inv_count;
}

// Column sums of a row-major M x N matrix: per (column block, row chunk)
// partials, then a fixed-order sum over chunks.
constexpr int kColRows = 256;
__global__ void colsum_partial_kernel(const float *__restrict__ X, int M, int N,
                                      float *__restrict__ part) {
  __shared__ float s[8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int n = blockIdx.x * 32 + tx;
  const int r0 = blockIdx.y * kColRows;
  float acc = 0.f;
  if (n < N)
    for (int r = r0 + ty; r < r0 + kColRows && r < M; r += 8) acc += X[(size_t)r * N + n];
  s[ty][tx] = acc;
  __syncthreads();
  if (ty == 0 && n < N) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += s[k][tx];
    part[(size_t)blockIdx.y * N + n] = t;
  }
}

__global__ void colsum_final_kernel(const float *__restrict__ part, int chunks, int N,
                                    float *__restrict__ out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float t = 0.f;
  for (int c = 0; c < chunks; ++c) t += part[(size_t)c * N + n];
  out[n] = t;
}

template <typename T>
__global__ void adam_kernel(T *__restrict__ p, const T *__restrict__ g, T *__restrict__ m,
                            T *__restrict__ v, int64_t count, T lr, T b1, T b2, T eps, T c1, T c2,
                            T gscale) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T gi = g[i] * gscale;
    const T mi = b1 * m[i] + (T(1) - b1) * gi;
    const T vi = b2 * v[i] + (T(1) - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrt(vi / c2) + eps);
  }
}

__global__ void features_kernel(const int64_t *__restrict__ hist, int hist_stride,
                                const int32_t *__restrict__ ns, const int32_t *__restrict__ ms,
                                int batch, int d_in, float *__restrict__ x) {
  const int64_t total = (int64_t)batch * d_in;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(i / d_in), c = (int)(i % d_in);
    const int n = ns[b], m = ms[b];
    float v = 0.f;
    if (c == d_in - 2) v = (float)n / 32.0f;
    else if (c == d_in - 1) v = (float)m / 128.0f;
    else if (c <= m && c < hist_stride) v = (float)((double)hist[(size_t)b * hist_stride + c] / (double)(1ull << n));
    x[i] = v;
  }
}

// ---------------------------------------------------------------------------
// workspace: z1, h1, z2, h2, dZ1, dZ2 [B x d_h]; o, dO [B x d_out];
//            column-sum partials; loss partials
// ---------------------------------------------------------------------------
struct MlpWs {
  float *z1, *h1, *z2, *h2, *dz1, *dz2, *o, *dO, *colpart;
  double *loss_parts;
};
constexpr int kHeadBlocks = 256;

static size_t mlp_ws_layout(int B, int d_h, int d_out, char *base, MlpWs *w) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = round_up(off + bytes, 256);
    return o;
  };
  const size_t bh = (size_t)B * d_h * sizeof(float), bo = (size_t)B * d_out * sizeof(float);
  const size_t chunks = ((size_t)B + kColRows - 1) / kColRows;
  const size_t dmax = d_h > d_out ? d_h : d_out;
  size_t oz1 = take(bh), oh1 = take(bh), oz2 = take(bh), oh2 = take(bh), odz1 = take(bh),
         odz2 = take(bh), oo = take(bo), odo = take(bo), ocp = take(chunks * dmax * sizeof(float)),
         olp = take(kHeadBlocks * sizeof(double));
  if (w) {
    w->z1 = reinterpret_cast<float *>(base + oz1);
    w->h1 = reinterpret_cast<float *>(base + oh1);
    w->z2 = reinterpret_cast<float *>(base + oz2);
    w->h2 = reinterpret_cast<float *>(base + oh2);
    w->dz1 = reinterpret_cast<float *>(base + odz1);
    w->dz2 = reinterpret_cast<float *>(base + odz2);
    w->o = reinterpret_cast<float *>(base + oo);
    w->dO = reinterpret_cast<float *>(base + odo);
    w->colpart = reinterpret_cast<float *>(base + ocp);
    w->loss_parts = reinterpret_cast<double *>(base + olp);
  }
  return off;
}

static int check_dims(int B, int d_in, int d_h, int d_out) {
  if (B < 1 || B > (1 << 24) || d_in < 3 || d_in > 4096 || d_h < 1 || d_h > 4096 || d_out < 1 ||
      d_out > 4096)
    return GQAOA_ERANGE;
  return GQAOA_OK;
}

static int colsum(const float *X, int M, int N, float *part, float *out, cudaStream_t st) {
  dim3 grid((N + 31) / 32, (M + kColRows - 1) / kColRows);
  colsum_partial_kernel<<<grid, 256, 0, st>>>(X, M, N, part);
  GQ_CHECK_LAUNCH();
  colsum_final_kernel<<<(N + 255) / 256, 256, 0, st>>>(part, (int)grid.y, N, out);
  GQ_CHECK_LAUNCH();
  return GQAOA_OK;
}

// Forward into the workspace (z1, h1, z2, h2, o); angles optional.
static int mlp_forward_ws(const float *params, int d_in, int d_h, int d_out, const float *x, int B,
                          const MlpWs &w, cudaStream_t st) {
  const float *W1 = params, *b1 = W1 + (size_t)d_h * d_in, *W2 = b1 + d_h,
              *b2 = W2 + (size_t)d_h * d_h, *W3 = b2 + d_h, *b3 = W3 + (size_t)d_out * d_h;
  GemmArgs g = {};
  g = GemmArgs{B, d_h, d_in, x, d_in, W1, d_in, w.h1, d_h, b1, w.z1, nullptr};
  if (gemm<false, true, kEpiBiasGelu>(g, st) != cudaSuccess) return GQAOA_ECUDA;
  g = GemmArgs{B, d_h, d_h, w.h1, d_h, W2, d_h, w.h2, d_h, b2, w.z2, nullptr};
  if (gemm<false, true, kEpiBiasGelu>(g, st) != cudaSuccess) return GQAOA_ECUDA;
  g = GemmArgs{B, d_out, d_h, w.h2, d_h, W3, d_h, w.o, d_out, b3, nullptr, nullptr};
  if (gemm<false, true, kEpiBias>(g, st) != cudaSuccess) return GQAOA_ECUDA;
  return GQAOA_OK;
}

}  // namespace gq

using namespace gq;

extern "C" int gqaoa_mlp_param_count(int d_in, int d_h, int d_out, size_t *count) {
  if (!count) return GQAOA_EINVAL;
  int rc = check_dims(1, d_in, d_h, d_out);
  if (rc) return rc;
  *count = (size_t)d_h * d_in + d_h + (size_t)d_h * d_h + d_h + (size_t)d_out * d_h + d_out;
  return GQAOA_OK;
}

extern "C" int gqaoa_mlp_workspace_size(int batch, int d_in, int d_h, int d_out, size_t *bytes) {
  if (!bytes) return GQAOA_EINVAL;
  int rc = check_dims(batch, d_in, d_h, d_out);
  if (rc) return rc;
  *bytes = mlp_ws_layout(batch, d_h, d_out, nullptr, nullptr);
  return GQAOA_OK;
}

extern "C" int gqaoa_mlp_forward(const float *params, int d_in, int d_h, int d_out, const float *x,
                                 int batch, float *angles, void *ws, size_t ws_bytes,
                                 void *stream) {
  gq::NvtxRange nvtx_range("gqaoa_mlp_forward");
  int rc = check_dims(batch, d_in, d_h, d_out);
  if (rc) return rc;
  if (!params || !x || !angles || !ws) return GQAOA_EINVAL;
  if (!aligned16(ws) || !aligned8(params) || !aligned8(x) || !aligned8(angles)) return GQAOA_EINVAL;
  if (ws_bytes < mlp_ws_layout(batch, d_h, d_out, nullptr, nullptr)) return GQAOA_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  MlpWs w;
  mlp_ws_layout(batch, d_h, d_out, static_cast<char *>(ws), &w);
  rc = mlp_forward_ws(params, d_in, d_h, d_out, x, batch, w, st);
  if (rc) return rc;
  const int64_t total = (int64_t)batch * d_out;
  head_kernel<<<kHeadBlocks, kThreads, 0, st>>>(w.o, nullptr, total, 0.f, angles, nullptr, nullptr);
  GQ_CHECK_LAUNCH();
  return GQAOA_OK;
}

extern "C" int gqaoa_mlp_backward(const float *params, int d_in, int d_h, int d_out, const float *x,
                                  const float *labels, int batch, float *grads, double *loss,
                                  void *ws, size_t ws_bytes, void *stream) {
  gq::NvtxRange nvtx_range("gqaoa_mlp_backward");
  int rc = check_dims(batch, d_in, d_h, d_out);
  if (rc) return rc;
  if (!params || !x || !labels || !grads || !loss || !ws) return GQAOA_EINVAL;
  if (!aligned16(ws) || !aligned8(params) || !aligned8(x) || !aligned8(labels) || !aligned8(grads) ||
      !aligned8(loss))
    return GQAOA_EINVAL;
  if (ws_bytes < mlp_ws_layout(batch, d_h, d_out, nullptr, nullptr)) return GQAOA_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  MlpWs w;
  mlp_ws_layout(batch, d_h, d_out, static_cast<char *>(ws), &w);
  rc = mlp_forward_ws(params, d_in, d_h, d_out, x, batch, w, st);
  if (rc) return rc;
  const float *W2 = params + (size_t)d_h * d_in + d_h;
  const float *W3 = W2 + (size_t)d_h * d_h + d_h;
  float *gW1 = grads, *gb1 = gW1 + (size_t)d_h * d_in, *gW2 = gb1 + d_h,
        *gb2 = gW2 + (size_t)d_h * d_h, *gW3 = gb2 + d_h, *gb3 = gW3 + (size_t)d_out * d_h;
  const int64_t total = (int64_t)batch * d_out;
  const double inv_count = 1.0 / (double)total;
  head_kernel<<<kHeadBlocks, kThreads, 0, st>>>(w.o, labels, total, (float)inv_count, nullptr, w.dO,
                                                w.loss_parts);
  GQ_CHECK_LAUNCH();
  loss_final_kernel<<<1, 32, 0, st>>>(w.loss_parts, kHeadBlocks, inv_count, loss);
  GQ_CHECK_LAUNCH();
  GemmArgs g;
  // dW3 = dO^T h2 ; db3 = colsum(dO)
  g = GemmArgs{d_out, d_h, batch, w.dO, d_out, w.h2, d_h, gW3, d_h, nullptr, nullptr, nullptr};
  if (gemm<true, false, kEpiStore>(g, st) != cudaSuccess) return GQAOA_ECUDA;
  if ((rc = colsum(w.dO, batch, d_out, w.colpart, gb3, st))) return rc;
  // dZ2 = (dO W3) * GELU'(z2)
  g = GemmArgs{batch, d_h, d_out, w.dO, d_out, W3, d_h, w.dz2, d_h, nullptr, nullptr, w.z2};
  if (gemm<false, false, kEpiGeluBwd>(g, st) != cudaSuccess) return GQAOA_ECUDA;
  g = GemmArgs{d_h, d_h, batch, w.dz2, d_h, w.h1, d_h, gW2, d_h, nullptr, nullptr, nullptr};
  if (gemm<true, false, kEpiStore>(g, st) != cudaSuccess) return GQAOA_ECUDA;
  if ((rc = colsum(w.dz2, batch, d_h, w.colpart, gb2, st))) return rc;
  // dZ1 = (dZ2 W2) * GELU'(z1)
  g = GemmArgs{batch, d_h, d_h, w.dz2, d_h, W2, d_h, w.dz1, d_h, nullptr, nullptr, w.z1};
  if (gemm<false, false, kEpiGeluBwd>(g, st) != cudaSuccess) return GQAOA_ECUDA;
  g = GemmArgs{d_h, d_in, batch, w.dz1, d_h, x, d_in, gW1, d_in, nullptr, nullptr, nullptr};
  if (gemm<true, false, kEpiStore>(g, st) != cudaSuccess) return GQAOA_ECUDA;
  if ((rc = colsum(w.dz1, batch, d_h, w.colpart, gb1, st))) return rc;
  return GQAOA_OK;
}

template <typename T>
static int adam_impl(T *params, const T *grads, T *m, T *v, int64_t count, double lr, double b1,
                     double b2, double eps, int step, double gscale, void *stream) {
  if (!params || !grads || !m || !v) return GQAOA_EINVAL;
  if (count < 0 || step < 1) return GQAOA_ERANGE;
  if (count == 0) return GQAOA_OK;
  const double c1 = 1.0 - pow(b1, (double)step), c2 = 1.0 - pow(b2, (double)step);
  int64_t grid = (count + kThreads - 1) / kThreads;
  if (grid > 4096) grid = 4096;
  adam_kernel<T><<<(unsigned)grid, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      params, grads, m, v, count, (T)lr, (T)b1, (T)b2, (T)eps, (T)c1, (T)c2, (T)gscale);
  GQ_CHECK_LAUNCH();
  return GQAOA_OK;
}

extern "C" int gqaoa_adam_f32(float *params, const float *grads, float *m, float *v, int64_t count,
                              double lr, double beta1, double beta2, double eps, int step,
                              double grad_scale, void *stream) {
  return adam_impl<float>(params, grads, m, v, count, lr, beta1, beta2, eps, step, grad_scale,
                          stream);
}

extern "C" int gqaoa_adam_f64(double *params, const double *grads, double *m, double *v,
                              int64_t count, double lr, double beta1, double beta2, double eps,
                              int step, double grad_scale, void *stream) {
  return adam_impl<double>(params, grads, m, v, count, lr, beta1, beta2, eps, step, grad_scale,
                           stream);
}

extern "C" int gqaoa_mlp_features(const int64_t *hist, int hist_stride, const int32_t *ns,
                                  const int32_t *ms, int batch, int d_in, float *x, void *stream) {
  if (!hist || !ns || !ms || !x) return GQAOA_EINVAL;
  if (batch < 1 || d_in < 3 || hist_stride < 1) return GQAOA_ERANGE;
  int64_t grid = ((int64_t)batch * d_in + kThreads - 1) / kThreads;
  if (grid > 4096) grid = 4096;
  features_kernel<<<(unsigned)grid, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      hist, hist_stride, ns, ms, batch, d_in, x);
  GQ_CHECK_LAUNCH();
  return GQAOA_OK;
}
