// Streaming G-QAOA kernels: K10 phase tables, K2 fused round, K3 reduction,
// K4 readout and K6 adjoint backward, for one instance or a batch of
// instances of equal n.
//
// Eq. 3 applies, per round k, the diagonal phase e^{-i gamma_k H_P} and then
// the Grover mixer e^{-i beta_k H_M}, H_M = |+><+| (Eq. 2). H_M is a rank-1
// projector, so
//   e^{-i beta H_M} psi = psi + alpha (sum_z psi(z) / N) 1,   alpha = e^{-i beta} - 1,
// and a round is   chi_k = T_k[C] psi_{k-1},   psi_k = chi_k + a_k,
//   T_k[c] = e^{-i gamma_k c},   a_k = alpha_k S_k / N,   S_k = sum_z chi_k(z).
//
// a_k needs a sum over all 2^n amplitudes, so it cannot be added in the pass
// that produces chi_k. The pass of round k therefore stores chi_k and, in the
// same read-modify-write, first adds the pending a_{k-1}:
//   read chi_{k-1}, C -> psi = chi_{k-1} + a_{k-1} -> chi_k = T_k[C] psi
//   -> write chi_k, accumulate S_k.
// 8 B read + 1 B cost + 8 B write = 17 B per amplitude-round. Round 1
// synthesises psi_0 = N^{-1/2} (9 B). A last pass writes psi_p = chi_p + a_p
// and reads out P(C=0), <H_P> and the norm.
//
// Reductions are deterministic. A thread sums a 16-amplitude tile in FP32,
// accumulates tiles in double-float (two FP32 words, ~48 bits), then the CTA
// combines threads in FP64 (warp shuffles, then warps in order) and a
// thread-block cluster combines its CTAs through distributed shared memory
// (rank 0 reads the others with ld.shared::cluster), giving one FP64 record
// per cluster. Warp 0 of every CTA of the next pass sums the records of its
// instance in index order with the same instructions, so every CTA derives
// the bit-identical a_k with no extra launch and no grid-wide barrier. FP64
// work is kept to a few operations per CTA: on this part the FP64 rate is a
// small fraction of the FP32 rate.
//
// Adjoint (Appendix C optimises the angles with a gradient method). For
// L = <psi_p|O|psi_p>, O = [C = 0] or O = C, lambda_p = O psi_p and for
// k = p..1 (Lambda_k = sum_z lambda_k):
//   dL/dbeta_k   = 2 Re[-i e^{-i beta_k} (S_k / N) conj(Lambda_k)]
//   mu_k         = lambda_k + conj(alpha_k) Lambda_k / N
//   dL/dgamma_k  = 2 sum_z C(z) Im[conj(mu_k(z)) chi_k(z)]
//   lambda_{k-1} = conj(T_k[C]) mu_k
// using checkpoints chi_k stored by the forward passes. One backward pass per
// round: read lambda_k, chi_k, C; write lambda_{k-1}; 25 B per amplitude.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "cdf.cuh"
#include "common.cuh"

namespace gq {

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------
constexpr int kClusterSize = 4;  // CTAs per cluster for single-instance passes
constexpr int kMaxDevices = 64;
constexpr int kMaxCpi = 1024;    // CTAs per instance, upper bound

static int g_sm_count[kMaxDevices];
static std::once_flag g_sm_once[kMaxDevices];

int sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 152;
  std::call_once(g_sm_once[dev], [dev]() {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
      v = 152;
    g_sm_count[dev] = v;
  });
  return g_sm_count[dev];
}

struct Geometry {
  uint64_t N;       // amplitudes per instance
  uint64_t ntiles;  // tiles per instance
  int B;            // instances
  int cpi;          // CTAs per instance
  int cluster;      // CTAs per cluster (1 or kClusterSize)
  int nparts;       // records per instance = cpi / cluster
  bool small;       // N < one tile: one CTA per instance, everything on chip
};

// One wave is `per_sm` CTAs of 256 threads per SM: 2 for every streaming
// pass (each thread keeps a tile, or for the adjoint a half-tile of lambda
// and of chi, in flight while it processes the previous one; <= 128
// registers). A single instance gets
// one wave in clusters of 4; a batch gets about two waves split evenly over
// instances, each CTA owning whole tiles of one instance.
constexpr int kFwdPerSm = 2;
constexpr int kBwdPerSm = 2;

// CTAs of one full wave of a clustered streaming pass: the number of clusters
// of kClusterSize the device keeps resident at once (clusters are placed
// within a GPC, so this can be fewer than SMs x per_sm / kClusterSize) times
// the cluster size. Queried once per device and pass kind; falls back to
// SMs x per_sm when no device answers (e.g. sizing a workspace on a host
// without a GPU, which then errs on the large side).
static int resident_cluster_ctas(int per_sm);

static Geometry make_geometry(int n, int B, int per_sm) {
  Geometry g;
  g.N = 1ull << n;
  g.B = B;
  g.small = g.N < (uint64_t)kTileAmps;
  g.ntiles = g.small ? 1 : g.N / kTileAmps;
  const uint64_t wave = (uint64_t)sm_count() * (uint64_t)per_sm;
  if (g.small) {
    g.cpi = 1; g.cluster = 1; g.nparts = 1;
    return g;
  }
  if (B == 1) {
    const uint64_t full = (uint64_t)resident_cluster_ctas(per_sm);
    uint64_t c = g.ntiles < full ? g.ntiles : full;
    c = (c + kClusterSize - 1) / kClusterSize * kClusterSize;
    if (c > kMaxCpi) c = kMaxCpi;
    g.cpi = (int)c;
    g.cluster = kClusterSize;
  } else {
    // CTAs per instance: enough for at least two waves, chosen so the last
    // wave is nearly full (B * cpi close to a multiple of the wave), since a
    // half-empty last wave of a streaming pass idles the HBM for its length.
    const uint64_t cmax = g.ntiles < (uint64_t)kMaxCpi ? g.ntiles : (uint64_t)kMaxCpi;
    uint64_t c0 = (2 * wave + B - 1) / (uint64_t)B;
    if (c0 < 1) c0 = 1;
    if (c0 > cmax) c0 = cmax;
    uint64_t best = c0;
    double best_eff = 0.0;
    for (uint64_t c = c0; c <= cmax && c <= 4 * c0 + 8; ++c) {
      const uint64_t ctas = (uint64_t)B * c;
      const double waves = (double)ctas / (double)wave;
      const double eff = waves / (double)((ctas + wave - 1) / wave);
      if (eff > best_eff + 1e-9) { best_eff = eff; best = c; }
      if (eff >= 0.95) break;
    }
    g.cpi = (int)best;
    g.cluster = 1;
  }
  g.nparts = g.cpi / g.cluster;
  return g;
}

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------
struct Ws {
  double2 *alpha;   // [B][p]        e^{-i beta_k} - 1
  float2 *phase;    // [B][p][256]   e^{-i gamma_k c}
  double *parts;    // [2][B][nparts][kPartStride]
  double *record;   // [B][p][4]     S_k (re, im), a_k (re, im)
  float2 *ckpt;     // [p][B][N]     chi_k checkpoints (gradient only)
  float2 *lambda;   // [B][N]        adjoint state (gradient only)
  size_t parts_half;  // doubles in one half of `parts`
};

static size_t ws_layout(const Geometry &g, int p, bool grad, char *base, Ws *w,
                        int max_nparts) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = round_up(off + bytes, 256);
    return o;
  };
  const size_t Bp = (size_t)g.B * (size_t)p;
  const size_t half = (size_t)g.B * (size_t)max_nparts * kPartStride;
  size_t o_alpha = take(sizeof(double2) * Bp);
  size_t o_phase = take(sizeof(float2) * 256 * Bp);
  size_t o_parts = take(sizeof(double) * 2 * half);
  size_t o_rec = take(sizeof(double) * 4 * Bp);
  size_t o_ckpt = 0, o_lam = 0;
  if (grad) {
    o_ckpt = take(sizeof(float2) * (size_t)p * g.B * g.N);
    o_lam = take(sizeof(float2) * (size_t)g.B * g.N);
  }
  if (w) {
    w->alpha = reinterpret_cast<double2 *>(base + o_alpha);
    w->phase = reinterpret_cast<float2 *>(base + o_phase);
    w->parts = reinterpret_cast<double *>(base + o_parts);
    w->record = reinterpret_cast<double *>(base + o_rec);
    w->ckpt = grad ? reinterpret_cast<float2 *>(base + o_ckpt) : nullptr;
    w->lambda = grad ? reinterpret_cast<float2 *>(base + o_lam) : nullptr;
    w->parts_half = half;
  }
  return off;
}

// ---------------------------------------------------------------------------
// K10: phase tables and mixer coefficients
// ---------------------------------------------------------------------------
// T[c] = e^{-i gamma c} for c < 256, rounded to complex64, and
// alpha = e^{-i beta} - 1 in FP64. GB300's FP64 rate is a small fraction of
// its FP32 rate, so FP64 is spent only on two sincos per table (gamma,
// beta); e^{-i 16 gamma} is e^{-i gamma} squared four times, and the powers
// e^{-i gamma r} and e^{-i 16 gamma q} (r, q < 16) and the entries
// T[16 q + r] = e^{-i 16 gamma q} e^{-i gamma r} are formed in double-float
// arithmetic (FP32 pairs, ~2^-44 relative error after the at most 34
// multiplications behind an entry), whose leading word is the entry rounded
// to FP32.
struct DFv {
  float hi, lo;
};
__device__ __forceinline__ DFv dfv_from(double x) {
  const float h = (float)x;
  return DFv{h, (float)(x - (double)h)};
}
// Renormalise a + b with |a| >= |b| (Dekker's Fast2Sum).
__device__ __forceinline__ DFv dfv_fast(float a, float b) {
  const float s = __fadd_rn(a, b);
  return DFv{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DFv dfv_mul(DFv a, DFv b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);  // the rounding error of p, exactly
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return dfv_fast(p, e);
}
__device__ __forceinline__ DFv dfv_add(DFv a, DFv b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return dfv_fast(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
struct DFc {
  DFv x, y;  // x + i y
};
__device__ __forceinline__ DFc dfc_mul(const DFc &a, const DFc &b) {
  const DFv yy = dfv_mul(a.y, b.y);
  return DFc{dfv_add(dfv_mul(a.x, b.x), DFv{-yy.hi, -yy.lo}),
             dfv_add(dfv_mul(a.x, b.y), dfv_mul(a.y, b.x))};
}
__device__ __forceinline__ DFc dfc_load(float4 v) { return DFc{{v.x, v.y}, {v.z, v.w}}; }

constexpr int kPhaseWarps = 8;  // warps per CTA; the CTA owns 32 tables at a time

// Warp 0's lane l takes table t0 + l for the sincos and its power chains,
// which go to shared rows ([table][power], padded so the lanes' float4 stores
// spread over the banks), while warp 1's lane l forms alpha; then the CTA's
// warps write the 32 tables, warp w the tables w, w + 8, ..., 32
// consecutive entries per store.
__global__ void __launch_bounds__(kPhaseWarps * 32)
phase_table_kernel(const double *__restrict__ gammas, const double *__restrict__ betas,
                   int64_t count, int entries, float2 *__restrict__ phase,
                   double2 *__restrict__ alpha) {
  __shared__ float4 P[32][33];  // [table][r] = e^{-i gamma r}, [table][16 + q] = e^{-i 16 gamma q}
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nq = entries / 16;  // rows of the 16 gamma chain in use
  const int64_t nblk = (count + 31) / 32;
  for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    if (warp == 1) {  // the mixer coefficients, beside warp 0's phase powers
      const int64_t t = blk * 32 + lane;
      if (t < count) {
        double sb, cb;
        sincos(betas[t], &sb, &cb);
        alpha[t] = make_double2(cb - 1.0, -sb);
      }
    }
    if (warp == 0) {
      const int64_t t = blk * 32 + lane;
      const bool live = t < count;
      const double g = live ? gammas[t] : 0.0;
      double s1, c1;
      sincos(g, &s1, &c1);
      const DFc e1 = {dfv_from(c1), dfv_from(-s1)};
      DFc e16 = dfc_mul(e1, e1);  // e^{-i 2 gamma}
      e16 = dfc_mul(e16, e16);
      e16 = dfc_mul(e16, e16);
      e16 = dfc_mul(e16, e16);    // e^{-i 16 gamma}
      DFc a1 = {{1.f, 0.f}, {0.f, 0.f}}, a16 = a1;
#pragma unroll 1
      for (int r = 0; r < 16; ++r) {
        P[lane][r] = make_float4(a1.x.hi, a1.x.lo, a1.y.hi, a1.y.lo);
        a1 = dfc_mul(a1, e1);
        if (r < nq) {
          P[lane][16 + r] = make_float4(a16.x.hi, a16.x.lo, a16.y.hi, a16.y.lo);
          a16 = dfc_mul(a16, e16);
        }
      }
    }
    __syncthreads();
    const int tn = (int)(count - blk * 32 < 32 ? count - blk * 32 : 32);
#pragma unroll 1
    for (int tt = warp; tt < tn; tt += kPhaseWarps) {
      const DFc er = dfc_load(P[tt][lane & 15]);
      float2 *dst = phase + (blk * 32 + tt) * entries;
#pragma unroll 8
      for (int i = 0; i < entries / 32; ++i) {
        // entry c = lane + 32 i = 16 q + r with r = lane & 15, q = (lane >> 4) + 2 i
        const DFc v = dfc_mul(dfc_load(P[tt][16 + (lane >> 4) + 2 * i]), er);
        dst[lane + 32 * i] = make_float2(v.x.hi, v.y.hi);
      }
    }
    __syncthreads();  // the rows are rewritten for the next block
  }
}

// ---------------------------------------------------------------------------
// common pieces of the streaming passes
// ---------------------------------------------------------------------------
struct PassArgs {
  const uint8_t *cost;      // instance b's table at cost + b * cost_bstride
  uint64_t cost_bstride;    // N, or 0 when every instance shares one table
  const float4 *src;        // instance b at src + b * N/2 (float4 = 2 amplitudes)
  float4 *dst;              // may equal src (in place)
  const float2 *phase;      // [B][p][256]
  const double2 *alpha;     // [B][p]
  const double *parts_in;   // [B][nparts][stride] of the previous pass
  double *parts_out;        // [B][nparts][stride] of this pass
  double *record;           // [B][p][4]
  double *trace;            // [B][p] or null
  double *value;            // [B]   (gradient)
  double *dgamma;           // [B][p] (gradient)
  double *dbeta;            // [B][p] (gradient)
  int p;
  int round;                // 0-based round index of this pass
  int cpi;
  int nparts;               // records per instance written by this pass
  int nparts_in;            // records per instance written by the previous pass
  uint64_t ntiles;          // tiles per instance
  uint64_t N;
  double inv_n;
  float amp0;               // N^{-1/2}
  unsigned target;          // the cost class read out (readout) or projected on (lambda init)
};

// Programmatic dependent launch. A streaming pass is launched while the
// previous one drains; it reads or writes no global memory before
// griddepcontrol.wait, and it lets the next pass launch only after that wait
// (so every kernel before the previous one has completed too). What overlaps
// is the launch and CTA set-up of pass k+1 with the tail of pass k.
__device__ __forceinline__ void pdl_wait_then_release() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Sum slot j of instance b's records in index order within warp 0.
__device__ __forceinline__ double w0_parts(const PassArgs &a, int b, int j) {
  const int lane = threadIdx.x & 31;
  const double *base = a.parts_in + (size_t)b * a.nparts_in * kPartStride;
  double v = 0.0;
  for (int i = lane; i < a.nparts_in; i += 32) v += base[(size_t)i * kPartStride + j];
  return warp_sum(v);
}

// CTA + cluster reduction of up to kPartStride double-float accumulators
// into this CTA's cluster record of instance b.
template <int kVals>
__device__ __forceinline__ void reduce_to_record(const PassArgs &a, int b, int local,
                                                 const DF (&acc)[kVals], double (*s_w)[kPartStride],
                                                 double *s_vals) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < kVals; ++j) {
    double x = warp_sum(acc[j].value());
    if (lane == 0) s_w[warp][j] = x;
  }
  __syncthreads();
  if (threadIdx.x < kVals) {
    double x = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) x += s_w[w][threadIdx.x];
    s_vals[threadIdx.x] = x;
  }
  __syncthreads();
  const unsigned cs = cluster_nctarank();
  cluster_reduce_store(s_vals, kVals,
                       a.parts_out + ((size_t)b * a.nparts + local / cs) * kPartStride);
}

__device__ __forceinline__ uint64_t tile_vbase(uint64_t tile, int warp, int lane) {
  return tile * (kTileAmps / 2) + (uint64_t)warp * (kWarpTileAmps / 2) + lane;
}

// A thread's share of one tile: 8 float4 (16 amplitudes) and their costs.
struct TileRegs {
  float4 v[kVecPerThread];
  uint16_t c2[kVecPerThread];
};

// Tiles first, first + stride, ... below ntiles, two in flight per thread:
// the loads of the next tile are issued before the current one is processed,
// so each thread keeps ~256 bytes of HBM reads outstanding.
template <typename Load, typename Proc>
__device__ __forceinline__ void pipelined_tiles(uint64_t first, uint64_t stride, uint64_t ntiles,
                                                Load load, Proc proc) {
  TileRegs A, Bt;
  uint64_t t = first;
  if (t < ntiles) load(A, t);
  for (; t < ntiles; t += 2 * stride) {
    const uint64_t t2 = t + stride;
    if (t2 < ntiles) load(Bt, t2);
    proc(A, t);
    if (t2 < ntiles) {
      const uint64_t t3 = t2 + stride;
      if (t3 < ntiles) load(A, t3);
      proc(Bt, t2);
    }
  }
}

// ---------------------------------------------------------------------------
// K2: fused round
// ---------------------------------------------------------------------------
enum RoundMode { kFromPlus = 0, kFromState = 1, kChained = 2 };

template <int kMode, bool kTrace>
__global__ void __launch_bounds__(kThreads, kFwdPerSm) round_kernel(const PassArgs a) {
  __shared__ float2 s_T[256];
  __shared__ float2 s_a;
  __shared__ double s_w[kWarps][kPartStride];
  __shared__ double s_vals[kPartStride];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int b = blockIdx.x / a.cpi, local = blockIdx.x % a.cpi;
  const size_t bk = (size_t)b * a.p + a.round;

  pdl_wait_then_release();
  s_T[threadIdx.x] = a.phase[bk * 256 + threadIdx.x];
  if (warp == 0) {
    double2 av = make_double2(0.0, 0.0);
    if (kMode == kChained) {
      const double Sre = w0_parts(a, b, 0), Sim = w0_parts(a, b, 1);
      const double2 al = a.alpha[bk - 1];
      av = make_double2((al.x * Sre - al.y * Sim) * a.inv_n, (al.x * Sim + al.y * Sre) * a.inv_n);
      double P = 0.0;
      if (kTrace) {
        const double A0 = w0_parts(a, b, 2), B0r = w0_parts(a, b, 3), B0i = w0_parts(a, b, 4);
        const double c0 = w0_parts(a, b, 5);
        // sum_{C=0} |chi + a|^2 = A0 + 2 Re(conj(a) B0) + h[0] |a|^2
        P = A0 + 2.0 * (av.x * B0r + av.y * B0i) + c0 * (av.x * av.x + av.y * av.y);
      }
      if (local == 0 && lane == 0) {
        double *rec = a.record + 4 * (bk - 1);
        rec[0] = Sre; rec[1] = Sim; rec[2] = av.x; rec[3] = av.y;
        if (kTrace) a.trace[bk - 1] = P;
      }
    }
    if (lane == 0) s_a = make_float2((float)av.x, (float)av.y);
  }
  __syncthreads();
  const float2 ad = s_a;

  constexpr int kVals = kTrace ? 6 : 2;
  DF acc[kVals];
#pragma unroll
  for (int j = 0; j < kVals; ++j) acc[j].zero();

  const uint16_t *__restrict__ cost2 =
      reinterpret_cast<const uint16_t *>(a.cost + (size_t)b * a.cost_bstride);
  const float4 *__restrict__ src = a.src + (size_t)b * (a.N / 2);
  float4 *dst = a.dst + (size_t)b * (a.N / 2);
  const bool reverse = (a.round & 1) != 0;  // alternate sweep direction: L2 reuse across rounds
  auto vbase = [&](uint64_t t) {
    return tile_vbase(reverse ? (a.ntiles - 1 - t) : t, warp, lane);
  };
  auto load = [&](TileRegs &T, uint64_t t) {
    const uint64_t vb = vbase(t);
#pragma unroll
    for (int j = 0; j < kVecPerThread; ++j) T.c2[j] = cost2[vb + 32 * j];
    if (kMode != kFromPlus) {
#pragma unroll
      for (int j = 0; j < kVecPerThread; ++j) T.v[j] = src[vb + 32 * j];
    }
  };
  auto proc = [&](TileRegs &T, uint64_t t) {
    const uint64_t vb = vbase(t);
    float tr = 0.f, ti = 0.f, ta = 0.f, tbr = 0.f, tbi = 0.f, tc = 0.f;
#pragma unroll
    for (int j = 0; j < kVecPerThread; ++j) {
      float2 p0, p1;
      if (kMode == kFromPlus) {
        p0 = make_float2(a.amp0, 0.f);
        p1 = p0;
      } else {
        p0 = make_float2(T.v[j].x + ad.x, T.v[j].y + ad.y);
        p1 = make_float2(T.v[j].z + ad.x, T.v[j].w + ad.y);
      }
      const unsigned c_0 = T.c2[j] & 0xFFu, c_1 = T.c2[j] >> 8;
      const float2 x0 = cmul(s_T[c_0], p0);
      const float2 x1 = cmul(s_T[c_1], p1);
      T.v[j] = make_float4(x0.x, x0.y, x1.x, x1.y);
      tr += x0.x + x1.x;
      ti += x0.y + x1.y;
      if (kTrace) {
        if (c_0 == 0) { ta += x0.x * x0.x + x0.y * x0.y; tbr += x0.x; tbi += x0.y; tc += 1.f; }
        if (c_1 == 0) { ta += x1.x * x1.x + x1.y * x1.y; tbr += x1.x; tbi += x1.y; tc += 1.f; }
      }
    }
#pragma unroll
    for (int j = 0; j < kVecPerThread; ++j) dst[vb + 32 * j] = T.v[j];
    acc[0].add(tr);
    acc[1].add(ti);
    if (kTrace) { acc[2].add(ta); acc[3].add(tbr); acc[4].add(tbi); acc[5 % kVals].add(tc); }
  };
  pipelined_tiles(local, a.cpi, a.ntiles, load, proc);
  reduce_to_record<kVals>(a, b, local, acc, s_w, s_vals);
}

// ---------------------------------------------------------------------------
// K4: readout. kPending: dst <- psi_p = src + a_p first (materialise).
// ---------------------------------------------------------------------------
template <bool kPending>
__global__ void __launch_bounds__(kThreads, kFwdPerSm) readout_kernel(const PassArgs a) {
  __shared__ float2 s_a;
  __shared__ double s_w[kWarps][kPartStride];
  __shared__ double s_vals[kPartStride];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int b = blockIdx.x / a.cpi, local = blockIdx.x % a.cpi;
  pdl_wait_then_release();
  if (warp == 0) {
    double2 av = make_double2(0.0, 0.0);
    if (kPending) {
      const size_t bk = (size_t)b * a.p + a.round;  // round = last round index
      const double Sre = w0_parts(a, b, 0), Sim = w0_parts(a, b, 1);
      const double2 al = a.alpha[bk];
      av = make_double2((al.x * Sre - al.y * Sim) * a.inv_n, (al.x * Sim + al.y * Sre) * a.inv_n);
      if (local == 0 && lane == 0) {
        double *rec = a.record + 4 * bk;
        rec[0] = Sre; rec[1] = Sim; rec[2] = av.x; rec[3] = av.y;
      }
    }
    if (lane == 0) s_a = make_float2((float)av.x, (float)av.y);
  }
  __syncthreads();
  const float2 ad = s_a;
  DF acc[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) acc[j].zero();
  const uint16_t *__restrict__ cost2 =
      reinterpret_cast<const uint16_t *>(a.cost + (size_t)b * a.cost_bstride);
  const float4 *__restrict__ src = a.src + (size_t)b * (a.N / 2);
  float4 *dst = a.dst + (size_t)b * (a.N / 2);
  const bool reverse = kPending && ((a.round + 1) & 1) != 0;
  auto vbase = [&](uint64_t t) {
    return tile_vbase(reverse ? (a.ntiles - 1 - t) : t, warp, lane);
  };
  auto load = [&](TileRegs &T, uint64_t t) {
    const uint64_t vb = vbase(t);
#pragma unroll
    for (int j = 0; j < kVecPerThread; ++j) {
      T.c2[j] = cost2[vb + 32 * j];
      T.v[j] = src[vb + 32 * j];
    }
  };
  auto proc = [&](TileRegs &T, uint64_t t) {
    float tp = 0.f, te = 0.f, tn = 0.f;
#pragma unroll
    for (int j = 0; j < kVecPerThread; ++j) {
      if (kPending)
        T.v[j] = make_float4(T.v[j].x + ad.x, T.v[j].y + ad.y, T.v[j].z + ad.x, T.v[j].w + ad.y);
      const float w0 = T.v[j].x * T.v[j].x + T.v[j].y * T.v[j].y;
      const float w1 = T.v[j].z * T.v[j].z + T.v[j].w * T.v[j].w;
      const unsigned c_0 = T.c2[j] & 0xFFu, c_1 = T.c2[j] >> 8;
      tn += w0 + w1;
      te += (float)c_0 * w0 + (float)c_1 * w1;
      tp += (c_0 == a.target ? w0 : 0.f) + (c_1 == a.target ? w1 : 0.f);
    }
    if (kPending) {
      const uint64_t vb = vbase(t);
#pragma unroll
      for (int j = 0; j < kVecPerThread; ++j) dst[vb + 32 * j] = T.v[j];
    }
    acc[0].add(tp);
    acc[1].add(te);
    acc[2].add(tn);
  };
  pipelined_tiles(local, a.cpi, a.ntiles, load, proc);
  reduce_to_record<3>(a, b, local, acc, s_w, s_vals);
}

// K4 fused with the sampler's first pass (gqaoa_evolve_sample): psi_p =
// chi_p + a_p is formed in registers exactly as readout_kernel<true> forms it
// and is not written back; the pass makes the readouts of readout_kernel and,
// per tile, the sampler's tile total and chunk prefixes of psi_p (cdf.cuh).
// One instance (B = 1). add_out receives a_p as the float pair the pass
// added, so the sampler can add it again when it walks a chunk.
__global__ void __launch_bounds__(kThreads, kFwdPerSm)
readout_sample_kernel(const PassArgs a, double *__restrict__ tsum, double *__restrict__ chunk_incl,
                      float2 *__restrict__ add_out) {
  __shared__ float2 s_a;
  __shared__ double s_w[kWarps][kPartStride];
  __shared__ double s_vals[kPartStride];
  __shared__ double s_incl[kChunksPerTile];
  __shared__ float2 s_wtot[kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int local = blockIdx.x;
  pdl_wait_then_release();
  if (warp == 0) {
    const size_t bk = (size_t)a.round;  // the last round
    const double Sre = w0_parts(a, 0, 0), Sim = w0_parts(a, 0, 1);
    const double2 al = a.alpha[bk];
    const double2 av = make_double2((al.x * Sre - al.y * Sim) * a.inv_n,
                                    (al.x * Sim + al.y * Sre) * a.inv_n);
    if (local == 0 && lane == 0) {
      double *rec = a.record + 4 * bk;
      rec[0] = Sre; rec[1] = Sim; rec[2] = av.x; rec[3] = av.y;
      *add_out = make_float2((float)av.x, (float)av.y);
    }
    if (lane == 0) s_a = make_float2((float)av.x, (float)av.y);
  }
  __syncthreads();
  const float2 ad = s_a;
  DF acc[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) acc[j].zero();
  const uint16_t *__restrict__ cost2 = reinterpret_cast<const uint16_t *>(a.cost);
  const float4 *__restrict__ src = a.src;
  const bool reverse = ((a.round + 1) & 1) != 0;
  auto tile_of = [&](uint64_t t) { return reverse ? (a.ntiles - 1 - t) : t; };
  auto load = [&](TileRegs &T, uint64_t t) {
    const uint64_t vb = tile_vbase(tile_of(t), warp, lane);
#pragma unroll
    for (int j = 0; j < kVecPerThread; ++j) {
      T.c2[j] = cost2[vb + 32 * j];
      T.v[j] = src[vb + 32 * j];
    }
  };
  auto proc = [&](TileRegs &T, uint64_t t) {
    float tp = 0.f, te = 0.f, tn = 0.f;
#pragma unroll
    for (int j = 0; j < kVecPerThread; ++j) {
      T.v[j] = make_float4(T.v[j].x + ad.x, T.v[j].y + ad.y, T.v[j].z + ad.x, T.v[j].w + ad.y);
      const float w0 = T.v[j].x * T.v[j].x + T.v[j].y * T.v[j].y;
      const float w1 = T.v[j].z * T.v[j].z + T.v[j].w * T.v[j].w;
      const unsigned c_0 = T.c2[j] & 0xFFu, c_1 = T.c2[j] >> 8;
      tn += w0 + w1;
      te += (float)c_0 * w0 + (float)c_1 * w1;
      tp += (c_0 == a.target ? w0 : 0.f) + (c_1 == a.target ? w1 : 0.f);
    }
    acc[0].add(tp);
    acc[1].add(te);
    acc[2].add(tn);
    const uint64_t tile = tile_of(t);
    float ch, cl;
    tile_chunk_scan_regs(T.v, s_incl, s_wtot, ch, cl, nullptr);
    chunk_incl[tile * kChunksPerTile + threadIdx.x] = s_incl[threadIdx.x];
    if (threadIdx.x == 0) tsum[tile] = tile_total(s_wtot);
    __syncthreads();  // s_wtot and s_incl are rewritten for the next tile
  };
  pipelined_tiles(local, a.cpi, a.ntiles, load, proc);
  reduce_to_record<3>(a, 0, local, acc, s_w, s_vals);
}

// One warp per instance: out[b][0..2] from the readout records, and the
// last trace entry.
__global__ void finalize_readout_kernel(const double *__restrict__ parts, int nparts, int p,
                                        double *__restrict__ out, double *__restrict__ trace) {
  const int b = blockIdx.x, lane = threadIdx.x;
  const double *base = parts + (size_t)b * nparts * kPartStride;
  double v[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    double x = 0.0;
    for (int i = lane; i < nparts; i += 32) x += base[(size_t)i * kPartStride + j];
    v[j] = warp_sum(x);
  }
  if (lane == 0) {
    if (out) { out[3 * b] = v[0]; out[3 * b + 1] = v[1]; out[3 * b + 2] = v[2]; }
    if (trace) trace[(size_t)b * p + p - 1] = v[0];
  }
}

// A thread's share of half a tile of an adjoint pass: 4 float4 of lambda,
// 4 of the checkpoint chi, and their costs.
constexpr int kHalfVec = kVecPerThread / 2;
struct HalfRegs {
  float4 l[kHalfVec];
  float4 x[kHalfVec];
  uint16_t c2[kHalfVec];
};

// ---------------------------------------------------------------------------
// K6: adjoint. lambda_p = O psi_p, psi_p = chi_p + a_p (chi_p = checkpoint).
// Records: 0,1 = Lambda_p; 2 = L = sum O |psi_p|^2.
// ---------------------------------------------------------------------------
template <int kObj>
__global__ void __launch_bounds__(kThreads, kBwdPerSm) lambda_init_kernel(const PassArgs a) {
  __shared__ float2 s_a;
  __shared__ double s_w[kWarps][kPartStride];
  __shared__ double s_vals[kPartStride];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int b = blockIdx.x / a.cpi, local = blockIdx.x % a.cpi;
  const size_t bk = (size_t)b * a.p + a.round;  // last forward round
  pdl_wait_then_release();
  if (warp == 0) {
    const double Sre = w0_parts(a, b, 0), Sim = w0_parts(a, b, 1);
    const double2 al = a.alpha[bk];
    const double2 av =
        make_double2((al.x * Sre - al.y * Sim) * a.inv_n, (al.x * Sim + al.y * Sre) * a.inv_n);
    if (local == 0 && lane == 0) {
      double *rec = a.record + 4 * bk;
      rec[0] = Sre; rec[1] = Sim; rec[2] = av.x; rec[3] = av.y;
    }
    if (lane == 0) s_a = make_float2((float)av.x, (float)av.y);
  }
  __syncthreads();
  const float2 ad = s_a;
  DF acc[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) acc[j].zero();
  const uint16_t *__restrict__ cost2 =
      reinterpret_cast<const uint16_t *>(a.cost + (size_t)b * a.cost_bstride);
  const float4 *__restrict__ src = a.src + (size_t)b * (a.N / 2);
  float4 *dst = a.dst + (size_t)b * (a.N / 2);
  // against the last forward pass's direction: its tail is still in L2
  const bool reverse = ((a.round + 1) & 1) != 0;
  auto vbase = [&](uint64_t t) {
    return tile_vbase(reverse ? (a.ntiles - 1 - t) : t, warp, lane);
  };
  auto load = [&](TileRegs &T, uint64_t t) {
    const uint64_t vb = vbase(t);
#pragma unroll
    for (int j = 0; j < kVecPerThread; ++j) {
      T.c2[j] = cost2[vb + 32 * j];
      T.v[j] = src[vb + 32 * j];
    }
  };
  auto proc = [&](TileRegs &T, uint64_t t) {
    const uint64_t vb = vbase(t);
    float tlr = 0.f, tli = 0.f, tL = 0.f;
#pragma unroll
    for (int j = 0; j < kVecPerThread; ++j) {
      const uint16_t c2 = T.c2[j];
      const float4 v = T.v[j];
      const float o0 = kObj == GQAOA_OBJ_P0 ? ((c2 & 0xFFu) == a.target ? 1.f : 0.f) : (float)(c2 & 0xFFu);
      const float o1 = kObj == GQAOA_OBJ_P0 ? ((c2 >> 8) == a.target ? 1.f : 0.f) : (float)(c2 >> 8);
      const float2 p0 = make_float2(v.x + ad.x, v.y + ad.y);
      const float2 p1 = make_float2(v.z + ad.x, v.w + ad.y);
      const float4 l = make_float4(o0 * p0.x, o0 * p0.y, o1 * p1.x, o1 * p1.y);
      dst[vb + 32 * j] = l;
      tlr += l.x + l.z;
      tli += l.y + l.w;
      tL += o0 * (p0.x * p0.x + p0.y * p0.y) + o1 * (p1.x * p1.x + p1.y * p1.y);
    }
    acc[0].add(tlr);
    acc[1].add(tli);
    acc[2].add(tL);
  };
  pipelined_tiles(local, a.cpi, a.ntiles, load, proc);
  reduce_to_record<3>(a, b, local, acc, s_w, s_vals);
}

// Backward pass of round r (0-based). src = lambda_r (in place -> lambda_{r-1}),
// chi = checkpoint chi_r. Records in: 0,1 = Lambda_r; 2 = G_{r+1} (or L when
// r = p-1). Records out: 0,1 = Lambda_{r-1}; 2 = G_r.
template <bool kFirst, bool kLast>
__global__ void __launch_bounds__(kThreads, kBwdPerSm)
backward_kernel(const PassArgs a, const float4 *__restrict__ chi_base) {
  __shared__ float2 s_T[256];
  __shared__ float2 s_b;
  __shared__ double s_w[kWarps][kPartStride];
  __shared__ double s_vals[kPartStride];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int b = blockIdx.x / a.cpi, local = blockIdx.x % a.cpi;
  const size_t bk = (size_t)b * a.p + a.round;
  pdl_wait_then_release();
  s_T[threadIdx.x] = a.phase[bk * 256 + threadIdx.x];
  if (warp == 0) {
    const double Lr = w0_parts(a, b, 0), Li = w0_parts(a, b, 1), G = w0_parts(a, b, 2);
    const double2 al = a.alpha[bk];
    // b_r = conj(alpha_r) Lambda_r / N
    const double2 bv =
        make_double2((al.x * Lr + al.y * Li) * a.inv_n, (al.x * Li - al.y * Lr) * a.inv_n);
    if (local == 0 && lane == 0) {
      const double *rec = a.record + 4 * bk;
      const double Sre = rec[0] * a.inv_n, Sim = rec[1] * a.inv_n;
      // e^{-i beta} = alpha + 1; w = e^{-i beta} (S/N) conj(Lambda)
      const double er = al.x + 1.0, ei = al.y;
      const double qr = er * Sre - ei * Sim, qi = er * Sim + ei * Sre;
      const double wi = qi * Lr - qr * Li;  // Im(w)
      a.dbeta[bk] = 2.0 * wi;  // 2 Re(-i w) = 2 Im(w)
      if (kFirst) a.value[b] = G;
      else a.dgamma[bk + 1] = 2.0 * G;
    }
    if (lane == 0) s_b = make_float2((float)bv.x, (float)bv.y);
  }
  __syncthreads();
  const float2 bd = s_b;
  DF acc[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) acc[j].zero();
  const uint16_t *__restrict__ cost2 =
      reinterpret_cast<const uint16_t *>(a.cost + (size_t)b * a.cost_bstride);
  const float4 *__restrict__ lam = a.src + (size_t)b * (a.N / 2);
  const float4 *__restrict__ chi = chi_base + (size_t)b * (a.N / 2);
  float4 *dst = a.dst + (size_t)b * (a.N / 2);
  // Half-tile units (4 float4 of lambda and of chi per thread), two in
  // flight: the loads of the next unit are issued before the current one is
  // processed. Alternate direction per pass: the previous pass's tail of
  // lambda is still in L2.
  const bool reverse = (a.round & 1) != 0;
  const uint64_t mine = a.ntiles > (uint64_t)local ? (a.ntiles - 1 - local) / a.cpi + 1 : 0;
  const uint64_t nu = 2 * mine;
  auto vbase = [&](uint64_t u) {
    const uint64_t t = local + (u >> 1) * a.cpi;
    return tile_vbase(reverse ? (a.ntiles - 1 - t) : t, warp, lane) +
           (u & 1) * (32 * kHalfVec);
  };
  auto load = [&](HalfRegs &H, uint64_t u) {
    const uint64_t vb = vbase(u);
#pragma unroll
    for (int j = 0; j < kHalfVec; ++j) H.c2[j] = cost2[vb + 32 * j];
#pragma unroll
    for (int j = 0; j < kHalfVec; ++j) H.l[j] = lam[vb + 32 * j];
#pragma unroll
    for (int j = 0; j < kHalfVec; ++j) H.x[j] = chi[vb + 32 * j];
  };
  auto proc = [&](HalfRegs &H, uint64_t u) {
    const uint64_t vb = vbase(u);
    float tg = 0.f, tlr = 0.f, tli = 0.f;
#pragma unroll
    for (int j = 0; j < kHalfVec; ++j) {
      const float4 l = H.l[j], x = H.x[j];
      const unsigned c_0 = H.c2[j] & 0xFFu, c_1 = H.c2[j] >> 8;
      const float2 m0 = make_float2(l.x + bd.x, l.y + bd.y);
      const float2 m1 = make_float2(l.z + bd.x, l.w + bd.y);
      // Im(conj(mu) chi) = mu.re chi.im - mu.im chi.re
      tg += (float)c_0 * (m0.x * x.y - m0.y * x.x) + (float)c_1 * (m1.x * x.w - m1.y * x.z);
      if (!kLast) {
        const float2 T0 = s_T[c_0], T1 = s_T[c_1];
        // conj(T) mu
        const float2 n0 = make_float2(fmaf(T0.x, m0.x, T0.y * m0.y), fmaf(T0.x, m0.y, -T0.y * m0.x));
        const float2 n1 = make_float2(fmaf(T1.x, m1.x, T1.y * m1.y), fmaf(T1.x, m1.y, -T1.y * m1.x));
        dst[vb + 32 * j] = make_float4(n0.x, n0.y, n1.x, n1.y);
        tlr += n0.x + n1.x;
        tli += n0.y + n1.y;
      }
    }
    acc[0].add(tlr);
    acc[1].add(tli);
    acc[2].add(tg);
  };
  HalfRegs A, Bh;
  uint64_t u = 0;
  if (u < nu) load(A, u);
  for (; u < nu; u += 2) {
    if (u + 1 < nu) load(Bh, u + 1);
    proc(A, u);
    if (u + 1 < nu) {
      if (u + 2 < nu) load(A, u + 2);
      proc(Bh, u + 1);
    }
  }
  reduce_to_record<3>(a, b, local, acc, s_w, s_vals);
}

// dgamma of round 0 from the last backward pass (one warp per instance).
__global__ void finalize_grad_kernel(const double *__restrict__ parts, int nparts, int p,
                                     double *__restrict__ dgamma) {
  const int b = blockIdx.x, lane = threadIdx.x;
  const double *base = parts + (size_t)b * nparts * kPartStride;
  double x = 0.0;
  for (int i = lane; i < nparts; i += 32) x += base[(size_t)i * kPartStride + 2];
  x = warp_sum(x);
  if (lane == 0) dgamma[(size_t)b * p] = 2.0 * x;
}

// ---------------------------------------------------------------------------
// small states (N <= 2048): one CTA per instance keeps the state in registers
// ---------------------------------------------------------------------------
constexpr int kSmallPer = 8;  // 256 threads x 8 = 2048 amplitudes

struct SmallArgs {
  const uint8_t *cost;
  uint64_t cost_bstride;
  int n;
  int p;
  const float2 *phase;   // [B][p][256]
  const double2 *alpha;  // [B][p]
  float2 *state;         // [B][N]
  bool from_state;
  double *out;           // [B][3] or null
  double *trace;         // [B][p] or null
  double *record;        // [B][p][4]
  float2 *ckpt;          // [p][B][N] or null (gradient forward)
  int B;
  unsigned target;       // the cost class of out[0] and of the projector objective
};

// Sum of two FP32 values per thread over the CTA, every thread getting the
// FP64 results: a double-float butterfly per warp, then the warps' partials
// in warp order, also in double-float. The rounds of the small-state kernels
// reduce this way so that their per-amplitude work stays on the FP32 pipe
// (GB300's FP64 rate is a small fraction of it). scr: 2 kWarps float2.
__device__ __forceinline__ double2 block_sum_df2(float x, float y, float2 *scr) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float xl = 0.f, yl = 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float xh2 = __shfl_xor_sync(0xffffffffu, x, o), xl2 = __shfl_xor_sync(0xffffffffu, xl, o);
    const float yh2 = __shfl_xor_sync(0xffffffffu, y, o), yl2 = __shfl_xor_sync(0xffffffffu, yl, o);
    float s, e;
    two_sum(x, xh2, s, e);
    x = s;
    xl = __fadd_rn(__fadd_rn(xl, xl2), e);
    two_sum(y, yh2, s, e);
    y = s;
    yl = __fadd_rn(__fadd_rn(yl, yl2), e);
  }
  __syncthreads();  // scr is free (its last readers are past this point)
  if (lane == 0) {
    scr[warp] = make_float2(x, xl);
    scr[kWarps + warp] = make_float2(y, yl);
  }
  __syncthreads();
  float hx = 0.f, lx = 0.f, hy = 0.f, ly = 0.f;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    const float2 px = scr[w], py = scr[kWarps + w];
    float s, e;
    two_sum(hx, px.x, s, e);
    hx = s;
    lx = __fadd_rn(lx, __fadd_rn(e, px.y));
    two_sum(hy, py.x, s, e);
    hy = s;
    ly = __fadd_rn(ly, __fadd_rn(e, py.y));
  }
  return make_double2((double)hx + (double)lx, (double)hy + (double)ly);
}

// One round of the small-state kernel on a thread's amplitudes; writes the
// round's record (S_k, a_k), the checkpoint chi_k if asked, and, if P is
// given, *P = P(C=0) of the round's state.
__device__ __forceinline__ void small_round(float2 (&s)[kSmallPer], const unsigned (&c)[kSmallPer],
                                            const float2 *T, const double2 al, int N, double inv_n,
                                            float2 *s_scr, float2 *ck, double *rec, double *P) {
  float lr = 0.f, li = 0.f;
#pragma unroll
  for (int j = 0; j < kSmallPer; ++j) {
    const int z = threadIdx.x + j * kThreads;
    if (z < N) {
      s[j] = cmul(T[c[j]], s[j]);
      if (ck) ck[z] = s[j];
      lr += s[j].x;
      li += s[j].y;
    }
  }
  const double2 S = block_sum_df2(lr, li, s_scr);
  const double Sre = S.x, Sim = S.y;
  const double ar = (al.x * Sre - al.y * Sim) * inv_n, ai = (al.x * Sim + al.y * Sre) * inv_n;
  const float2 af = make_float2((float)ar, (float)ai);
  float lp = 0.f;
#pragma unroll
  for (int j = 0; j < kSmallPer; ++j) {
    const int z = threadIdx.x + j * kThreads;
    if (z < N) {
      s[j] = make_float2(s[j].x + af.x, s[j].y + af.y);
      if (P && c[j] == 0) lp += fmaf(s[j].x, s[j].x, s[j].y * s[j].y);
    }
  }
  if (P) *P = block_sum_df2(lp, 0.f, s_scr).x;
  if (threadIdx.x == 0) { rec[0] = Sre; rec[1] = Sim; rec[2] = ar; rec[3] = ai; }
}

__global__ void __launch_bounds__(kThreads) evolve_small_kernel(const SmallArgs a) {
  __shared__ double s_scr[kWarps];
  __shared__ float2 s_df[2 * kWarps];
  const int b = blockIdx.x;
  const int N = 1 << a.n;
  const double inv_n = 1.0 / (double)N;
  const uint8_t *cost = a.cost + (size_t)b * a.cost_bstride;
  float2 *state = a.state + (size_t)b * N;
  float2 s[kSmallPer];
  unsigned c[kSmallPer];
  const float amp0 = (float)(1.0 / sqrt((double)N));
#pragma unroll
  for (int j = 0; j < kSmallPer; ++j) {
    const int z = threadIdx.x + j * kThreads;
    c[j] = z < N ? cost[z] : 0u;
    s[j] = z < N ? (a.from_state ? state[z] : make_float2(amp0, 0.f)) : make_float2(0.f, 0.f);
  }
  for (int k = 0; k < a.p; ++k) {
    const size_t bk = (size_t)b * a.p + k;
    double P = 0.0;
    float2 *ck = a.ckpt ? a.ckpt + ((size_t)k * a.B + b) * N : nullptr;
    small_round(s, c, a.phase + bk * 256, a.alpha[bk], N, inv_n, s_df, ck, a.record + 4 * bk,
                a.trace ? &P : nullptr);
    if (a.trace && threadIdx.x == 0) a.trace[bk] = P;
  }
  double lp = 0.0, le = 0.0, ln = 0.0;
#pragma unroll
  for (int j = 0; j < kSmallPer; ++j) {
    const int z = threadIdx.x + j * kThreads;
    if (z < N) {
      if (!a.ckpt) state[z] = s[j];
      const double w = (double)s[j].x * s[j].x + (double)s[j].y * s[j].y;
      ln += w;
      le += (double)c[j] * w;
      if (c[j] == a.target) lp += w;
    }
  }
  const double P = block_sum(lp, s_scr);
  const double E = block_sum(le, s_scr);
  const double Nm = block_sum(ln, s_scr);
  if (threadIdx.x == 0 && a.out) { a.out[3 * b] = P; a.out[3 * b + 1] = E; a.out[3 * b + 2] = Nm; }
}

// Small-state adjoint: one CTA per instance; forward checkpoints were written
// by evolve_small_kernel (ckpt mode), records hold S_k and a_k.
__global__ void __launch_bounds__(kThreads)
grad_small_kernel(const SmallArgs a, int objective, double *__restrict__ value,
                  double *__restrict__ dgamma, double *__restrict__ dbeta) {
  __shared__ double s_scr[kWarps];
  __shared__ float2 s_df[2 * kWarps];
  const int b = blockIdx.x;
  const int N = 1 << a.n;
  const double inv_n = 1.0 / (double)N;
  const uint8_t *cost = a.cost + (size_t)b * a.cost_bstride;
  unsigned c[kSmallPer];
  float2 l[kSmallPer];
  const size_t last = (size_t)b * a.p + (a.p - 1);
  const float2 ap = make_float2((float)a.record[4 * last + 2], (float)a.record[4 * last + 3]);
  const float2 *chip = a.ckpt + ((size_t)(a.p - 1) * a.B + b) * N;
  double lv = 0.0;
#pragma unroll
  for (int j = 0; j < kSmallPer; ++j) {
    const int z = threadIdx.x + j * kThreads;
    c[j] = z < N ? cost[z] : 0u;
    l[j] = make_float2(0.f, 0.f);
    if (z < N) {
      const float2 ps = make_float2(chip[z].x + ap.x, chip[z].y + ap.y);
      const float o = objective == GQAOA_OBJ_P0 ? (c[j] == a.target ? 1.f : 0.f) : (float)c[j];
      l[j] = make_float2(o * ps.x, o * ps.y);
      lv += (double)o * ((double)ps.x * ps.x + (double)ps.y * ps.y);
    }
  }
  const double L = block_sum(lv, s_scr);
  if (threadIdx.x == 0) value[b] = L;
  for (int k = a.p - 1; k >= 0; --k) {
    const size_t bk = (size_t)b * a.p + k;
    float lr = 0.f, li = 0.f;
#pragma unroll
    for (int j = 0; j < kSmallPer; ++j) {
      const int z = threadIdx.x + j * kThreads;
      if (z < N) { lr += l[j].x; li += l[j].y; }
    }
    const double2 Ls = block_sum_df2(lr, li, s_df);
    const double Lr = Ls.x, Li = Ls.y;
    const double2 al = a.alpha[bk];
    const float2 bv = make_float2((float)((al.x * Lr + al.y * Li) * inv_n),
                                  (float)((al.x * Li - al.y * Lr) * inv_n));
    const float2 *T = a.phase + bk * 256;
    const float2 *chi = a.ckpt + ((size_t)k * a.B + b) * N;
    float g = 0.f;
#pragma unroll
    for (int j = 0; j < kSmallPer; ++j) {
      const int z = threadIdx.x + j * kThreads;
      if (z < N) {
        const float2 mu = make_float2(l[j].x + bv.x, l[j].y + bv.y);
        const float2 x = chi[z];
        g = fmaf((float)c[j], fmaf(mu.x, x.y, -mu.y * x.x), g);
        const float2 t = T[c[j]];
        l[j] = make_float2(fmaf(t.x, mu.x, t.y * mu.y), fmaf(t.x, mu.y, -t.y * mu.x));
      }
    }
    const double G = block_sum_df2(g, 0.f, s_df).x;
    if (threadIdx.x == 0) {
      const double *rec = a.record + 4 * bk;
      const double Sre = rec[0] * inv_n, Sim = rec[1] * inv_n;
      const double er = al.x + 1.0, ei = al.y;
      const double qr = er * Sre - ei * Sim, qi = er * Sim + ei * Sre;
      dbeta[bk] = 2.0 * (qi * Lr - qr * Li);
      dgamma[bk] = 2.0 * G;
    }
  }
}

// ---------------------------------------------------------------------------
// host-side launch helpers
// ---------------------------------------------------------------------------
static std::once_flag g_res_once[kMaxDevices][2];
static int g_res_ctas[kMaxDevices][2];

template <typename Kernel>
static int query_cluster_ctas(Kernel kernel, int per_sm) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kClusterSize, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kClusterSize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, kernel, &cfg) != cudaSuccess || clusters < 1) {
    cudaGetLastError();  // clear a failed query: fall back to the SM count
    return sm_count() * per_sm;
  }
  return clusters * kClusterSize;
}

static int resident_cluster_ctas(int per_sm) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return sm_count() * per_sm;
  }
  const int kind = per_sm == kFwdPerSm ? 0 : 1;
  std::call_once(g_res_once[dev][kind], [dev, kind, per_sm]() {
    g_res_ctas[dev][kind] = kind == 0 ? query_cluster_ctas(round_kernel<kChained, false>, per_sm)
                                      : query_cluster_ctas(backward_kernel<false, false>, per_sm);
  });
  return g_res_ctas[dev][kind];
}
template <typename Kernel, typename... Args>
static cudaError_t launch_pass(const Geometry &g, Kernel kernel, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((size_t)g.B * g.cpi), 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  int na = 0;
  attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[na].val.programmaticStreamSerializationAllowed = 1;
  ++na;
  if (g.cluster > 1) {
    attr[na].id = cudaLaunchAttributeClusterDimension;
    attr[na].val.clusterDim.x = (unsigned)g.cluster;
    attr[na].val.clusterDim.y = 1;
    attr[na].val.clusterDim.z = 1;
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

static int check_common(int n, int m, int B, int p) {
  if (n < 1 || n > GQAOA_MAX_N || m < 0 || m > GQAOA_MAX_M || p < 1 || p > (1 << 20) || B < 1 ||
      B > (1 << 24))
    return GQAOA_ERANGE;
  if ((size_t)B * (size_t)p > ((size_t)1 << 32)) return GQAOA_ERANGE;
  return GQAOA_OK;
}

static void init_pass(PassArgs &pa, const Geometry &g, const Ws &w, const uint8_t *cost,
                      uint64_t cost_bstride, int p) {
  pa = PassArgs{};
  pa.cost = cost;
  pa.cost_bstride = cost_bstride;
  pa.phase = w.phase;
  pa.alpha = w.alpha;
  pa.record = w.record;
  pa.p = p;
  pa.cpi = g.cpi;
  pa.nparts = g.nparts;
  pa.nparts_in = g.nparts;
  pa.ntiles = g.ntiles;
  pa.N = g.N;
  pa.inv_n = 1.0 / (double)g.N;
  pa.amp0 = (float)(1.0 / sqrt((double)g.N));
}

static double *parts_half(const Ws &w, int i) { return w.parts + (size_t)(i & 1) * w.parts_half; }

// Phase tables e^{-i gamma c} (c < entries, a multiple of 32 up to 256; table
// t at phase + t * entries) and alpha = e^{-i beta} - 1 for `count` angle
// pairs (also used by the on-chip sweep and the cost-class model).
int phase_tables(const double *gammas, const double *betas, int64_t count, int entries,
                 float2 *phase, double2 *alpha, cudaStream_t st) {
  if (entries < 32 || entries > 256 || entries % 32 != 0) return GQAOA_EINVAL;
  const int64_t nblk = (count + 31) / 32;  // blocks of 32 tables, one per CTA
  const int64_t cap = (int64_t)sm_count() * 8;
  const int64_t grid = nblk < cap ? nblk : cap;
  phase_table_kernel<<<(unsigned)grid, kPhaseWarps * 32, 0, st>>>(gammas, betas, count, entries,
                                                                  phase, alpha);
  GQ_CHECK_LAUNCH();
  return GQAOA_OK;
}

static int launch_phase_tables(const double *gammas, const double *betas, int64_t bp, const Ws &w,
                               cudaStream_t st) {
  return phase_tables(gammas, betas, bp, 256, w.phase, w.alpha, st);
}

// Forward rounds. In place on `state` (ckpt == null) or chi_k -> ckpt[k].
static int run_forward(const Geometry &g, const Ws &w, const uint8_t *cost, uint64_t cost_bstride,
                       int p, float2 *state, bool from_state, double *trace, float2 *ckpt,
                       cudaStream_t st) {
  PassArgs pa;
  init_pass(pa, g, w, cost, cost_bstride, p);
  pa.trace = trace;
  const size_t inst = (size_t)g.B * g.N;
  for (int k = 0; k < p; ++k) {
    pa.round = k;
    pa.parts_in = parts_half(w, k + 1);
    pa.parts_out = parts_half(w, k);
    if (ckpt) {
      pa.src = reinterpret_cast<const float4 *>(k == 0 ? state : ckpt + (size_t)(k - 1) * inst);
      pa.dst = reinterpret_cast<float4 *>(ckpt + (size_t)k * inst);
    } else {
      pa.src = reinterpret_cast<const float4 *>(state);
      pa.dst = reinterpret_cast<float4 *>(state);
    }
    cudaError_t e;
    const bool tr = trace != nullptr;
    if (k == 0) {
      if (from_state)
        e = tr ? launch_pass(g, round_kernel<kFromState, true>, st, pa)
               : launch_pass(g, round_kernel<kFromState, false>, st, pa);
      else
        e = tr ? launch_pass(g, round_kernel<kFromPlus, true>, st, pa)
               : launch_pass(g, round_kernel<kFromPlus, false>, st, pa);
    } else {
      e = tr ? launch_pass(g, round_kernel<kChained, true>, st, pa)
             : launch_pass(g, round_kernel<kChained, false>, st, pa);
    }
    if (e != cudaSuccess) return GQAOA_ECUDA;
  }
  return GQAOA_OK;
}

static int evolve_impl(const uint8_t *cost, uint64_t cost_bstride, int n, int m, int B,
                       const double *gammas, const double *betas, int p, void *state, double *out,
                       double *trace, void *ws, size_t ws_bytes, unsigned flags, cudaStream_t st) {
  int rc = check_common(n, m, B, p);
  if (rc) return rc;
  if (!cost || !gammas || !betas || !state || !ws) return GQAOA_EINVAL;
  if (flags & ~(GQAOA_STATE_IN | GQAOA_READOUT_CLASS(255))) return GQAOA_EINVAL;
  const unsigned target = (flags >> 8) & 0xFFu;  // the class read out as out[0]
  if (target != 0u && trace) return GQAOA_EINVAL;  // the per-round trace is P(C=0)
  if (!aligned16(state) || !aligned16(cost) || !aligned8(gammas) || !aligned8(betas) ||
      (out && !aligned8(out)) || (trace && !aligned8(trace)) || !aligned16(ws))
    return GQAOA_EINVAL;
  const Geometry g = make_geometry(n, B, kFwdPerSm);
  if (!g.small && cost_bstride % 16 != 0) return GQAOA_EINVAL;
  if (ws_bytes < ws_layout(g, p, false, nullptr, nullptr, g.nparts)) return GQAOA_ENOMEM;
  Ws w;
  ws_layout(g, p, false, static_cast<char *>(ws), &w, g.nparts);
  const bool from_state = (flags & GQAOA_STATE_IN) != 0;
  rc = launch_phase_tables(gammas, betas, (int64_t)B * p, w, st);
  if (rc) return rc;
  if (g.small) {
    SmallArgs sa = {cost, cost_bstride, n, p, w.phase, w.alpha, static_cast<float2 *>(state),
                    from_state, out, trace, w.record, nullptr, B, target};
    evolve_small_kernel<<<B, kThreads, 0, st>>>(sa);
    GQ_CHECK_LAUNCH();
    return GQAOA_OK;
  }
  rc = run_forward(g, w, cost, cost_bstride, p, static_cast<float2 *>(state), from_state, trace,
                   nullptr, st);
  if (rc) return rc;
  PassArgs pa;
  init_pass(pa, g, w, cost, cost_bstride, p);
  pa.round = p - 1;
  pa.parts_in = parts_half(w, p - 1);
  pa.parts_out = parts_half(w, p);
  pa.src = static_cast<const float4 *>(state);
  pa.dst = static_cast<float4 *>(state);
  pa.target = target;
  if (launch_pass(g, readout_kernel<true>, st, pa) != cudaSuccess) return GQAOA_ECUDA;
  finalize_readout_kernel<<<B, 32, 0, st>>>(pa.parts_out, g.nparts, p, out, trace);
  GQ_CHECK_LAUNCH();
  return GQAOA_OK;
}

bool adjoint_cluster_fits(int n, int B);
int adjoint_cluster(const uint8_t *cost, uint64_t cost_bstride, int n, int B, int p,
                    const float2 *phase, const double2 *alpha, double *record, float2 *ckpt,
                    int objective, unsigned target, double *value, double *dgamma,
                    double *dbeta, unsigned *status, cudaStream_t st);

static int grad_impl(const uint8_t *cost, uint64_t cost_bstride, int n, int m, int B,
                     const double *gammas, const double *betas, int p, int objective, double *value,
                     double *dgamma, double *dbeta, void *ws, size_t ws_bytes, cudaStream_t st) {
  int rc = check_common(n, m, B, p);
  if (rc) return rc;
  if (!cost || !gammas || !betas || !value || !dgamma || !dbeta || !ws) return GQAOA_EINVAL;
  const bool streaming = (objective & GQAOA_GRAD_STREAMING) != 0;
  objective &= ~GQAOA_GRAD_STREAMING;
  // GQAOA_OBJ_CLASS(c): the projector objective on cost class c (P0 is class 0)
  unsigned target = 0u;
  if (objective >= GQAOA_OBJ_CLASS(0) && objective <= GQAOA_OBJ_CLASS(255)) {
    target = (unsigned)(objective - GQAOA_OBJ_CLASS(0));
    objective = GQAOA_OBJ_P0;
  } else if (objective != GQAOA_OBJ_P0 && objective != GQAOA_OBJ_ENERGY) {
    return GQAOA_EINVAL;
  }
  if (!aligned16(cost) || !aligned8(gammas) || !aligned8(betas) || !aligned8(value) ||
      !aligned8(dgamma) || !aligned8(dbeta) || !aligned16(ws))
    return GQAOA_EINVAL;
  const Geometry g = make_geometry(n, B, kFwdPerSm);   // forward passes
  const Geometry gb = make_geometry(n, B, kBwdPerSm);  // adjoint passes
  if (!g.small && cost_bstride % 16 != 0) return GQAOA_EINVAL;
  const int maxp = g.nparts > gb.nparts ? g.nparts : gb.nparts;
  if (ws_bytes < ws_layout(g, p, true, nullptr, nullptr, maxp)) return GQAOA_ENOMEM;
  Ws w;
  ws_layout(g, p, true, static_cast<char *>(ws), &w, maxp);
  rc = launch_phase_tables(gammas, betas, (int64_t)B * p, w, st);
  if (rc) return rc;
  if (!streaming && adjoint_cluster_fits(n, B))  // every round of a row on one cluster
    return adjoint_cluster(cost, cost_bstride, n, B, p, w.phase, w.alpha, w.record, w.ckpt,
                           objective, target, value, dgamma, dbeta,
                           reinterpret_cast<unsigned *>(w.parts), st);  // parts: unused here
  if (g.small) {
    SmallArgs sa = {cost, cost_bstride, n, p, w.phase, w.alpha, w.lambda, false, nullptr,
                    nullptr, w.record, w.ckpt, B, target};
    evolve_small_kernel<<<B, kThreads, 0, st>>>(sa);
    GQ_CHECK_LAUNCH();
    grad_small_kernel<<<B, kThreads, 0, st>>>(sa, objective, value, dgamma, dbeta);
    GQ_CHECK_LAUNCH();
    return GQAOA_OK;
  }
  // forward: chi_k -> ckpt[k]; round 0 synthesises |+> (src unused)
  rc = run_forward(g, w, cost, cost_bstride, p, w.lambda, false, nullptr, w.ckpt, st);
  if (rc) return rc;
  const size_t inst = (size_t)g.B * g.N;
  PassArgs pa;
  init_pass(pa, gb, w, cost, cost_bstride, p);
  pa.value = value;
  pa.dgamma = dgamma;
  pa.dbeta = dbeta;
  pa.target = target;
  // lambda_p = O psi_p (reads the last forward pass's records)
  pa.nparts_in = g.nparts;
  pa.round = p - 1;
  pa.parts_in = parts_half(w, p - 1);
  pa.parts_out = parts_half(w, p);
  pa.src = reinterpret_cast<const float4 *>(w.ckpt + (size_t)(p - 1) * inst);
  pa.dst = reinterpret_cast<float4 *>(w.lambda);
  cudaError_t e = objective == GQAOA_OBJ_P0 ? launch_pass(gb, lambda_init_kernel<GQAOA_OBJ_P0>, st, pa)
                                            : launch_pass(gb, lambda_init_kernel<GQAOA_OBJ_ENERGY>, st, pa);
  if (e != cudaSuccess) return GQAOA_ECUDA;
  pa.nparts_in = gb.nparts;
  int half = p;
  for (int r = p - 1; r >= 0; --r) {
    pa.round = r;
    pa.parts_in = parts_half(w, half);
    pa.parts_out = parts_half(w, half + 1);
    ++half;
    pa.src = reinterpret_cast<const float4 *>(w.lambda);
    pa.dst = reinterpret_cast<float4 *>(w.lambda);
    const float4 *chi = reinterpret_cast<const float4 *>(w.ckpt + (size_t)r * inst);
    const bool first = r == p - 1, last = r == 0;
    if (first && last) e = launch_pass(gb, backward_kernel<true, true>, st, pa, chi);
    else if (first) e = launch_pass(gb, backward_kernel<true, false>, st, pa, chi);
    else if (last) e = launch_pass(gb, backward_kernel<false, true>, st, pa, chi);
    else e = launch_pass(gb, backward_kernel<false, false>, st, pa, chi);
    if (e != cudaSuccess) return GQAOA_ECUDA;
  }
  finalize_grad_kernel<<<B, 32, 0, st>>>(parts_half(w, half), gb.nparts, p, dgamma);
  GQ_CHECK_LAUNCH();
  return GQAOA_OK;
}

}  // namespace gq

using namespace gq;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" int gqaoa_evolve_workspace_size(int n, int p, size_t *bytes) {
  return gqaoa_evolve_batched_workspace_size(n, 1, p, bytes);
}

extern "C" int gqaoa_evolve_batched_workspace_size(int n, int batch, int p, size_t *bytes) {
  if (!bytes) return GQAOA_EINVAL;
  int rc = check_common(n, 0, batch, p);
  if (rc) return rc;
  const Geometry g = make_geometry(n, batch, kFwdPerSm);
  *bytes = ws_layout(g, p, false, nullptr, nullptr, g.nparts);
  return GQAOA_OK;
}

extern "C" int gqaoa_evolve(const uint8_t *cost, int n, int m, const double *gammas,
                            const double *betas, int p, void *state, double *out, double *trace,
                            void *ws, size_t ws_bytes, unsigned flags, void *stream) {
  gq::NvtxRange nvtx_range("gqaoa_evolve");
  return evolve_impl(cost, 0, n, m, 1, gammas, betas, p, state, out, trace, ws, ws_bytes, flags,
                     static_cast<cudaStream_t>(stream));
}

extern "C" int gqaoa_evolve_batched(const uint8_t *cost, int64_t cost_stride, int n, int m,
                                    int batch, const double *gammas, const double *betas, int p,
                                    void *state, double *out, double *trace, void *ws,
                                    size_t ws_bytes, unsigned flags, void *stream) {
  gq::NvtxRange nvtx_range("gqaoa_evolve_batched");
  if (cost_stride < 0) return GQAOA_EINVAL;
  return evolve_impl(cost, (uint64_t)cost_stride, n, m, batch, gammas, betas, p, state, out, trace,
                     ws, ws_bytes, flags, static_cast<cudaStream_t>(stream));
}

extern "C" int gqaoa_batched_geometry(int n, int batch, int adjoint, int *ctas_per_instance,
                                      int *records_per_instance) {
  if (!ctas_per_instance || !records_per_instance) return GQAOA_EINVAL;
  int rc = check_common(n, 0, batch, 1);
  if (rc) return rc;
  const Geometry g = make_geometry(n, batch, adjoint ? kBwdPerSm : kFwdPerSm);
  *ctas_per_instance = g.cpi;
  *records_per_instance = g.nparts;
  return GQAOA_OK;
}

namespace gq {
// The sampler's part of gqaoa_evolve_sample (sample.cu): direct mode, its
// workspace layout and the passes after the tile totals.
bool sample_direct_ok(uint64_t ntiles, int64_t shots);
size_t sample_direct_ws(uint64_t ntiles, int64_t shots, char *base, double **tsum,
                        double **chunk_incl);
int sample_direct_tail(const float4 *state, const float2 *add, uint64_t ntiles, uint64_t seed,
                       int64_t shots, uint64_t *out_idx, void *ws, cudaStream_t st);
}  // namespace gq

// Layout of gqaoa_evolve_sample's workspace: the evolution's, then a_p (256
// bytes), then the sampler's.
static size_t evolve_sample_layout(int n, int p, int64_t shots, size_t *o_add, size_t *o_samp) {
  size_t ev = 0, sa = 0;
  gqaoa_evolve_workspace_size(n, p, &ev);
  gqaoa_sample_workspace_size(n, shots, &sa);
  const size_t a0 = round_up(ev, 256), s0 = a0 + 256;
  if (o_add) *o_add = a0;
  if (o_samp) *o_samp = s0;
  return s0 + sa;
}

extern "C" int gqaoa_evolve_sample_workspace_size(int n, int p, int64_t shots, size_t *bytes) {
  if (!bytes) return GQAOA_EINVAL;
  int rc = check_common(n, 0, 1, p);
  if (rc) return rc;
  if (shots < 0 || shots >= (1ll << 32)) return GQAOA_ERANGE;
  *bytes = evolve_sample_layout(n, p, shots, nullptr, nullptr);
  return GQAOA_OK;
}

extern "C" int gqaoa_evolve_sample(const uint8_t *cost, int n, int m, const double *gammas,
                                   const double *betas, int p, void *state, double *out,
                                   double *trace, uint64_t seed, int64_t shots, uint64_t *out_idx,
                                   void *ws, size_t ws_bytes, unsigned flags, void *stream) {
  gq::NvtxRange nvtx_range("gqaoa_evolve_sample");
  int rc = check_common(n, m, 1, p);
  if (rc) return rc;
  if (shots < 0 || shots >= (1ll << 32)) return GQAOA_ERANGE;
  if (!cost || !gammas || !betas || !state || !ws || (shots > 0 && !out_idx)) return GQAOA_EINVAL;
  if (flags & ~(GQAOA_STATE_IN | GQAOA_READOUT_CLASS(255))) return GQAOA_EINVAL;
  const unsigned target = (flags >> 8) & 0xFFu;
  if (target != 0u && trace) return GQAOA_EINVAL;
  if (!aligned16(state) || !aligned16(cost) || !aligned8(gammas) || !aligned8(betas) ||
      (out && !aligned8(out)) || (trace && !aligned8(trace)) || !aligned16(ws) ||
      (out_idx && !aligned8(out_idx)))
    return GQAOA_EINVAL;
  size_t o_add = 0, o_samp = 0;
  if (ws_bytes < evolve_sample_layout(n, p, shots, &o_add, &o_samp)) return GQAOA_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char *base = static_cast<char *>(ws);
  size_t ev_bytes = 0, sa_bytes = 0;
  gqaoa_evolve_workspace_size(n, p, &ev_bytes);
  gqaoa_sample_workspace_size(n, shots, &sa_bytes);
  const Geometry g = make_geometry(n, 1, kFwdPerSm);
  if (g.small || shots == 0 || !sample_direct_ok(g.ntiles, shots)) {
    // one CTA per state, no shots, or many shots per tile: the evolution
    // materialises psi_p and the sampler runs on it
    rc = evolve_impl(cost, 0, n, m, 1, gammas, betas, p, state, out, trace, ws, ev_bytes, flags,
                     st);
    if (rc) return rc;
    return gqaoa_sample(state, n, seed, shots, out_idx, base + o_samp, sa_bytes, stream);
  }
  Ws w;
  ws_layout(g, p, false, base, &w, g.nparts);
  rc = launch_phase_tables(gammas, betas, p, w, st);
  if (rc) return rc;
  rc = run_forward(g, w, cost, 0, p, static_cast<float2 *>(state), (flags & GQAOA_STATE_IN) != 0,
                   trace, nullptr, st);
  if (rc) return rc;
  double *tsum = nullptr, *chunk_incl = nullptr;
  sample_direct_ws(g.ntiles, shots, base + o_samp, &tsum, &chunk_incl);
  float2 *add = reinterpret_cast<float2 *>(base + o_add);
  PassArgs pa;
  init_pass(pa, g, w, cost, 0, p);
  pa.round = p - 1;
  pa.parts_in = parts_half(w, p - 1);
  pa.parts_out = parts_half(w, p);
  pa.src = static_cast<const float4 *>(state);
  pa.target = target;
  if (launch_pass(g, readout_sample_kernel, st, pa, tsum, chunk_incl, add) != cudaSuccess)
    return GQAOA_ECUDA;
  finalize_readout_kernel<<<1, 32, 0, st>>>(pa.parts_out, g.nparts, p, out, trace);
  GQ_CHECK_LAUNCH();
  return sample_direct_tail(static_cast<const float4 *>(state), add, g.ntiles, seed, shots,
                            out_idx, base + o_samp, st);
}

extern "C" int gqaoa_grad_workspace_size(int n, int p, size_t *bytes) {
  return gqaoa_grad_batched_workspace_size(n, 1, p, bytes);
}

extern "C" int gqaoa_grad_batched_workspace_size(int n, int batch, int p, size_t *bytes) {
  if (!bytes) return GQAOA_EINVAL;
  int rc = check_common(n, 0, batch, p);
  if (rc) return rc;
  const Geometry g = make_geometry(n, batch, kFwdPerSm);
  const Geometry gb = make_geometry(n, batch, kBwdPerSm);
  *bytes = ws_layout(g, p, true, nullptr, nullptr, g.nparts > gb.nparts ? g.nparts : gb.nparts);
  return GQAOA_OK;
}

extern "C" int gqaoa_grad(const uint8_t *cost, int n, int m, const double *gammas,
                          const double *betas, int p, int objective, double *value, double *dgamma,
                          double *dbeta, void *ws, size_t ws_bytes, void *stream) {
  gq::NvtxRange nvtx_range("gqaoa_grad");
  return grad_impl(cost, 0, n, m, 1, gammas, betas, p, objective, value, dgamma, dbeta, ws,
                   ws_bytes, static_cast<cudaStream_t>(stream));
}

extern "C" int gqaoa_grad_batched(const uint8_t *cost, int64_t cost_stride, int n, int m,
                                  int batch, const double *gammas, const double *betas, int p,
                                  int objective, double *value, double *dgamma, double *dbeta,
                                  void *ws, size_t ws_bytes, void *stream) {
  gq::NvtxRange nvtx_range("gqaoa_grad_batched");
  if (cost_stride < 0) return GQAOA_EINVAL;
  return grad_impl(cost, (uint64_t)cost_stride, n, m, batch, gammas, betas, p, objective, value,
                   dgamma, dbeta, ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

extern "C" int gqaoa_prob_workspace_size(int n, size_t *bytes) {
  if (!bytes) return GQAOA_EINVAL;
  if (n < 1 || n > GQAOA_MAX_N) return GQAOA_ERANGE;
  const Geometry g = make_geometry(n, 1, kFwdPerSm);
  *bytes = sizeof(double) * (size_t)g.nparts * kPartStride;
  return GQAOA_OK;
}

__global__ void __launch_bounds__(kThreads)
readout_small_kernel(const float2 *__restrict__ state, const uint8_t *__restrict__ cost, int n,
                     double *__restrict__ out) {
  __shared__ double s_scr[kWarps];
  const int N = 1 << n;
  double lp = 0.0, le = 0.0, ln = 0.0;
  for (int z = threadIdx.x; z < N; z += blockDim.x) {
    const float2 v = state[z];
    const double w = (double)v.x * v.x + (double)v.y * v.y;
    ln += w;
    le += (double)cost[z] * w;
    if (cost[z] == 0) lp += w;
  }
  const double P = block_sum(lp, s_scr);
  const double E = block_sum(le, s_scr);
  const double Nm = block_sum(ln, s_scr);
  if (threadIdx.x == 0) { out[0] = P; out[1] = E; out[2] = Nm; }
}

extern "C" int gqaoa_prob(const void *state, const uint8_t *cost, int n, double *out, void *ws,
                          size_t ws_bytes, void *stream) {
  gq::NvtxRange nvtx_range("gqaoa_prob");
  if (n < 1 || n > GQAOA_MAX_N) return GQAOA_ERANGE;
  if (!state || !cost || !out) return GQAOA_EINVAL;
  if (!aligned16(state) || !aligned16(cost) || !aligned8(out)) return GQAOA_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Geometry g = make_geometry(n, 1, kFwdPerSm);
  if (g.small) {
    readout_small_kernel<<<1, kThreads, 0, st>>>(static_cast<const float2 *>(state), cost, n, out);
    GQ_CHECK_LAUNCH();
    return GQAOA_OK;
  }
  if (!ws || !aligned16(ws)) return GQAOA_EINVAL;
  if (ws_bytes < sizeof(double) * (size_t)g.nparts * kPartStride) return GQAOA_ENOMEM;
  PassArgs pa = {};
  pa.cost = cost;
  pa.src = static_cast<const float4 *>(state);
  pa.dst = static_cast<float4 *>(const_cast<void *>(state));  // not written without kPending
  pa.parts_out = static_cast<double *>(ws);
  pa.p = 1;
  pa.cpi = g.cpi;
  pa.nparts = g.nparts;
  pa.nparts_in = g.nparts;
  pa.ntiles = g.ntiles;
  pa.N = g.N;
  pa.inv_n = 1.0 / (double)g.N;
  if (launch_pass(g, readout_kernel<false>, st, pa) != cudaSuccess) return GQAOA_ECUDA;
  finalize_readout_kernel<<<1, 32, 0, st>>>(pa.parts_out, g.nparts, 1, out, nullptr);
  GQ_CHECK_LAUNCH();
  return GQAOA_OK;
}
