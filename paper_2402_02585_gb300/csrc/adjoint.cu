// Cluster-resident adjoint gradient (Eq. 3 rounds, forward then backward,
// for states of 2^10..2^16 amplitudes).
//
// The streaming adjoint makes one launch per round and direction; for a
// state of at most 2^16 amplitudes a round is a few microseconds of work on
// the whole GPU, so the launch boundaries set the time. Here one thread-block
// cluster owns one instance (row) for the whole call: each thread keeps 16
// amplitudes in registers, the forward rounds write the checkpoints chi_k
// (each thread later rereads only its own), and the backward rounds follow
// in the same launch. A round's sums are butterflies over the warp's lanes
// (FP32: at most 512 amplitudes a warp), then (warp 0) over the CTA's warps
// and over the cluster's CTAs in double-float (FP32 pairs, ~48 bits, so the
// mixer sum keeps FP64 accuracy on the FP32 pipe); every CTA's partial is
// stored into the shared memory of every peer and every warp sums them, so
// every warp of every CTA holds the same totals bit for bit and no further
// barrier is needed. The objective's value is double-float at every stage.
// FP32 amplitudes and mixer coefficients: the rounds use no FP64, a closing
// kernel forms the gradients from the double-float sums they left.
//
// Forward round k: chi_k = T_k[c] psi_{k-1} (checkpointed), S_k = sum chi_k,
// a_k = alpha_k S_k / N, psi_k = chi_k + a_k. Backward, from
// lambda = O psi_p: with L = sum lambda and mu = lambda + conj(alpha_k) L / N,
// dE/dgamma_k = 2 sum_z c(z) Im(conj(mu) chi_k), and lambda <- conj(T_k) mu;
// dE/dbeta_k = 2 Im(conj(e^{-i beta_k} S_k / N) L). The sum of the updated
// lambda (the next round's L) is reduced together with the gamma term, so a
// backward round takes one cluster reduction.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.cuh"

namespace gq {

int sm_count();

namespace {

constexpr int kAdjPer = 16;  // amplitudes per thread
constexpr int kAdjVals = 3;  // values per reduction

struct AdjArgs {
  const uint8_t *cost;    // row b at cost + b * cost_bstride
  uint64_t cost_bstride;
  const float2 *phase;    // [B][p][256]
  const double2 *alpha;   // [B][p]
  double *record;         // [B][p][4]: S_k (re, im as double-float pairs), float alpha_k, G_k
  float2 *ckpt;           // [p][B][N]
  double *value;          // [B]
  double *dgamma;         // [B][p]
  double *dbeta;          // [B][p]
  int n;
  int p;
  int B;
  int objective;          // GQAOA_OBJ_P0 (projector on `target`) or GQAOA_OBJ_ENERGY
  unsigned target;
  unsigned *status;       // nonzero once a bounded wait gave up (outputs then NaN)
};

// (hi, lo) += x in double-float arithmetic.
__device__ __forceinline__ void adj_df_add(float &hi, float &lo, float x) {
  float s, e;
  two_sum(hi, x, s, e);
  hi = s;
  lo = __fadd_rn(lo, e);
}

// The exchange of one cluster reduction (st.async into every CTA's receive
// slot, mbarrier-counted): a CTA's partials are three double-float pairs, 24 bytes.
constexpr uint32_t kAdjSlotBytes = 24;

struct AdjSync {
  unsigned t;  // calls so far: this call uses buffer t & 1, in its use (t >> 1)
  bool ok;     // false once a wait of this thread has given up
};

// Store d[0..2] at the receive slot `slot` (a local shared address) of CTA
// `peer` and complete 24 bytes on that CTA's mbarrier at local address mb.
__device__ __forceinline__ void adj_send(uint32_t slot, uint32_t mb, unsigned peer,
                                         const float2 (&d)[kAdjVals]) {
  const uint32_t rs = mapa_shared(slot, peer), rm = mapa_shared(mb, peer);
  st_async_v4(rs, make_float4(d[0].x, d[0].y, d[1].x, d[1].y), rm);
  st_async_v2(rs + 16, d[2], rm);
}

// Double-float sum over each aligned group of kG lanes (kG a power of two up
// to 32): every lane ends with its group's sum, the same bits in every group
// that holds the same values (TwoSum's error term does not depend on the
// order of its operands).
template <int kG>
__device__ __forceinline__ void adj_df_group(float &hi, float &lo) {
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

// Sum over each aligned group of kG lanes (a power of two up to 32): FP32 in
// v.x, or (kDF) the double-float pair (v.x, v.y).
template <int kG, bool kDF>
__device__ __forceinline__ void adj_group(float2 &v) {
  if (kDF) {
    adj_df_group<kG>(v.x, v.y);
  } else {
    float x = v.x;
#pragma unroll
    for (int o = kG / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    v = make_float2(x, 0.f);
  }
}

// Cluster-wide sums of kV <= kAdjVals values: v[k] holds this thread's
// partial on entry (an FP32 value in .x, or a double-float pair with kDF);
// on exit v[k] is the cluster's total as a double-float pair, the same bits
// in every thread: each stage is a butterfly, whose partner lanes add the
// same two operands (the warp's lanes in FP32, or double-float with kDF;
// the CTA's warps and the cluster's CTAs in double-float).
// The buffers alternate between calls (sy.t counts them): the partials of
// one call are read while the next call's are written. Slots are 32 bytes
// (v[0], v[1] at 0, v[2] at 16). between() runs while the partials are in
// flight (after this CTA's sends, before its wait), so global loads and
// stores placed there overlap the exchange.
struct AdjNothing {
  __device__ __forceinline__ void operator()() const {}
};

template <int kThreads, int kCluster, int kV, bool kDF = false, typename Between = AdjNothing>
__device__ __forceinline__ void adj_cluster_sum(float2 (&v)[kAdjVals],
                                                float2 (*s_wp)[kThreads / 32][kAdjVals],
                                                float2 (*s_ps)[kCluster][4], uint64_t *s_mb,
                                                unsigned rank, AdjSync &sy, unsigned *status,
                                                Between between = Between()) {
  constexpr int kW = kThreads / 32;
  const int buf = sy.t & 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kV; ++k) adj_group<32, kDF>(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < kV; ++k) s_wp[buf][warp][k] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
    // every group of kW lanes holds the kW warp partials
    float2 d[kAdjVals];
#pragma unroll
    for (int k = 0; k < kAdjVals; ++k) {
      d[k] = make_float2(0.f, 0.f);
      if (k < kV) {
        d[k] = s_wp[buf][lane & (kW - 1)][k];
        adj_group<kW, true>(d[k]);
      }
    }
    if (kCluster == 1) {
      if (lane == 0) {
#pragma unroll
        for (int k = 0; k < kV; ++k) s_ps[buf][0][k] = d[k];
      }
    } else if (lane < kCluster && sy.ok) {
      adj_send(smem_addr(&s_ps[buf][rank][0]), smem_addr(&s_mb[buf]), (unsigned)lane, d);
    }
  }
  if (kCluster > 1) {
    between();
    if (sy.ok) {
      if (!mbar_wait(smem_addr(&s_mb[buf]), (sy.t >> 1) & 1u, status)) {
        sy.ok = false;
        atomicExch(status, 1u);
      }
    }
    // warp-uniform from here on, so warp 0's arming and sends stay in step
    sy.ok = __all_sync(0xffffffffu, sy.ok);
    // arm this mbarrier for its next use (two calls on; a peer can send
    // into it only after this CTA's partials of the call in between)
    if (threadIdx.x == 0 && sy.ok) mbar_arm(smem_addr(&s_mb[buf]), kCluster * kAdjSlotBytes);
  } else {
    __syncthreads();
    between();
  }
#pragma unroll
  for (int k = 0; k < kV; ++k) {
    float2 d = s_ps[buf][lane & (kCluster - 1)][k];
    adj_group<kCluster, true>(d);
    v[k] = d;
  }
  ++sy.t;
}

// The mixer coefficients as FP32 pairs, into the records' spare slots
// (record[4 bk + 2], read as a float2), so the rounds convert no FP64; and
// the launch's status word cleared.
__global__ void adj_alpha_kernel(const double2 *__restrict__ alpha, uint64_t count,
                                 double *__restrict__ record, unsigned *status) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *status = 0u;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const double2 al = alpha[i];
    *reinterpret_cast<float2 *>(record + 4 * i + 2) = make_float2((float)al.x, (float)al.y);
  }
}

template <int kThreads, int kCluster>
__global__ void __launch_bounds__(kThreads, 512 / kThreads)
adjoint_cluster_kernel(const __grid_constant__ AdjArgs a) {
  constexpr int kW = kThreads / 32;
  __shared__ float2 s_wp[2][kW][kAdjVals];
  __shared__ __align__(16) float2 s_ps[2][kCluster][4];  // receive slots
  __shared__ __align__(8) uint64_t s_mb[2];              // their mbarriers
  // phase tables, double-buffered: a round reads s_T[k & 1] while its table
  // for two rounds on is in flight in registers (tn) of threads 0..255, each
  // holding kTab entries (t, t + kThreads, ...)
  constexpr int kTab = kThreads >= 256 ? 1 : 256 / kThreads;
  __shared__ float2 s_T[2][256];
  const bool tabler = threadIdx.x < 256;
  const unsigned rank = kCluster > 1 ? cluster_ctarank() : 0u;
  const uint64_t cl = blockIdx.x / kCluster, ncl = gridDim.x / kCluster;
  const uint64_t N = 1ull << a.n;
  const float inv_n = (float)(1.0 / (double)N);  // a power of two: exact
  const float amp0 = (float)(1.0 / sqrt((double)N));
  const bool writer = rank == 0 && threadIdx.x == 0;
  AdjSync sy = {0u, true};
  if (kCluster > 1) {
    if (threadIdx.x == 0) {
      mbar_init(smem_addr(&s_mb[0]));
      mbar_init(smem_addr(&s_mb[1]));
      mbar_init_fence();
      mbar_arm(smem_addr(&s_mb[0]), kCluster * kAdjSlotBytes);
      mbar_arm(smem_addr(&s_mb[1]), kCluster * kAdjSlotBytes);
    }
    cluster_sync();  // every CTA's mbarriers initialised before any partial is sent
  }
  // slot j of this thread is amplitude z0 + j kThreads
  const uint64_t z0 = (uint64_t)rank * kAdjPer * kThreads + threadIdx.x;
  for (uint64_t b = cl; b < (uint64_t)a.B; b += ncl) {
    const uint8_t *cost = a.cost + b * a.cost_bstride + z0;
    unsigned c[kAdjPer];
    float2 s[kAdjPer];
#pragma unroll
    for (int j = 0; j < kAdjPer; ++j) {
      c[j] = cost[j * kThreads];
      s[j] = make_float2(amp0, 0.f);
    }
    const float2 *tab = a.phase + b * (uint64_t)a.p * 256 + threadIdx.x;  // + 256 k: round k
    // the rounds' FP32 mixer coefficients, each loaded one round before its
    // use (after an exchange's acquire a load could not be hoisted, and its
    // latency would sit on every round's critical path)
    const float2 *alf = reinterpret_cast<const float2 *>(a.record + 4 * b * (uint64_t)a.p + 2);
    float2 aln = alf[0];  // round k at alf[4 k] (a record is four doubles)
    float2 tn[kTab];
    if (tabler) {
#pragma unroll
      for (int i = 0; i < kTab; ++i) {
        s_T[0][threadIdx.x + i * kThreads] = tab[i * kThreads];
        tn[i] = a.p > 1 ? tab[256 + i * kThreads] : make_float2(0.f, 0.f);
      }
    }
    __syncthreads();
    // forward: chi_k into the checkpoints, psi_k = chi_k + a_k
    for (int k = 0; k < a.p; ++k) {
      const uint64_t bk = b * (uint64_t)a.p + k;
      const float2 *T = s_T[k & 1];
      float2 *ck = a.ckpt + ((uint64_t)k * a.B + b) * N + z0;
      float sr = 0.f, si = 0.f;
#pragma unroll
      for (int j = 0; j < kAdjPer; ++j) {
        s[j] = cmul(T[c[j]], s[j]);
        sr += s[j].x;
        si += s[j].y;
      }
      // round k + 1's table (its buffer was last read in round k - 1, before
      // that round's barriers; this round's barrier publishes it)
      if (tabler) {
#pragma unroll
        for (int i = 0; i < kTab; ++i) {
          if (k + 1 < a.p) s_T[(k + 1) & 1][threadIdx.x + i * kThreads] = tn[i];
          if (k + 2 < a.p) tn[i] = tab[(uint64_t)(k + 2) * 256 + i * kThreads];
        }
      }
      float2 v[kAdjVals] = {make_float2(sr, 0.f), make_float2(si, 0.f), make_float2(0.f, 0.f)};
      // the checkpoints chi_k, stored while the partials are exchanged
      adj_cluster_sum<kThreads, kCluster, 2>(v, s_wp, s_ps, s_mb, rank, sy, a.status, [&]() {
#pragma unroll
        for (int j = 0; j < kAdjPer; ++j) ck[j * kThreads] = s[j];
      });
      const float Sr = v[0].x + v[0].y, Si = v[1].x + v[1].y;
      const float2 al = aln;
      if (k + 1 < a.p) aln = alf[4 * (k + 1)];  // else kept: backward round p - 1 uses it
      const float2 af = make_float2((al.x * Sr - al.y * Si) * inv_n, (al.x * Si + al.y * Sr) * inv_n);
#pragma unroll
      for (int j = 0; j < kAdjPer; ++j) s[j] = make_float2(s[j].x + af.x, s[j].y + af.y);
      if (writer)  // S_k as double-float pairs, read by adj_finalize_kernel
        *reinterpret_cast<float4 *>(a.record + 4 * bk) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    }
    // lambda_p = O psi_p, the objective sum_z O |psi_p|^2 (double-float:
    // each square split exactly by an FMA) and L = sum lambda
    float2 l[kAdjPer];
    float vh = 0.f, vl = 0.f, lr = 0.f, li = 0.f;
#pragma unroll
    for (int j = 0; j < kAdjPer; ++j) {
      const float o = a.objective == GQAOA_OBJ_P0 ? (c[j] == a.target ? 1.f : 0.f) : (float)c[j];
      l[j] = make_float2(o * s[j].x, o * s[j].y);
      const float px = s[j].x * s[j].x, ex = fmaf(s[j].x, s[j].x, -px);
      const float py = s[j].y * s[j].y, ey = fmaf(s[j].y, s[j].y, -py);
      float wh, wl;
      two_sum(px, py, wh, wl);
      wl = __fadd_rn(wl, __fadd_rn(ex, ey));
      const float ph = o * wh, pe = fmaf(o, wh, -ph);  // o is an integer below 256
      adj_df_add(vh, vl, ph);
      vl = __fadd_rn(vl, fmaf(o, wl, pe));
      lr += l[j].x;
      li += l[j].y;
    }
    // the last round's checkpoints are loaded before the reduction, and each
    // backward round loads the next one's after its own are consumed, so the
    // loads' latency overlaps the reductions
    float2 x[kAdjPer];
    {
      const float2 *ck = a.ckpt + ((uint64_t)(a.p - 1) * a.B + b) * N + z0;
#pragma unroll
      for (int j = 0; j < kAdjPer; ++j) x[j] = ck[j * kThreads];
    }
    // the backward rounds read the tables in reverse: s_T[(p - 1) & 1] still
    // holds round p - 1's; round p - 2's is in flight
    if (tabler && a.p > 1) {
#pragma unroll
      for (int i = 0; i < kTab; ++i) tn[i] = tab[(uint64_t)(a.p - 2) * 256 + i * kThreads];
    }
    float2 v[kAdjVals] = {make_float2(vh, vl), make_float2(lr, 0.f), make_float2(li, 0.f)};
    adj_cluster_sum<kThreads, kCluster, 3, true>(v, s_wp, s_ps, s_mb, rank, sy, a.status);
    if (writer) a.value[b] = (double)v[0].x + (double)v[0].y;
    // backward rounds
    for (int k = a.p - 1; k >= 0; --k) {
      const uint64_t bk = b * (uint64_t)a.p + k;
      const float2 Ld = v[1], Li2 = v[2];  // this round's L (double-float)
      const float Lr = Ld.x + Ld.y, Li = Li2.x + Li2.y;
      const float2 al = aln;
      if (k > 0) aln = alf[4 * (k - 1)];
      const float2 bv = make_float2((al.x * Lr + al.y * Li) * inv_n, (al.x * Li - al.y * Lr) * inv_n);
      const float2 *T = s_T[k & 1];
      float g = 0.f, nlr = 0.f, nli = 0.f;
      // round k - 1's checkpoint slot j is loaded as soon as round k's is
      // used, so each load has the rest of the round and its exchange to land
      const float2 *ckn = a.ckpt + ((uint64_t)(k > 0 ? k - 1 : 0) * a.B + b) * N + z0;
#pragma unroll
      for (int j = 0; j < kAdjPer; ++j) {
        const float2 mu = make_float2(l[j].x + bv.x, l[j].y + bv.y);
        g = fmaf((float)c[j], fmaf(mu.x, x[j].y, -mu.y * x[j].x), g);
        if (k > 0) x[j] = ckn[j * kThreads];
        const float2 t = T[c[j]];
        l[j] = make_float2(fmaf(t.x, mu.x, t.y * mu.y), fmaf(t.x, mu.y, -t.y * mu.x));
        nlr += l[j].x;
        nli += l[j].y;
      }
      // round k - 1's table (its buffer was last read in round k + 1, or in
      // forward round p - 2 for k = p - 1)
      if (tabler) {
#pragma unroll
        for (int i = 0; i < kTab; ++i) {
          if (k >= 1) s_T[(k - 1) & 1][threadIdx.x + i * kThreads] = tn[i];
          if (k >= 2) tn[i] = tab[(uint64_t)(k - 2) * 256 + i * kThreads];
        }
      }
      v[0] = make_float2(g, 0.f);
      v[1] = make_float2(nlr, 0.f);
      v[2] = make_float2(nli, 0.f);
      adj_cluster_sum<kThreads, kCluster, 3>(v, s_wp, s_ps, s_mb, rank, sy, a.status);
      if (writer) {  // the round's sums, finished in FP64 by adj_finalize_kernel
        *reinterpret_cast<float2 *>(a.record + 4 * bk + 3) = v[0];  // G_k
        *reinterpret_cast<float2 *>(a.dbeta + bk) = Ld;             // L_k (re)
        *reinterpret_cast<float2 *>(a.dgamma + bk) = Li2;           // L_k (im)
      }
    }
  }
  if (kCluster > 1) cluster_sync();  // no CTA leaves while a peer may still store into it
}

// The gradients in FP64 from the double-float sums the rounds left (one
// thread per instance and round, off the rounds' critical path):
// dE/dbeta_k = 2 Im(conj(e^{-i beta_k} S_k / N) L_k), dE/dgamma_k = 2 G_k.
// If a bounded wait of the rounds gave up, every value and derivative of the
// call is NaN instead.
__global__ void adj_finalize_kernel(const double2 *__restrict__ alpha, const double *record,
                                    uint64_t count, int n, int B, const unsigned *status,
                                    double *value, double *dgamma, double *dbeta) {
  const double inv_n = ldexp(1.0, -n);
  if (*status) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x) {
      dgamma[i] = dbeta[i] = __longlong_as_double(0x7ff8000000000000ll);
      if (i < (uint64_t)B) value[i] = __longlong_as_double(0x7ff8000000000000ll);
    }
    return;
  }
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const float4 S = *reinterpret_cast<const float4 *>(record + 4 * i);
    const float2 G = *reinterpret_cast<const float2 *>(record + 4 * i + 3);
    const float2 Lr = *reinterpret_cast<const float2 *>(dbeta + i);
    const float2 Li = *reinterpret_cast<const float2 *>(dgamma + i);
    const double Sre = ((double)S.x + (double)S.y) * inv_n, Sim = ((double)S.z + (double)S.w) * inv_n;
    const double2 al = alpha[i];
    const double er = al.x + 1.0, ei = al.y;  // e^{-i beta_k}
    const double qr = er * Sre - ei * Sim, qi = er * Sim + ei * Sre;
    const double Lrd = (double)Lr.x + (double)Lr.y, Lid = (double)Li.x + (double)Li.y;
    dbeta[i] = 2.0 * (qi * Lrd - qr * Lid);
    dgamma[i] = 2.0 * ((double)G.x + (double)G.y);
  }
}

template <int kThreads, int kCluster>
int launch_adjoint(const AdjArgs &args, cudaStream_t st) {
  auto kernel = adjoint_cluster_kernel<kThreads, kCluster>;
  if (kCluster > 8 &&
      cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return GQAOA_ECUDA;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kCluster, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;  // resident clusters (CTAs for kCluster = 1)
  if (kCluster == 1) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&clusters, kernel, kThreads, 0) != cudaSuccess)
      return GQAOA_ECUDA;
    clusters *= sm_count();
  } else if (cudaOccupancyMaxActiveClusters(&clusters, kernel, &cfg) != cudaSuccess) {
    return GQAOA_ECUDA;
  }
  if (clusters < 1) return GQAOA_ERANGE;  // this shape cannot be placed
  const uint64_t units = (uint64_t)args.B < (uint64_t)clusters ? (uint64_t)args.B : (uint64_t)clusters;
  cfg.gridDim = dim3((unsigned)(units * kCluster), 1, 1);
  cfg.stream = st;
  cfg.numAttrs = kCluster > 1 ? 1 : 0;
  if (cudaLaunchKernelEx(&cfg, kernel, args) != cudaSuccess) return GQAOA_ECUDA;
  return GQAOA_OK;
}

}  // namespace

// Whether the cluster-resident adjoint takes B states of 2^n amplitudes
// (10 <= n <= 16, any batch: each instance's rounds run back to back on one
// cluster and move only the checkpoints through memory, which beats the
// streaming passes at every batch size measured).
bool adjoint_cluster_fits(int n, int B) { return n >= 10 && n <= 16 && B >= 1; }

// Objective and adjoint gradient of B rows of 2^n amplitudes (10 <= n <= 16)
// in one launch (plus the FP32 mixer coefficients' conversion). phase,
// alpha: the rows' tables ([B][p][256], [B][p]); record [B][p][4] and ckpt
// [p][B][2^n] and the status word are workspace. objective: GQAOA_OBJ_P0
// with target, or GQAOA_OBJ_ENERGY.
int adjoint_cluster(const uint8_t *cost, uint64_t cost_bstride, int n, int B, int p,
                    const float2 *phase, const double2 *alpha, double *record, float2 *ckpt,
                    int objective, unsigned target, double *value, double *dgamma,
                    double *dbeta, unsigned *status, cudaStream_t st) {
  if (!adjoint_cluster_fits(n, B)) return GQAOA_ERANGE;
  const uint64_t count = (uint64_t)B * (uint64_t)p;
  const unsigned grid = (unsigned)(count < 256ull * 1024 ? (count + 255) / 256 : 1024);
  adj_alpha_kernel<<<grid, 256, 0, st>>>(alpha, count, record, status);
  GQ_CHECK_LAUNCH();
  AdjArgs args = {cost, cost_bstride, phase, alpha, record, ckpt, value, dgamma, dbeta,
                  n, p, B, objective, target, status};
  // 16 amplitudes a thread; several CTAs per SM, so each SM interleaves
  // several rows' rounds: 64- or 128-thread CTAs alone at n = 10, 11, then
  // clusters of 128-thread CTAs (n = 12..15: 2, 4, 8, 16 CTAs) and 16 CTAs
  // of 256 threads at n = 16. 16 is a non-portable cluster size: where it
  // cannot be placed, the shape with half as many CTAs of twice the threads.
  int rc;
  switch (n) {
    case 10: rc = launch_adjoint<64, 1>(args, st); break;
    case 11: rc = launch_adjoint<128, 1>(args, st); break;
    case 12: rc = launch_adjoint<128, 2>(args, st); break;
    case 13: rc = launch_adjoint<128, 4>(args, st); break;
    case 14: rc = launch_adjoint<128, 8>(args, st); break;
    case 15:
      rc = launch_adjoint<128, 16>(args, st);
      if (rc == GQAOA_ECUDA || rc == GQAOA_ERANGE) {
        (void)cudaGetLastError();
        rc = launch_adjoint<256, 8>(args, st);
      }
      break;
    default:
      rc = launch_adjoint<256, 16>(args, st);
      if (rc == GQAOA_ECUDA || rc == GQAOA_ERANGE) {
        (void)cudaGetLastError();
        rc = launch_adjoint<512, 8>(args, st);
      }
      break;
  }
  if (rc) return rc;
  adj_finalize_kernel<<<grid, 256, 0, st>>>(alpha, record, count, n, B, status, value, dgamma,
                                           dbeta);
  GQ_CHECK_LAUNCH();
  return GQAOA_OK;
}

}  // namespace gq
