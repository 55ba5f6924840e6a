// K7: batched single-angle-pair sweep with the state held on chip.
//
// The single-angle-pair protocol (Eq. 5) applies the same (gamma, beta) in
// every round; Appendix C scans it on a grid for every instance. A sweep is
// B instances x A angle points, each evolved for p rounds from |+> with P(C=0)
// read out after the rounds listed in `rounds` (a prefix sweep: one p-round run
// gives every shorter p).
//
// One work item = (instance, angle point) and is owned by one CTA (n <= 14)
// or one thread-block cluster of 2..16 CTAs (n = 15..19). Each thread holds
// 16 consecutive amplitudes and their 16 cost bytes in registers for the
// whole evolution (n = 19: 16 more in shared memory), so a round costs no
// memory traffic at all: per amplitude one shared-memory phase lookup, a
// complex multiply-add and a partial sum.
// The mixer needs S = sum_z chi(z) every round: FP32 over a thread's 16
// values and the warp's butterfly, then double-float (two FP32 words) across
// warps and, for clusters, across CTAs: warp 0 stores its CTA's partial into
// a receive slot of every CTA of the cluster with st.async, each store
// completing its bytes on the receiver's mbarrier, and waits on its own
// mbarrier (no cluster barrier in the rounds). Warp 0 of every CTA forms the
// same a = alpha S / N from the same partials, so the CTAs of a cluster agree
// bit for bit without a broadcast. Persistent grid: each CTA/cluster loops
// over items instance-major, so consecutive items reuse the instance's cost
// table from L2.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.cuh"

namespace gq {

int phase_tables(const double *gammas, const double *betas, int64_t count, int entries,
                 float2 *phase, double2 *alpha, cudaStream_t st);
int sm_count();

constexpr int kSweepMaxRounds = 16;
constexpr int kSlots = 6;  // S.re, S.im, A0, B0.re, B0.im, count of C = 0
constexpr uint32_t kSweepSlotBytes = kSlots * 8;  // a CTA partial: six double-float pairs

struct SweepArgs {
  const uint8_t *cost;   // [B][N]
  const float2 *phase;   // [A][256]
  const double2 *alpha;  // [A]
  double *out;           // [B][A][R]
  float4 *scratch;       // cluster-resident path: [kL2Slots][N / 2]
  unsigned *status;      // nonzero once a bounded wait gave up (its outputs are then NaN)
  uint64_t nitems;       // B * A
  int n;
  int A;
  int p;
  int R;
  int rounds[kSweepMaxRounds];  // ascending, 1-based
};

// Double-float butterfly over the warp (every lane ends with the same sum).
__device__ __forceinline__ void df_warp(float &hi, float &lo) {
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
__device__ __forceinline__ float warp_fsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One round over a thread's 16 amplitudes: chi = T[c] (s + a), then the
// partial sums. kExtra adds the readout sums over C = 0 and the C = 0 count
// (only readout rounds and the first round pay for them).
template <bool kExtra>
__device__ __forceinline__ void round_body(float2 (&s)[16], const uint32_t (&cw)[4],
                                           const float2 *s_T, float2 ad, float (&v)[kSlots],
                                           bool ro, bool first) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const unsigned c = (cw[j >> 2] >> (8 * (j & 3))) & 0xFFu;
    const float2 x = cmul(s_T[c], make_float2(s[j].x + ad.x, s[j].y + ad.y));
    s[j] = x;
    v[0] += x.x;
    v[1] += x.y;
    if (kExtra && c == 0) {
      if (ro) { v[2] += x.x * x.x + x.y * x.y; v[3] += x.x; v[4] += x.y; }
      if (first) v[5] += 1.f;
    }
  }
}

// The same round over a thread's 16 shared-memory amplitudes (the second half
// of the state when it does not fit in registers). Layout [j][thread], so a
// warp's accesses for one j are consecutive words: no bank conflicts.
template <bool kExtra, int kThreads>
__device__ __forceinline__ void round_body_smem(float2 *s_state, const uint32_t *s_cost,
                                                const float2 *s_T, float2 ad, float (&v)[kSlots],
                                                bool ro, bool first) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t cw = s_cost[q * kThreads + threadIdx.x];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float2 *sp = s_state + (4 * q + k) * kThreads + threadIdx.x;
      const unsigned c = (cw >> (8 * k)) & 0xFFu;
      const float2 y = *sp;
      const float2 x = cmul(s_T[c], make_float2(y.x + ad.x, y.y + ad.y));
      *sp = x;
      v[0] += x.x;
      v[1] += x.y;
      if (kExtra && c == 0) {
        if (ro) { v[2] += x.x * x.x + x.y * x.y; v[3] += x.x; v[4] += x.y; }
        if (first) v[5] += 1.f;
      }
    }
  }
}

// 64 registers per thread, so small CTAs run several per SM (1024 threads in
// all) and one CTA's reduction overlaps another's rounds. kSmemHalf: the
// instance's second half lives in shared memory (16 more amplitudes per
// thread), which lets a 16-CTA cluster hold 2^19 amplitudes.
template <int kThreads, int kCluster, bool kSmemHalf>
__global__ void __launch_bounds__(kThreads, (kThreads >= 1024 ? 1 : 1024 / kThreads))
sweep_kernel(const __grid_constant__ SweepArgs a) {
  constexpr int kW = kThreads / 32;
  extern __shared__ __align__(16) unsigned char s_dyn[];
  float2 *s_state = reinterpret_cast<float2 *>(s_dyn);                              // [16][kThreads]
  uint32_t *s_cost = reinterpret_cast<uint32_t *>(s_dyn + 16 * kThreads * sizeof(float2));  // [4][kThreads]
  __shared__ float2 s_T[256];
  __shared__ float s_wp[2][kW][kSlots];        // warp partials (FP32)
  __shared__ __align__(16) float2 s_ps[kCluster > 1 ? 2 : 1][kCluster][kSlots];  // receive slots
  __shared__ __align__(8) uint64_t s_mb[2];    // their mbarriers (warp 0 exchanges)
  __shared__ float2 s_a;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned rank = kCluster > 1 ? cluster_ctarank() : 0u;
  const uint64_t cluster_id = blockIdx.x / kCluster, nclusters = gridDim.x / kCluster;
  const uint64_t N = 1ull << a.n;
  const float inv_n = (float)(1.0 / (double)N);
  const float amp0 = (float)(1.0 / sqrt((double)N));
  int buf = 0;
  unsigned xt = 0;  // warp 0: cluster exchanges so far (buffer xt & 1, its use xt >> 1)
  bool ok = true;   // warp 0: false once its wait gave up
  if (kCluster > 1) {
    if (threadIdx.x == 0) {
      mbar_init(smem_addr(&s_mb[0]));
      mbar_init(smem_addr(&s_mb[1]));
      mbar_init_fence();
      mbar_arm(smem_addr(&s_mb[0]), kSweepSlotBytes * kCluster);
      mbar_arm(smem_addr(&s_mb[1]), kSweepSlotBytes * kCluster);
    }
    cluster_sync();  // every CTA's mbarriers initialised before any partial is sent
  }

  for (uint64_t item = cluster_id; item < a.nitems; item += nclusters) {
    const uint64_t b = item / (uint64_t)a.A;
    const int ai = (int)(item % (uint64_t)a.A);
    const uint4 cw = *reinterpret_cast<const uint4 *>(
        a.cost + b * N + 16ull * ((uint64_t)rank * kThreads + threadIdx.x));
    if (kSmemHalf) {
      const uint4 cw2 = *reinterpret_cast<const uint4 *>(
          a.cost + b * N + N / 2 + 16ull * ((uint64_t)rank * kThreads + threadIdx.x));
      s_cost[0 * kThreads + threadIdx.x] = cw2.x;
      s_cost[1 * kThreads + threadIdx.x] = cw2.y;
      s_cost[2 * kThreads + threadIdx.x] = cw2.z;
      s_cost[3 * kThreads + threadIdx.x] = cw2.w;
    }
    for (int i = threadIdx.x; i < 256; i += kThreads) s_T[i] = a.phase[(size_t)ai * 256 + i];
    const double2 ald = a.alpha[ai];
    const float alr = (float)ald.x, ali = (float)ald.y;
    __syncthreads();
    const uint32_t cwords[4] = {cw.x, cw.y, cw.z, cw.w};
    float2 s[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) s[j] = make_float2(amp0, 0.f);
    if (kSmemHalf) {
#pragma unroll
      for (int j = 0; j < 16; ++j) s_state[j * kThreads + threadIdx.x] = make_float2(amp0, 0.f);
    }
    float2 ad = make_float2(0.f, 0.f);  // pending mixer add
    float cnt0 = 0.f;  // C = 0 count of the instance (warp 0 keeps it)
    int ridx = 0;
    for (int r = 0; r < a.p; ++r) {
      const bool ro = ridx < a.R && a.rounds[ridx] == r + 1;
      const bool first = r == 0;
      float v[kSlots] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (ro || first) {
        round_body<true>(s, cwords, s_T, ad, v, ro, first);
        if (kSmemHalf) round_body_smem<true, kThreads>(s_state, s_cost, s_T, ad, v, ro, first);
      } else {
        round_body<false>(s, cwords, s_T, ad, v, false, false);
        if (kSmemHalf) round_body_smem<false, kThreads>(s_state, s_cost, s_T, ad, v, false, false);
      }
      const int nv = (ro || first) ? kSlots : 2;
#pragma unroll
      for (int k = 0; k < kSlots; ++k)
        if (k < nv) v[k] = warp_fsum(v[k]);
      if (lane == 0) {
#pragma unroll
        for (int k = 0; k < kSlots; ++k)
          if (k < nv) s_wp[buf][warp][k] = v[k];
      }
      __syncthreads();
      float hi[kSlots], lo[kSlots];
      if (warp == 0) {
        // double-float sum over this CTA's warps
#pragma unroll
        for (int k = 0; k < kSlots; ++k) {
          hi[k] = (k < nv && lane < kW) ? s_wp[buf][lane][k] : 0.f;
          lo[k] = 0.f;
          if (k < nv) df_warp(hi[k], lo[k]);
        }
        if (kCluster > 1) {
          // this CTA's partial into a receive slot of every CTA of the
          // cluster (all six slots, zero past nv), then the cluster's sum
          const int xb = xt & 1;
          if (lane < kCluster && ok) {
            const uint32_t rs = mapa_shared(smem_addr(&s_ps[xb][rank][0]), (unsigned)lane);
            const uint32_t rm = mapa_shared(smem_addr(&s_mb[xb]), (unsigned)lane);
            st_async_v4(rs, make_float4(hi[0], lo[0], hi[1], lo[1]), rm);
            st_async_v4(rs + 16, make_float4(hi[2], lo[2], hi[3], lo[3]), rm);
            st_async_v4(rs + 32, make_float4(hi[4], lo[4], hi[5], lo[5]), rm);
          }
          if (ok && !mbar_wait(smem_addr(&s_mb[xb]), (xt >> 1) & 1u, a.status)) {
            ok = false;
            atomicExch(a.status, 1u);
          }
          ok = __all_sync(0xffffffffu, ok);
          // armed for its next use, two rounds on
          if (lane == 0 && ok) mbar_arm(smem_addr(&s_mb[xb]), kSweepSlotBytes * kCluster);
          ++xt;
          // double-float butterfly over the cluster's CTAs
#pragma unroll
          for (int k = 0; k < kSlots; ++k) {
            const float2 d = (k < nv && lane < kCluster) ? s_ps[xb][lane][k] : make_float2(0.f, 0.f);
            hi[k] = d.x;
            lo[k] = d.y;
            if (k < nv) df_warp(hi[k], lo[k]);
          }
        }
      }
      if (warp == 0) {
        const float Sr = hi[0] + lo[0], Si = hi[1] + lo[1];
        const float ar = (alr * Sr - ali * Si) * inv_n, aim = (alr * Si + ali * Sr) * inv_n;
        if (lane == 0) s_a = make_float2(ar, aim);
        if (first) cnt0 = hi[5] + lo[5];
        if (ro && rank == 0 && lane == 0) {
          // sum_{C=0} |chi + a|^2 = A0 + 2 Re(conj(a) B0) + h[0] |a|^2
          const double A0 = (double)hi[2] + lo[2], Br = (double)hi[3] + lo[3],
                       Bi = (double)hi[4] + lo[4];
          const double P = A0 + 2.0 * ((double)ar * Br + (double)aim * Bi) +
                           (double)cnt0 * ((double)ar * ar + (double)aim * aim);
          a.out[(b * (uint64_t)a.A + ai) * a.R + ridx] =
              ok ? P : __longlong_as_double(0x7ff8000000000000ll);
        }
      }
      __syncthreads();
      ad = s_a;
      if (ro) ++ridx;
      buf ^= 1;
    }
  }
  if (kCluster > 1) cluster_sync();  // no CTA leaves while a peer may read its shared memory
}

// ---------------------------------------------------------------------------
// Cluster-resident sweep: states too large for a cluster's registers and
// shared memory (n >= 20). One item per 16-CTA cluster of 512-thread CTAs,
// one CTA per SM; CTA r owns the r-th sixteenth of the state (Q float4, two
// amplitudes each). The CTA's warps split into two roles that run side by
// side, so the SM's L2 port and its ALUs are busy at the same time:
//  * on-chip warps (8): thread u holds the float4 j 256 + u of the sixteenth
//    for j < kL2RegVec in registers and for kL2RegVec <= j < kL2OnChip in
//    shared memory, for the whole evolution (16896 float4 per CTA, 52 % of an
//    n = 20 state);
//  * streaming warps (8): thread u owns the float4 kL2OnChip 256 + j 256 + u
//    for the rest of the sixteenth; they live in the cluster's slot of the
//    workspace and stream through a ring of kL2RegVec / kL2Batch register
//    batches (the same registers that hold state in the on-chip warps).
// Every warp access is 512 contiguous bytes, and each thread rereads only
// what it wrote, so the slot needs no synchronisation beyond program order.
// At most kL2Slots items are in flight (one per resident cluster, seven on
// GB300), whose slots total 27 MiB at n = 20: the per-round
// read-modify-write of them is served by the 129 MB L2, whose
// read-modify-write bandwidth is about twice that of HBM (and per SM about
// 95 GB/s, whatever the loads in flight, which is why the on-chip share
// matters).
//
// The mixer sum: FP32 over at most 8 amplitudes, double-float per thread,
// FP32 across a warp's lanes (butterfly), double-float per CTA (warp 0).
// Warp 0 then stores its CTA's partial into a receive slot of every CTA of
// the cluster with st.async (lane r stores to CTA r), each store completing
// its bytes on the receiver's mbarrier; every thread waits on its own CTA's
// mbarrier (acquire at cluster scope, no fence: the streaming warps' stores
// to the L2 slots need not complete first) and every warp sums the
// kL2Cluster partials with the same butterfly, so all warps of all CTAs
// hold the same a_k bit for bit with no further barrier.
// ---------------------------------------------------------------------------
constexpr int kL2Threads = 512;
constexpr int kL2Warps = kL2Threads / 32;
constexpr int kL2RoleThreads = kL2Threads / 2;  // threads per role
constexpr int kL2Cluster = 16;
constexpr int kL2Slots = 16;
constexpr int kL2RegVec = 18;   // float4 per on-chip thread held in registers
constexpr int kL2SmemVec = 48;  // float4 per on-chip thread held in shared memory
constexpr int kL2OnChip = kL2RegVec + kL2SmemVec;
constexpr int kL2Batch = 2;     // float4 per streaming batch
constexpr int kL2Ring = kL2RegVec / kL2Batch;  // batches in a streaming thread's ring
// a batch's two float4 take their four cost bytes from one 32-bit word of the
// cost ring, and a thread's streamed share (2^(n-13) - kL2OnChip float4 for
// n = 20..24) must split into whole batches
static_assert(kL2Batch == 2 && kL2RegVec % kL2Batch == 0 && kL2OnChip % kL2Batch == 0,
              "cluster-resident sweep: ring layout");
constexpr size_t kL2DynSmem =
    (size_t)kL2SmemVec * kL2RoleThreads * (sizeof(float4) + sizeof(uint16_t));

// chi = T[c] (psi + a) for one float4 (two amplitudes, cost bytes in c2),
// adding to the FP32 partials v.
template <bool kExtra>
__device__ __forceinline__ void l2_vec(float4 &x, unsigned c2, const float2 *s_T, float2 ad,
                                       float (&v)[kSlots], bool ro, bool first) {
  const unsigned c0 = c2 & 0xFFu, c1 = (c2 >> 8) & 0xFFu;
  const float2 x0 = cmul(s_T[c0], make_float2(x.x + ad.x, x.y + ad.y));
  const float2 x1 = cmul(s_T[c1], make_float2(x.z + ad.x, x.w + ad.y));
  x = make_float4(x0.x, x0.y, x1.x, x1.y);
  v[0] += x0.x + x1.x;
  v[1] += x0.y + x1.y;
  if (kExtra) {
    if (c0 == 0) {
      if (ro) { v[2] += x0.x * x0.x + x0.y * x0.y; v[3] += x0.x; v[4] += x0.y; }
      if (first) v[5] += 1.f;
    }
    if (c1 == 0) {
      if (ro) { v[2] += x1.x * x1.x + x1.y * x1.y; v[3] += x1.x; v[4] += x1.y; }
      if (first) v[5] += 1.f;
    }
  }
}

template <bool kExtra>
__device__ __forceinline__ void l2_fold(float (&v)[kSlots], DF (&acc)[kSlots]) {
#pragma unroll
  for (int k = 0; k < kSlots; ++k)
    if (kExtra || k < 2) {
      acc[k].add(v[k]);
      v[k] = 0.f;
    }
}

// A streaming thread's round: nb batches of kL2Batch float4 from its slot
// (gp: its first float4; gc: their cost bytes), kL2Ring - 1 batches ahead.
template <bool kExtra, bool kFirst>
__device__ __forceinline__ void l2_stream_round(float4 (&ring)[kL2RegVec],
                                                uint32_t (&cring)[kL2Ring], float4 *gp,
                                                const uint16_t *gc, int nb, const float2 *s_T,
                                                float2 ad, float amp0, DF (&acc)[kSlots],
                                                bool ro) {
  constexpr bool first = kFirst;
  constexpr int T = kL2RoleThreads;
  constexpr int kStep = kL2Batch * T;
  const float4 plus = make_float4(amp0, 0.f, amp0, 0.f);
  const float4 *lp = gp;  // next batch to load
  const uint16_t *lc = gc;
  float4 *sp = gp;        // next batch to store
  float v[kSlots] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  auto load = [&](int slot) {
    cring[slot] = (uint32_t)lc[0] | ((uint32_t)lc[T] << 16);
#pragma unroll
    for (int k = 0; k < kL2Batch; ++k)
      ring[slot * kL2Batch + k] = first ? plus : __ldcg(lp + k * T);
    lp += kStep;
    lc += kStep;
  };
#pragma unroll
  for (int d = 0; d + 1 < kL2Ring; ++d)
    if (d < nb) load(d);
#pragma unroll 1
  for (int g0 = 0; g0 < nb; g0 += kL2Ring) {
#pragma unroll
    for (int d = 0; d < kL2Ring; ++d) {
      const int g = g0 + d;
      if (g < nb) {
        constexpr int kAhead = kL2Ring - 1;
        if (g + kAhead < nb) load((d + kAhead) % kL2Ring);  // the slot batch g - 1 freed
#pragma unroll
        for (int k = 0; k < kL2Batch; ++k)
          l2_vec<kExtra>(ring[d * kL2Batch + k], cring[d] >> (16 * k), s_T, ad, v, ro, first);
#pragma unroll
        for (int k = 0; k < kL2Batch; ++k) __stcg(sp + k * T, ring[d * kL2Batch + k]);
        sp += kStep;
        if ((d & 3) == 3) l2_fold<kExtra>(v, acc);
      }
    }
  }
  l2_fold<kExtra>(v, acc);
}

// An on-chip thread's round: its kL2RegVec register float4, then its
// kL2SmemVec shared-memory float4 ([j][thread] layout: conflict-free).
template <bool kExtra, bool kFirst>
__device__ __forceinline__ void l2_onchip_round(float4 (&xr)[kL2RegVec],
                                                const uint32_t (&cr)[kL2Ring], float4 *s_state,
                                                const uint16_t *s_cost, int u, const float2 *s_T,
                                                float2 ad, float amp0, DF (&acc)[kSlots],
                                                bool ro) {
  constexpr bool first = kFirst;
  constexpr int T = kL2RoleThreads;
  const float4 plus = make_float4(amp0, 0.f, amp0, 0.f);
  float v[kSlots] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < kL2RegVec; ++k) {
    if (first) xr[k] = plus;
    l2_vec<kExtra>(xr[k], cr[k >> 1] >> (16 * (k & 1)), s_T, ad, v, ro, first);
    if ((k & 7) == 7) l2_fold<kExtra>(v, acc);
  }
  l2_fold<kExtra>(v, acc);
#pragma unroll 1
  for (int j0 = 0; j0 < kL2SmemVec; j0 += 8) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      float4 y = first ? plus : s_state[(j0 + k) * T + u];
      l2_vec<kExtra>(y, s_cost[(j0 + k) * T + u], s_T, ad, v, ro, first);
      s_state[(j0 + k) * T + u] = y;
    }
    l2_fold<kExtra>(v, acc);
  }
  l2_fold<kExtra>(v, acc);
}

__global__ void __launch_bounds__(kL2Threads, 1) sweep_l2_kernel(const __grid_constant__ SweepArgs a) {
  constexpr int T = kL2RoleThreads;
  extern __shared__ __align__(16) unsigned char s_dyn[];
  float4 *s_state = reinterpret_cast<float4 *>(s_dyn);  // [kL2SmemVec][T]
  uint16_t *s_cost =
      reinterpret_cast<uint16_t *>(s_dyn + sizeof(float4) * kL2SmemVec * T);  // [kL2SmemVec][T]
  __shared__ float2 s_T[256];
  __shared__ float2 s_wp[2][kL2Warps][kSlots];    // warp partials (double-float)
  __shared__ __align__(16) float2 s_ps[2][kL2Cluster][kSlots];  // receive slots: CTA partials
  __shared__ __align__(8) uint64_t s_mb[2];                     // their mbarriers
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool streaming = threadIdx.x < T;          // warps 0..7 stream, 8..15 stay on chip
  const int u = streaming ? threadIdx.x : threadIdx.x - T;
  const unsigned rank = cluster_ctarank();
  const uint64_t cluster_id = blockIdx.x / kL2Cluster, nclusters = gridDim.x / kL2Cluster;
  const uint64_t N = 1ull << a.n, Nv = N / 2;
  const uint64_t Q = Nv / kL2Cluster;                         // float4 per CTA
  const int nb = (int)(Q / T - kL2OnChip) / kL2Batch;         // streaming batches per thread
  const float inv_n = (float)(1.0 / (double)N);
  const float amp0 = (float)(1.0 / sqrt((double)N));
  const uint64_t seg0 = (uint64_t)rank * Q;
  float4 *gp = a.scratch + cluster_id * Nv + seg0 + (uint64_t)kL2OnChip * T + u;
  unsigned xt = 0;  // exchanges so far: this round's uses buffer xt & 1, in its use xt >> 1
  bool ok = true;   // false once a wait of this thread has given up
  if (threadIdx.x == 0) {
    mbar_init(smem_addr(&s_mb[0]));
    mbar_init(smem_addr(&s_mb[1]));
    mbar_init_fence();
    mbar_arm(smem_addr(&s_mb[0]), kSweepSlotBytes * kL2Cluster);
    mbar_arm(smem_addr(&s_mb[1]), kSweepSlotBytes * kL2Cluster);
  }
  cluster_sync();  // every CTA's mbarriers initialised before any partial is sent

  for (uint64_t item = cluster_id; item < a.nitems; item += nclusters) {
    const uint64_t b = item / (uint64_t)a.A;
    const int ai = (int)(item % (uint64_t)a.A);
    const uint16_t *cseg = reinterpret_cast<const uint16_t *>(a.cost + b * N) + seg0 + u;
    const uint16_t *gc = cseg + kL2OnChip * T;
    float4 xr[kL2RegVec];   // on-chip: state; streaming: the load ring
    uint32_t cr[kL2Ring];   // on-chip: cost pairs of xr; streaming: the ring's
    if (!streaming) {
#pragma unroll
      for (int k = 0; k < kL2Ring; ++k)
        cr[k] = (uint32_t)cseg[(2 * k) * T] | ((uint32_t)cseg[(2 * k + 1) * T] << 16);
      for (int j = 0; j < kL2SmemVec; ++j) s_cost[j * T + u] = cseg[(kL2RegVec + j) * T];
    }
    for (int i = threadIdx.x; i < 256; i += kL2Threads) s_T[i] = a.phase[(size_t)ai * 256 + i];
    const double2 ald = a.alpha[ai];
    const float alr = (float)ald.x, ali = (float)ald.y;
    __syncthreads();
    float2 ad = make_float2(0.f, 0.f);  // pending mixer add
    float cnt0 = 0.f;                   // C = 0 count of the instance
    int ridx = 0;
    for (int r = 0; r < a.p; ++r) {
      const bool ro = ridx < a.R && a.rounds[ridx] == r + 1;
      const bool first = r == 0;
      const bool extra = ro || first;
      const int nv = extra ? kSlots : 2;
      DF acc[kSlots];
#pragma unroll
      for (int k = 0; k < kSlots; ++k) acc[k].zero();
      if (streaming) {
        if (first)
          l2_stream_round<true, true>(xr, cr, gp, gc, nb, s_T, ad, amp0, acc, ro);
        else if (extra)
          l2_stream_round<true, false>(xr, cr, gp, gc, nb, s_T, ad, amp0, acc, ro);
        else
          l2_stream_round<false, false>(xr, cr, gp, gc, nb, s_T, ad, amp0, acc, false);
      } else {
        if (first)
          l2_onchip_round<true, true>(xr, cr, s_state, s_cost, u, s_T, ad, amp0, acc, ro);
        else if (extra)
          l2_onchip_round<true, false>(xr, cr, s_state, s_cost, u, s_T, ad, amp0, acc, ro);
        else
          l2_onchip_round<false, false>(xr, cr, s_state, s_cost, u, s_T, ad, amp0, acc, false);
      }
      const int buf = xt & 1;
      float hi[kSlots], lo[kSlots];
#pragma unroll
      for (int k = 0; k < kSlots; ++k) {
        hi[k] = k < nv ? warp_fsum(acc[k].hi + acc[k].lo) : 0.f;
        lo[k] = 0.f;
      }
      if (lane == 0) {
#pragma unroll
        for (int k = 0; k < kSlots; ++k)
          if (k < nv) s_wp[buf][warp][k] = make_float2(hi[k], lo[k]);
      }
      __syncthreads();
      if (warp == 0) {
        // this CTA's partial, pushed to every CTA of the cluster
#pragma unroll
        for (int k = 0; k < kSlots; ++k) {
          const float2 d = (k < nv && lane < kL2Warps) ? s_wp[buf][lane][k] : make_float2(0.f, 0.f);
          hi[k] = d.x;
          lo[k] = d.y;
          if (k < nv) df_warp(hi[k], lo[k]);
        }
        if (lane < kL2Cluster && ok) {  // all six slots, zero past nv: 48 bytes per peer
          const uint32_t rs = mapa_shared(smem_addr(&s_ps[buf][rank][0]), (unsigned)lane);
          const uint32_t rm = mapa_shared(smem_addr(&s_mb[buf]), (unsigned)lane);
          st_async_v4(rs, make_float4(hi[0], lo[0], hi[1], lo[1]), rm);
          st_async_v4(rs + 16, make_float4(hi[2], lo[2], hi[3], lo[3]), rm);
          st_async_v4(rs + 32, make_float4(hi[4], lo[4], hi[5], lo[5]), rm);
        }
      }
      // every CTA's partial in this CTA's receive slots (no cluster barrier:
      // the streaming warps' stores need not complete first)
      if (ok && !mbar_wait(smem_addr(&s_mb[buf]), (xt >> 1) & 1u, a.status)) {
        ok = false;
        atomicExch(a.status, 1u);
      }
      ok = __all_sync(0xffffffffu, ok);
      // armed for its next use, two rounds on (a peer sends into it only
      // after this CTA's partial of the round in between)
      if (threadIdx.x == 0 && ok) mbar_arm(smem_addr(&s_mb[buf]), kSweepSlotBytes * kL2Cluster);
      ++xt;
      // every warp: the cluster sum in rank order
#pragma unroll
      for (int k = 0; k < kSlots; ++k) {
        const float2 d = (k < nv && lane < kL2Cluster) ? s_ps[buf][lane][k] : make_float2(0.f, 0.f);
        hi[k] = d.x;
        lo[k] = d.y;
        if (k < nv) df_warp(hi[k], lo[k]);
      }
      const float Sr = hi[0] + lo[0], Si = hi[1] + lo[1];
      const float ar = (alr * Sr - ali * Si) * inv_n, aim = (alr * Si + ali * Sr) * inv_n;
      if (first) cnt0 = hi[5] + lo[5];
      if (ro && rank == 0 && threadIdx.x == 0) {
        // sum_{C=0} |chi + a|^2 = A0 + 2 Re(conj(a) B0) + h[0] |a|^2
        const double A0 = (double)hi[2] + lo[2], Br = (double)hi[3] + lo[3],
                     Bi = (double)hi[4] + lo[4];
        const double P = A0 + 2.0 * ((double)ar * Br + (double)aim * Bi) +
                         (double)cnt0 * ((double)ar * ar + (double)aim * aim);
        a.out[(b * (uint64_t)a.A + ai) * a.R + ridx] =
            ok ? P : __longlong_as_double(0x7ff8000000000000ll);
      }
      ad = make_float2(ar, aim);
      if (ro) ++ridx;
    }
    __syncthreads();  // s_T and s_cost are rewritten for the next item
  }
  cluster_sync();  // no CTA leaves while a peer may still store into its shared memory
}

static int launch_sweep_l2(const SweepArgs &args, cudaStream_t st) {
  auto kernel = sweep_l2_kernel;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kL2DynSmem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return GQAOA_ECUDA;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kL2Cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kL2Cluster, 1, 1);
  cfg.blockDim = dim3(kL2Threads, 1, 1);
  cfg.dynamicSmemBytes = kL2DynSmem;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, kernel, &cfg) != cudaSuccess) return GQAOA_ECUDA;
  if (clusters < 1) return GQAOA_ECUDA;
  uint64_t units = clusters < kL2Slots ? (uint64_t)clusters : (uint64_t)kL2Slots;
  if (args.nitems < units) units = args.nitems;
  cfg.gridDim = dim3((unsigned)(units * kL2Cluster), 1, 1);
  cfg.stream = st;
  if (cudaLaunchKernelEx(&cfg, kernel, args) != cudaSuccess) return GQAOA_ECUDA;
  return GQAOA_OK;
}

struct SweepShape {
  int threads;
  int cluster;
  bool smem_half;
};

// amps_per_thread: 16 (all in registers) or 32 (16 more in shared memory);
// up to 1024 threads per CTA, then clusters of up to 16 CTAs.
static SweepShape sweep_shape(int n, int amps_per_thread) {
  const int amps = 1 << n;
  int threads = amps / amps_per_thread;
  int cluster = 1;
  if (threads > 1024) {
    cluster = threads / 1024;
    threads = 1024;
  }
  return SweepShape{threads, cluster, amps_per_thread == 32};
}

template <int kThreads, int kCluster, bool kSmemHalf = false>
static int launch_sweep(const SweepArgs &args, cudaStream_t st) {
  auto kernel = sweep_kernel<kThreads, kCluster, kSmemHalf>;
  const size_t dyn = kSmemHalf ? (size_t)kThreads * (16 * sizeof(float2) + 4 * sizeof(uint32_t)) : 0;
  if (kSmemHalf &&
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess)
    return GQAOA_ECUDA;
  int per_unit = 0;  // resident CTAs (cluster == 1) or clusters
  if (kCluster == 1) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_unit, kernel, kThreads, dyn) != cudaSuccess)
      return GQAOA_ECUDA;
    per_unit *= sm_count();
  } else {
    if (kCluster > 8 &&
        cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
      return GQAOA_ECUDA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kCluster, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = dyn;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&per_unit, kernel, &cfg) != cudaSuccess) return GQAOA_ECUDA;
  }
  if (per_unit < 1) return GQAOA_ECUDA;
  uint64_t units = args.nitems < (uint64_t)per_unit ? args.nitems : (uint64_t)per_unit;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(units * kCluster), 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = kCluster > 1 ? 1 : 0;
  if (cudaLaunchKernelEx(&cfg, kernel, args) != cudaSuccess) return GQAOA_ECUDA;
  return GQAOA_OK;
}

// [A][256] phase tables | [A] mixer coefficients | the status word (256 B
// block) | the cluster-resident path's L2 slots.
static size_t sweep_ws_layout(int n, int A, bool resident, char *base, float2 **phase,
                              double2 **alpha, unsigned **status, float4 **scratch) {
  const size_t o_alpha = round_up(sizeof(float2) * 256 * (size_t)A, 256);
  const size_t o_status = o_alpha + round_up(sizeof(double2) * (size_t)A, 256);
  const size_t o_scratch = o_status + 256;
  const size_t scratch_bytes = resident ? (size_t)kL2Slots * (sizeof(float2) << n) : 0;
  if (base) {
    *phase = reinterpret_cast<float2 *>(base);
    *alpha = reinterpret_cast<double2 *>(base + o_alpha);
    *status = reinterpret_cast<unsigned *>(base + o_status);
    *scratch = resident ? reinterpret_cast<float4 *>(base + o_scratch) : nullptr;
  }
  return o_scratch + scratch_bytes;
}

// 0 picks 16 (n <= 18), 32 (n = 19) or the cluster-resident path (n >= 20).
static int sweep_mode(int n, int amps_per_thread) {
  if (amps_per_thread != 0) return amps_per_thread;
  return n <= 18 ? 16 : (n == 19 ? 32 : GQAOA_SWEEP_L2);
}

static int sweep_check_n(int n, int mode) {
  if (mode == GQAOA_SWEEP_L2)
    return (n < GQAOA_SWEEP_L2_MIN_N || n > GQAOA_SWEEP_L2_MAX_N) ? GQAOA_ERANGE : GQAOA_OK;
  if (mode != 16 && mode != 32) return GQAOA_EINVAL;
  if (n < GQAOA_SWEEP_MIN_N || n > GQAOA_SWEEP_MAX_N) return GQAOA_ERANGE;
  if ((mode == 16 && n > 18) || (mode == 32 && n < 10)) return GQAOA_ERANGE;
  return GQAOA_OK;
}

}  // namespace gq

using namespace gq;

extern "C" int gqaoa_sweep_workspace_size(int n, int angles, int amps_per_thread, size_t *bytes) {
  if (!bytes) return GQAOA_EINVAL;
  if (angles < 1 || angles > (1 << 24)) return GQAOA_ERANGE;
  const int mode = sweep_mode(n, amps_per_thread);
  const int rc = sweep_check_n(n, mode);
  if (rc) return rc;
  *bytes = sweep_ws_layout(n, angles, mode == GQAOA_SWEEP_L2, nullptr, nullptr, nullptr, nullptr,
                           nullptr);
  return GQAOA_OK;
}

extern "C" int gqaoa_sweep(const uint8_t *cost, int n, int m, int batch, const double *gammas,
                           const double *betas, int angles, int p, const int32_t *rounds,
                           int nrounds, int amps_per_thread, double *out, void *ws,
                           size_t ws_bytes, void *stream) {
  gq::NvtxRange nvtx_range("gqaoa_sweep");
  if (m < 0 || m > GQAOA_MAX_M || batch < 1 || angles < 1 || angles > (1 << 24) || p < 1 ||
      p > (1 << 20) || nrounds < 1 || nrounds > kSweepMaxRounds)
    return GQAOA_ERANGE;
  if (n < GQAOA_SWEEP_MIN_N || n > GQAOA_SWEEP_L2_MAX_N) return GQAOA_ERANGE;
  const int mode = sweep_mode(n, amps_per_thread);
  int rc = sweep_check_n(n, mode);
  if (rc) return rc;
  if (!cost || !gammas || !betas || !rounds || !out || !ws) return GQAOA_EINVAL;
  if (!aligned16(cost) || !aligned8(gammas) || !aligned8(betas) || !aligned8(out) ||
      !aligned16(ws))
    return GQAOA_EINVAL;
  for (int i = 0; i < nrounds; ++i) {
    if (rounds[i] < 1 || rounds[i] > p) return GQAOA_ERANGE;
    if (i > 0 && rounds[i] <= rounds[i - 1]) return GQAOA_EINVAL;
  }
  const bool resident = mode == GQAOA_SWEEP_L2;
  if (ws_bytes < sweep_ws_layout(n, angles, resident, nullptr, nullptr, nullptr, nullptr, nullptr))
    return GQAOA_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SweepArgs args = {};
  float2 *phase = nullptr;
  double2 *alpha = nullptr;
  float4 *scratch = nullptr;
  unsigned *status = nullptr;
  sweep_ws_layout(n, angles, resident, static_cast<char *>(ws), &phase, &alpha, &status, &scratch);
  rc = phase_tables(gammas, betas, angles, 256, phase, alpha, st);
  if (rc) return rc;
  GQ_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned), st));
  args.cost = cost;
  args.phase = phase;
  args.alpha = alpha;
  args.out = out;
  args.scratch = scratch;
  args.status = status;
  args.nitems = (uint64_t)batch * (uint64_t)angles;
  args.n = n;
  args.A = angles;
  args.p = p;
  args.R = nrounds;
  for (int i = 0; i < nrounds; ++i) args.rounds[i] = rounds[i];
  if (resident) return launch_sweep_l2(args, st);
  const SweepShape sh = sweep_shape(n, mode);
  if (sh.smem_half) {
    switch (sh.threads * 100 + sh.cluster) {
      case 32 * 100 + 1: return launch_sweep<32, 1, true>(args, st);
      case 64 * 100 + 1: return launch_sweep<64, 1, true>(args, st);
      case 128 * 100 + 1: return launch_sweep<128, 1, true>(args, st);
      case 256 * 100 + 1: return launch_sweep<256, 1, true>(args, st);
      case 512 * 100 + 1: return launch_sweep<512, 1, true>(args, st);
      case 1024 * 100 + 1: return launch_sweep<1024, 1, true>(args, st);
      case 1024 * 100 + 2: return launch_sweep<1024, 2, true>(args, st);
      case 1024 * 100 + 4: return launch_sweep<1024, 4, true>(args, st);
      case 1024 * 100 + 8: return launch_sweep<1024, 8, true>(args, st);
      case 1024 * 100 + 16: return launch_sweep<1024, 16, true>(args, st);
      default: return GQAOA_ERANGE;
    }
  }
  switch (sh.threads * 100 + sh.cluster) {
    case 32 * 100 + 1: return launch_sweep<32, 1>(args, st);
    case 64 * 100 + 1: return launch_sweep<64, 1>(args, st);
    case 128 * 100 + 1: return launch_sweep<128, 1>(args, st);
    case 256 * 100 + 1: return launch_sweep<256, 1>(args, st);
    case 512 * 100 + 1: return launch_sweep<512, 1>(args, st);
    case 1024 * 100 + 1: return launch_sweep<1024, 1>(args, st);
    case 1024 * 100 + 2: return launch_sweep<1024, 2>(args, st);
    case 1024 * 100 + 4: return launch_sweep<1024, 4>(args, st);
    case 1024 * 100 + 8: return launch_sweep<1024, 8>(args, st);
    case 1024 * 100 + 16: return launch_sweep<1024, 16>(args, st);
    default: return GQAOA_ERANGE;
  }
}
