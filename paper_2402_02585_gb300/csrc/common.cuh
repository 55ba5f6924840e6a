// Shared device helpers of the G-QAOA CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "gqaoa.h"

namespace gq {

// ---------------------------------------------------------------------------
// error plumbing
// ---------------------------------------------------------------------------
#define GQ_CHECK_LAUNCH()                                                      \
  do {                                                                         \
    if (cudaPeekAtLastError() != cudaSuccess) return GQAOA_ECUDA;              \
  } while (0)

#define GQ_CUDA(call)                                                          \
  do {                                                                         \
    if ((call) != cudaSuccess) return GQAOA_ECUDA;                             \
  } while (0)

// NVTX range around a C-ABI call, so profilers show each call as one range
// over its kernels (header-only NVTX; a no-op unless a tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
inline bool aligned8(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }
inline size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------------------
// launch geometry of the streaming kernels
// ---------------------------------------------------------------------------
constexpr int kThreads = 256;          // threads per CTA
constexpr int kWarps = kThreads / 32;  // warps per CTA
constexpr int kVecPerThread = 8;       // float4 (2 amplitudes) per thread per tile
constexpr int kWarpTileAmps = 32 * kVecPerThread * 2;  // 512 amplitudes
constexpr int kTileAmps = kWarps * kWarpTileAmps;      // 4096 amplitudes per CTA tile
constexpr int kPartStride = 8;         // doubles per partial record

// ---------------------------------------------------------------------------
// small complex helpers (float2 = complex64, double2 = complex128)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Error-free sum of two floats (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Double-float accumulator: hi + lo carries ~48 significant bits, so the
// running sum of many FP32 terms loses nothing measurable before it is
// converted to FP64. It runs on the FP32 pipe, which matters on a part whose
// FP64 rate is a small fraction of its FP32 rate.
struct DF {
  float hi, lo;
  __device__ __forceinline__ void zero() { hi = 0.f; lo = 0.f; }
  __device__ __forceinline__ void add(float x) {
    float s, e;
    two_sum(hi, x, s, e);
    hi = s;
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// ---------------------------------------------------------------------------
// deterministic reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of one double per thread over the CTA in a fixed order; every thread
// gets the result. `scratch` holds kWarps doubles; it is reused on return.
__device__ __forceinline__ double block_sum(double v, double *scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) t += scratch[w];
  return t;
}

// ---------------------------------------------------------------------------
// thread-block cluster primitives (inline PTX; plain DSMEM loads, no multicast)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned cluster_ctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_nctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Load a double from the shared memory of CTA `rank` of this cluster at the
// same offset as the local shared address `p`.
__device__ __forceinline__ double ld_dsmem_f64(const double *p, unsigned rank) {
  uint32_t local = static_cast<uint32_t>(__cvta_generic_to_shared(p));
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(rank));
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(remote) : "memory");
  return v;
}

// Reduce `nvals` (<= kPartStride) per-CTA doubles held in shared `vals`
// over the cluster and write one record to `out_rec` (global). Rank 0 sums
// the CTAs in rank order. Must be called by all threads of every CTA.
__device__ __forceinline__ void cluster_reduce_store(const double *vals, int nvals,
                                                     double *out_rec) {
  const unsigned cs = cluster_nctarank();
  if (cs == 1) {
    if (threadIdx.x < nvals) out_rec[threadIdx.x] = vals[threadIdx.x];
    return;
  }
  cluster_sync();  // every CTA's vals visible cluster-wide
  if (cluster_ctarank() == 0 && threadIdx.x < nvals) {
    double acc = 0.0;
    for (unsigned r = 0; r < cs; ++r) acc += ld_dsmem_f64(vals + threadIdx.x, r);
    out_rec[threadIdx.x] = acc;
  }
  cluster_sync();  // keep every CTA's shared memory alive until rank 0 is done
}

// ---------------------------------------------------------------------------
// cluster exchange through st.async and transaction-counted mbarriers
// ---------------------------------------------------------------------------
// A CTA stores its partials into a receive slot of every CTA of the cluster
// with st.async, each store completing its bytes on the receiver's mbarrier;
// a receiver that armed the phase for (CTAs x slot bytes) holds every
// partial once that phase completes. No cluster barrier and no fence: the
// phase completion, observed with acquire semantics at cluster scope,
// orders the data. Waits are bounded (kMbarWaitNs); a wait that gives up
// returns false, after which the caller stops exchanging and marks what it
// writes invalid.
constexpr uint32_t kMbarWaitNs = 2000000000u;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// The shared::cluster address of CTA `rank`'s copy of local shared address `local`.
__device__ __forceinline__ uint32_t mapa_shared(uint32_t local, unsigned rank) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(rank));
  return remote;
}

__device__ __forceinline__ uint32_t globaltimer_lo() {
  uint32_t t;
  asm volatile("mov.u32 %0, %%globaltimer_lo;" : "=r"(t));
  return t;
}

// An mbarrier with arrival count 1 (the arming thread).
__device__ __forceinline__ void mbar_init(uint32_t mb) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
}

// Makes the initialised mbarriers visible to the cluster's st.async; a
// cluster barrier must follow before any peer stores into them.
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// The one arrival of the current phase, expecting `bytes` of complete_tx.
__device__ __forceinline__ void mbar_arm(uint32_t mb, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(mb),
      "r"(bytes)
      : "memory");
}

// 16 (8) bytes to the shared::cluster address `remote` (16- (8-) byte
// aligned), completing as many bytes on the mbarrier at shared::cluster
// address `rmb` of the same CTA.
__device__ __forceinline__ void st_async_v4(uint32_t remote, float4 v, uint32_t rmb) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];"
      ::"r"(remote), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(rmb) : "memory");
}
__device__ __forceinline__ void st_async_v2(uint32_t remote, float2 v, uint32_t rmb) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];"
               ::"r"(remote), "f"(v.x), "f"(v.y), "r"(rmb) : "memory");
}

// Wait for the phase of parity `parity` of the mbarrier at mb to complete
// (acquire at cluster scope: the peers' st.async data is then visible).
// Bounded: gives up after kMbarWaitNs of polling, or soon after any other
// thread of the launch has given up (*status nonzero); false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t mb, unsigned parity,
                                          const volatile unsigned *status) {
  uint32_t t0 = 0;  // differences of the timer's low word are exact below 4.29 s
  for (unsigned i = 1;; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(mb), "r"(parity)
        : "memory");
    if (done) return true;
    if ((i & 255u) == 0) {
      if (*status) return false;
      const uint32_t t = globaltimer_lo();
      if (i == 256) t0 = t;
      else if (t - t0 > kMbarWaitNs) return false;
    }
  }
}

}  // namespace gq
