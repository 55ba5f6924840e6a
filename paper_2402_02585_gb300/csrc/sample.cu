// K5: fair sampling of shots z ~ |psi(z)|^2 (Section IV; Table I's
// shots-to-all-solutions metric needs exactly this).
//
// Definition: shot s is the smallest z with CDF(z) > u_s * CDF(N-1), where
// CDF(z) = sum_{y <= z} |psi(y)|^2 in index order and u_s is a uniform
// double in [0,1) from Philox4x32-10 (Salmon et al., SC 2011) with counter
// (s, s >> 32, 0, 0) and key (seed, seed >> 32).
//
// CDF arithmetic. The weights of a complex64 state are formed without
// rounding loss that matters: w(z) = re^2 + im^2 as a double-float pair (FP32
// hi + lo; each square is split exactly into its product and the product's
// error by an FMA, the two products are added with TwoSum), about 2^-46
// relative. The state is cut into tiles of 4096 amplitudes and a tile into
// 256 chunks of 16 consecutive amplitudes:
//   chunk    = double-float sum of its 16 weights in index order,
//   in-tile  = inclusive scan over the chunks in double-float arithmetic
//              (warp shuffles, then warps in order), each prefix rounded to
//              FP64, tile total = the last one,
//   tiles    = exclusive scan over the tile totals in FP64 pairs (TwoSum
//              carries each addition's rounding error), rounded to FP64, by
//              many CTAs in two launches,
//   in-chunk = double-float running sums of the chunk's weights, compared as
//              FP64.
// Every CDF value is therefore within a few FP64 rounding units of the exact
// prefix sum of the state's weights, at any n: equal-magnitude amplitudes
// (a whole cost class has one magnitude) cannot make rounding errors pile up
// the way FP32 sums would.
//
// Pass 1 computes tile totals; two launches scan them. With few shots per
// tile (up to 64 on average) pass 1 also stores every tile's chunk prefixes
// and each shot is resolved on its own: binary searches over the tile and
// chunk prefixes, then a walk over its chunk's 16 weights. With more shots,
// each shot finds its tile by binary search, shots are bucketed by tile with
// a counting sort (its counts scanned the same way), and pass 2 re-reads
// only the tiles that received shots, rebuilds the same chunk sums and scan,
// and resolves the shots with the same searches and walk. With at most eight
// tiles (n <= 15) every CTA keeps all tile scans in shared memory and
// resolves its shots directly instead (no bucketing).
// Both passes compute the tile totals with the same instructions in the same
// order, so the levels agree exactly; a target that rounding puts past the
// end of a chunk or tile goes to its last amplitude of nonzero weight.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "cdf.cuh"
#include "common.cuh"

namespace gq {

// ---------------------------------------------------------------------------
// Philox4x32-10: ten rounds of two 32x32 multiplies, key bumped by the Weyl
// constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double shot_uniform(uint64_t seed, uint64_t s) {
  uint32_t c0 = (uint32_t)s, c1 = (uint32_t)(s >> 32), c2 = 0u, c3 = 0u;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  const uint64_t x = ((uint64_t)c1 << 32) | c0;
  return (double)(x >> 11) * (1.0 / 9007199254740992.0);
}

// One tile from global memory (see tile_chunk_scan_regs).
__device__ __forceinline__ void tile_chunk_scan(const float4 *__restrict__ st, uint64_t tile,
                                                double *s_incl, float2 *s_wtot, float &ch,
                                                float &cl, float *cum) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t vbase = tile * (kSampTile / 2) + (uint64_t)warp * 256 + lane;
  float4 v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = st[vbase + 32 * j];
  tile_chunk_scan_regs(v, s_incl, s_wtot, ch, cl, cum);
}

// Pass 1: tile totals and, when chunk_incl is not null, every tile's
// in-tile chunk prefixes (chunk_incl[t * 256 + i] = s_incl[i] of tile t).
__global__ void __launch_bounds__(kThreads)
tile_sum_kernel(const float4 *__restrict__ st, uint64_t ntiles, double *__restrict__ tsum,
                double *__restrict__ chunk_incl) {
  __shared__ double s_incl[kChunksPerTile];
  __shared__ float2 s_wtot[kWarps];
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    float ch, cl;
    tile_chunk_scan(st, t, s_incl, s_wtot, ch, cl, nullptr);
    if (chunk_incl) chunk_incl[t * kChunksPerTile + threadIdx.x] = s_incl[threadIdx.x];
    if (threadIdx.x == 0) tsum[t] = tile_total(s_wtot);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Exclusive scans over per-tile values (tile totals, shot counts) by many
// CTAs in two launches: CTA g scans its 256 values and their total; then
// CTA g adds the total of the CTAs before it, summed once per CTA in a fixed
// order, so the result does not depend on scheduling. (FP64 runs at a few
// operations per clock per SM on GB300, so every FP64-pair addition is
// spread over many CTAs and none is repeated per thread.) Tile totals are added in FP64 pairs
// (the rounding error of each addition kept in the second word, TwoSum), so
// a prefix over 2^22 tiles stays within a rounding unit of the exact sum;
// counts are exact integers.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;

struct DD {
  double hi, lo;
};
__device__ __forceinline__ DD dd_add(DD a, DD b) {
  const double s = __dadd_rn(a.hi, b.hi);
  const double bb = __dsub_rn(s, a.hi);
  const double e = __dadd_rn(__dsub_rn(a.hi, __dsub_rn(s, bb)), __dsub_rn(b.hi, bb));
  const double t = __dadd_rn(e, __dadd_rn(a.lo, b.lo));
  const double h = __dadd_rn(s, t);
  return DD{h, __dsub_rn(t, __dsub_rn(h, s))};
}

struct SumDD {  // tile totals -> FP64 prefixes
  using In = double;
  using Acc = DD;
  using Out = double;
  static __device__ __forceinline__ Acc zero() { return DD{0.0, 0.0}; }
  static __device__ __forceinline__ Acc from(In v) { return DD{v, 0.0}; }
  static __device__ __forceinline__ Acc add(Acc a, Acc b) { return dd_add(a, b); }
  static __device__ __forceinline__ Acc shfl_up(Acc a, int o) {
    return DD{__shfl_up_sync(0xffffffffu, a.hi, o), __shfl_up_sync(0xffffffffu, a.lo, o)};
  }
  static __device__ __forceinline__ Acc shfl_xor(Acc a, int o) {
    return DD{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
  }
  static __device__ __forceinline__ Out out(Acc a) { return __dadd_rn(a.hi, a.lo); }
};

struct SumU32 {  // shot counts -> offsets
  using In = uint32_t;
  using Acc = uint32_t;
  using Out = uint32_t;
  static __device__ __forceinline__ Acc zero() { return 0u; }
  static __device__ __forceinline__ Acc from(In v) { return v; }
  static __device__ __forceinline__ Acc add(Acc a, Acc b) { return a + b; }
  static __device__ __forceinline__ Acc shfl_up(Acc a, int o) {
    return __shfl_up_sync(0xffffffffu, a, o);
  }
  static __device__ __forceinline__ Acc shfl_xor(Acc a, int o) {
    return __shfl_xor_sync(0xffffffffu, a, o);
  }
  static __device__ __forceinline__ Out out(Acc a) { return a; }
};

template <class A>
__global__ void __launch_bounds__(kScanThreads)
scan_local_kernel(const typename A::In *__restrict__ in, uint64_t count,
                  typename A::Acc *__restrict__ loc, typename A::Acc *__restrict__ gtot) {
  using Acc = typename A::Acc;
  __shared__ Acc s_warp[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t i = (uint64_t)blockIdx.x * kScanThreads + threadIdx.x;
  Acc inc = i < count ? A::from(in[i]) : A::zero();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const Acc y = A::shfl_up(inc, o);
    if (lane >= o) inc = A::add(y, inc);
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  constexpr int kW = kScanThreads / 32;
  if (warp == 0) {
    Acc w = lane < kW ? s_warp[lane] : A::zero();
#pragma unroll
    for (int o = 1; o < kW; o <<= 1) {
      const Acc y = A::shfl_up(w, o);
      if (lane >= o) w = A::add(y, w);
    }
    if (lane < kW) s_warp[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  Acc ex = A::shfl_up(inc, 1);
  if (lane == 0) ex = A::zero();
  if (warp > 0) ex = A::add(s_warp[warp - 1], ex);
  if (i < count) loc[i] = ex;
  if (threadIdx.x == 0) gtot[blockIdx.x] = s_warp[kW - 1];
}

template <class A>
__global__ void __launch_bounds__(kScanThreads)
scan_finish_kernel(const typename A::Acc *__restrict__ loc, uint64_t count,
                   const typename A::Acc *__restrict__ gtot, typename A::Out *__restrict__ out) {
  using Acc = typename A::Acc;
  __shared__ Acc s_base;
  // total of the CTAs before this one, by warp 0: strided partial sums per
  // lane, then a fixed butterfly
  if (threadIdx.x < 32) {
    Acc acc = A::zero();
    for (uint32_t g = threadIdx.x; g < blockIdx.x; g += 32) acc = A::add(acc, gtot[g]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = A::add(acc, A::shfl_xor(acc, o));
    if (threadIdx.x == 0) s_base = acc;
  }
  __syncthreads();
  const Acc base = s_base;
  const uint64_t i = (uint64_t)blockIdx.x * kScanThreads + threadIdx.x;
  if (i < count) out[i] = A::out(A::add(base, loc[i]));
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
    out[count] = A::out(A::add(base, gtot[blockIdx.x]));
}

// Smallest tile i with prefix[i+1] > t; past the end -> last tile of nonzero weight.
__device__ __forceinline__ uint32_t find_tile(const double *__restrict__ prefix, uint64_t ntiles,
                                              double t) {
  uint64_t lo = 0, hi = ntiles;  // answer in [lo, hi)
  while (lo < hi) {
    const uint64_t mid = lo + (hi - lo) / 2;
    if (gt_nonneg(prefix[mid + 1], t)) hi = mid; else lo = mid + 1;
  }
  if (lo >= ntiles) {
    lo = ntiles - 1;
    while (lo > 0 && !(prefix[lo + 1] > prefix[lo])) --lo;
  }
  return (uint32_t)lo;
}

// Shots -> tiles, and per-tile shot counts.
__global__ void shot_tile_kernel(const double *__restrict__ prefix, uint64_t ntiles, uint64_t seed,
                                 int64_t shots, uint32_t *__restrict__ shot_tile,
                                 uint32_t *__restrict__ count) {
  const double total = prefix[ntiles];
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < shots;
       s += (int64_t)gridDim.x * blockDim.x) {
    const double t = shot_uniform(seed, (uint64_t)s) * total;
    const uint32_t tile = find_tile(prefix, ntiles, t);
    shot_tile[s] = tile;
    atomicAdd(&count[tile], 1u);
  }
}

__global__ void scatter_kernel(const uint32_t *__restrict__ shot_tile, int64_t shots,
                               const uint32_t *__restrict__ offset, uint32_t *__restrict__ cursor,
                               uint32_t *__restrict__ bucket) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < shots;
       s += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t tile = shot_tile[s];
    const uint32_t pos = offset[tile] + atomicAdd(&cursor[tile], 1u);
    bucket[pos] = (uint32_t)s;
  }
}

// Chunk of the tile: smallest i with incl[i] > r; a target that rounding puts
// past the tile's end goes to its last chunk of nonzero weight.
__device__ __forceinline__ int find_chunk(const double *incl, const float *chunk, double r) {
  int lo = 0, hi = kChunksPerTile;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (gt_nonneg(incl[mid], r)) hi = mid; else lo = mid + 1;
  }
  if (lo >= kChunksPerTile) {
    lo = kChunksPerTile - 1;
    while (lo > 0 && !(chunk[lo] > 0.f)) --lo;
  }
  return lo;
}

// Pass 2: resolve the shots of every tile that received any.
__global__ void __launch_bounds__(kThreads)
resolve_kernel(const float4 *__restrict__ st, uint64_t ntiles, const double *__restrict__ prefix,
               const uint32_t *__restrict__ offset, const uint32_t *__restrict__ bucket,
               uint64_t seed, uint64_t *__restrict__ out) {
  __shared__ double s_incl[kChunksPerTile];
  __shared__ float2 s_wtot[kWarps];
  __shared__ float s_chunk[kChunksPerTile];
  const double total = prefix[ntiles];
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint32_t b0 = offset[t], b1 = offset[t + 1];
    if (b0 == b1) continue;  // uniform across the CTA
    float ch, cl;
    tile_chunk_scan(st, t, s_incl, s_wtot, ch, cl, nullptr);
    s_chunk[threadIdx.x] = ch;
    __syncthreads();
    const double tbase = prefix[t];
    for (uint32_t q = b0 + threadIdx.x; q < b1; q += blockDim.x) {
      const uint32_t s = bucket[q];
      const double r = shot_uniform(seed, s) * total - tbase;
      const int c = find_chunk(s_incl, s_chunk, r);
      const double rl = r - (c > 0 ? s_incl[c - 1] : 0.0);
      const uint64_t base = t * kSampTile + (uint64_t)c * kChunk;  // the tile is in L2 now
      out[s] = base + chunk_pick(st + base / 2, rl, make_float2(0.f, 0.f));
    }
    __syncthreads();
  }
}

// Few shots per tile (at most kDirectShotsPerTile on average, e.g. 10^6 shots
// over the 65536 tiles of n = 28): pass 1 has stored every tile's chunk
// prefixes, so a shot needs neither the counting sort nor a re-read of its
// whole tile. Each thread takes a grid-stride range of shots and resolves
// each from the tile prefixes, its tile's 256 chunk prefixes and its chunk's
// 16 amplitudes (128 bytes), with the searches and the chunk walk of pass 2:
// the same shots, about a twentieth of the memory traffic.
constexpr uint64_t kDirectShotsPerTile = 64;

// `add`: when not null, the pending mixer term a_p of a state st = psi_p - a_p
// (gqaoa_evolve_sample), added to every amplitude as the chunk is walked.
__global__ void __launch_bounds__(kThreads)
resolve_direct_kernel(const float4 *__restrict__ st, uint64_t ntiles,
                      const double *__restrict__ prefix, const double *__restrict__ chunk_incl,
                      const float2 *__restrict__ add, uint64_t seed, int64_t shots,
                      uint64_t *__restrict__ out) {
  const double total = prefix[ntiles];
  const float2 ad = add ? *add : make_float2(0.f, 0.f);
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < shots;
       s += (int64_t)gridDim.x * blockDim.x) {
    const double tt = shot_uniform(seed, (uint64_t)s) * total;
    const uint32_t t = find_tile(prefix, ntiles, tt);
    const double r = tt - prefix[t];
    const double *incl = chunk_incl + (uint64_t)t * kChunksPerTile;
    int lo = 0, hi = kChunksPerTile;  // chunk: smallest i with incl[i] > r
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (gt_nonneg(incl[mid], r)) hi = mid; else lo = mid + 1;
    }
    if (lo >= kChunksPerTile) {  // rounding past the tile end: last chunk of nonzero weight
      lo = kChunksPerTile - 1;
      while (lo > 0 && !(incl[lo] > incl[lo - 1])) --lo;
    }
    const double rl = r - (lo > 0 ? incl[lo - 1] : 0.0);
    const uint64_t base = (uint64_t)t * kSampTile + (uint64_t)lo * kChunk;
    out[s] = base + chunk_pick(st + base / 2, rl, ad);
  }
}

// Few tiles (N <= kResidentTiles x 4096): shots far outnumber tiles, and the
// counting sort would serialise on a handful of counters. Every CTA instead
// rebuilds the chunk scans of all tiles in shared memory (the instructions of
// pass 2) and resolves a grid-stride range of shots directly, with the same
// tile and chunk searches. Inside a chunk it first searches FP32 running sums
// of the weights' leading words, which lie within 2^-19 of the chunk's sum of
// the exact running sums; only a target within 2^-17 of the chunk's sum of
// one of them (about one shot in 10^4) is decided by chunk_pick on the
// chunk's amplitudes reloaded from global memory (L2-resident at these
// sizes), so every shot is the one pass 2 would give. A tile scan takes 20 KB
// of shared memory, so up to four tiles (n <= 14) leave room for two CTAs per
// SM.
constexpr int kResidentTiles = 8;
struct TileScan {
  float cum[kChunksPerTile * kPad];  // per chunk (row of kPad): FP32 running sums
  double incl[kChunksPerTile];
  float chunk[kChunksPerTile];       // leading word of each chunk's sum
};

// chunk_pick on global memory, kept out of line: the resident path takes it
// for about one shot in 10^4, and inlined it would crowd the common path.
__device__ __noinline__ int chunk_pick_global(const float4 *row, double rl) {
  return chunk_pick(row, rl, make_float2(0.f, 0.f));
}

__device__ __forceinline__ uint64_t resolve_shot(const float4 *__restrict__ st, const TileScan *ts,
                                                 const double *s_prefix, uint64_t ntiles,
                                                 double total, uint64_t seed, uint64_t s) {
  const double u = shot_uniform(seed, s);
  const uint32_t t = find_tile(s_prefix, ntiles, u * total);
  const TileScan &T = ts[t];
  const double r = u * total - s_prefix[t];
  const int c = find_chunk(T.incl, T.chunk, r);
  const double rl = r - (c > 0 ? T.incl[c - 1] : 0.0);
  const float rlf = (float)rl;
  const float *row = T.cum + c * kPad;
  int a = 0, b = kChunk;  // first FP32 running sum above rl
  while (a < b) {
    const int mid = (a + b) >> 1;
    if (row[mid] > rlf) b = mid; else a = mid + 1;
  }
  const float tol = T.chunk[c] * 0x1p-17f;
  const bool clear = a < kChunk && row[a] > rlf + tol && (a == 0 || row[a - 1] < rlf - tol);
  const uint64_t base = (uint64_t)t * kSampTile + (uint64_t)c * kChunk;
  const int pick = clear ? a : chunk_pick_global(st + base / 2, rl);
  return base + pick;
}

__global__ void __launch_bounds__(kThreads)
resolve_resident_kernel(const float4 *__restrict__ st, uint64_t ntiles,
                        const double *__restrict__ prefix, uint64_t seed, int64_t shots,
                        uint64_t *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  TileScan *ts = reinterpret_cast<TileScan *>(s_dyn);  // [ntiles]
  __shared__ float2 s_wtot[kWarps];
  __shared__ double s_prefix[kResidentTiles + 1];
  if (threadIdx.x <= ntiles) s_prefix[threadIdx.x] = prefix[threadIdx.x];
  for (uint64_t t = 0; t < ntiles; ++t) {
    float ch, cl;
    tile_chunk_scan(st, t, ts[t].incl, s_wtot, ch, cl, ts[t].cum);
    ts[t].chunk[threadIdx.x] = ch;
  }
  __syncthreads();
  const double total = s_prefix[ntiles];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // two shots per thread in flight: independent chains of shared-memory loads
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < shots; s += 2 * stride) {
    const int64_t s2 = s + stride;
    const uint64_t z = resolve_shot(st, ts, s_prefix, ntiles, total, seed, (uint64_t)s);
    uint64_t z2 = 0;
    if (s2 < shots) z2 = resolve_shot(st, ts, s_prefix, ntiles, total, seed, (uint64_t)s2);
    out[s] = z;
    if (s2 < shots) out[s2] = z2;
  }
}

// Small states (N <= 2048): FP64 CDF in shared memory (exact squares of the
// complex64 parts, running sum with Neumaier's compensation), built by every
// CTA, shots in a grid-stride range.
__global__ void __launch_bounds__(kThreads)
sample_small_kernel(const float2 *__restrict__ st, int n, uint64_t seed, int64_t shots,
                    uint64_t *__restrict__ out) {
  __shared__ double s_cdf[2048];
  const int N = 1 << n;
  for (int z = threadIdx.x; z < N; z += blockDim.x) {
    const float2 v = st[z];
    s_cdf[z] = (double)v.x * v.x + (double)v.y * v.y;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double run = 0.0, carry = 0.0;
    for (int z = 0; z < N; ++z) {
      const double w = s_cdf[z];
      const double t = run + w;
      carry += fabs(run) >= fabs(w) ? (run - t) + w : (w - t) + run;
      run = t;
      s_cdf[z] = run + carry;
    }
  }
  __syncthreads();
  const double total = s_cdf[N - 1];
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < shots;
       s += (int64_t)gridDim.x * blockDim.x) {
    const double t = shot_uniform(seed, (uint64_t)s) * total;
    int lo = 0, hi = N - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (gt_nonneg(s_cdf[mid], t)) hi = mid; else lo = mid + 1;
    }
    out[s] = (uint64_t)lo;
  }
}

struct SampleWs {
  double *chunk_incl;  // [ntiles][256] (direct mode only)
  double *tsum;        // [ntiles]
  double *prefix;      // [ntiles + 1]
  DD *scan_loc;        // [ntiles]   in-CTA prefixes of the tile-total scan
  DD *scan_tot;        // [groups]   CTA totals of the tile-total scan
  uint32_t *count;     // [ntiles]
  uint32_t *cursor;    // [ntiles]
  uint32_t *offset;    // [ntiles + 1]
  uint32_t *cnt_loc;   // [ntiles]   the same for the shot counts
  uint32_t *cnt_tot;   // [groups]
  uint32_t *shot_tile; // [shots]
  uint32_t *bucket;    // [shots]
};

// Direct mode (few shots per tile, more tiles than the resident path takes):
// the chunk prefixes instead of the counting sort's buffers.
static bool sample_direct(uint64_t ntiles, int64_t shots) {
  return ntiles > (uint64_t)kResidentTiles && (uint64_t)shots <= kDirectShotsPerTile * ntiles;
}

static size_t sample_ws_layout(uint64_t ntiles, int64_t shots, char *base, SampleWs *w) {
  const bool direct = sample_direct(ntiles, shots);
  if (direct) shots = 0;  // no per-shot buffers
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = round_up(off + bytes, 256);
    return o;
  };
  const uint64_t groups = (ntiles + kScanThreads - 1) / kScanThreads;
  size_t o1 = take(sizeof(double) * ntiles);
  size_t o2 = take(sizeof(double) * (ntiles + 1));
  size_t o3 = take(sizeof(DD) * ntiles);
  size_t o4 = take(sizeof(DD) * groups);
  size_t o5 = take(sizeof(uint32_t) * ntiles * 2);  // count and cursor, adjacent
  size_t o6 = take(sizeof(uint32_t) * (ntiles + 1));
  size_t o7 = take(sizeof(uint32_t) * ntiles);
  size_t o8 = take(sizeof(uint32_t) * groups);
  size_t o9 = take(sizeof(uint32_t) * (size_t)shots);
  size_t o10 = take(sizeof(uint32_t) * (size_t)shots);
  size_t o11 = direct ? take(sizeof(double) * ntiles * kChunksPerTile) : 0;
  if (w) {
    w->chunk_incl = direct ? reinterpret_cast<double *>(base + o11) : nullptr;
    w->tsum = reinterpret_cast<double *>(base + o1);
    w->prefix = reinterpret_cast<double *>(base + o2);
    w->scan_loc = reinterpret_cast<DD *>(base + o3);
    w->scan_tot = reinterpret_cast<DD *>(base + o4);
    w->count = reinterpret_cast<uint32_t *>(base + o5);
    w->cursor = w->count + ntiles;
    w->offset = reinterpret_cast<uint32_t *>(base + o6);
    w->cnt_loc = reinterpret_cast<uint32_t *>(base + o7);
    w->cnt_tot = reinterpret_cast<uint32_t *>(base + o8);
    w->shot_tile = reinterpret_cast<uint32_t *>(base + o9);
    w->bucket = reinterpret_cast<uint32_t *>(base + o10);
  }
  return off;
}

int sm_count();

// Resident CTAs per SM of the tile passes (shared memory bounds them),
// queried once per device; 4 if no device answers.
static int tile_pass_per_sm() {
  constexpr int kMaxDev = 64;
  static std::once_flag once[kMaxDev];
  static int per_sm[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 4;
  std::call_once(once[dev], [dev]() {
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, tile_sum_kernel, kThreads, 0) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, resolve_kernel, kThreads, 0) !=
            cudaSuccess)
      a = b = 4;
    per_sm[dev] = std::max(1, std::min(a, b));
  });
  return per_sm[dev];
}

// gqaoa_evolve_sample's use of the direct mode: whether it applies, the
// buffers a fused pass fills (tile totals and chunk prefixes in the layout of
// gqaoa_sample's workspace), and the passes after them.
bool sample_direct_ok(uint64_t ntiles, int64_t shots) { return sample_direct(ntiles, shots); }

size_t sample_direct_ws(uint64_t ntiles, int64_t shots, char *base, double **tsum,
                        double **chunk_incl) {
  SampleWs w;
  const size_t bytes = sample_ws_layout(ntiles, shots, base, &w);
  *tsum = w.tsum;
  *chunk_incl = w.chunk_incl;
  return bytes;
}

int sample_direct_tail(const float4 *state, const float2 *add, uint64_t ntiles, uint64_t seed,
                       int64_t shots, uint64_t *out_idx, void *ws, cudaStream_t st) {
  SampleWs w;
  sample_ws_layout(ntiles, shots, static_cast<char *>(ws), &w);
  const unsigned groups = (unsigned)((ntiles + kScanThreads - 1) / kScanThreads);
  scan_local_kernel<SumDD><<<groups, kScanThreads, 0, st>>>(w.tsum, ntiles, w.scan_loc,
                                                            w.scan_tot);
  GQ_CHECK_LAUNCH();
  scan_finish_kernel<SumDD><<<groups, kScanThreads, 0, st>>>(w.scan_loc, ntiles, w.scan_tot,
                                                             w.prefix);
  GQ_CHECK_LAUNCH();
  const int64_t need = (shots + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)(sm_count() > 0 ? sm_count() : 152) * 8;
  resolve_direct_kernel<<<(unsigned)(need < cap ? need : cap), kThreads, 0, st>>>(
      state, ntiles, w.prefix, w.chunk_incl, add, seed, shots, out_idx);
  GQ_CHECK_LAUNCH();
  return GQAOA_OK;
}

}  // namespace gq

using namespace gq;

extern "C" int gqaoa_sample_workspace_size(int n, int64_t shots, size_t *bytes) {
  if (!bytes) return GQAOA_EINVAL;
  if (n < 1 || n > GQAOA_MAX_N || shots < 0 || shots >= (1ll << 32)) return GQAOA_ERANGE;
  const uint64_t N = 1ull << n;
  *bytes = N < (uint64_t)kSampTile ? 256 : sample_ws_layout(N / kSampTile, shots, nullptr, nullptr);
  return GQAOA_OK;
}

extern "C" int gqaoa_sample(const void *state, int n, uint64_t seed, int64_t shots,
                            uint64_t *out_idx, void *ws, size_t ws_bytes, void *stream) {
  gq::NvtxRange nvtx_range("gqaoa_sample");
  if (n < 1 || n > GQAOA_MAX_N || shots < 0 || shots >= (1ll << 32)) return GQAOA_ERANGE;
  if (!state || (shots > 0 && !out_idx)) return GQAOA_EINVAL;
  if (!aligned16(state) || (out_idx && !aligned8(out_idx))) return GQAOA_EINVAL;
  if (shots == 0) return GQAOA_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint64_t N = 1ull << n;
  const int sms0 = sm_count() > 0 ? sm_count() : 152;
  // CTAs for a grid-stride pass over the shots (each builds its own tables)
  const auto shot_ctas = [&](int per_sm) {
    const int64_t need = (shots + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)sms0 * per_sm;
    return (unsigned)(need < cap ? need : cap);
  };
  if (N < (uint64_t)kSampTile) {
    sample_small_kernel<<<shot_ctas(8), kThreads, 0, st>>>(static_cast<const float2 *>(state), n,
                                                           seed, shots, out_idx);
    GQ_CHECK_LAUNCH();
    return GQAOA_OK;
  }
  const uint64_t ntiles = N / kSampTile;
  if (!ws || !aligned16(ws)) return GQAOA_EINVAL;
  if (ws_bytes < sample_ws_layout(ntiles, shots, nullptr, nullptr)) return GQAOA_ENOMEM;
  SampleWs w;
  sample_ws_layout(ntiles, shots, static_cast<char *>(ws), &w);
  const float4 *s4 = static_cast<const float4 *>(state);
  // the tile passes run one wave of resident CTAs, each striding over tiles
  const uint64_t twave = (uint64_t)sms0 * (uint64_t)tile_pass_per_sm();
  const unsigned tgrid = (unsigned)(ntiles < twave ? ntiles : twave);
  const int sms = sms0;
  const unsigned groups = (unsigned)((ntiles + kScanThreads - 1) / kScanThreads);
  tile_sum_kernel<<<tgrid, kThreads, 0, st>>>(s4, ntiles, w.tsum, w.chunk_incl);
  GQ_CHECK_LAUNCH();
  scan_local_kernel<SumDD><<<groups, kScanThreads, 0, st>>>(w.tsum, ntiles, w.scan_loc,
                                                            w.scan_tot);
  GQ_CHECK_LAUNCH();
  scan_finish_kernel<SumDD><<<groups, kScanThreads, 0, st>>>(w.scan_loc, ntiles, w.scan_tot,
                                                             w.prefix);
  GQ_CHECK_LAUNCH();
  if (ntiles <= (uint64_t)kResidentTiles) {
    const size_t dyn = sizeof(TileScan) * ntiles;
    if (cudaFuncSetAttribute(resolve_resident_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)dyn) != cudaSuccess)
      return GQAOA_ECUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, resolve_resident_kernel, kThreads,
                                                      dyn) != cudaSuccess || per_sm < 1)
      return GQAOA_ECUDA;
    resolve_resident_kernel<<<shot_ctas(per_sm), kThreads, dyn, st>>>(s4, ntiles, w.prefix, seed,
                                                                       shots, out_idx);
    GQ_CHECK_LAUNCH();
    return GQAOA_OK;
  }
  if (w.chunk_incl) {
    resolve_direct_kernel<<<shot_ctas(8), kThreads, 0, st>>>(s4, ntiles, w.prefix, w.chunk_incl,
                                                             nullptr, seed, shots, out_idx);
    GQ_CHECK_LAUNCH();
    return GQAOA_OK;
  }
  GQ_CUDA(cudaMemsetAsync(w.count, 0, sizeof(uint32_t) * ntiles * 2, st));
  const unsigned sgrid =
      (unsigned)((shots + kThreads - 1) / kThreads < (int64_t)sms * 16 ? (shots + kThreads - 1) / kThreads
                                                                      : (int64_t)sms * 16);
  shot_tile_kernel<<<sgrid, kThreads, 0, st>>>(w.prefix, ntiles, seed, shots, w.shot_tile, w.count);
  GQ_CHECK_LAUNCH();
  scan_local_kernel<SumU32><<<groups, kScanThreads, 0, st>>>(w.count, ntiles, w.cnt_loc,
                                                             w.cnt_tot);
  GQ_CHECK_LAUNCH();
  scan_finish_kernel<SumU32><<<groups, kScanThreads, 0, st>>>(w.cnt_loc, ntiles, w.cnt_tot,
                                                              w.offset);
  GQ_CHECK_LAUNCH();
  scatter_kernel<<<sgrid, kThreads, 0, st>>>(w.shot_tile, shots, w.offset, w.cursor, w.bucket);
  GQ_CHECK_LAUNCH();
  resolve_kernel<<<tgrid, kThreads, 0, st>>>(s4, ntiles, w.prefix, w.offset, w.bucket, seed, out_idx);
  GQ_CHECK_LAUNCH();
  return GQAOA_OK;
}
