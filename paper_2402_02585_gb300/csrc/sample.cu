// K5: fair sampling of shots z ~ |psi(z)|^2 (Section IV; Table I's
// shots-to-all-solutions metric needs exactly this).
//
// Definition: shot s is the smallest z with CDF(z) > u_s * CDF(N-1), where
// CDF(z) = sum_{y <= z} |psi(y)|^2 in index order and u_s is a uniform
// double in [0,1) from Philox4x32-10 (Salmon et al., SC 2011) with counter
// (s, s >> 32, 0, 0) and key (seed, seed >> 32).
//
// Two-level CDF. The state is cut into tiles of 4096 amplitudes and a tile
// into 256 chunks of 16 consecutive amplitudes.
//   w(z)     = |psi(z)|^2 in FP32 (the state is complex64),
//   chunk    = FP32 running sum of its 16 w in index order,
//   in-tile  = inclusive scan over the chunks in double-float arithmetic
//              (FP32 pairs: warp shuffles, then warps in order), each prefix
//              rounded to FP64, tile total = the last one,
//   tiles    = FP64 exclusive scan over tile totals.
// Pass 1 computes tile totals; a single-CTA pass scans them; each shot then
// finds its tile by binary search, shots are bucketed by tile with a
// counting sort, and pass 2 re-reads only the tiles that received shots,
// rebuilds the same chunk sums and scan, and resolves each shot by a binary
// search over chunks and a walk over 16 amplitudes. With at most eight tiles
// (n <= 15) every CTA keeps all tile scans in shared memory and resolves its
// shots directly instead (same arithmetic, no bucketing). Both passes compute the
// tile totals with the same instructions in the same order, so the levels
// agree exactly; a target that rounding puts past the end of a chunk or tile
// goes to its last amplitude of nonzero weight.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace gq {

constexpr int kSampTile = 4096;
constexpr int kChunk = 16;
constexpr int kChunksPerTile = kSampTile / kChunk;  // 256 = one per thread
constexpr int kPad = kChunk + 1;                    // shared row stride (bank spread)

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

// a > b for non-negative doubles (CDF values and targets), decided on the
// integer pipe: IEEE 754 orders non-negative values as their bit patterns
// read as integers, so this equals the FP64 comparison without using GB300's
// narrow FP64 pipe, which the shot searches would otherwise saturate.
__device__ __forceinline__ bool gt_nonneg(double a, double b) {
  return __double_as_longlong(a) > __double_as_longlong(b);
}

// (h, l) += (yh, yl) in double-float arithmetic (non-negative terms here).
__device__ __forceinline__ void df_add(float &h, float &l, float yh, float yl) {
  float s, e;
  two_sum(h, yh, s, e);
  h = s;
  l = __fadd_rn(__fadd_rn(l, yl), e);
}

// Per tile: chunk sums (FP32, index order) and their inclusive scan in
// double-float arithmetic (FP32 pairs, ~48 bits; FP64 would be issue-bound on
// GB300's FP64 pipe here), stored as FP64.
// On return s_incl[i] holds the inclusive prefix of chunk i within the tile
// and s_w the tile's w values (row stride kPad). Called by all 256 threads.
__device__ __forceinline__ void tile_chunk_scan(const float4 *__restrict__ st, uint64_t tile,
                                                float *s_w, double *s_incl, float2 *s_wtot,
                                                float *chunk_out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // coalesced loads: warp covers 512 amplitudes, lane holds amplitudes
  // 64j + 2 lane and 64j + 2 lane + 1 of its warp tile
  const uint64_t vbase = tile * (kSampTile / 2) + (uint64_t)warp * 256 + lane;
  float *sw = s_w + warp * 32 * kPad;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float4 v = st[vbase + 32 * j];
    const int a = 64 * j + 2 * lane;  // amplitude index within the warp tile
    sw[(a / kChunk) * kPad + (a % kChunk)] = fmaf(v.x, v.x, v.y * v.y);
    sw[((a + 1) / kChunk) * kPad + ((a + 1) % kChunk)] = fmaf(v.z, v.z, v.w * v.w);
  }
  __syncwarp();
  float c = 0.f;
#pragma unroll
  for (int i = 0; i < kChunk; ++i) c += sw[lane * kPad + i];
  *chunk_out = c;
  // inclusive scan over the warp's 32 chunks
  float xh = c, xl = 0.f;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float yh = __shfl_up_sync(0xffffffffu, xh, o);
    const float yl = __shfl_up_sync(0xffffffffu, xl, o);
    if (lane >= o) df_add(xh, xl, yh, yl);
  }
  if (lane == 31) s_wtot[warp] = make_float2(xh, xl);
  __syncthreads();
  float bh = 0.f, bl = 0.f;  // the warps before this one, in order
  for (int w = 0; w < warp; ++w) df_add(bh, bl, s_wtot[w].x, s_wtot[w].y);
  df_add(bh, bl, xh, xl);
  s_incl[threadIdx.x] = (double)bh + (double)bl;
  __syncthreads();
}

__device__ __forceinline__ double tile_total(const float2 *s_wtot) {
  float th = 0.f, tl = 0.f;
  for (int w = 0; w < kWarps; ++w) df_add(th, tl, s_wtot[w].x, s_wtot[w].y);
  return (double)th + (double)tl;
}

// Pass 1: tile totals.
__global__ void __launch_bounds__(kThreads)
tile_sum_kernel(const float4 *__restrict__ st, uint64_t ntiles, double *__restrict__ tsum) {
  __shared__ float s_w[kWarps * 32 * kPad];
  __shared__ double s_incl[kChunksPerTile];
  __shared__ float2 s_wtot[kWarps];
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    float c;
    tile_chunk_scan(st, t, s_w, s_incl, s_wtot, &c);
    if (threadIdx.x == 0) tsum[t] = tile_total(s_wtot);
    __syncthreads();
  }
}

// Single-CTA exclusive FP64 scan of tile totals: prefix[0..ntiles].
__global__ void __launch_bounds__(1024)
scan_tiles_kernel(const double *__restrict__ tsum, uint64_t ntiles, double *__restrict__ prefix) {
  __shared__ double s_part[1024];
  const uint64_t per = (ntiles + blockDim.x - 1) / blockDim.x;
  const uint64_t lo = threadIdx.x * per;
  const uint64_t hi = lo + per < ntiles ? lo + per : ntiles;
  double acc = 0.0;
#pragma unroll 8
  for (uint64_t i = lo; i < hi; ++i) acc += tsum[i];
  s_part[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double run = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) {
      const double v = s_part[i];
      s_part[i] = run;
      run += v;
    }
    prefix[ntiles] = run;
  }
  __syncthreads();
  double run = s_part[threadIdx.x];
#pragma unroll 8
  for (uint64_t i = lo; i < hi; ++i) {
    prefix[i] = run;
    run += tsum[i];
  }
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

// Single-CTA exclusive scan of the per-tile counts (uint32, exact in any
// order): thread t sums its contiguous range, a shuffle scan over the threads
// gives its offset, then it writes its range.
__global__ void __launch_bounds__(1024)
scan_counts_kernel(const uint32_t *__restrict__ count, uint64_t ntiles,
                   uint32_t *__restrict__ offset) {
  __shared__ uint32_t s_warp[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t per = (ntiles + blockDim.x - 1) / blockDim.x;
  const uint64_t lo = threadIdx.x * per;
  const uint64_t hi = lo + per < ntiles ? lo + per : ntiles;
  uint32_t acc = 0;
#pragma unroll 8
  for (uint64_t i = lo; i < hi; ++i) acc += count[i];
  // exclusive scan of acc over the CTA
  uint32_t x = acc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    s_warp[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  uint32_t run = (warp > 0 ? s_warp[warp - 1] : 0u) + x - acc;
  if (threadIdx.x == blockDim.x - 1) offset[ntiles] = run + acc;
#pragma unroll 8
  for (uint64_t i = lo; i < hi; ++i) {
    offset[i] = run;
    run += count[i];
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

// Pass 2: resolve the shots of every tile that received any.
__global__ void __launch_bounds__(kThreads)
resolve_kernel(const float4 *__restrict__ st, uint64_t ntiles, const double *__restrict__ prefix,
               const uint32_t *__restrict__ offset, const uint32_t *__restrict__ bucket,
               uint64_t seed, uint64_t *__restrict__ out) {
  __shared__ float s_w[kWarps * 32 * kPad];
  __shared__ double s_incl[kChunksPerTile];
  __shared__ float2 s_wtot[kWarps];
  __shared__ float s_chunk[kChunksPerTile];
  const double total = prefix[ntiles];
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint32_t b0 = offset[t], b1 = offset[t + 1];
    if (b0 == b1) continue;  // uniform across the CTA
    float c;
    tile_chunk_scan(st, t, s_w, s_incl, s_wtot, &c);
    s_chunk[threadIdx.x] = c;
    __syncthreads();
    const double tbase = prefix[t];
    for (uint32_t q = b0 + threadIdx.x; q < b1; q += blockDim.x) {
      const uint32_t s = bucket[q];
      const double r = shot_uniform(seed, s) * total - tbase;
      // chunk: smallest i with s_incl[i] > r
      int lo = 0, hi = kChunksPerTile;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (gt_nonneg(s_incl[mid], r)) hi = mid; else lo = mid + 1;
      }
      if (lo >= kChunksPerTile) {  // rounding past the tile end
        lo = kChunksPerTile - 1;
        while (lo > 0 && !(s_chunk[lo] > 0.f)) --lo;
      }
      const double rl = r - (lo > 0 ? s_incl[lo - 1] : 0.0);
      // for a float f, f > rl exactly when f > rl rounded down to a float, so
      // the walk compares in FP32 and decides as an FP64 comparison would
      const float rlf = __double2float_rd(rl);
      // walk the chunk in index order with the same FP32 running sum
      const int warp_of = lo >> 5, lane_of = lo & 31;
      const float *row = s_w + warp_of * 32 * kPad + lane_of * kPad;
      float cum = 0.f;
      int pick = -1, last_nz = 0;
#pragma unroll
      for (int i = 0; i < kChunk; ++i) {
        const float wi = row[i];
        cum += wi;
        if (wi > 0.f) last_nz = i;
        if (pick < 0 && cum > rlf) pick = i;
      }
      if (pick < 0) pick = last_nz;
      // amplitude index: tile, warp tile of the chunk, position in the warp tile
      out[s] = t * kSampTile + (uint64_t)warp_of * 512 + (uint64_t)lane_of * kChunk + pick;
    }
    __syncthreads();
  }
}

// Few tiles (N <= kResidentTiles x 4096): shots far outnumber tiles, and the
// counting sort would serialise on a handful of counters. Every CTA instead
// rebuilds the chunk scans of all tiles in shared memory (the instructions of
// pass 2) and resolves a grid-stride range of shots directly, with the same
// tile search. The walk over a chunk's 16 weights is replaced by a binary
// search over their FP32 running sums, computed once in the walk's order:
// the sums never decrease, so the first sum above the target is the index
// the walk would stop at, and the shots are the ones pass 2 would give.
constexpr int kResidentTiles = 8;
struct TileScan {
  float cum[kWarps * 32 * kPad];  // per chunk (row of kPad): running sums of its 16 weights
  double incl[kChunksPerTile];
  float chunk[kChunksPerTile];
  uint8_t last_nz[kChunksPerTile];  // last weight > 0 in the chunk (0 if none)
};

__device__ __forceinline__ uint64_t resolve_shot(const TileScan *ts, const double *s_prefix,
                                                 uint64_t ntiles, double total, uint64_t seed,
                                                 uint64_t s) {
  const double u = shot_uniform(seed, s);
  const uint32_t t = find_tile(s_prefix, ntiles, u * total);
  const TileScan &T = ts[t];
  const double r = u * total - s_prefix[t];
  int lo = 0, hi = kChunksPerTile;  // chunk: smallest i with incl[i] > r
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (gt_nonneg(T.incl[mid], r)) hi = mid; else lo = mid + 1;
  }
  if (lo >= kChunksPerTile) {  // rounding past the tile end
    lo = kChunksPerTile - 1;
    while (lo > 0 && !(T.chunk[lo] > 0.f)) --lo;
  }
  const double rl = r - (lo > 0 ? T.incl[lo - 1] : 0.0);
  const float rlf = __double2float_rd(rl);  // f > rl  <=>  f > rlf for every float f
  const int warp_of = lo >> 5, lane_of = lo & 31;
  const float *row = T.cum + warp_of * 32 * kPad + lane_of * kPad;
  int a = 0, b = kChunk;  // first running sum above rl
  while (a < b) {
    const int mid = (a + b) >> 1;
    if (row[mid] > rlf) b = mid; else a = mid + 1;
  }
  const int pick = a < kChunk ? a : (int)T.last_nz[lo];
  return t * kSampTile + (uint64_t)warp_of * 512 + (uint64_t)lane_of * kChunk + pick;
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
    float c;
    tile_chunk_scan(st, t, ts[t].cum, ts[t].incl, s_wtot, &c);
    ts[t].chunk[threadIdx.x] = c;
    // this thread's chunk: weights -> running sums (the walk's FP32 order)
    float *row = ts[t].cum + (threadIdx.x >> 5) * 32 * kPad + (threadIdx.x & 31) * kPad;
    float run = 0.f;
    int last = 0;
    for (int i = 0; i < kChunk; ++i) {
      const float wi = row[i];
      run += wi;
      if (wi > 0.f) last = i;
      row[i] = run;
    }
    ts[t].last_nz[threadIdx.x] = (uint8_t)last;
    __syncthreads();
  }
  const double total = s_prefix[ntiles];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // two shots per thread in flight: independent chains of shared-memory loads
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < shots; s += 2 * stride) {
    const int64_t s2 = s + stride;
    const uint64_t z = resolve_shot(ts, s_prefix, ntiles, total, seed, (uint64_t)s);
    uint64_t z2 = 0;
    if (s2 < shots) z2 = resolve_shot(ts, s_prefix, ntiles, total, seed, (uint64_t)s2);
    out[s] = z;
    if (s2 < shots) out[s2] = z2;
  }
}

// Small states (N <= 2048): exact FP64 CDF in shared memory, built by every
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
    double run = 0.0;
    for (int z = 0; z < N; ++z) {
      run += s_cdf[z];
      s_cdf[z] = run;
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
  double *tsum;        // [ntiles]
  double *prefix;      // [ntiles + 1]
  uint32_t *count;     // [ntiles]
  uint32_t *cursor;    // [ntiles]
  uint32_t *offset;    // [ntiles + 1]
  uint32_t *shot_tile; // [shots]
  uint32_t *bucket;    // [shots]
};

static size_t sample_ws_layout(uint64_t ntiles, int64_t shots, char *base, SampleWs *w) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = round_up(off + bytes, 256);
    return o;
  };
  size_t o1 = take(sizeof(double) * ntiles);
  size_t o2 = take(sizeof(double) * (ntiles + 1));
  size_t o3 = take(sizeof(uint32_t) * ntiles * 2);  // count and cursor, adjacent
  size_t o5 = take(sizeof(uint32_t) * (ntiles + 1));
  size_t o6 = take(sizeof(uint32_t) * (size_t)shots);
  size_t o7 = take(sizeof(uint32_t) * (size_t)shots);
  if (w) {
    w->tsum = reinterpret_cast<double *>(base + o1);
    w->prefix = reinterpret_cast<double *>(base + o2);
    w->count = reinterpret_cast<uint32_t *>(base + o3);
    w->cursor = w->count + ntiles;
    w->offset = reinterpret_cast<uint32_t *>(base + o5);
    w->shot_tile = reinterpret_cast<uint32_t *>(base + o6);
    w->bucket = reinterpret_cast<uint32_t *>(base + o7);
  }
  return off;
}

int sm_count();

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
  const int sms = sms0;
  const unsigned tgrid = (unsigned)(ntiles < (uint64_t)sms * 8 ? ntiles : (uint64_t)sms * 8);
  tile_sum_kernel<<<tgrid, kThreads, 0, st>>>(s4, ntiles, w.tsum);
  GQ_CHECK_LAUNCH();
  scan_tiles_kernel<<<1, 1024, 0, st>>>(w.tsum, ntiles, w.prefix);
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
  GQ_CUDA(cudaMemsetAsync(w.count, 0, sizeof(uint32_t) * ntiles * 2, st));
  const unsigned sgrid =
      (unsigned)((shots + kThreads - 1) / kThreads < (int64_t)sms * 16 ? (shots + kThreads - 1) / kThreads
                                                                      : (int64_t)sms * 16);
  shot_tile_kernel<<<sgrid, kThreads, 0, st>>>(w.prefix, ntiles, seed, shots, w.shot_tile, w.count);
  GQ_CHECK_LAUNCH();
  scan_counts_kernel<<<1, 1024, 0, st>>>(w.count, ntiles, w.offset);
  GQ_CHECK_LAUNCH();
  scatter_kernel<<<sgrid, kThreads, 0, st>>>(w.shot_tile, shots, w.offset, w.cursor, w.bucket);
  GQ_CHECK_LAUNCH();
  resolve_kernel<<<tgrid, kThreads, 0, st>>>(s4, ntiles, w.prefix, w.offset, w.bucket, seed, out_idx);
  GQ_CHECK_LAUNCH();
  return GQAOA_OK;
}
