// The sampling CDF's arithmetic, shared by the sampler (sample.cu) and the
// fused readout-and-tile pass of gqaoa_evolve_sample (stream.cu), so both
// build the same CDF from the same complex64 values.
//
// A tile is 4096 amplitudes, a chunk 16 consecutive amplitudes (256 chunks
// per tile); a CTA of 256 threads holds a tile as 8 float4 per thread, load j
// of lane l of warp w being float4 tile * 2048 + w * 256 + 32 j + l (the
// layout of the streaming passes). Weights |re + i im|^2 are double-float
// pairs (FP32 hi + lo), chunk sums and in-tile prefixes double-float, the
// prefixes rounded to FP64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace gq {

constexpr int kSampTile = 4096;
constexpr int kChunk = 16;
constexpr int kChunksPerTile = kSampTile / kChunk;  // 256 = one per thread
constexpr int kPad = kChunk + 1;  // floats per row of the resident running sums

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

// Renormalise (h, l) so that h is the FP32 rounding of h + l (Fast2Sum,
// |h| >= |l|).
__device__ __forceinline__ void df_norm(float &h, float &l) {
  const float s = __fadd_rn(h, l);
  l = __fsub_rn(l, __fsub_rn(s, h));
  h = s;
}

// |re + i im|^2 as a normalised double-float (h, l): re^2 = p1 + e1 and
// im^2 = p2 + e2 exactly (e = fma(x, x, -p)), p1 + p2 = s + e exactly
// (TwoSum), and the three small words are added in FP32, which leaves a
// relative error below 2^-46.
__device__ __forceinline__ void weight_df(float re, float im, float &h, float &l) {
  const float p1 = __fmul_rn(re, re), e1 = fmaf(re, re, -p1);
  const float p2 = __fmul_rn(im, im), e2 = fmaf(im, im, -p2);
  float s, e;
  two_sum(p1, p2, s, e);
  h = s;
  l = __fadd_rn(e, __fadd_rn(e1, e2));
  df_norm(h, l);
}

// The first of a chunk's 16 amplitudes (row: 8 float4 in global memory, each
// plus the pending mixer term `add`, added in FP32 as a materialising pass
// would) whose running weight sum exceeds rl: the sums are formed in
// double-float in index order and compared as FP64. A target that rounding
// puts past the chunk's sum goes to its last amplitude of nonzero weight.
__device__ __forceinline__ int chunk_pick(const float4 *row, double rl, float2 add) {
  float h = 0.f, l = 0.f;
  int pick = -1, last_nz = 0;
#pragma unroll
  for (int i = 0; i < kChunk / 2; ++i) {
    const float4 v = row[i];
    float wh, wl;
    weight_df(__fadd_rn(v.x, add.x), __fadd_rn(v.y, add.y), wh, wl);
    df_add(h, l, wh, wl);
    if (wh > 0.f) last_nz = 2 * i;
    if (pick < 0 && gt_nonneg((double)h + (double)l, rl)) pick = 2 * i;
    weight_df(__fadd_rn(v.z, add.x), __fadd_rn(v.w, add.y), wh, wl);
    df_add(h, l, wh, wl);
    if (wh > 0.f) last_nz = 2 * i + 1;
    if (pick < 0 && gt_nonneg((double)h + (double)l, rl)) pick = 2 * i + 1;
  }
  return pick >= 0 ? pick : last_nz;
}

// One tile held in registers (v: this thread's 8 float4 in the layout above),
// called by all 256 threads: every chunk's sum in double-float and the
// inclusive in-tile scan of the chunk sums in double-float, rounded to FP64
// into s_incl[i] (chunk i = tile amplitudes 16 i .. 16 i + 15; lane l of warp
// w owns chunk 32 w + l). (ch, cl) receives the thread's own chunk sum,
// normalised. With cum != nullptr, cum[i * kPad + k] also receives the FP32
// running sums of the weights' leading words over chunk i (the resident
// sampler's first filter).
// Load j of lane l holds amplitudes 64 j + 2 l and 64 j + 2 l + 1 of its
// warp's 512, i.e. slot l mod 8 of the warp's chunk 4 j + l / 8, so the 8
// lanes l / 8 = g hold one chunk. Its sum is a butterfly over those 8 lanes
// (every lane ends with the same sum: the double-float addition is
// commutative), and the owning lane 4 j + g takes it from lane 8 g.
__device__ __forceinline__ void tile_chunk_scan_regs(const float4 (&v)[8], double *s_incl,
                                                     float2 *s_wtot, float &ch, float &cl,
                                                     float *cum) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 3, slot = lane & 7;
  float mh = 0.f, ml = 0.f;  // the sum of this lane's own chunk
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float w0h, w0l, w1h, w1l;
    weight_df(v[j].x, v[j].y, w0h, w0l);
    weight_df(v[j].z, v[j].w, w1h, w1l);
    if (cum) {
      // FP32 running sums within the chunk: exclusive scan of the lanes'
      // pair sums over the 8-lane group, then the lane's two amplitudes
      const float x = w0h + w1h;
      float inc = x;
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        const float y = __shfl_up_sync(0xffffffffu, inc, o, 8);
        if (slot >= o) inc += y;
      }
      float ex = __shfl_up_sync(0xffffffffu, inc, 1, 8);
      if (slot == 0) ex = 0.f;
      float *row = cum + (warp * 32 + 4 * j + g) * kPad + 2 * slot;
      row[0] = ex + w0h;
      row[1] = (ex + w0h) + w1h;
    }
    float ph = w0h, pl = w0l;
    df_add(ph, pl, w1h, w1l);
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      const float yh = __shfl_xor_sync(0xffffffffu, ph, o);
      const float yl = __shfl_xor_sync(0xffffffffu, pl, o);
      df_add(ph, pl, yh, yl);
    }
    const float th = __shfl_sync(0xffffffffu, ph, 8 * (lane & 3));
    const float tl = __shfl_sync(0xffffffffu, pl, 8 * (lane & 3));
    if ((lane >> 2) == j) {
      mh = th;
      ml = tl;
    }
  }
  df_norm(mh, ml);
  ch = mh;
  cl = ml;
  // inclusive scan over the warp's 32 chunks
  float xh = mh, xl = ml;
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

// The tile's total from the warp totals tile_chunk_scan_regs left in s_wtot.
__device__ __forceinline__ double tile_total(const float2 *s_wtot) {
  float th = 0.f, tl = 0.f;
  for (int w = 0; w < kWarps; ++w) df_add(th, tl, s_wtot[w].x, s_wtot[w].y);
  return (double)th + (double)tl;
}

}  // namespace gq
