// Fair-sampling metrics of Section IV (Table I) over a measurement stream.
//
// Section IV measures how evenly G-QAOA samples the solutions by (i) the
// shots needed to observe every solution at least once and (ii) the draws
// from the solution distribution needed before a chi-square test rejects
// uniform sampling. Both are computed here for many independent runs of one
// shot stream (from gqaoa_sample): run r takes the shots r, r + R, r + 2R,
// ... in order (the shots are independent, and this interleaving makes a
// warp's reads consecutive words). "Solution" generalises to any target cost
// class (the lowest non-empty class for Max-SAT).
//
// One kernel labels the target assignments 0..M-1 (in any order: both
// metrics are invariant under relabelling), one thread per run then walks its
// shots with per-solution counts in the workspace ([M][R], so a warp's
// counters of one label are consecutive). The chi-square decision uses the
// exact integer numerator of d X^2 = M sum_j O_j^2 - d^2. For small states,
// few targets and short runs the labels, counts and per-draw-count thresholds
// sit in shared memory instead (fairness_smem_kernel, the same decisions).
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace gq {
namespace {

__device__ __forceinline__ int64_t round_up_dev(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

__global__ void label_targets_kernel(const uint8_t *__restrict__ cost, uint64_t N, unsigned target,
                                     int32_t *__restrict__ label, unsigned *__restrict__ count) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t z = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; z < N; z += stride)
    label[z] = cost[z] == target ? (int32_t)atomicAdd(count, 1u) : -1;
}

__global__ void __launch_bounds__(256)
fairness_kernel(const uint64_t *__restrict__ shots, int64_t runs, int64_t per_run, uint64_t N,
                const int32_t *__restrict__ label, const unsigned *__restrict__ count, int M,
                double crit, int64_t min_draws, int32_t *__restrict__ counts,
                int64_t *__restrict__ to_all, int64_t *__restrict__ to_rej) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= runs) return;
  if (*count != (unsigned)M) {  // `targets` is not the number of target assignments
    to_all[r] = -1;
    to_rej[r] = -1;
    return;
  }
  for (int j = 0; j < M; ++j) counts[(int64_t)j * runs + r] = 0;  // the workspace keeps old runs
  int64_t seen = 0, d = 0, s2 = 0, ta = 0, tr = 0;
  for (int64_t t = 0; t < per_run; ++t) {
    const uint64_t z = shots[t * runs + r];
    const int32_t j = z < N ? label[z] : -1;
    if (j < 0) continue;
    int32_t *cj = counts + (int64_t)j * runs + r;
    const int64_t c = *cj;
    *cj = (int32_t)(c + 1);
    seen += c == 0;
    s2 += 2 * c + 1;  // sum of squared counts, updated for O_j -> O_j + 1
    ++d;
    if (ta == 0 && seen == M) ta = t + 1;
    if (tr == 0 && d >= min_draws) {
      const int64_t num = (int64_t)M * s2 - d * d;  // d X^2, exact
      if ((double)num > crit * (double)d) tr = d;
    }
    if (ta != 0 && tr != 0) break;
  }
  to_all[r] = ta;
  to_rej[r] = tr;
}

// The same metrics with the labels, the counts and the chi-square thresholds
// in shared memory (small states, few targets, short runs): labels as int16,
// counts as uint16 [M][kSmemRuns], and thr[d] = floor(fl(crit * d)). With
// M <= kSmemMaxTargets and d <= kSmemMaxPerRun the numerator
// num = M sum O^2 - d^2 <= M d^2 stays below 2^33, so double(num) is exact and
// the test double(num) > crit * double(d) is the integer test num > thr[d].
// Each run's next shot is loaded one step ahead. Same loop, same decisions as
// fairness_kernel.
constexpr int kSmemRuns = 128;
constexpr int64_t kSmemMaxPerRun = 4095;
constexpr int kSmemMaxTargets = 384;
constexpr size_t kSmemMaxBytes = 96 * 1024;

size_t fairness_smem_bytes(uint64_t N, int M, int64_t per_run) {
  return round_up(sizeof(int64_t) * (size_t)(per_run + 1), 16) + round_up(sizeof(int16_t) * N, 16) +
         sizeof(uint16_t) * (size_t)M * kSmemRuns;
}

__device__ __forceinline__ int64_t chi2_threshold(double crit, int64_t d) {
  const double P = crit * (double)d;
  if (!(P < 0x1p62)) return INT64_MAX;  // also NaN and +inf: never exceeded
  if (P < -0x1p62) return INT64_MIN;
  return (int64_t)floor(P);
}

__global__ void __launch_bounds__(kSmemRuns)
fairness_smem_kernel(const uint64_t *__restrict__ shots, int64_t runs, int64_t per_run, uint64_t N,
                     const int32_t *__restrict__ label, const unsigned *__restrict__ count, int M,
                     double crit, int64_t min_draws, int64_t *__restrict__ to_all,
                     int64_t *__restrict__ to_rej) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  int64_t *thr = reinterpret_cast<int64_t *>(s_dyn);  // [per_run + 1]
  int16_t *lab = reinterpret_cast<int16_t *>(s_dyn + round_up_dev(8 * (per_run + 1), 16));  // [N]
  uint16_t *cnt = reinterpret_cast<uint16_t *>(
      reinterpret_cast<unsigned char *>(lab) + round_up_dev(2 * (int64_t)N, 16));  // [M][kSmemRuns]
  for (int64_t d = threadIdx.x; d <= per_run; d += blockDim.x) thr[d] = chi2_threshold(crit, d);
  for (uint64_t z = threadIdx.x; z < N; z += blockDim.x) lab[z] = (int16_t)label[z];
  for (int j = 0; j < M; ++j) cnt[j * kSmemRuns + threadIdx.x] = 0;
  __syncthreads();
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= runs) return;
  if (*count != (unsigned)M) {
    to_all[r] = -1;
    to_rej[r] = -1;
    return;
  }
  int64_t seen = 0, d = 0, s2 = 0, ta = 0, tr = 0;
  uint64_t z = per_run > 0 ? shots[r] : 0;
  for (int64_t t = 0; t < per_run; ++t) {
    const uint64_t zn = t + 1 < per_run ? shots[(t + 1) * runs + r] : 0;
    const int32_t j = z < N ? lab[z] : -1;
    z = zn;
    if (j < 0) continue;
    uint16_t *cj = cnt + j * kSmemRuns + threadIdx.x;
    const int64_t c = *cj;
    *cj = (uint16_t)(c + 1);
    seen += c == 0;
    s2 += 2 * c + 1;
    ++d;
    if (ta == 0 && seen == M) ta = t + 1;
    if (tr == 0 && d >= min_draws) {
      const int64_t num = (int64_t)M * s2 - d * d;
      if (num > thr[d]) tr = d;
    }
    if (ta != 0 && tr != 0) break;
  }
  to_all[r] = ta;
  to_rej[r] = tr;
}

size_t fairness_ws_layout(int n, int64_t runs, int targets, char *base, int32_t **label,
                          unsigned **count, int32_t **counts) {
  const size_t o_count = round_up(sizeof(int32_t) << n, 256);
  const size_t o_counts = o_count + 256;
  if (base) {
    *label = reinterpret_cast<int32_t *>(base);
    *count = reinterpret_cast<unsigned *>(base + o_count);
    *counts = reinterpret_cast<int32_t *>(base + o_counts);
  }
  return o_counts + round_up(sizeof(int32_t) * (size_t)runs * (size_t)targets, 256);
}

}  // namespace
}  // namespace gq

using namespace gq;

extern "C" int gqaoa_fairness_workspace_size(int n, int64_t runs, int targets, size_t *bytes) {
  if (!bytes) return GQAOA_EINVAL;
  if (n < 1 || n > 30 || runs < 1 || runs > (1ll << 32) || targets < 1 ||
      (int64_t)targets > (1ll << n))
    return GQAOA_ERANGE;
  *bytes = fairness_ws_layout(n, runs, targets, nullptr, nullptr, nullptr, nullptr);
  return GQAOA_OK;
}

extern "C" int gqaoa_fairness(const uint64_t *shots, int64_t runs, int64_t shots_per_run,
                              const uint8_t *cost, int n, int target, int targets,
                              double chi2_crit, int64_t min_draws, int64_t *to_all,
                              int64_t *to_reject, void *ws, size_t ws_bytes, void *stream) {
  gq::NvtxRange nvtx_range("gqaoa_fairness");
  if (n < 1 || n > 30 || runs < 1 || runs > (1ll << 32) || shots_per_run < 0 ||
      target < 0 || target > 255 || targets < 1 || (int64_t)targets > (1ll << n) ||
      min_draws < 1)
    return GQAOA_ERANGE;
  if (shots_per_run > 0 && runs > (INT64_MAX / shots_per_run)) return GQAOA_ERANGE;
  // M sum O^2 <= M d^2 must stay inside int64
  if ((double)targets * (double)shots_per_run * (double)shots_per_run > 4e18) return GQAOA_ERANGE;
  if (!cost || !to_all || !to_reject || !ws || (shots_per_run > 0 && !shots))
    return GQAOA_EINVAL;
  if (!aligned8(to_all) || !aligned8(to_reject) || !aligned16(ws) || (shots && !aligned8(shots)))
    return GQAOA_EINVAL;
  if (ws_bytes < fairness_ws_layout(n, runs, targets, nullptr, nullptr, nullptr, nullptr))
    return GQAOA_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int32_t *label = nullptr, *counts = nullptr;
  unsigned *count = nullptr;
  fairness_ws_layout(n, runs, targets, static_cast<char *>(ws), &label, &count, &counts);
  const uint64_t N = 1ull << n;
  GQ_CUDA(cudaMemsetAsync(count, 0, sizeof(unsigned), st));
  uint64_t blocks = (N + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  label_targets_kernel<<<(unsigned)blocks, 256, 0, st>>>(cost, N, (unsigned)target, label, count);
  GQ_CHECK_LAUNCH();
  const size_t smem = fairness_smem_bytes(N, targets, shots_per_run);
  if (n <= 15 && shots_per_run <= kSmemMaxPerRun && targets <= kSmemMaxTargets &&
      smem <= kSmemMaxBytes) {
    if (cudaFuncSetAttribute(fairness_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return GQAOA_ECUDA;
    const uint64_t rb = ((uint64_t)runs + kSmemRuns - 1) / kSmemRuns;
    fairness_smem_kernel<<<(unsigned)rb, kSmemRuns, smem, st>>>(
        shots, runs, shots_per_run, N, label, count, targets, chi2_crit, min_draws, to_all,
        to_reject);
    GQ_CHECK_LAUNCH();
    return GQAOA_OK;
  }
  const uint64_t rb = ((uint64_t)runs + 255) / 256;
  fairness_kernel<<<(unsigned)rb, 256, 0, st>>>(shots, runs, shots_per_run, N, label, count,
                                                targets, chi2_crit, min_draws, counts, to_all,
                                                to_reject);
  GQ_CHECK_LAUNCH();
  return GQAOA_OK;
}
