// gqaoa_evolve_noalloc: gqaoa_evolve for callers that cannot allocate.
//
// Some callers of this library have no way to allocate device memory or to
// hand it a workspace: a plugin reached through a fixed interface that passes
// only inputs and outputs, code running inside a framework that owns all
// device memory under a hard budget, or code that issues work while a stream
// is being captured in the global capture mode, where cudaMalloc is refused.
// This entry point serves them: its scratch is a file-scope __device__ array
// of fixed size, so the call allocates nothing; the caller still passes the
// cost table, the angles, the state and the outputs.
//
// The array lives in every GPU that loads this library until the process
// exits. In host code its name is only a host-side stand-in, so the device
// address is looked up once per device with cudaGetSymbolAddress (with that
// device current) on the first call made on that device; make that first
// call before any stream capture. Every call on a device shares the one
// array: calls whose GPU work overlaps (different streams, or host threads
// racing) corrupt each other's scratch and must be serialised by the caller.
// No word of the scratch has to start at zero: within a call every word is
// written before it is read, so the contents left by the previous call do
// not matter.
#include <cuda_runtime.h>

#include <mutex>

#include "gqaoa.h"

namespace {

constexpr size_t kScratchBytes = (size_t)GQAOA_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices];

// Device address of the scratch array on the current device, looked up once.
int scratch_address(void **addr) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GQAOA_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return GQAOA_ERANGE;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GQAOA_ECUDA;
    g_scratch_addr[dev] = p;
  }
  *addr = g_scratch_addr[dev];
  return GQAOA_OK;
}

}  // namespace

extern "C" int gqaoa_evolve_noalloc(const uint8_t *cost, int n, int m, const double *gammas,
                                    const double *betas, int p, void *state, double *out,
                                    double *trace, unsigned flags, void *stream) {
  if (p < 1 || p > GQAOA_NOALLOC_MAX_P) return GQAOA_ERANGE;
  size_t need = 0;
  int rc = gqaoa_evolve_workspace_size(n, p, &need);
  if (rc != GQAOA_OK) return rc;
  if (need > kScratchBytes) return GQAOA_ENOMEM;
  void *scratch = nullptr;
  rc = scratch_address(&scratch);
  if (rc != GQAOA_OK) return rc;
  return gqaoa_evolve(cost, n, m, gammas, betas, p, state, out, trace, scratch, kScratchBytes,
                      flags, stream);
}
