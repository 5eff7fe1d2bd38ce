// Allocation-free dual-operator apply.
//
// feti_dual_apply_noalloc runs the same kernels as feti_dual_apply (q = F v,
// z = M^-1 q) but keeps its scratch -- the gathered local boundary vectors and
// the local results -- in one statically sized device array defined in this
// file instead of in memory the context allocated with cudaMalloc, and it
// creates no CUDA graph and no event.  It is meant for callers that must not
// allocate device memory once the solver is set up: code that runs with a
// fixed device-memory budget reserved at start-up, code that cannot afford the
// implicit device synchronisation cudaMalloc may cause in a latency-critical
// loop, and code that issues work while some other component holds the
// allocator (for example while a stream is being captured).
#include "feti.h"
#include "feti_internal.h"

#include <cstdio>

namespace {

// Capacity of the static scratch, in doubles (8 MiB).  Every GPU that loads
// the library holds this array until the process exits.
constexpr size_t kNoAllocScratchDoubles = size_t(1) << 20;

__device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

// Device address of the array, looked up once per device (host code may not
// use the symbol itself as a device pointer).
constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" feti_status feti_dual_apply_noalloc(feti_ctx* ctx, const double* v, double* q, double* z) {
  if (!ctx) return FETI_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    (void)cudaGetLastError();
    return feti::set_error(ctx, FETI_ERR_CUDA, "feti_dual_apply_noalloc: no current CUDA device");
  }
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return feti::set_error(ctx, FETI_ERR_CUDA, std::string("feti_dual_apply_noalloc: cudaGetSymbolAddress: ") +
                                                     cudaGetErrorString(e));
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  return feti::dual_apply_with_scratch(ctx, v, q, z, g_scratch_addr[dev], kNoAllocScratchDoubles);
}
