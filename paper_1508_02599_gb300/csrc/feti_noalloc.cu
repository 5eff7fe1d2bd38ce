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
//
// Set-up: feti_create calls noalloc_scratch_lookup with the context's device
// current.  The lookup (cudaGetSymbolAddress) makes the runtime load this
// file's device module -- and so reserve the array -- at that point, never
// inside a later feti_dual_apply_noalloc call; the context keeps the address
// and the device it belongs to.
#include "feti.h"
#include "feti_internal.h"

#include <string>

namespace {

// Capacity of the static scratch, in doubles (8 MiB).  Every GPU that loads
// the library holds this array until the process exits.
constexpr size_t kNoAllocScratchDoubles = size_t(1) << 20;

__device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

}  // namespace

namespace feti {

// Device address of the static scratch on the current device.  Host code may
// not use the symbol itself as a device pointer: in host code the name
// stands for a host-side shadow, not for device memory.
cudaError_t noalloc_scratch_lookup(double** out, size_t* capacity) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    *out = nullptr;
    *capacity = 0;
    return e != cudaSuccess ? e : cudaErrorInvalidSymbol;
  }
  *out = static_cast<double*>(p);
  *capacity = kNoAllocScratchDoubles;
  return cudaSuccess;
}

}  // namespace feti

extern "C" feti_status feti_dual_apply_noalloc(feti_ctx* ctx, const double* v, double* q, double* z) {
  if (!ctx) return FETI_ERR_INVALID_ARG;
  return feti::dual_apply_noalloc(ctx, v, q, z);
}
