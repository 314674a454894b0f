// deconv_solve_noalloc: a whole solve whose scratch lives in a file-scope
// device array instead of caller-provided workspace.
//
// For callers that cannot allocate device memory themselves: code running
// inside a host framework that owns the CUDA allocator and forbids
// cudaMalloc, real-time paths where an allocation could block, and plugins
// loaded into a process whose device memory was reserved up front.  The
// array below is reserved once, when the library's code is loaded on a
// device, and stays reserved on every GPU that loads the library until the
// process exits.
//
// The entry point is composed from the existing public calls
// (deconv_workspace_size, deconv_plan_create, deconv_solve, deconv_sync,
// deconv_plan_destroy) with the plan workspace placed in the array.  It never
// calls cudaMalloc, cudaFree, cudaMallocAsync or any allocating library
// routine, and it launches the iterations directly (in chunks short enough
// that deconv_solve never instantiates a CUDA graph).
#include "deconv.h"

namespace {

constexpr size_t kScratchBytes = 32u << 20;  // 32 MiB
constexpr int kChunk = 20;  // deconv_solve replays a graph only for runs longer than this

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch in the current device's context.  In host
// code the symbol g_scratch names a host-side stand-in, never the device
// memory, so the address comes from cudaGetSymbolAddress with the device
// current.  It is looked up on every call (the lookup is cheap): a cached
// address would go stale if the context were torn down and recreated
// (cudaDeviceReset), and a later call would launch on unmapped memory.
deconv_status scratch_address(void **out) {
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return DECONV_ECUDA;
  *out = p;
  return DECONV_OK;
}

}  // namespace

extern "C" deconv_status deconv_solve_noalloc(const deconv_dims *dims, const void *h, const uint8_t *mask,
                                              const void *y, void *x, double lambda, double mu, int32_t iters,
                                              void *stream) {
  if (!dims || !h || !mask || !y || !x || iters < 0) return DECONV_EINVAL;
  size_t need = 0;
  deconv_status st = deconv_workspace_size(dims, &need);
  if (st != DECONV_OK) return st;
  if (need > kScratchBytes) return DECONV_ENOMEM;  // problem too large for the static scratch
  void *ws = nullptr;
  st = scratch_address(&ws);
  if (st != DECONV_OK) return st;
  deconv_plan plan = nullptr;
  // Plan creation clears everything that must start at zero (the dual
  // variables and the device error word) and rewrites every table.
  st = deconv_plan_create(&plan, dims, h, mask, lambda, mu, ws, kScratchBytes, stream);
  if (st != DECONV_OK) return st;
  int done = 0;
  do {
    const int n = iters - done < kChunk ? iters - done : kChunk;
    st = deconv_solve(plan, done == 0 ? y : nullptr, x, n, done == 0 ? 0 : 1, nullptr);
    done += n;
  } while (st == DECONV_OK && done < iters);
  const deconv_status sync = deconv_sync(plan);
  deconv_plan_destroy(plan);
  return st != DECONV_OK ? st : sync;
}
