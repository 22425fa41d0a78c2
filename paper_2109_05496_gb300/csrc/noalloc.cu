// ctv_denoise_noalloc: ctv_denoise for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all or cannot afford it: applications
// that hand all device memory to their own pool allocator and forbid raw
// allocations, plugin hosts whose callbacks must not allocate, and
// latency-critical loops where an allocation (which may synchronise the device)
// is not acceptable. For them this entry point takes only the input and output
// images and keeps its scratch (the per-image statistics record and the two
// ping-pong dual buffer sets of the FGP passes) in the file-scope device array
// below, of a fixed size chosen for images of up to CTV_NOALLOC_MAX_PIXELS pixels.
//
// The array is placed on a device when the library's module is loaded there
// and stays until that device's context is destroyed. Host code only holds a
// stand-in symbol for it, so every call looks up the array's device address with
// cudaGetSymbolAddress, with the caller's device current, and passes it to the
// kernels. The lookup allocates nothing and, once the module is loaded, is cheap;
// doing it on every call (rather than caching it) keeps the address right after a
// cudaDeviceReset or under another context, where the module is loaded again and
// the array can move. The first call on a device loads the module (and places
// the array), so it must come before any stream capture.
#include <cuda_runtime.h>
#include <string.h>

#include "ctv.h"
#include "ctv_device.cuh"
#include "ctv_host.h"

namespace {

// the workspace of the largest accepted image: the statistics record, the slots
// of the gap reduction and two sets of (q, r), float4 per pixel (every m x n with
// m n <= CTV_NOALLOC_MAX_PIXELS needs at most this much)
constexpr size_t kNoAllocScratchBytes = ctv::denoise_workspace_bytes_c(1, 512, 512) + 64 * 1024;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch in the current context.
ctv_status scratch_for_current_device(void** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return CTV_ECUDA;
  *out = p;
  return CTV_OK;
}


}  // namespace

extern "C" {

int ctv_denoise_noalloc(const void* b, void* x, int m, int n, int ld, float lambda, const ctv_constraint* C,
                        int tv_type, const ctv_opts* opts, ctv_stats* stats, ctv_stream stream) {
  if (m <= 0 || n <= 0) return CTV_EINVAL;
  if ((long long)m * (long long)n > (long long)CTV_NOALLOC_MAX_PIXELS) return CTV_ETOOBIG;
  if (opts != nullptr && opts->warm_start) return CTV_EINVAL;   // no dual state is kept between calls
  void* scratch = nullptr;
  const ctv_status st = scratch_for_current_device(&scratch);
  if (st != CTV_OK) return st;
  const size_t need = ctv::denoise_workspace_bytes(1, m, n);
  if (need > kNoAllocScratchBytes) return CTV_ETOOBIG;
  ctv::DenoiseCall c;
  memset(&c, 0, sizeof(c));
  c.b = b;
  c.x = x;
  c.batch = 1;
  c.m = m;
  c.n = n;
  c.ld = ld;
  c.lam = lambda;
  c.C = C;
  c.tv = tv_type;
  c.opts = opts;
  c.dual_state = nullptr;
  c.workspace = scratch;
  c.workspace_bytes = kNoAllocScratchBytes;
  c.stats = stats;
  c.stream = stream;
  c.plain_launches = 1;   // a stop graph would allocate driver resources when instantiated
  return ctv::run_denoise(c);
}

}  // extern "C"
