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
// The array lives in every GPU that loads this library, for as long as the
// library stays loaded. Host code only holds a stand-in symbol for it, so its
// device address is looked up once per device with cudaGetSymbolAddress (on the
// first call made with that device current) and passed to the kernels.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "ctv.h"
#include "ctv_device.cuh"
#include "ctv_host.h"

namespace {

// statistics record (rounded up to 256 B) + two sets of (q, r), float4 per pixel
constexpr size_t kNoAllocScratchBytes = 256 + 4 * sizeof(float4) * (size_t)CTV_NOALLOC_MAX_PIXELS;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on the current device (looked up once).
ctv_status scratch_for_current_device(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CTV_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return CTV_ECUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return CTV_OK;
}

static_assert(sizeof(ctv::DevStats) <= 256, "statistics record must fit its 256-byte slot");

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
