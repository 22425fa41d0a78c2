// Library-wide C ABI helpers: status strings, the ABI version and the
// asynchronous error word.
#include <cuda_runtime.h>

#include "ctv.h"
#include "ctv_host.h"

extern "C" {

int ctv_get_last_error(ctv_stream stream) {
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return CTV_ECUDA;
  // every unit's word is read (and cleared); the first recorded failure is reported
  const int words[3] = {ctv::take_async_status_denoise(), ctv::take_async_status_plan(),
                        ctv::take_async_status_pr()};
  int out = CTV_OK;
  for (int w : words) {
    if (w < 0) return CTV_ECUDA;
    if (out == CTV_OK && w != 0) out = w;
  }
  return out;
}

const char* ctv_status_string(int status) {
  switch (status) {
    case CTV_OK: return "ok";
    case CTV_EINVAL: return "invalid argument";
    case CTV_ENOMEM: return "out of device memory";
    case CTV_ECUDA: return "CUDA error";
    case CTV_ETIMEOUT: return "bounded device wait ran out (unused: no kernel of this library waits)";
    case CTV_ENONFINITE: return "non-finite input (NaN or infinity)";
    case CTV_EUNSUPPORTED: return "unsupported";
    case CTV_ETOOBIG: return "image exceeds the fixed scratch of ctv_denoise_noalloc (CTV_NOALLOC_MAX_PIXELS)";
  }
  return "unknown status";
}

int ctv_abi_version(void) { return 1; }

}  // extern "C"
