// Library-wide C ABI helpers: status strings and the ABI version.
#include "ctv.h"

extern "C" {

const char* ctv_status_string(int status) {
  switch (status) {
    case CTV_OK: return "ok";
    case CTV_EINVAL: return "invalid argument";
    case CTV_ENOMEM: return "out of device memory";
    case CTV_ECUDA: return "CUDA error";
    case CTV_ETIMEOUT: return "bounded device wait ran out";
    case CTV_ENONFINITE: return "non-finite input";
    case CTV_EUNSUPPORTED: return "unsupported";
    case CTV_ETOOBIG: return "image exceeds the fixed scratch of ctv_denoise_noalloc (CTV_NOALLOC_MAX_PIXELS)";
  }
  return "unknown status";
}

int ctv_abi_version(void) { return 1; }

}  // extern "C"
