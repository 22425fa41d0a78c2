// The library's asynchronous error word.
//
// Some failures are only visible on the device: a NaN or an infinity in an input
// image reaches the kernels after the call has returned. Kernels that read the
// inputs test them as they load them (no extra bytes) and record the first such
// failure in a status word on the device, which ctv_get_last_error reads and
// clears after synchronising the caller's stream.
//
// Every translation unit that includes this header gets its own copy of the word
// (internal linkage: the library is compiled without relocatable device code, so
// a kernel can only name a device variable of its own unit). Each such unit
// exports a host function that reads and clears its copy on the current device,
// and ctv_get_last_error asks all of them. Host code never passes the word's
// address to a kernel, so launch paths do no symbol lookups.
#pragma once

#include <cuda_runtime.h>

namespace ctv {
namespace {

__device__ int tu_async_status;

// First failure wins: later ones leave the recorded code unchanged.
__device__ __forceinline__ void raise_async(int code) { atomicCAS(&tu_async_status, 0, code); }

// Returns this unit's recorded code on the current device (0: none) and clears
// it; -1 if the word cannot be read. Call only while no kernel of the unit runs.
inline int take_unit_async_status() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, tu_async_status, sizeof(int)) != cudaSuccess) return -1;
  if (v != 0) {
    const int zero = 0;
    if (cudaMemcpyToSymbol(tu_async_status, &zero, sizeof(int)) != cudaSuccess) return -1;
  }
  return v;
}

}  // namespace
}  // namespace ctv
