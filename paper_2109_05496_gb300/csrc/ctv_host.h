// Internal host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <vector>

#include "ctv.h"

namespace ctv {

struct ConsDev;

// One denoising request, single image (lam) or equally sized batch (lam_dev).
struct DenoiseCall {
  const void* b;
  void* x;
  int batch, m, n, ld;
  long long batch_stride;
  float lam;
  const float* lam_dev;
  const ctv_constraint* C;
  int tv;
  const ctv_opts* opts;
  void* dual_state;
  void* workspace;
  size_t workspace_bytes;
  ctv_stats* stats;
  ctv_stream stream;
  int plain_launches;   // nonzero: never build a stop graph (callers that must not allocate)
  // Algorithm 1's momentum folded into the finalize (one image; phase retrieval):
  // when the solve ends with the x-only finalize, it also writes
  // z = x + mom_beta (x - mom_xprev) (x_prev with x's row stride) to mom_z (row
  // stride mom_ld) and sets *mom_written; otherwise the caller forms z itself.
  float2* mom_z;
  int mom_ld;
  const float2* mom_xprev;
  float mom_beta;
  int* mom_written;
};

// Facts that hold for one device - a kernel's shared-memory limit, the SM count,
// an occupancy, the tuned configurations - are kept per device ordinal, so that
// one process can drive several GPUs. Ordinals at or above kMaxDevices are not
// cached (every call then recomputes).
constexpr int kMaxDevices = 64;
inline int device_slot() {
  int d = -1;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return -1;
  return d;
}
// Raises a kernel's dynamic shared-memory limit to `bytes` once per device.
template <typename F>
inline cudaError_t smem_attr_once(F* kernel, size_t bytes, bool (&done)[kMaxDevices]) {
  const int d = device_slot();
  if (d >= 0 && done[d]) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && d >= 0) done[d] = true;
  return e;
}

ctv_status run_denoise(const DenoiseCall& c);
size_t denoise_workspace_bytes(int batch, int m, int n);

// Workspace of a solve: per image a statistics record (DevStats, at most 256 B)
// and a slot array of block partial sums of the duality-gap reduction (4
// doubles per block, as many blocks as a launch over the image can have: one per
// 16 x 16 pixels or more), then two dual buffer sets (q, r) of float4 per pixel.
constexpr size_t ws_align256(size_t v) { return (v + 255) & ~(size_t)255; }
constexpr size_t gap_slots_per_image(int m, int n) { return (size_t)((m + 15) / 16) * (size_t)((n + 15) / 16); }
constexpr size_t denoise_workspace_bytes_c(int batch, int m, int n) {
  return (batch <= 0 || m <= 0 || n <= 0)
             ? 0
             : ws_align256((size_t)batch * 256) + ws_align256((size_t)batch * gap_slots_per_image(m, n) * 32) +
                   4 * ws_align256((size_t)batch * (size_t)m * (size_t)n * 16);
}
bool convert_constraint(const ctv_constraint* C, int m, int n, ConsDev* out);
void nesterov_betas(int K, std::vector<double>* beta);
// cons: the constraint specialisation (CONS_*) of the solve's C
// check_every: the solve's gap-check interval (0: none), which can change the
// best iterations per pass
int default_config(int m, int n, int iters, int tv, int cons, int check_every = 0);
int tuned_config(int m, int n, int tv);   // -1 when the size class / TV type is not tuned
int size_class(int m, int n);
int num_configs();
bool config_info(int i, int* T, int* RW, int* RH, int* NT);

// Readers of the asynchronous error word of the units whose kernels test their
// inputs (async_status.cuh): return the first recorded ctv_status code on the
// current device (0: none) and clear it; -1 if the word cannot be read.
int take_async_status_denoise();
int take_async_status_plan();
int take_async_status_pr();

// Measurement hooks (prof.cu): count every launch; time fused passes when enabled.
void count_launch();
void count_launches(int n);
// whether ctv_profile_enable(1 or 2) is in force (pass launches are then bracketed by events)
bool prof_active();
// 0 off, 1 every pass launch timed, 2 every run of consecutive pass launches timed
int prof_mode();
int prof_begin(cudaStream_t s);
void prof_end(int slot, cudaStream_t s, double units, int launches);

}  // namespace ctv
