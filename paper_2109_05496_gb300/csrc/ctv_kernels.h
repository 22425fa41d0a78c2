// Kernel parameter blocks and launchers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "ctv.h"
#include "ctv_host.h"
#include "ctv_device.cuh"
#include "gap_device.cuh"

namespace ctv {

// Check intervals a stop graph can hold (solves with more run as plain launches).
#define CTV_MAX_STOP_INTERVALS 64

// One launch of the fused FGP pass over an equally sized batch (blockIdx.z = image).
struct PassParams {
  const float2* b;
  long long b_stride;
  int ld;
  const float4* q_in;
  const float4* r_in;
  float4* q_out;
  float4* r_out;
  long long d_stride;
  int m, n;
  float lam;
  const float* lam_dev;
  float alpha;
  ConsDev C;
  const DevStats* st;
  float beta[8];
  int nsteps;
  int first;
  int reverse;   // blocks take the tiles in reverse order (bit-identical results)
  // a pass that ends a check interval with the duality-gap terms evaluated in it
  // (gap_eval != 0, strip configurations only): each block stores its sums in its
  // slot of the image's slot array and fgp_gap_finish_kernel evaluates them
  int gap_eval;
  DevStats* gst;
  float* slots;
  long long slot_stride;
};

// One launch of the finalize / gap evaluation over an equally sized batch.
struct GapParams {
  const float2* b;
  long long b_stride;
  int ld;
  const float4* qA;
  const float4* qB;
  long long d_stride;
  int default_set;   // 0: qA, 1: qB, 2: dual_in
  const float4* dual_in;
  int zero_q;        // q = 0 (no iteration has run)
  float2* x;         // nullable
  long long x_stride;
  float4* q_export;  // nullable, stride d_stride
  int m, n;
  float lam;
  const float* lam_dev;
  float alpha;
  ConsDev C;
  // x-only finalize of one image: optionally z = x + mom_beta (x - mom_xprev) too
  float2* mom_z;
  int mom_ld;
  const float2* mom_xprev;
  float mom_beta;
  DevStats* st;
  float* slots;           // block partial sums of the reduction (slot_stride floats per image)
  long long slot_stride;
  int iter;
  double gap_tol;
  int final_call;
  // inside a stop graph: the handles of the later check intervals, cleared when
  // the test passes (a conditional handle belongs to one conditional node)
  int n_cond;
  cudaGraphConditionalHandle cond[CTV_MAX_STOP_INTERVALS];
};

cudaError_t launch_pass(int tv, int cfg, const PassParams& p, dim3 grid, cudaStream_t s);
// Streaming multiprocessors of the current device (queried once per device).
int sm_count();
// Resident blocks per SM of `kernel` at `threads` threads on the current device
// (queried once per device into `cached`).
int occupancy_once(const void* kernel, int threads, int (&cached)[kMaxDevices]);
// Per-TV-type launchers, instantiated one translation unit per type (pass_tv*.cu).
template <int TV>
cudaError_t launch_pass_tv(int cfg, int cons, const PassParams& p, dim3 grid, cudaStream_t s);
// The same with the duality gap evaluated in the pass (pass_gap_tv*.cu); only for
// configurations with pass_gap_eval_ok(cfg).
template <int TV>
cudaError_t launch_pass_gap_tv(int cfg, int cons, const PassParams& p, dim3 grid, cudaStream_t s);
bool pass_gap_eval_ok(int cfg);
// Constraint specialisation (CONS_*) of a constraint descriptor.
inline int cons_mode(const ConsDev& c) {
  if (c.box) return CONS_GEN;
  if (c.sup == 0) return c.amp ? CONS_AMP : CONS_NONE;
  if (c.sup == 1) return CONS_RECT;
  return CONS_GEN;
}
// Evaluation of a reduction stored in per-block slots (gap_store_slot): one block
// per image adds the nblk slots and turns them into primal, dual and gap, applies
// the stopping test of a check or records the final statistics, and inside a stop
// graph clears the later intervals' handles when the test passes.
struct GapFinishParams {
  DevStats* st;
  const float* slots;
  long long slot_stride;
  unsigned nblk;
  float lam;
  const float* lam_dev;
  int set;   // the dual set holding q at this check (recorded at a stop)
  int iter;
  double gap_tol;
  int final_call;
  int n_cond;
  cudaGraphConditionalHandle cond[CTV_MAX_STOP_INTERVALS];
};
cudaError_t launch_gap_finish(const GapFinishParams& f, int batch, cudaStream_t s);
// The gap / finalize evaluation (two kernels: the evaluation and its finish).
cudaError_t launch_gap(int tv, const GapParams& p, int batch, cudaStream_t s);
// x = P_C(b - lam L^T q) only (no objective terms, no statistics record)
cudaError_t launch_finalize(const GapParams& p, int batch, cudaStream_t s);
// Grid of the fused pass for configuration cfg over an m x n image batch.
dim3 pass_grid(int cfg, int m, int n, int batch);

}  // namespace ctv
