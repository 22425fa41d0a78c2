// The fused FGP pass kernel over an equally sized batch and its launcher for one
// TV type; each pass_tv<k>.cu instantiates it for one type so that the many
// configuration x constraint specialisations compile in parallel.
#pragma once

#include <cuda_runtime.h>
#include <string.h>

#include "ctv_configs.cuh"
#include "ctv_device.cuh"
#include "ctv_host.h"
#include "ctv_kernels.h"

namespace ctv {

#ifndef CTV_PDL
#define CTV_PDL 1
#endif

template <int KIND, int TV, int T, int A, int B, int C, int CONS, bool GAPEV>
__global__ void __launch_bounds__(CfgGeom<KIND, A, B, C>::NT, CfgGeom<KIND, A, B, C>::MINB)
    fgp_pass_kernel(PassParams p) {
  using G = CfgGeom<KIND, A, B, C>;
#if CTV_PDL
  // Programmatic dependent launch: the next pass may be scheduled onto SMs this
  // grid's last wave leaves idle (launch_dependents), and this grid's blocks wait
  // for the previous kernel's results before their first load (wait). Both are
  // no-ops for a launch without the programmatic attribute.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
  const int z = blockIdx.z;
  if (p.st != nullptr && *(volatile const int*)&p.st[z].stop) return;
  Img I;
  I.b = p.b + z * p.b_stride;
  I.ld = p.ld;
  I.q_in = p.q_in + z * p.d_stride;
  I.r_in = p.r_in + z * p.d_stride;
  I.q_out = p.q_out + z * p.d_stride;
  I.r_out = p.r_out + z * p.d_stride;
  I.m = p.m;
  I.n = p.n;
  const float lam = p.lam_dev != nullptr ? p.lam_dev[z] : p.lam;
  I.lam = lam > 0.f ? lam : 0.f;
  I.alpha = p.alpha;
  I.C = p.C;
  I.r_hist = nullptr;
  I.hist_plane = 0;
  const int bx = p.reverse ? gridDim.x - 1 - blockIdx.x : blockIdx.x;
  const int by = p.reverse ? gridDim.y - 1 - blockIdx.y : blockIdx.y;
  if constexpr (!GAPEV) {
    run_tile<KIND, TV, T, A, B, C, false, CONS>(I, by * (G::RH - 2 * T), bx * (G::RW - 2 * T),
                                                p.beta, p.nsteps, p.first != 0);
  } else {
    GapSums gs = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, false};
    run_tile<KIND, TV, T, A, B, C, false, CONS, true>(I, by * (G::RH - 2 * T),
                                                      bx * (G::RW - 2 * T), p.beta, p.nsteps,
                                                      p.first != 0, &gs);
    // the block's sums as FP32 pairs into its slot (fgp_gap_finish_kernel, launched
    // after this pass, evaluates them)
    __shared__ float2 red[3 * (G::NT / 32)];
    gap_block_store<G::NT>(gs, I.lam, p.gst + z, p.slots + z * p.slot_stride, blockIdx.y * gridDim.x + blockIdx.x,
                           red);
  }
}

template <int KIND, int TV, int T, int A, int B, int C, int CONS, bool GAPEV>
static cudaError_t launch_pass_t(const PassParams& p, dim3 grid, cudaStream_t s) {
  using G = CfgGeom<KIND, A, B, C>;
  static bool attr_done[kMaxDevices] = {};
  cudaError_t e = smem_attr_once(fgp_pass_kernel<KIND, TV, T, A, B, C, CONS, GAPEV>, G::SMEM, attr_done);
  if (e != cudaSuccess) return e;
#if CTV_PDL
  cudaLaunchConfig_t lc;
  memset(&lc, 0, sizeof(lc));
  lc.gridDim = grid;
  lc.blockDim = dim3(G::NT);
  lc.dynamicSmemBytes = G::SMEM;
  lc.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  return cudaLaunchKernelEx(&lc, fgp_pass_kernel<KIND, TV, T, A, B, C, CONS, GAPEV>, p);
#else
  fgp_pass_kernel<KIND, TV, T, A, B, C, CONS, GAPEV><<<grid, G::NT, G::SMEM, s>>>(p);
  return cudaGetLastError();
#endif
}

// Region kernels (kind 0) use the general constraint path; column-strip kernels
// (kind 1) are specialised per constraint kind.
template <int KIND, int TV, int T, int A, int B, int C, bool GAPEV>
static cudaError_t launch_pass_cons(int cons, const PassParams& p, dim3 grid, cudaStream_t s) {
  if constexpr (KIND == 0) {
    if constexpr (GAPEV) return cudaErrorInvalidValue;
    else return launch_pass_t<KIND, TV, T, A, B, C, CONS_GEN, false>(p, grid, s);
  } else {
    if constexpr (GAPEV && !GapEvalOk<KIND, C>::value) {
      return cudaErrorInvalidValue;
    } else {
      switch (cons) {
        case CONS_NONE: return launch_pass_t<KIND, TV, T, A, B, C, CONS_NONE, GAPEV>(p, grid, s);
        case CONS_AMP: return launch_pass_t<KIND, TV, T, A, B, C, CONS_AMP, GAPEV>(p, grid, s);
        case CONS_RECT: return launch_pass_t<KIND, TV, T, A, B, C, CONS_RECT, GAPEV>(p, grid, s);
        default: return launch_pass_t<KIND, TV, T, A, B, C, CONS_GEN, GAPEV>(p, grid, s);
      }
    }
  }
}

template <int TV>
cudaError_t launch_pass_tv(int cfg, int cons, const PassParams& p, dim3 grid, cudaStream_t s) {
  switch (cfg) {
#define CTV_CFG_CASE(id, kind, T, A, B, C) \
  case id: return launch_pass_cons<kind, TV, T, A, B, C, false>(cons, p, grid, s);
    CTV_PASS_CONFIGS(CTV_CFG_CASE)
#undef CTV_CFG_CASE
  }
  return cudaErrorInvalidValue;
}

template <int TV>
cudaError_t launch_pass_gap_tv(int cfg, int cons, const PassParams& p, dim3 grid, cudaStream_t s) {
  switch (cfg) {
#define CTV_CFG_CASE(id, kind, T, A, B, C) \
  case id: return launch_pass_cons<kind, TV, T, A, B, C, true>(cons, p, grid, s);
    CTV_PASS_CONFIGS(CTV_CFG_CASE)
#undef CTV_CFG_CASE
  }
  return cudaErrorInvalidValue;
}

}  // namespace ctv
