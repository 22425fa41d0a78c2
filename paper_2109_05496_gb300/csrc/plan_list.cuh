// The batched plan's pass over a work list of tiles of many images (plan.cu),
// compiled per TV type in plan_list_tv{0..3}.cu so the build runs in parallel.
#pragma once

#include <cuda_runtime.h>

#include "ctv_configs.cuh"
#include "ctv_device.cuh"
#include "ctv_kernels.h"

namespace ctv {

struct PlanImg {
  const float2* b;
  float2* x;
  int ld;
  int m, n;
  float lam, alpha;
  int tv;
  ConsDev C;
  float4* q[2];
  float4* r[2];
  DevStats* st;
  int tiles_x;     // pass tiles per tile row
  int gtiles_x;    // gap tiles per tile row
  unsigned gnblk;  // gap blocks of this image
};

struct WorkItem {
  int img;
  int tile;
};

struct ListPassParams {
  const PlanImg* imgs;
  const WorkItem* items;
  int in_set;
  int out_set;
  int first;
  int nsteps;
  int can_stop;   // the plan has gap checks: a block first tests its image's stop flag
  float beta[8];
};

template <int KIND, int TV, int CONS, int T, int A, int B, int C>
__global__ void __launch_bounds__(CfgGeom<KIND, A, B, C>::NT, CfgGeom<KIND, A, B, C>::MINB)
    fgp_pass_list_kernel(ListPassParams p) {
  using G = CfgGeom<KIND, A, B, C>;
  const WorkItem w = p.items[blockIdx.x];
  // fields read from global memory one by one (a register copy of the
  // descriptor indexed by the runtime set number would live in local memory)
  const PlanImg& d = p.imgs[w.img];
  if (p.can_stop && *(volatile const int*)&d.st->stop) return;
  Img I;
  I.b = d.b;
  I.ld = d.ld;
  I.q_in = d.q[p.in_set];
  I.r_in = d.r[p.in_set];
  I.q_out = d.q[p.out_set];
  I.r_out = d.r[p.out_set];
  I.m = d.m;
  I.n = d.n;
  I.lam = d.lam;
  I.alpha = d.alpha;
  I.C = d.C;
  I.r_hist = nullptr;
  I.hist_plane = 0;
  const int j0 = (w.tile / d.tiles_x) * (G::RH - 2 * T), k0 = (w.tile % d.tiles_x) * (G::RW - 2 * T);
  // The extrapolation weights go through shared memory: indexing the parameter
  // array by the runtime step number would copy the whole parameter block into
  // local memory. (Some tile bodies have no barrier of their own, so one orders
  // these stores before the first use.)
  __shared__ float beta_s[8];
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < 8; ++i) beta_s[i] = p.beta[i];
  }
  __syncthreads();
  run_tile<KIND, TV, T, A, B, C, false, CONS>(I, j0, k0, beta_s, p.nsteps, p.first != 0);
}

// configurations a plan can use (a subset of the pass table, to bound build time)
#define CTV_PLAN_CONFIGS(X)   \
  X(2, 0, 4, 64, 32, 256)     \
  X(5, 1, 6, 2, 8, 8)         \
  X(6, 1, 8, 2, 8, 8)         \
  X(7, 1, 3, 2, 8, 4)         \
  X(11, 1, 4, 2, 8, 4)        \
  X(14, 1, 6, 2, 16, 4)       \
  X(18, 1, 8, 2, 16, 4)

template <int KIND, int TV, int CONS, int T, int A, int B, int C>
static cudaError_t launch_list_t(const ListPassParams& p, int nblocks, cudaStream_t s, bool set_attr) {
  using G = CfgGeom<KIND, A, B, C>;
  if (set_attr) {
    return cudaFuncSetAttribute(fgp_pass_list_kernel<KIND, TV, CONS, T, A, B, C>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
  }
  fgp_pass_list_kernel<KIND, TV, CONS, T, A, B, C><<<nblocks, G::NT, G::SMEM, s>>>(p);
  return cudaGetLastError();
}

template <int KIND, int TV, int T, int A, int B, int C>
static cudaError_t launch_list_cons(int cons, const ListPassParams& p, int nblocks, cudaStream_t s, bool set_attr) {
  if constexpr (KIND == 0) {
    return launch_list_t<KIND, TV, CONS_GEN, T, A, B, C>(p, nblocks, s, set_attr);
  } else {
    switch (cons) {
      case CONS_NONE: return launch_list_t<KIND, TV, CONS_NONE, T, A, B, C>(p, nblocks, s, set_attr);
      case CONS_AMP: return launch_list_t<KIND, TV, CONS_AMP, T, A, B, C>(p, nblocks, s, set_attr);
      case CONS_RECT: return launch_list_t<KIND, TV, CONS_RECT, T, A, B, C>(p, nblocks, s, set_attr);
      default: return launch_list_t<KIND, TV, CONS_GEN, T, A, B, C>(p, nblocks, s, set_attr);
    }
  }
}

// One launch over work items of images of type TV in configuration cfg (set_attr:
// raise the kernel's dynamic shared-memory limit instead of launching).
template <int TV>
cudaError_t launch_plan_list_tv(int cfg, int cons, const ListPassParams& p, int nblocks, cudaStream_t s,
                                bool set_attr) {
  switch (cfg) {
#define CTV_CFG_CASE(id, kind, T, A, B, C) \
  case id: return launch_list_cons<kind, TV, T, A, B, C>(cons, p, nblocks, s, set_attr);
    CTV_PLAN_CONFIGS(CTV_CFG_CASE)
#undef CTV_CFG_CASE
  }
  return cudaErrorInvalidValue;
}

extern template cudaError_t launch_plan_list_tv<0>(int, int, const ListPassParams&, int, cudaStream_t, bool);
extern template cudaError_t launch_plan_list_tv<1>(int, int, const ListPassParams&, int, cudaStream_t, bool);
extern template cudaError_t launch_plan_list_tv<2>(int, int, const ListPassParams&, int, cudaStream_t, bool);
extern template cudaError_t launch_plan_list_tv<3>(int, int, const ListPassParams&, int, cudaStream_t, bool);

}  // namespace ctv
