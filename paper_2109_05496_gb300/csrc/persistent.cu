// All passes of Algorithm 2 in one launch, for images small enough that every
// tile of the fused pass has its own resident block.
//
// Small images are latency-bound: a 256 x 256 solve of 100 iterations needs 25
// launches of a few microseconds each that occupy only part of the GPU. Here
// each block keeps one tile for the whole solve and runs the same column-strip
// body as the regular pass, T iterations at a time, with a grid-wide barrier
// between passes (the dual state of the halos is exchanged through global
// memory, which stays in L2 at these sizes). The launch is cooperative, so all
// blocks are resident; every wait on the barrier is bounded, and a wait that
// runs out records CTV_ETIMEOUT in the image's statistics and ends the kernel
// (the host then sees the status; nothing hangs). Nesterov's t_k is recomputed
// in FP64 by every block, which gives the host table's values bit for bit.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "ctv.h"
#include "ctv_configs.cuh"
#include "ctv_device.cuh"
#include "ctv_host.h"
#include "ctv_kernels.h"

namespace ctv {

struct PersistParams {
  PassParams p;              // b, pointers of the two dual sets (q_in/r_in = set 0, q_out/r_out = set 1), ...
  int K;
  int warm;                  // first pass reads the warm-start dual (dual_q) instead of zeros
  const float4* dual_q;
  unsigned int* bar;         // [0] arrivals, [1] generation (zeroed before the launch)
  int* status;               // CTV_ETIMEOUT on a wait that ran out
};

// Grid-wide barrier with a bounded wait; returns false (everywhere) if any block
// gave up waiting.
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, int* status, unsigned nblocks) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = bar + 1;
    const unsigned int g0 = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == nblocks - 1) {
      bar[0] = 0u;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*gen == g0) {
        if (++spins > (1LL << 22)) {      // several tenths of a second
          atomicExch(status, (int)CTV_ETIMEOUT);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    ok = *(volatile int*)status == 0;
  }
  __syncthreads();
  return ok != 0;
}

template <int TV, int T, int WX, int WY, int PPT, int CONS>
__global__ void __launch_bounds__(32 * WX * WY) fgp_persistent_kernel(PersistParams pp) {
  constexpr int RW = 32 * WX, RH = PPT * WY;
  const PassParams& p = pp.p;
  const int tiles_x = (p.n + (RW - 2 * T) - 1) / (RW - 2 * T);
  const int tile = blockIdx.x;
  const int j0 = (tile / tiles_x) * (RH - 2 * T), k0 = (tile % tiles_x) * (RW - 2 * T);
  float4* qs[2] = {const_cast<float4*>(p.q_in), p.q_out};
  float4* rs[2] = {const_cast<float4*>(p.r_in), p.r_out};
  Img I;
  I.b = p.b;
  I.ld = p.ld;
  I.m = p.m;
  I.n = p.n;
  I.lam = p.lam > 0.f ? p.lam : 0.f;
  I.alpha = p.alpha;
  I.C = p.C;
  I.r_hist = nullptr;
  I.hist_plane = 0;
  double t = 1.0;
  float beta[8];
  int k = 1, out = 0;
  while (k <= pp.K) {
    const int steps = min(T, pp.K - k + 1);
    for (int i = 0; i < steps; ++i) {
      const double tn = (1.0 + sqrt(1.0 + 4.0 * t * t)) / 2.0;
      beta[i] = (float)((t - 1.0) / tn);
      t = tn;
    }
    const bool first = k == 1 && !pp.warm;
    I.q_in = (k == 1) ? pp.dual_q : qs[out ^ 1];
    I.r_in = (k == 1) ? pp.dual_q : rs[out ^ 1];
    I.q_out = qs[out];
    I.r_out = rs[out];
    fgp_strip_tile<TV, T, WX, WY, PPT, false, CONS>(I, j0, k0, beta, steps, first);
    k += steps;
    out ^= 1;
    if (k <= pp.K && !grid_barrier(pp.bar, pp.status, gridDim.x)) return;
  }
}

// persistent geometries: X(id, T, WX, WY, PPT)
#define CTV_PERSIST_CONFIGS(X) \
  X(15, 4, 1, 4, 8)            \
  X(16, 4, 2, 8, 4)

template <int TV, int T, int WX, int WY, int PPT, int CONS>
static ctv_status launch_persist_t(PersistParams& pp, int tiles, cudaStream_t s) {
  constexpr int NT = 32 * WX * WY;
  constexpr size_t SMEM = CfgGeom<1, WX, WY, PPT>::SMEM;
  auto kern = fgp_persistent_kernel<TV, T, WX, WY, PPT, CONS>;
  static bool attr_done = false;
  if (!attr_done) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM) != cudaSuccess)
      return CTV_ECUDA;
    attr_done = true;
  }
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CTV_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CTV_ECUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, SMEM) != cudaSuccess) return CTV_ECUDA;
  if (tiles > per_sm * sms) return CTV_EUNSUPPORTED;   // not all tiles can be resident: use the regular passes
  void* args[] = {&pp};
  if (cudaLaunchCooperativeKernel((const void*)kern, dim3(tiles), dim3(NT), args, SMEM, s) != cudaSuccess)
    return CTV_ECUDA;
  return CTV_OK;
}

template <int T, int WX, int WY, int PPT, int CONS>
static ctv_status launch_persist_tv(int tv, PersistParams& pp, int tiles, cudaStream_t s) {
  switch (tv) {
    case TV1_ISO: return launch_persist_t<TV1_ISO, T, WX, WY, PPT, CONS>(pp, tiles, s);
    case TV1_ANISO: return launch_persist_t<TV1_ANISO, T, WX, WY, PPT, CONS>(pp, tiles, s);
    case TV2_ISO: return launch_persist_t<TV2_ISO, T, WX, WY, PPT, CONS>(pp, tiles, s);
    default: return launch_persist_t<TV2_ANISO, T, WX, WY, PPT, CONS>(pp, tiles, s);
  }
}

template <int T, int WX, int WY, int PPT>
static ctv_status launch_persist_cons(int tv, int cons, PersistParams& pp, int tiles, cudaStream_t s) {
  switch (cons) {
    case CONS_NONE: return launch_persist_tv<T, WX, WY, PPT, CONS_NONE>(tv, pp, tiles, s);
    case CONS_AMP: return launch_persist_tv<T, WX, WY, PPT, CONS_AMP>(tv, pp, tiles, s);
    case CONS_RECT: return launch_persist_tv<T, WX, WY, PPT, CONS_RECT>(tv, pp, tiles, s);
    default: return launch_persist_tv<T, WX, WY, PPT, CONS_GEN>(tv, pp, tiles, s);
  }
}

bool is_persistent_config(int cfg) {
#define CTV_PERSIST_ID(id, T, WX, WY, PPT) if (cfg == id) return true;
  CTV_PERSIST_CONFIGS(CTV_PERSIST_ID)
#undef CTV_PERSIST_ID
  return false;
}

// All K iterations of one image in one cooperative launch. Returns
// CTV_EUNSUPPORTED (before launching anything) when the tiles cannot all be
// resident, so that the caller can run the regular passes instead.
ctv_status run_persistent(int cfg, int tv, const PassParams& p, int K, bool warm, const float4* dual_q,
                          unsigned int* bar, int* status, int* last_set, cudaStream_t s) {
  PersistParams pp;
  memset(&pp, 0, sizeof(pp));
  pp.p = p;
  pp.K = K;
  pp.warm = warm ? 1 : 0;
  pp.dual_q = dual_q;
  pp.bar = bar;
  pp.status = status;
  int T = 1, RW = 0, RH = 0;
  config_info(cfg, &T, &RW, &RH, nullptr);
  const int tiles = ((p.n + (RW - 2 * T) - 1) / (RW - 2 * T)) * ((p.m + (RH - 2 * T) - 1) / (RH - 2 * T));
  const int cons = cons_mode(p.C);
  ctv_status st = CTV_EINVAL;
  switch (cfg) {
#define CTV_PERSIST_CASE(id, T_, WX, WY, PPT) \
  case id: st = launch_persist_cons<T_, WX, WY, PPT>(tv, cons, pp, tiles, s); break;
    CTV_PERSIST_CONFIGS(CTV_PERSIST_CASE)
#undef CTV_PERSIST_CASE
  }
  if (st == CTV_OK) {
    const int passes = (K + T - 1) / T;
    *last_set = (passes - 1) & 1;   // pass i writes set i % 2
  }
  return st;
}

}  // namespace ctv
