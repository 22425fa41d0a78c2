// Kernel configurations of the fused FGP pass, shared by the single-image,
// batched and plan front ends.
//
// X(id, kind, T, A, B, C):
//   kind 0  fgp_tile:       region A x B pixels (RW x RH), C threads, T iterations per launch
//   kind 1  fgp_strip_tile: A warps across, B warps down, C pixels per thread
//                           (region 32A x BC pixels, 32AB threads)
#pragma once

#include "ctv_device.cuh"

#define CTV_PASS_CONFIGS(X)  \
  X(0, 0, 1, 64, 16, 256)    \
  X(1, 0, 2, 64, 32, 256)    \
  X(2, 0, 4, 64, 32, 256)    \
  X(3, 1, 4, 2, 4, 8)        \
  X(4, 1, 4, 2, 8, 8)        \
  X(5, 1, 6, 2, 8, 8)        \
  X(6, 1, 8, 2, 8, 8)        \
  X(7, 1, 3, 2, 8, 4)        \
  X(8, 1, 6, 4, 4, 8)        \
  X(9, 1, 4, 1, 4, 8)        \
  X(10, 1, 2, 1, 4, 8)       \
  X(11, 1, 4, 2, 8, 4)       \
  X(12, 1, 2, 2, 8, 4)       \
  X(13, 1, 4, 2, 16, 4)      \
  X(14, 1, 6, 2, 16, 4)      \
  X(15, 1, 4, 1, 16, 2)      \
  X(16, 1, 4, 1, 32, 1)      \
  X(17, 1, 8, 1, 32, 1)      \
  X(18, 1, 8, 2, 16, 4)

namespace ctv {

template <int KIND, int A, int B, int C>
struct CfgGeom {
  static constexpr int RW = KIND == 0 ? A : 32 * A;
  static constexpr int RH = KIND == 0 ? B : B * C;
  static constexpr int NT = KIND == 0 ? C : 32 * A * B;
  static constexpr size_t SMEM = KIND == 0 ? (size_t)RW * RH * (sizeof(float4) + sizeof(float2))
                                           : (size_t)RW * RH * 3 * sizeof(float2) + (size_t)B * RW * sizeof(float2);
  // Resident blocks per SM the pass kernel is compiled for: one row per thread
  // fits in 32 registers (two 1024-thread blocks per SM), up to four rows in 64
  // (two 512-thread blocks); deeper strips need more registers and run one
  // block (of their size) per SM.
  static constexpr int MINB = KIND != 1 ? 1
                              : C == 1 ? 65536 / (NT * 32)
                              : (C <= 4 && NT <= 512) ? 65536 / (NT * 64) : 1;
};

template <int KIND, int TV, int T, int A, int B, int C, bool HIST = false, int CONS = CONS_GEN, bool GAPEV = false>
__device__ __forceinline__ void run_tile(const Img& I, int j0, int k0, const float* beta, int nsteps, bool first,
                                         GapSums* gs = nullptr) {
  if constexpr (KIND == 0) {
    static_assert(!GAPEV, "region tiles do not evaluate the gap");
    fgp_tile<TV, T, A, B, C, HIST>(I, j0, k0, beta, nsteps, first);
  } else {
    fgp_strip_tile<TV, T, A, B, C, HIST, CONS, GAPEV>(I, j0, k0, beta, nsteps, first, gs);
  }
}

// Configurations whose pass can end a check interval with the duality-gap
// evaluation fused in (column strips of at most four rows per thread, within
// their register budget).
template <int KIND, int C>
struct GapEvalOk {
  static constexpr bool value = KIND == 1 && C <= 4;
};

}  // namespace ctv
