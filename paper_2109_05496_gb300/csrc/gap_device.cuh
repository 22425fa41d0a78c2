// Device code of the finalize / duality-gap evaluation (Eq. (18), problem (1),
// App. A): x = P_C(b - lam L^T q), the primal and dual values and their gap,
// reduced in FP64.
#pragma once

#include "ctv_device.cuh"

namespace ctv {

// Evaluation of one image at a dual point q (shared by the finalize step and the
// duality-gap checks).
struct GapImg {
  const float2* b;      // row stride ld
  int ld;
  const float4* q;      // dense m x n; nullptr means q = 0
  float2* x;            // nullable: receives x = P_C(b - lam L^T q), row stride ld
  float4* q_export;     // nullable: receives q (dense m x n)
  int m, n;
  float lam, alpha;
  ConsDev C;
};

constexpr int GAP_RW = 64, GAP_RH = 16, GAP_NT = 256;

// One GAP_RW x GAP_RH region with a one-pixel halo; its interior of
// (GAP_RW - 2) x (GAP_RH - 2) pixels starting at (j0, k0) is evaluated: x at a
// pixel needs q at the pixel, above and to the left (Eq. (18)); the TV summand
// needs x below and to the right. Returns, in thread 0, the block's sums of
//   acc[0] = ||x - b||^2, acc[1] = TV(x), acc[2] = ||b||^2 - ||w||^2 + ||w - P_C(w)||^2
// (w = b - lam L^T q), i.e. 2 P - 2 lam TV and 2 D of App. A.
// gap_tile_add adds this thread's share of the three sums (FP32 over its pixels
// of the tile) into the compensated sums acc (no block reduction; the caller
// synchronises before reusing qs and xs) and sets nf when one of the thread's
// values of b is a NaN or an infinity.
template <int TV>
__device__ __forceinline__ void gap_tile_add(const GapImg& g, int j0, int k0, float4* qs, float2* xs,
                                             GapSums& acc, bool& nf) {
  constexpr int RW = GAP_RW, RH = GAP_RH, NT = GAP_NT, R = RW * RH, PPT = R / NT;
  const int m = g.m, n = g.n;
  const int gj0 = j0 - 1, gk0 = k0 - 1;
  const int tid = threadIdx.x;
  const float4 z4 = f4(0.f, 0.f, 0.f, 0.f);
  const float lam = g.lam;
  // b of the thread's own pixels is loaded with q, so that a tile waits on one
  // round of global loads; both later phases take it from registers
  float2 bv[PPT];
#pragma unroll
  for (int s = 0; s < PPT; ++s) {
    const int i = tid + s * NT;
    const int gj = gj0 + i / RW, gk = gk0 + i % RW;
    float4 v = z4;
    bv[s] = make_float2(0.f, 0.f);
    if ((unsigned)gj < (unsigned)m && (unsigned)gk < (unsigned)n) {
      if (g.q != nullptr) v = __ldg(g.q + (long long)gj * n + gk);
      bv[s] = __ldg(g.b + (long long)gj * g.ld + gk);
      nf |= nonfinite2(bv[s]);
    }
    qs[i] = v;
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < PPT; ++s) {
    const int i = tid + s * NT;
    const int lj = i / RW, lk = i % RW;
    const int gj = gj0 + lj, gk = gk0 + lk;
    float2 xv = make_float2(0.f, 0.f);
    if ((unsigned)gj < (unsigned)m && (unsigned)gk < (unsigned)n) {
      const float4 qc = qs[i];
      const float4 qu = lj > 0 ? qs[i - RW] : z4;
      const float4 ql = lk > 0 ? qs[i - 1] : z4;
      const float2 bb = bv[s];
      xv = proj_C(make_float2(fmaf(-lam, qc.x - qu.x + qc.z - ql.z, bb.x), fmaf(-lam, qc.y - qu.y + qc.w - ql.w, bb.y)),
                  gj, gk, g.C);
    }
    xs[i] = xv;
  }
  __syncthreads();
  float fa0 = 0.f, fa1 = 0.f, fa2 = 0.f;   // per-thread partial sums over PPT pixels, then FP64
#pragma unroll
  for (int s = 0; s < PPT; ++s) {
    const int i = tid + s * NT;
    const int lj = i / RW, lk = i % RW;
    const int gj = gj0 + lj, gk = gk0 + lk;
    if (lj >= 1 && lj < RH - 1 && lk >= 1 && lk < RW - 1 && (unsigned)gj < (unsigned)m && (unsigned)gk < (unsigned)n) {
      const float4 qc = qs[i];
      const float4 qu = qs[i - RW];
      const float4 ql = qs[i - 1];
      const float2 bb = bv[s];
      const float dlr = lam * (qc.x - qu.x + qc.z - ql.z);   // lam (L^T q)
      const float dli = lam * (qc.y - qu.y + qc.w - ql.w);
      const float wr = bb.x - dlr, wi = bb.y - dli;
      const float2 xc = xs[i];
      float d1r = 0.f, d1i = 0.f, d2r = 0.f, d2i = 0.f;
      if (gj < m - 1) { const float2 xd = xs[i + RW]; d1r = xc.x - xd.x; d1i = xc.y - xd.y; }
      if (gk < n - 1) { const float2 xr = xs[i + 1]; d2r = xc.x - xr.x; d2i = xc.y - xr.y; }
      const float er = xc.x - bb.x, ei = xc.y - bb.y;
      fa0 += er * er + ei * ei;
      fa1 += tv_term<TV>(d1r, d1i, d2r, d2i, g.alpha);
      // ||b||^2 - ||w||^2 = 2 <b, lam L^T q> - ||lam L^T q||^2, plus ||w - P_C(w)||^2
      const float hr = wr - xc.x, hi = wi - xc.y;
      fa2 += (2.f * (bb.x * dlr + bb.y * dli) - (dlr * dlr + dli * dli)) + (hr * hr + hi * hi);
      if (g.x != nullptr) g.x[(long long)gj * g.ld + gk] = xc;
      if (g.q_export != nullptr) g.q_export[(long long)gj * n + gk] = qc;
    }
  }
  kahan_add(acc.s[0], acc.c[0], fa0);
  kahan_add(acc.s[1], acc.c[1], fa1);
  kahan_add(acc.s[2], acc.c[2], fa2);
}

// Turns the three sums of a completed reduction into primal, dual and gap
// (P = 1/2 ||x - b||^2 + lam TV(x), D = 1/2 (||b||^2 - ||w||^2 + ||w - P_C(w)||^2)),
// applies the stopping test (checks) or records the final iteration count.
__device__ __forceinline__ void gap_finish(DevStats* st, double fid, double tvs, double dual2, float lam,
                                           bool bad_lam, int set, int stopped, int iter, double gap_tol,
                                           int final_call) {
  const double P = 0.5 * fid + (double)lam * tvs;
  const double D = 0.5 * dual2;
  st->primal = P;
  st->dual = D;
  st->gap = P - D;
  if (bad_lam) st->status = 1;   // CTV_EINVAL
  if (*(volatile unsigned int*)&st->nonfinite) st->status = 5;   // CTV_ENONFINITE
  if (!final_call) {
    st->iters = iter;
    if (gap_tol > 0.0 && P - D <= gap_tol * fmax(P, 1e-30)) {
      st->stop = 1;
      st->stop_set = set;
      st->stop_iter = iter;
    }
  } else {
    st->iters = stopped ? st->stop_iter : iter;
  }
}

// Adds the block sums into st and lets the commit that completes the reduction
// (nblk units in all; this one covers `units` of them) evaluate it and reset the
// accumulators. Thread 0 holds the block sums; nonfinite (any thread's flag,
// block-reduced by the caller) marks the image's record. FP64 atomics on one
// address: for reductions with few commits per image (batched plans).
__device__ __forceinline__ void gap_commit(DevStats* st, const double (&acc)[3], unsigned nblk, unsigned units,
                                           float lam, bool bad_lam, int set, int stopped, int iter, double gap_tol,
                                           int final_call, int* last, bool nonfinite) {
  if (threadIdx.x == 0) {
    if (nonfinite) atomicOr(&st->nonfinite, 1u);
    atomicAdd(&st->acc[0], acc[0]);
    atomicAdd(&st->acc[1], acc[1]);
    atomicAdd(&st->acc[2], acc[2]);
    __threadfence();
    *last = (atomicAdd(&st->blocks_done, units) + units == nblk) ? 1 : 0;
  }
  __syncthreads();
  if (*last && threadIdx.x == 0) {
    __threadfence();
    volatile double* a = st->acc;
    gap_finish(st, a[0], a[1], a[2], lam, bad_lam, set, stopped, iter, gap_tol, final_call);
    a[0] = 0.0;
    a[1] = 0.0;
    a[2] = 0.0;
    __threadfence();
    st->blocks_done = 0u;
  }
}

// For reductions over thousands of blocks: every block stores its sums - FP32
// pairs (hi, lo) summed without rounding loss - in its own slot (8 floats at
// slots + 8 blk), with no fence and no atomic, and a one-block kernel launched
// after the reduction (fgp_gap_finish_kernel) adds all slots, always in the same
// order, in FP32 pairs and evaluates them. A per-block memory fence and ticket
// atomic at the end of every block would put their latency on each wave's
// critical path, and FP64 work per block is slow on this GPU (its FP64 rate is a
// small fraction of its FP32 rate). Thread 0 holds the block's pairs.
__device__ __forceinline__ void gap_store_slot(DevStats* st, float* slots, unsigned blk, const float (&hi)[3],
                                               const float (&lo)[3], bool nonfinite) {
  if (threadIdx.x == 0) {
    if (nonfinite) atomicOr(&st->nonfinite, 1u);
    float4* sl = reinterpret_cast<float4*>(slots + 8 * (size_t)blk);
    sl[0] = make_float4(hi[0], lo[0], hi[1], lo[1]);
    sl[1] = make_float4(hi[2], lo[2], 0.f, 0.f);
  }
}

// The duality-gap sums of one block of a pass that evaluates the gap (fused
// check) into its slot. The primal's two terms are combined per thread
// (fid + 2 lam TV, so that P = (fid + 2 lam TV) / 2, evaluated by gap_finish with
// a zero TV sum), leaving two sums to reduce; within a warp they add in plain
// FP32 (a warp's partial covers up to 128 pixels, its relative rounding error is
// below 5 units in the last place, 3e-7, and unbiased, so about 2e-9 of the
// image's total over its tens of thousands of warps), across warps in FP32
// pairs. Measured side by side on 2048^2 solves with checks every 10
// iterations: 54.8 us per check with three sums reduced in pairs at every level,
// 49.4 us in this form.
template <int NT>
__device__ __forceinline__ void gap_block_store(const GapSums& gs, float lam, DevStats* st, float* slots,
                                                unsigned blk, float2* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // (the fused epilogue adds its few terms per thread without compensation)
  float h[2] = {fmaf(2.f * lam, gs.s[1], gs.s[0]) - fmaf(2.f * lam, gs.c[1], gs.c[0]), gs.s[2] - gs.c[2]};
  float l[2];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int a = 0; a < 2; ++a) h[a] += __shfl_down_sync(0xffffffffu, h[a], off);
  }
  const unsigned nfw = __ballot_sync(0xffffffffu, gs.nf);
  if (lane == 0) {
    red[warp] = make_float2(h[0], 0.f);
    red[NT / 32 + warp] = make_float2(h[1], 0.f);
    red[2 * (NT / 32) + warp] = make_float2(nfw != 0u ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  if (warp == 0) {
    bool nf = false;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const float2 v = lane < NT / 32 ? red[a * (NT / 32) + lane] : make_float2(0.f, 0.f);
      h[a] = v.x;
      l[a] = v.y;
      warp_sum_pair(h[a], l[a]);
    }
    if (lane < NT / 32) nf = red[2 * (NT / 32) + lane].x != 0.f;
    nf = __any_sync(0xffffffffu, nf);
    const float hi3[3] = {h[0], 0.f, h[1]}, lo3[3] = {l[0], 0.f, l[1]};
    gap_store_slot(st, slots, blk, hi3, lo3, nf);
  }
}

}  // namespace ctv
