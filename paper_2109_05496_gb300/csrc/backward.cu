// Differentiation through K unrolled iterations of Algorithm 2.
//
// Forward (ctv_unrolled_forward): the fused FGP passes over an equally sized
// batch, split at every ckpt_every iterations, where the state (q_k, r_{k+1}) is
// kept as a checkpoint, followed by x = P_C(b - lam L^T q_K) (Eq. (18)).
//
// Backward (ctv_unrolled_backward), given xbar = dLoss/dx:
//   finalize:   what = J_PC(w_K)^T xbar, w_K = b - lam L^T q_K;
//               bbar = what, lambar = -<L^T q_K, what>, qbar_K = -lam L what
//   step k = K..1 (forward map (q_{k-1}, r_k) -> (q_k, r_{k+1})):
//     d = L^T r_k, w = b - lam d, x = P_C(w), e = L x, g = r_k + e / (8 lam)
//     qbar_k = qbar-carry + (1 + beta_k) rbar_{k+1},  the carry being qbar_K at
//              k = K and -beta_{k+1} rbar_{k+2} below it (r_{k+1} = (1+beta_k) q_k - beta_k q_{k-1})
//     gbar = J_PS(g)^T qbar_k   (zero on the padded dual slots)
//     ebar = gbar / (8 lam),  xbar_k = L^T ebar,  what = J_PC(w)^T xbar_k
//     bbar += what,  lambar += -<gbar, e>/(8 lam^2) - <d, what>
//     rbar_k = gbar - lam L what
// Each segment of ckpt_every iterations is first recomputed from its
// checkpoint by the fused pass, storing every r_k of the segment, then walked
// backwards two reverse steps per launch (adj2_stream_kernel; a single step,
// adj_stream_kernel, where a segment has an odd number left). Both kernels
// stream warps down bands of rows with a two-pixel halo per step, since a
// reverse step reads two stencils deep. (Running the next segment's recompute
// on a second stream during the walk back was measured: both kernels fill the
// GPU, so it saved nothing.) All Jacobians are those of the projections, which
// are symmetric; at a projection's boundary the interior branch (identity) is
// taken, and the projection onto a radius-0 ball has Jacobian 0.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ctv.h"
#include "ctv_configs.cuh"
#include "ctv_device.cuh"
#include "ctv_host.h"
#include "ctv_kernels.h"

namespace ctv {

// xhat = J_PC(w)^T xbar
__device__ __forceinline__ float2 proj_C_adj(float2 w, float2 xb, int gj, int gk, const ConsDev& c) {
  if (c.sup == 1) {
    if (gj < c.j0 || gj >= c.j1 || gk < c.k0 || gk >= c.k1) return make_float2(0.f, 0.f);
  } else if (c.sup == 2) {
    if (c.mask[(long long)gj * c.mask_ld + gk] == 0) return make_float2(0.f, 0.f);
  }
  if (c.amp) {
    const float a2 = w.x * w.x + w.y * w.y;
    if (a2 > c.amax * c.amax) {
      const float inv = rsqrtf(a2);
      const float nx = w.x * inv, ny = w.y * inv;
      const float dot = nx * xb.x + ny * xb.y;
      const float s = c.amax * inv;
      return make_float2(s * (xb.x - nx * dot), s * (xb.y - ny * dot));
    }
  } else if (c.box) {
    if (w.x < c.re_lo || w.x > c.re_hi) xb.x = 0.f;
    if (w.y < c.im_lo || w.y > c.im_hi) xb.y = 0.f;
  }
  return xb;
}

// qbar_k = yc Y + rc rbar_{k+1} and the running dL/db sum with a fixed rounding
// sequence (yc Y rounded, then one FMA; plain rounded adds), so that every
// reverse-step kernel, whatever the compiler fuses around it, gives the same bits
__device__ __forceinline__ float4 q_scale(float c, float4 y) {
  const float2 a = __fmul2_rn(make_float2(c, c), make_float2(y.x, y.y));
  const float2 b = __fmul2_rn(make_float2(c, c), make_float2(y.z, y.w));
  return f4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float4 q_axpy(float c, float4 y, float4 q) {
  const float2 a = __ffma2_rn(make_float2(c, c), make_float2(y.x, y.y), make_float2(q.x, q.y));
  const float2 b = __ffma2_rn(make_float2(c, c), make_float2(y.z, y.w), make_float2(q.z, q.w));
  return f4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float2 add_rn(float2 a, float2 b) { return __fadd2_rn(a, b); }

// (a, b) <- J^T (a, b) for the projection of the pair (u, v) onto the ball of radius rad
__device__ __forceinline__ void ball2_adj(float u, float v, float rad, float& a, float& b) {
  if (rad <= 0.f) { a = 0.f; b = 0.f; return; }
  const float nn = u * u + v * v;
  if (nn > rad * rad) {
    const float inv = rsqrtf(nn);
    const float nu = u * inv, nv = v * inv;
    const float dot = nu * a + nv * b;
    const float s = rad * inv;
    a = s * (a - nu * dot);
    b = s * (b - nv * dot);
  }
}

// gbar = J_PS(g)^T qbar for the type-II TV types, whose balls pair the real
// parts of the two differences and the imaginary parts (Eq. (35)) or clamp each
// component (Eq. (37)); g = (r1, s1, r2, s2). (Type I: proj_S_adj2.)
template <int TV>
__device__ __forceinline__ float4 proj_S_adj_type2(float4 g, float4 qb, float alpha) {
  static_assert(TV == TV2_ISO || TV == TV2_ANISO, "type-II TV only");
  if (TV == TV2_ISO) {
    ball2_adj(g.x, g.z, alpha, qb.x, qb.z);
    ball2_adj(g.y, g.w, 1.f - alpha, qb.y, qb.w);
  } else {
    const float a = alpha, c = 1.f - alpha;
    if (a <= 0.f || g.x * g.x > a * a) qb.x = 0.f;
    if (a <= 0.f || g.z * g.z > a * a) qb.z = 0.f;
    if (c <= 0.f || g.y * g.y > c * c) qb.y = 0.f;
    if (c <= 0.f || g.w * g.w > c * c) qb.w = 0.f;
  }
  return qb;
}

constexpr int ADJ_RW = 64, ADJ_RH = 24, ADJ_NT = 512;

struct AdjParams {
  const float2* b;        // dense m x n per image, image stride px
  const float4* r;        // r_k (nullptr: 0)
  const float4* Y;        // carry: qbar_K or rbar_{k+2} (nullptr: 0)
  float yc;               // coefficient of Y
  const float4* rbn;      // rbar_{k+1} (nullptr: 0)
  float rc;               // 1 + beta_k
  float4* rb_out;         // rbar_k
  // two-step reverse pass only: step k-1, whose carry is rbn (coefficient
  // -beta_k) and whose rbar_{k+1} is the rbar_k computed in the same pass
  const float4* r_lo;     // r_{k-1} (nullptr: 0)
  float yc_lo;            // -beta_k
  float rc_lo;            // 1 + beta_{k-1}
  float4* rb_out_lo;      // rbar_{k-1}
  const float2* xbar;     // finalize only
  const float4* qK;       // finalize only
  float4* qbK;            // finalize only: qbar_K
  float2* bbar;
  double* lamacc;
  long long px;
  int m, n;
  const float* lam_dev;
  float alpha;
  ConsDev C;
};

// Finalize adjoint: region with a one-pixel halo.
template <int TV>
__global__ void __launch_bounds__(ADJ_NT) adj_final_kernel(AdjParams p) {
  constexpr int RW = ADJ_RW, RH = ADJ_RH, NT = ADJ_NT, R = RW * RH, PPT = R / NT;
  __shared__ float4 QS[R];
  __shared__ float2 XW[R];
  __shared__ double red[NT / 32];
  const int z = blockIdx.z;
  const long long off = (long long)z * p.px;
  const float lam = fmaxf(p.lam_dev[z], 0.f);
  const int m = p.m, n = p.n;
  const int gj0 = blockIdx.y * (RH - 2) - 1, gk0 = blockIdx.x * (RW - 2) - 1;
  const int tid = threadIdx.x;
  const float4 z4 = f4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int s = 0; s < PPT; ++s) {
    const int i = tid + s * NT;
    const int gj = gj0 + i / RW, gk = gk0 + i % RW;
    float4 q = z4;
    if (p.qK != nullptr && (unsigned)gj < (unsigned)m && (unsigned)gk < (unsigned)n)
      q = __ldg(p.qK + off + (long long)gj * n + gk);
    QS[i] = q;
  }
  __syncthreads();
  float lacc = 0.f;
#pragma unroll
  for (int s = 0; s < PPT; ++s) {
    const int i = tid + s * NT;
    const int lj = i / RW, lk = i % RW;
    const int gj = gj0 + lj, gk = gk0 + lk;
    float2 wh = make_float2(0.f, 0.f);
    if ((unsigned)gj < (unsigned)m && (unsigned)gk < (unsigned)n) {
      const long long o = off + (long long)gj * n + gk;
      const float4 qc = QS[i];
      const float4 qu = lj > 0 ? QS[i - RW] : z4;
      const float4 ql = lk > 0 ? QS[i - 1] : z4;
      const float dr = qc.x - qu.x + qc.z - ql.z, di = qc.y - qu.y + qc.w - ql.w;
      const float2 b2 = __ldg(p.b + o);
      const float2 w = make_float2(b2.x - lam * dr, b2.y - lam * di);
      wh = proj_C_adj(w, __ldg(p.xbar + o), gj, gk, p.C);
      if (lj >= 1 && lj < RH - 1 && lk >= 1 && lk < RW - 1) {
        p.bbar[o] = wh;
        lacc -= dr * wh.x + di * wh.y;
      }
    }
    XW[i] = wh;
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < PPT; ++s) {
    const int i = tid + s * NT;
    const int lj = i / RW, lk = i % RW;
    const int gj = gj0 + lj, gk = gk0 + lk;
    if (lj >= 1 && lj < RH - 1 && lk >= 1 && lk < RW - 1 && (unsigned)gj < (unsigned)m && (unsigned)gk < (unsigned)n) {
      const float2 wc = XW[i];
      float d1r = 0.f, d1i = 0.f, d2r = 0.f, d2i = 0.f;
      if (gj < m - 1) { const float2 wd = XW[i + RW]; d1r = wc.x - wd.x; d1i = wc.y - wd.y; }
      if (gk < n - 1) { const float2 wr = XW[i + 1]; d2r = wc.x - wr.x; d2i = wc.y - wr.y; }
      p.qbK[off + (long long)gj * n + gk] = f4(-lam * d1r, -lam * d1i, -lam * d2r, -lam * d2i);
    }
  }
  double v[1] = {(double)lacc};
  block_sum<NT, 1>(v, red);
  if (tid == 0) atomicAdd(p.lamacc + z, v[0]);
}

__global__ void lambar_finish_kernel(const double* acc, float* out, int batch) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < batch) out[i] = (float)acc[i];
}

// ---------------------------------------------------------------------------
// Recompute pass that also stores r after every iteration (HIST tiles)
// ---------------------------------------------------------------------------
template <int KIND, int TV, int T, int A, int B, int C, int CONS>
__global__ void __launch_bounds__(CfgGeom<KIND, A, B, C>::NT) fgp_hist_pass_kernel(PassParams p, float4* hist,
                                                                                long long hist_plane) {
  using G = CfgGeom<KIND, A, B, C>;
  const int z = blockIdx.z;
  Img I;
  I.b = p.b + z * p.b_stride;
  I.ld = p.ld;
  I.q_in = p.q_in + z * p.d_stride;
  I.r_in = p.r_in + z * p.d_stride;
  I.q_out = p.q_out != nullptr ? p.q_out + z * p.d_stride : nullptr;
  I.r_out = p.r_out != nullptr ? p.r_out + z * p.d_stride : nullptr;
  I.m = p.m;
  I.n = p.n;
  const float lam = p.lam_dev != nullptr ? p.lam_dev[z] : p.lam;
  I.lam = lam > 0.f ? lam : 0.f;
  I.alpha = p.alpha;
  I.C = p.C;
  I.r_hist = hist + z * p.d_stride;
  I.hist_plane = hist_plane;
  const int bx = p.reverse ? gridDim.x - 1 - blockIdx.x : blockIdx.x;
  const int by = p.reverse ? gridDim.y - 1 - blockIdx.y : blockIdx.y;
  run_tile<KIND, TV, T, A, B, C, true, CONS>(I, by * (G::RH - 2 * T), bx * (G::RW - 2 * T), p.beta,
                                             p.nsteps, p.first != 0);
}

// configurations available to the recompute (a subset of the pass table)
#define CTV_HIST_CONFIGS(X) \
  X(2, 0, 4, 64, 32, 256)   \
  X(3, 1, 4, 2, 4, 8)       \
  X(5, 1, 6, 2, 8, 8)       \
  X(14, 1, 6, 2, 16, 4)

template <int KIND, int TV, int T, int A, int B, int C, int CONS>
static cudaError_t launch_hist_c(const PassParams& p, dim3 grid, float4* hist, long long plane, cudaStream_t s) {
  using G = CfgGeom<KIND, A, B, C>;
  static bool attr_done[kMaxDevices] = {};
  cudaError_t e = smem_attr_once(fgp_hist_pass_kernel<KIND, TV, T, A, B, C, CONS>, G::SMEM, attr_done);
  if (e != cudaSuccess) return e;
  fgp_hist_pass_kernel<KIND, TV, T, A, B, C, CONS><<<grid, G::NT, G::SMEM, s>>>(p, hist, plane);
  return cudaGetLastError();
}

// P_C specialised per constraint kind, as in the forward pass (the region tile has one form)
template <int KIND, int TV, int T, int A, int B, int C>
static cudaError_t launch_hist_t(const PassParams& p, dim3 grid, float4* hist, long long plane, cudaStream_t s) {
  if constexpr (KIND == 0) {
    return launch_hist_c<KIND, TV, T, A, B, C, CONS_GEN>(p, grid, hist, plane, s);
  } else {
    switch (cons_mode(p.C)) {
      case CONS_NONE: return launch_hist_c<KIND, TV, T, A, B, C, CONS_NONE>(p, grid, hist, plane, s);
      case CONS_AMP: return launch_hist_c<KIND, TV, T, A, B, C, CONS_AMP>(p, grid, hist, plane, s);
      case CONS_RECT: return launch_hist_c<KIND, TV, T, A, B, C, CONS_RECT>(p, grid, hist, plane, s);
      default: return launch_hist_c<KIND, TV, T, A, B, C, CONS_GEN>(p, grid, hist, plane, s);
    }
  }
}

template <int TV>
static cudaError_t launch_hist_tv(int cfg, const PassParams& p, dim3 grid, float4* hist, long long plane,
                                  cudaStream_t s) {
  switch (cfg) {
#define CTV_HIST_CASE(id, kind, T, A, B, C) \
  case id: return launch_hist_t<kind, TV, T, A, B, C>(p, grid, hist, plane, s);
    CTV_HIST_CONFIGS(CTV_HIST_CASE)
#undef CTV_HIST_CASE
  }
  return cudaErrorInvalidValue;
}

static cudaError_t launch_hist(int tv, int cfg, const PassParams& p, dim3 grid, float4* hist, long long plane,
                               cudaStream_t s) {
  switch (tv) {
    case TV1_ISO: return launch_hist_tv<TV1_ISO>(cfg, p, grid, hist, plane, s);
    case TV1_ANISO: return launch_hist_tv<TV1_ANISO>(cfg, p, grid, hist, plane, s);
    case TV2_ISO: return launch_hist_tv<TV2_ISO>(cfg, p, grid, hist, plane, s);
    case TV2_ANISO: return launch_hist_tv<TV2_ANISO>(cfg, p, grid, hist, plane, s);
  }
  return cudaErrorInvalidValue;
}

static bool hist_config_ok(int cfg) {
#define CTV_HIST_ID(id, kind, T, A, B, C) if (cfg == id) return true;
  CTV_HIST_CONFIGS(CTV_HIST_ID)
#undef CTV_HIST_ID
  return false;
}

// ---------------------------------------------------------------------------
// Reverse step streamed down the rows by independent warps: no shared memory
// and no block barriers. A warp owns 28 columns (lanes 2..29 of a 32-column
// window that starts two columns to the left of them) and a band of ADJS_H
// rows, which it walks top to bottom one row per iteration, keeping in
// registers the rows each stencil phase still needs and taking horizontal
// neighbours from the adjacent lanes. With row i arriving, phase A
// (x = P_C(b - lam L^T r)) runs on row i, phases B (gbar, ebar) and C (what,
// dL/db) on row i-1 and phase D (rbar) on row i-2; the next row's loads are
// issued before the current row is computed.
// ---------------------------------------------------------------------------
#ifndef ADJS_H
#define ADJS_H 16           // rows per warp
#endif
#ifndef ADJS_PF
#define ADJS_PF 1           // rows of loads issued ahead
#endif
#ifndef ADJS_WARPS
#define ADJS_WARPS 4        // warps per block (adjacent column windows)
#endif
constexpr int ADJS_OWN = 28;    // columns owned by a warp
#ifndef ADJS_MINB
#define ADJS_MINB 6
#endif

__device__ __forceinline__ float2 shfl_up2(float2 v) {
  return make_float2(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1));
}
__device__ __forceinline__ float2 shfl_dn2(float2 v) {
  return make_float2(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1));
}

// Registers a warp carries down its band: row i-1 for phases B and C, row i-2
// for phase D, and r1 of row i-1 for phase A.
struct AdjsState {
  float4 Rm, Qm, gbmm;
  float2 r1p, wm, dm, xm, e2m, eb1m, whmm, d2mm;
  float lacc;
};

// Phases A-D for arriving row i with inputs R = r_k, B = b, Q = qbar_k of row
// i: what of row i-1 and rbar of row i-2 are returned (rbar computed on every
// lane and row; only the caller knows which are valid and owned); own_m says
// whether row i-1 of this lane counts toward dL/dlambda. EDGE = false: the
// warp's 32 columns lie in [0, n - 1) and the rows in [0, m - 1), so no bounds
// or edge tests are needed.
// The reverse sweep differentiates the branch of each projection that the
// forward pass took, so every quantity that feeds x or a projection's test is
// computed with the forward's own expressions (same association, same fused
// multiply-adds); only the Jacobian products that follow use packed arithmetic.

// J^T of the projection of the pair u onto the ball of radius rad, applied to a (packed)
__device__ __forceinline__ float2 ball2_adj2(float2 u, float rad, float2 a) {
  if (rad <= 0.f) return make_float2(0.f, 0.f);
  const float nn = u.x * u.x + u.y * u.y;
  if (nn > rad * rad) {
    const float inv = rsqrtf(nn);
    const float2 nu = mul2(u, p2(inv));
    return mul2(p2(rad * inv), fma2(nu, p2(-dot2(nu, a)), a));
  }
  return a;
}

// J^T of the amplitude bound's projection (as proj_C_adj: the interior branch
// wherever |w| <= amax, including w = 0 when amax = 0)
__device__ __forceinline__ float2 amp_adj2(float2 w, float amax, float2 xb) {
  const float a2 = w.x * w.x + w.y * w.y;
  if (a2 > amax * amax) {
    const float inv = rsqrtf(a2);
    const float2 nw = mul2(w, p2(inv));
    return mul2(p2(amax * inv), fma2(nw, p2(-dot2(nw, xb)), xb));
  }
  return xb;
}

// xhat = J_PC(w)^T xbar, specialised like proj_C_t
template <int CONS>
__device__ __forceinline__ float2 proj_C_adj_t2(float2 w, float2 xb, int gj, int gk, bool kin, const ConsDev& c) {
  if (CONS == CONS_NONE) return xb;
  if (CONS == CONS_RECT && (!kin || gj < c.j0 || gj >= c.j1)) return make_float2(0.f, 0.f);
  if (CONS == CONS_AMP || (CONS == CONS_RECT && c.amp)) return amp_adj2(w, c.amax, xb);
  if (CONS == CONS_RECT) return xb;
  return proj_C_adj(w, xb, gj, gk, c);
}

// gbar = J_PS(g)^T qbar with g and qbar as (d1, d2) halves
template <int TV>
__device__ __forceinline__ void proj_S_adj2(float2 g1, float2 g2, float2& q1, float2& q2, float alpha) {
  if constexpr (TV == TV1_ISO) {
    const float nn = g1.x * g1.x + g1.y * g1.y + g2.x * g2.x + g2.y * g2.y;
    if (nn > 1.f) {
      const float inv = rsqrtf(nn);
      const float2 n1 = mul2(g1, p2(inv)), n2 = mul2(g2, p2(inv));
      const float2 dt = fma2(n2, q2, mul2(n1, q1));
      const float2 md = p2(-(dt.x + dt.y));
      q1 = mul2(p2(inv), fma2(n1, md, q1));
      q2 = mul2(p2(inv), fma2(n2, md, q2));
    }
  } else if constexpr (TV == TV1_ANISO) {
    q1 = ball2_adj2(g1, 1.f, q1);
    q2 = ball2_adj2(g2, 1.f, q2);
  } else {
    const float4 r = proj_S_adj_type2<TV>(f4(g1.x, g1.y, g2.x, g2.y), f4(q1.x, q1.y, q2.x, q2.y), alpha);
    q1 = lo2(r);
    q2 = hi2(r);
  }
}

// Phases A-D for arriving row i with inputs R = r_k, B = b, Q = qbar_k of row
// i: what of row i-1 and rbar of row i-2 are returned (rbar computed on every
// lane and row; only the caller knows which are valid and owned); own_m says
// whether row i-1 of this lane counts toward dL/dlambda. EDGE = false: the
// warp's 32 columns lie in [0, n - 1) and the rows in [0, m - 1), so no bounds
// or edge tests are needed. The complex halves go through packed FP32x2
// instructions.
template <int TV, int CONS, bool EDGE>
__device__ __forceinline__ void adjs_core(const AdjParams& p, AdjsState& S, int i, const float4 R, const float2 B,
                                          const float4 Q, bool colin, bool own_m, bool kin, bool has_right, int gk,
                                          float lam, float c8, float2& wh_out, float4& rbar_out) {
  const int m = p.m;
  const float2 z2 = make_float2(0.f, 0.f);
  const bool rin = colin && (!EDGE || (unsigned)i < (unsigned)m);
  const int im = i - 1;
  const bool inm = colin && (!EDGE || (unsigned)im < (unsigned)m);
  const float2 nlam = p2(-lam), vc8 = p2(c8);
  // A (row i): d = L^T r, w = b - lam d, x = P_C(w); e2 = x - x(right)
  const float2 R1 = lo2(R), R2 = hi2(R);
  const float2 left = shfl_up2(R2);
  float2 d = z2, w = z2, x = z2;
  if (rin) {
    // (L^T p)[j,k] = p1[j,k] - p1[j-1,k] + p2[j,k] - p2[j,k-1], summed left to right as in the forward
    d = sub2(add2(sub2(R1, S.r1p), R2), left);
    w = fma2(nlam, d, B);
    x = proj_C_t<CONS>(w, i, gk, kin, p.C);
  }
  const float2 xr = shfl_dn2(x);
  const float2 e2 = rin && has_right ? sub2(x, xr) : z2;
  // B (row i-1): g = r + L x / (8 lam), gbar = J_PS(g)^T qbar, ebar = gbar / (8 lam)
  float2 gb1 = z2, gb2 = z2;
  if (inm) {
    const float2 e1 = !EDGE || im < m - 1 ? sub2(S.xm, x) : z2;
    const float2 g1 = fma2(vc8, e1, lo2(S.Rm)), g2 = fma2(vc8, S.e2m, hi2(S.Rm));
    gb1 = lo2(S.Qm);
    gb2 = hi2(S.Qm);
    proj_S_adj2<TV>(g1, g2, gb1, gb2, p.alpha);
    if (EDGE && im == m - 1) gb1 = z2;
    if (!has_right) gb2 = z2;
    if (own_m) {
      const float2 t = fma2(gb2, S.e2m, mul2(gb1, e1));
      S.lacc -= 8.f * c8 * c8 * (t.x + t.y);
    }
  }
  const float2 eb1 = mul2(vc8, gb1), eb2 = mul2(vc8, gb2);
  // C (row i-1): xbar = L^T ebar, what = J_PC(w)^T xbar
  const float2 ebl = shfl_up2(eb2);
  float2 wh = z2;
  if (inm) {
    const float2 xb = add2(sub2(eb1, S.eb1m), sub2(eb2, ebl));
    wh = proj_C_adj_t2<CONS>(S.wm, xb, im, gk, kin, p.C);
    if (own_m) S.lacc -= dot2(S.dm, wh);
  }
  const float2 whr = shfl_dn2(wh);
  const float2 d2 = inm && has_right ? sub2(wh, whr) : z2;
  // D (row i-2): rbar = gbar - lam L what
  const float2 d1 = !EDGE || i - 2 < m - 1 ? sub2(S.whmm, wh) : z2;
  const float2 rb1 = fma2(nlam, d1, lo2(S.gbmm)), rb2 = fma2(nlam, S.d2mm, hi2(S.gbmm));
  rbar_out = f4(rb1.x, rb1.y, rb2.x, rb2.y);
  wh_out = wh;
  S.r1p = R1;
  S.Rm = R;
  S.Qm = Q;
  S.wm = w;
  S.dm = d;
  S.xm = x;
  S.e2m = e2;
  S.eb1m = eb1;
  S.gbmm = f4(gb1.x, gb1.y, gb2.x, gb2.y);
  S.whmm = wh;
  S.d2mm = d2;
}

// One reverse step on arriving row i: dL/db of row i-1 (bbo: its value before
// this step) and rbar_k of row i-2 are written for the owned pixels of the band.
template <int TV, int CONS, bool EDGE>
__device__ __forceinline__ void adjs_row(const AdjParams& p, AdjsState& S, int i, const float4 R, const float2 B,
                                         const float4 Q, const float2 bbo, bool colin, bool own, bool kin,
                                         bool has_right, int gk, int j0, int j1, long long col, float lam,
                                         float c8) {
  const int n = p.n;
  const int im = i - 1, i2 = i - 2;
  const bool own_m = own && im >= j0 && im < j1;
  float2 wh;
  float4 rb;
  adjs_core<TV, CONS, EDGE>(p, S, i, R, B, Q, colin, own_m, kin, has_right, gk, lam, c8, wh, rb);
  if (own_m) p.bbar[col + (long long)im * n] = add_rn(bbo, wh);
  if (own && i2 >= j0 && i2 < j1) p.rb_out[col + (long long)i2 * n] = rb;
}

__device__ __forceinline__ void adjs_init(const AdjParams& p, const float4* r, AdjsState& S, bool colin, bool edge,
                                          int j0, long long col) {
  const float4 z4 = f4(0.f, 0.f, 0.f, 0.f);
  const float2 z2 = make_float2(0.f, 0.f);
  S.Rm = S.Qm = S.gbmm = z4;
  S.r1p = S.wm = S.dm = S.xm = S.e2m = S.eb1m = S.whmm = S.d2mm = z2;
  S.lacc = 0.f;
  // r1 of row j0-2 (upper neighbour of the first row phase A computes)
  if (r != nullptr && colin && (!edge || j0 - 2 >= 0)) {
    const float4 t = __ldg(r + col + (long long)(j0 - 2) * p.n);
    S.r1p = make_float2(t.x, t.y);
  }
}

// Band with asynchronous copies (cp.async) of the next ADJS_D - 1 rows into a
// per-warp ring of shared-memory slots: the loads are in flight for several
// rows without holding registers. Every lane reads back only its own column.
#ifndef ADJS_D
#define ADJS_D 3            // ring slots (rows in flight + the row being consumed)
#endif
struct AdjsSlot {
  float4 R[32], Y[32], N[32];
  float2 B[32], BB[32];
};

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Issue the copies of row gj (zero-filled outside the image; dL/db only for
// owned pixels of the band) and close the group.
__device__ __forceinline__ void adjs_issue(const AdjParams& p, AdjsSlot* sl, int lane, int gj, bool colin, bool own,
                                          int j0, int j1, long long col) {
  const bool in = colin && (unsigned)gj < (unsigned)p.m;
  const long long o = in ? col + (long long)gj * p.n : 0;
  const int s16 = in ? 16 : 0, s8 = in ? 8 : 0;
  if (p.r != nullptr) cp_async16(&sl->R[lane], p.r + o, s16);
  cp_async8(&sl->B[lane], p.b + o, s8);
  if (p.Y != nullptr) cp_async16(&sl->Y[lane], p.Y + o, s16);
  if (p.rbn != nullptr) cp_async16(&sl->N[lane], p.rbn + o, s16);
  const bool bo = own && gj >= j0 && gj < j1;
  cp_async8(&sl->BB[lane], p.bbar + (bo ? o : 0), bo ? 8 : 0);
  cp_async_commit();
}

template <int TV, int CONS, bool EDGE>
__device__ __forceinline__ float adjs_band_async(const AdjParams& p, AdjsSlot* ring, int lane, int gk, int j0,
                                                 int j1, long long col, float lam, float c8) {
  const int n = p.n;
  const bool colin = !EDGE || (unsigned)gk < (unsigned)n;
  const bool own = colin && lane >= 2 && lane < 2 + ADJS_OWN;
  const bool kin = gk >= p.C.k0 && gk < p.C.k1;
  const bool has_right = !EDGE || gk < n - 1;
  const float4 z4 = f4(0.f, 0.f, 0.f, 0.f);
  AdjsState S;
  adjs_init(p, p.r, S, colin, EDGE, j0, col);
  // prologue: rows j0-1 .. j0+D-3 in slots 0 .. D-2
#pragma unroll
  for (int t = 0; t < ADJS_D - 1; ++t) adjs_issue(p, ring + t, lane, j0 - 1 + t, colin, own, j0, j1, col);
  float2 bbn = make_float2(0.f, 0.f);
  int slot = 0;
  for (int i = j0 - 1; i <= j1 + 1; ++i) {
    // refill the slot consumed last iteration with row i+D-1 (an empty group past the band)
    const int fill = slot == 0 ? ADJS_D - 1 : slot - 1;
    if (i + ADJS_D - 1 <= j1 + 1) adjs_issue(p, ring + fill, lane, i + ADJS_D - 1, colin, own, j0, j1, col);
    else cp_async_commit();
    cp_async_wait<ADJS_D - 1>();
    const AdjsSlot* sl = ring + slot;
    const float4 R = p.r != nullptr ? sl->R[lane] : z4;
    const float2 B = sl->B[lane];
    float4 Q = z4;
    if (p.Y != nullptr) {
      const float4 y = sl->Y[lane];
      Q = q_scale(p.yc, y);
    }
    if (p.rbn != nullptr) {
      const float4 y = sl->N[lane];
      Q = q_axpy(p.rc, y, Q);
    }
    const float2 bbo = bbn;
    bbn = sl->BB[lane];
    adjs_row<TV, CONS, EDGE>(p, S, i, R, B, Q, bbo, colin, own, kin, has_right, gk, j0, j1, col, lam, c8);
    slot = slot == ADJS_D - 1 ? 0 : slot + 1;
  }
  cp_async_wait<0>();
  return S.lacc;
}

template <int TV, int CONS>
__global__ void __launch_bounds__(32 * ADJS_WARPS, ADJS_MINB) adj_stream_kernel(AdjParams p) {
  const int lane = threadIdx.x & 31;
  const int wc = blockIdx.x * ADJS_WARPS + (threadIdx.x >> 5);
  const int m = p.m, n = p.n;
  if (wc * ADJS_OWN >= n) return;   // whole warp past the last column
  const int z = blockIdx.z;
  const float lam = fmaxf(p.lam_dev[z], 0.f);
  const float c8 = lam > 0.f ? 1.f / (8.f * lam) : 0.f;
  const int gk0 = wc * ADJS_OWN - 2;
  const int gk = gk0 + lane;
  const int j0 = blockIdx.y * ADJS_H;
  const int j1 = min(j0 + ADJS_H, m);
  const long long col = (long long)z * p.px + gk;
  const bool inside = gk0 >= 0 && gk0 + 32 <= n - 1 && j0 - 2 >= 0 && j1 + 2 <= m - 1;
  extern __shared__ AdjsSlot adjs_ring[];
  AdjsSlot* ring = adjs_ring + (threadIdx.x >> 5) * ADJS_D;
  const float lacc = inside ? adjs_band_async<TV, CONS, false>(p, ring, lane, gk, j0, j1, col, lam, c8)
                            : adjs_band_async<TV, CONS, true>(p, ring, lane, gk, j0, j1, col, lam, c8);
  double v = (double)lacc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) atomicAdd(p.lamacc + z, v);
}

// ---------------------------------------------------------------------------
// Two reverse steps (k, then k-1) in one streaming pass. Step k runs as in
// adj_stream_kernel; step k-1 follows two rows behind, its qbar_{k-1} =
// -beta_k rbar_{k+1} + (1 + beta_{k-1}) rbar_k taking rbar_k from step k's
// phase D of the same iteration. Both rbar_k and rbar_{k-1} are written, and
// dL/db is read and written once for both steps. The lower step's valid lanes
// shrink to 3..28, so a warp owns 26 columns; the ring keeps each row's slot
// until the lower step has read it two iterations later.
// ---------------------------------------------------------------------------
#ifndef CTV_ADJ_PAIR
#define CTV_ADJ_PAIR 1
#endif
#ifndef ADJ2_H
#define ADJ2_H 32           // rows per warp
#endif
#ifndef ADJ2_D
#define ADJ2_D 5            // ring slots
#endif
#ifndef ADJ2_MINB
#define ADJ2_MINB 4
#endif
constexpr int ADJ2_OWN = 26;

struct Adj2Slot {
  float4 R[32], RL[32], Y[32], N[32];
  float2 B[32], BB[32];
};

__device__ __forceinline__ void adj2_issue(const AdjParams& p, Adj2Slot* sl, int lane, int gj, bool colin, bool own,
                                          int j0, int j1, long long col) {
  const bool in = colin && (unsigned)gj < (unsigned)p.m;
  const long long o = in ? col + (long long)gj * p.n : 0;
  const int s16 = in ? 16 : 0, s8 = in ? 8 : 0;
  if (p.r != nullptr) cp_async16(&sl->R[lane], p.r + o, s16);
  if (p.r_lo != nullptr) cp_async16(&sl->RL[lane], p.r_lo + o, s16);
  cp_async8(&sl->B[lane], p.b + o, s8);
  if (p.Y != nullptr) cp_async16(&sl->Y[lane], p.Y + o, s16);
  if (p.rbn != nullptr) cp_async16(&sl->N[lane], p.rbn + o, s16);
  const bool bo = own && gj >= j0 && gj < j1;
  cp_async8(&sl->BB[lane], p.bbar + (bo ? o : 0), bo ? 8 : 0);
  cp_async_commit();
}

template <int TV, int CONS, bool EDGE>
__device__ __forceinline__ float adj2_band(const AdjParams& p, Adj2Slot* ring, int lane, int gk, int j0, int j1,
                                           long long col, float lam, float c8) {
  const int n = p.n;
  const bool colin = !EDGE || (unsigned)gk < (unsigned)n;
  const bool own = colin && lane >= 3 && lane < 3 + ADJ2_OWN;
  const bool kin = gk >= p.C.k0 && gk < p.C.k1;
  const bool has_right = !EDGE || gk < n - 1;
  const float4 z4 = f4(0.f, 0.f, 0.f, 0.f);
  const float2 z2 = make_float2(0.f, 0.f);
  AdjsState U, Lo;
  adjs_init(p, p.r, U, colin, EDGE, j0 - 1, col);     // step k: first arriving row j0-2
  adjs_init(p, p.r_lo, Lo, colin, EDGE, j0, col);     // step k-1: first arriving row j0-1
  const int base = j0 - 2;   // row of slot 0
#pragma unroll
  for (int t = 0; t < ADJ2_D - 3; ++t) adj2_issue(p, ring + t, lane, base + t, colin, own, j0, j1, col);
  float2 acc1 = z2, acc2 = z2;   // dL/db + what_k of rows i-2 and i-3
  int slot = 0;                  // slot of row i
  for (int i = base; i <= j1 + 3; ++i) {
    // refill the slot of row i-3 (read for the last time last iteration) with row i-3+D
    const int fill = slot >= 3 ? slot - 3 : slot + ADJ2_D - 3;
    if (i - 3 + ADJ2_D <= j1 + 3) adj2_issue(p, ring + fill, lane, i - 3 + ADJ2_D, colin, own, j0, j1, col);
    else cp_async_commit();
    cp_async_wait<ADJ2_D - 3>();
    const int s1 = slot >= 1 ? slot - 1 : slot + ADJ2_D - 1;
    const int s2 = slot >= 2 ? slot - 2 : slot + ADJ2_D - 2;
    // step k on row i
    const Adj2Slot* sl = ring + slot;
    const float4 R = p.r != nullptr ? sl->R[lane] : z4;
    float4 Q = z4;
    if (p.Y != nullptr) {
      const float4 y = sl->Y[lane];
      Q = q_scale(p.yc, y);
    }
    if (p.rbn != nullptr) {
      const float4 y = sl->N[lane];
      Q = q_axpy(p.rc, y, Q);
    }
    const int im = i - 1;
    float2 whU;
    float4 rbU;
    adjs_core<TV, CONS, EDGE>(p, U, i, R, sl->B[lane], Q, colin, own && im >= j0 && im < j1, kin, has_right, gk,
                              lam, c8, whU, rbU);
    const int i2 = i - 2;
    if (own && i2 >= j0 && i2 < j1) p.rb_out[col + (long long)i2 * n] = rbU;
    const float2 bo = ring[s1].BB[lane];   // dL/db of row i-1 before this pass
    const float2 acc0 = add_rn(bo, whU);
    // step k-1 on row i-2
    if (i >= j0 + 1) {
      const Adj2Slot* sl2 = ring + s2;
      const float4 RL = p.r_lo != nullptr ? sl2->RL[lane] : z4;
      // same operation order as the single step's yc Y + rc rbar_{k+1}, so that
      // pairing steps changes no bit of the result
      float4 QL = z4;
      if (p.rbn != nullptr) {
        const float4 y = sl2->N[lane];
        QL = q_scale(p.yc_lo, y);
      }
      QL = q_axpy(p.rc_lo, rbU, QL);
      const int i3 = i - 3, i4 = i - 4;
      float2 whL;
      float4 rbL;
      adjs_core<TV, CONS, EDGE>(p, Lo, i2, RL, sl2->B[lane], QL, colin, own && i3 >= j0 && i3 < j1, kin, has_right,
                                gk, lam, c8, whL, rbL);
      if (own && i3 >= j0 && i3 < j1) p.bbar[col + (long long)i3 * n] = add_rn(acc2, whL);
      if (own && i4 >= j0 && i4 < j1) p.rb_out_lo[col + (long long)i4 * n] = rbL;
    }
    acc2 = acc1;
    acc1 = acc0;
    slot = slot == ADJ2_D - 1 ? 0 : slot + 1;
  }
  cp_async_wait<0>();
  return U.lacc + Lo.lacc;
}

template <int TV, int CONS>
__global__ void __launch_bounds__(32 * ADJS_WARPS, ADJ2_MINB) adj2_stream_kernel(AdjParams p) {
  const int lane = threadIdx.x & 31;
  const int wc = blockIdx.x * ADJS_WARPS + (threadIdx.x >> 5);
  const int m = p.m, n = p.n;
  if (wc * ADJ2_OWN >= n) return;   // whole warp past the last column
  const int z = blockIdx.z;
  const float lam = fmaxf(p.lam_dev[z], 0.f);
  const float c8 = lam > 0.f ? 1.f / (8.f * lam) : 0.f;
  const int gk0 = wc * ADJ2_OWN - 3;
  const int gk = gk0 + lane;
  const int j0 = blockIdx.y * ADJ2_H;
  const int j1 = min(j0 + ADJ2_H, m);
  const long long col = (long long)z * p.px + gk;
  const bool inside = gk0 >= 0 && gk0 + 32 <= n - 1 && j0 - 3 >= 0 && j1 + 4 <= m - 1;
  extern __shared__ Adj2Slot adj2_ring[];
  Adj2Slot* ring = adj2_ring + (threadIdx.x >> 5) * ADJ2_D;
  const float lacc = inside ? adj2_band<TV, CONS, false>(p, ring, lane, gk, j0, j1, col, lam, c8)
                            : adj2_band<TV, CONS, true>(p, ring, lane, gk, j0, j1, col, lam, c8);
  double v = (double)lacc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) atomicAdd(p.lamacc + z, v);
}

template <int TV, int CONS>
static cudaError_t launch_adj_stream_t(const AdjParams& p, int batch, cudaStream_t s) {
  const int ncw = (p.n + ADJS_OWN - 1) / ADJS_OWN;
  dim3 grid((ncw + ADJS_WARPS - 1) / ADJS_WARPS, (p.m + ADJS_H - 1) / ADJS_H, batch);
  constexpr size_t smem = sizeof(AdjsSlot) * ADJS_D * ADJS_WARPS;
  static bool attr_done[kMaxDevices] = {};
  cudaError_t e = smem_attr_once(adj_stream_kernel<TV, CONS>, smem, attr_done);
  if (e != cudaSuccess) return e;
  adj_stream_kernel<TV, CONS><<<grid, 32 * ADJS_WARPS, smem, s>>>(p);
  return cudaGetLastError();
}

template <int TV>
static cudaError_t launch_adj_stream_tv(int cons, const AdjParams& p, int batch, cudaStream_t s) {
  switch (cons) {
    case CONS_NONE: return launch_adj_stream_t<TV, CONS_NONE>(p, batch, s);
    case CONS_AMP: return launch_adj_stream_t<TV, CONS_AMP>(p, batch, s);
    case CONS_RECT: return launch_adj_stream_t<TV, CONS_RECT>(p, batch, s);
    default: return launch_adj_stream_t<TV, CONS_GEN>(p, batch, s);
  }
}

template <int TV, int CONS>
static cudaError_t launch_adj2_t(const AdjParams& p, int batch, cudaStream_t s) {
  const int ncw = (p.n + ADJ2_OWN - 1) / ADJ2_OWN;
  dim3 grid((ncw + ADJS_WARPS - 1) / ADJS_WARPS, (p.m + ADJ2_H - 1) / ADJ2_H, batch);
  constexpr size_t smem = sizeof(Adj2Slot) * ADJ2_D * ADJS_WARPS;
  static bool attr_done[kMaxDevices] = {};
  cudaError_t e = smem_attr_once(adj2_stream_kernel<TV, CONS>, smem, attr_done);
  if (e != cudaSuccess) return e;
  adj2_stream_kernel<TV, CONS><<<grid, 32 * ADJS_WARPS, smem, s>>>(p);
  return cudaGetLastError();
}

template <int TV>
static cudaError_t launch_adj2_tv(int cons, const AdjParams& p, int batch, cudaStream_t s) {
  switch (cons) {
    case CONS_NONE: return launch_adj2_t<TV, CONS_NONE>(p, batch, s);
    case CONS_AMP: return launch_adj2_t<TV, CONS_AMP>(p, batch, s);
    case CONS_RECT: return launch_adj2_t<TV, CONS_RECT>(p, batch, s);
    default: return launch_adj2_t<TV, CONS_GEN>(p, batch, s);
  }
}

// steps k and k-1 in one pass (p.r_lo, p.yc_lo, p.rc_lo, p.rb_out_lo set)
static cudaError_t launch_adj_pair(int tv, const AdjParams& p, int batch, cudaStream_t s) {
  const int cons = cons_mode(p.C);
  switch (tv) {
    case TV1_ISO: return launch_adj2_tv<TV1_ISO>(cons, p, batch, s);
    case TV1_ANISO: return launch_adj2_tv<TV1_ANISO>(cons, p, batch, s);
    case TV2_ISO: return launch_adj2_tv<TV2_ISO>(cons, p, batch, s);
    default: return launch_adj2_tv<TV2_ANISO>(cons, p, batch, s);
  }
}

static cudaError_t launch_adj_step(int tv, const AdjParams& p, int batch, cudaStream_t s) {
  const int cons = cons_mode(p.C);
  switch (tv) {
    case TV1_ISO: return launch_adj_stream_tv<TV1_ISO>(cons, p, batch, s);
    case TV1_ANISO: return launch_adj_stream_tv<TV1_ANISO>(cons, p, batch, s);
    case TV2_ISO: return launch_adj_stream_tv<TV2_ISO>(cons, p, batch, s);
    default: return launch_adj_stream_tv<TV2_ANISO>(cons, p, batch, s);
  }
}

static cudaError_t launch_adj_final(int tv, const AdjParams& p, int batch, cudaStream_t s) {
  dim3 grid((p.n + ADJ_RW - 3) / (ADJ_RW - 2), (p.m + ADJ_RH - 3) / (ADJ_RH - 2), batch);
  switch (tv) {
    case TV1_ISO: adj_final_kernel<TV1_ISO><<<grid, ADJ_NT, 0, s>>>(p); break;
    case TV1_ANISO: adj_final_kernel<TV1_ANISO><<<grid, ADJ_NT, 0, s>>>(p); break;
    case TV2_ISO: adj_final_kernel<TV2_ISO><<<grid, ADJ_NT, 0, s>>>(p); break;
    default: adj_final_kernel<TV2_ANISO><<<grid, ADJ_NT, 0, s>>>(p); break;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Workspace layout
// ---------------------------------------------------------------------------
static size_t al(size_t v) { return (v + 255) & ~(size_t)255; }

struct UnrolledLayout {
  DevStats* st;
  double* lamacc;
  std::vector<float4*> ckq, ckr;   // slot s: state after s * ckpt iterations (slot 0 unused: zero state)
  float4* finq;
  float4* finr;
  float4* setq[2];
  float4* setr[2];
  float4* hist;                    // ckpt planes: r_k of the segment being walked back
  float4* rb[4];                   // rbar carries of the reverse walk
  size_t bytes;
};

static UnrolledLayout layout(char* base, int batch, int m, int n, int K, int ckpt) {
  UnrolledLayout L;
  const size_t plane = al((size_t)batch * m * n * sizeof(float4));
  const int nseg = (K + ckpt - 1) / ckpt;
  size_t off = 0;
  L.st = (DevStats*)(base + off); off += al((size_t)batch * sizeof(DevStats));
  L.lamacc = (double*)(base + off); off += al((size_t)batch * sizeof(double));
  L.ckq.assign((size_t)nseg, nullptr);
  L.ckr.assign((size_t)nseg, nullptr);
  for (int s = 1; s < nseg; ++s) {
    L.ckq[(size_t)s] = (float4*)(base + off); off += plane;
    L.ckr[(size_t)s] = (float4*)(base + off); off += plane;
  }
  L.finq = (float4*)(base + off); off += plane;
  L.finr = (float4*)(base + off); off += plane;
  for (int i = 0; i < 2; ++i) {
    L.setq[i] = (float4*)(base + off); off += plane;
    L.setr[i] = (float4*)(base + off); off += plane;
  }
  L.hist = (float4*)(base + off); off += (size_t)ckpt * plane;
  for (int i = 0; i < 4; ++i) {
    L.rb[i] = (float4*)(base + off); off += plane;
  }
  L.bytes = off;
  return L;
}

static int unrolled_config(const ctv_opts* o) {
  if (o != nullptr && o->config >= 0 && hist_config_ok(o->config)) return o->config;
  return 5;
}

struct UnrolledArgs {
  const void* b;
  int batch, m, n;
  const float* lams;
  const ctv_constraint* C;
  int tv;
  const ctv_opts* opts;
  int ckpt;
  void* ws;
  size_t ws_bytes;
};

static ctv_status check_unrolled(const UnrolledArgs& a, ConsDev* C) {
  if (a.b == nullptr || a.lams == nullptr || a.ws == nullptr || a.opts == nullptr) return CTV_EINVAL;
  if (a.batch <= 0 || a.batch > 65535 || a.m <= 0 || a.n <= 0) return CTV_EINVAL;
  if (a.opts->max_iters < 1 || a.ckpt < 1 || a.opts->warm_start || a.opts->plain_gp) return CTV_EINVAL;
  if (!(a.opts->alpha >= 0.f && a.opts->alpha <= 1.f)) return CTV_EINVAL;
  if (a.tv < 0 || a.tv > 3) return CTV_EINVAL;
  if (((uintptr_t)a.b & 7) || ((uintptr_t)a.ws & 255)) return CTV_EINVAL;
  if (!convert_constraint(a.C, a.m, a.n, C)) return CTV_EINVAL;
  const UnrolledLayout L = layout(nullptr, a.batch, a.m, a.n, a.opts->max_iters, a.ckpt);
  if (a.ws_bytes < L.bytes) return CTV_EINVAL;
  return CTV_OK;
}

static PassParams base_pass(const UnrolledArgs& a, const ConsDev& C) {
  PassParams p;
  memset(&p, 0, sizeof(p));
  p.b = (const float2*)a.b;
  p.b_stride = (long long)a.m * a.n;
  p.ld = a.n;
  p.d_stride = (long long)a.m * a.n;
  p.m = a.m;
  p.n = a.n;
  p.lam_dev = a.lams;
  p.alpha = a.opts->alpha;
  p.C = C;
  p.st = nullptr;
  return p;
}

}  // namespace ctv

extern "C" {

size_t ctv_unrolled_workspace_size(int batch, int m, int n, int iters, int ckpt_every) {
  if (batch <= 0 || m <= 0 || n <= 0 || iters < 1 || ckpt_every < 1) return 0;
  return ctv::layout(nullptr, batch, m, n, iters, ckpt_every).bytes;
}

int ctv_unrolled_forward(const void* b, void* x, int batch, int m, int n, const float* lambdas,
                         const ctv_constraint* C, int tv_type, const ctv_opts* opts, int ckpt_every,
                         void* workspace, size_t workspace_bytes, ctv_stream stream) {
  using namespace ctv;
  UnrolledArgs a{b, batch, m, n, lambdas, C, tv_type, opts, ckpt_every, workspace, workspace_bytes};
  ConsDev cons;
  ctv_status st = check_unrolled(a, &cons);
  if (st != CTV_OK) return st;
  if (x == nullptr || ((uintptr_t)x & 7)) return CTV_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int K = opts->max_iters, c = ckpt_every;
  UnrolledLayout L = layout((char*)workspace, batch, m, n, K, c);
  const int cfg = unrolled_config(opts);
  int T = 1;
  config_info(cfg, &T, nullptr, nullptr, nullptr);
  std::vector<double> beta;
  nesterov_betas(K, &beta);
  PassParams p = base_pass(a, cons);
  const dim3 grid = pass_grid(cfg, m, n, batch);
  const long long plane = (long long)(al((size_t)batch * m * n * sizeof(float4)) / sizeof(float4));
  // The passes of the last checkpoint segment run as recompute passes and keep
  // its r_k history (plane j holds r_{k0+2+j}, as the backward walk reads it),
  // so the backward starts walking at once instead of recomputing that segment.
  const int k0_last = ((K + c - 1) / c - 1) * c;
  int k = 1, out = 0;
  const float4* qin = nullptr;
  const float4* rin = nullptr;
  bool first = true;
  while (k <= K) {
    const int steps = std::min(std::min(T, K - k + 1), c - ((k - 1) % c));
    const int kend = k + steps - 1;
    float4* qo;
    float4* ro;
    if (kend == K) { qo = L.finq; ro = L.finr; }
    else if (kend % c == 0) { qo = L.ckq[(size_t)(kend / c)]; ro = L.ckr[(size_t)(kend / c)]; }
    else { qo = L.setq[out]; ro = L.setr[out]; out ^= 1; }
    for (int i = 0; i < 8; ++i) p.beta[i] = i < steps ? (float)beta[(size_t)k + i] : 0.f;
    p.nsteps = steps;
    p.first = first ? 1 : 0;
    p.reverse = p.reverse ^ 1;   // alternate tile order (the previous pass's last tiles are in L2)
    p.q_in = qin;
    p.r_in = rin;
    p.q_out = qo;
    p.r_out = ro;
    if (k > k0_last) {
      if (launch_hist(tv_type, cfg, p, grid, L.hist + (long long)(k - k0_last - 1) * plane, plane, s) != cudaSuccess)
        return CTV_ECUDA;
    } else if (launch_pass(tv_type, cfg, p, grid, s) != cudaSuccess) {
      return CTV_ECUDA;
    }
    count_launch();
    qin = qo;
    rin = ro;
    first = false;
    k = kend + 1;
  }
  // x_K = P_C(b - lam L^T q_K) (Eq. (18)); nobody reads objective terms here
  GapParams g;
  memset(&g, 0, sizeof(g));
  g.b = (const float2*)b;
  g.b_stride = (long long)m * n;
  g.ld = n;
  g.qA = L.finq;
  g.qB = L.finq;
  g.d_stride = (long long)m * n;
  g.default_set = 0;
  g.x = (float2*)x;
  g.x_stride = (long long)m * n;
  g.m = m;
  g.n = n;
  g.lam_dev = lambdas;
  g.alpha = opts->alpha;
  g.C = cons;
  g.iter = K;
  g.final_call = 1;
  if (launch_finalize(g, batch, s) != cudaSuccess) return CTV_ECUDA;
  count_launch();
  return CTV_OK;
}

int ctv_unrolled_backward(const void* b, const void* xbar, void* bbar, float* lambdabar, int batch, int m, int n,
                          const float* lambdas, const ctv_constraint* C, int tv_type, const ctv_opts* opts,
                          int ckpt_every, void* workspace, size_t workspace_bytes, ctv_stream stream) {
  using namespace ctv;
  UnrolledArgs a{b, batch, m, n, lambdas, C, tv_type, opts, ckpt_every, workspace, workspace_bytes};
  ConsDev cons;
  ctv_status st = check_unrolled(a, &cons);
  if (st != CTV_OK) return st;
  if (xbar == nullptr || bbar == nullptr || lambdabar == nullptr) return CTV_EINVAL;
  if (((uintptr_t)xbar & 7) || ((uintptr_t)bbar & 7) || ((uintptr_t)lambdabar & 3)) return CTV_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int K = opts->max_iters, c = ckpt_every;
  UnrolledLayout L = layout((char*)workspace, batch, m, n, K, c);
  const int cfg = unrolled_config(opts);
  int T = 1;
  config_info(cfg, &T, nullptr, nullptr, nullptr);
  std::vector<double> beta;
  nesterov_betas(K, &beta);
  beta.push_back(0.0);   // beta_{K+1} is never used with a nonzero carry
  const long long px = (long long)m * n;
  const long long plane = (long long)(al((size_t)batch * px * sizeof(float4)) / sizeof(float4));
  if (cudaMemsetAsync(L.lamacc, 0, (size_t)batch * sizeof(double), s) != cudaSuccess) return CTV_ECUDA;

  AdjParams ap;
  memset(&ap, 0, sizeof(ap));
  ap.b = (const float2*)b;
  ap.bbar = (float2*)bbar;
  ap.lamacc = L.lamacc;
  ap.px = px;
  ap.m = m;
  ap.n = n;
  ap.lam_dev = lambdas;
  ap.alpha = opts->alpha;
  ap.C = cons;
  ap.xbar = (const float2*)xbar;
  ap.qK = L.finq;
  ap.qbK = L.rb[0];
  if (launch_adj_final(tv_type, ap, batch, s) != cudaSuccess) return CTV_ECUDA;
  count_launch();

  int yi = 0;        // index of the carry buffer (qbar_K first)
  float yc = 1.f;
  int nbi = -1;      // index of rbar_{k+1} (-1: zero)
  PassParams p = base_pass(a, cons);
  const dim3 grid = pass_grid(cfg, m, n, batch);
  const int nseg = (K + c - 1) / c;
  // each segment: recompute it from its checkpoint (storing every r_k), then walk
  // it back; the forward left the history of the last segment in place
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int k0 = sg * c, k1 = std::min(k0 + c, K);
    // recompute iterations k0+1 .. k1-1, keeping r_{k0+2} .. r_{k1}
    const float4* qin = sg == 0 ? nullptr : L.ckq[(size_t)sg];
    const float4* rin = sg == 0 ? nullptr : L.ckr[(size_t)sg];
    bool first = sg == 0;
    int kk = sg == nseg - 1 ? k1 : k0 + 1, out = 0;
    while (kk <= k1 - 1) {
      const int steps = std::min(T, k1 - 1 - kk + 1);
      for (int i = 0; i < 8; ++i) p.beta[i] = i < steps ? (float)beta[(size_t)kk + i] : 0.f;
      p.nsteps = steps;
      p.first = first ? 1 : 0;
      p.reverse = p.reverse ^ 1;   // alternate tile order, as in the forward
      p.q_in = qin;
      p.r_in = rin;
      // the last recompute pass of a segment keeps only its r_k history
      const bool last = kk + steps > k1 - 1;
      p.q_out = last ? nullptr : L.setq[out];
      p.r_out = last ? nullptr : L.setr[out];
      if (launch_hist(tv_type, cfg, p, grid, L.hist + (long long)(kk - k0 - 1) * plane, plane, s) != cudaSuccess)
        return CTV_ECUDA;
      count_launch();
      qin = L.setq[out];
      rin = L.setr[out];
      out ^= 1;
      first = false;
      kk += steps;
    }
    auto r_of = [&](int k) -> const float4* {
      if (k == k0 + 1) return sg == 0 ? nullptr : L.ckr[(size_t)sg];
      return L.hist + (long long)(k - k0 - 2) * plane;
    };
    for (int k = k1; k >= k0 + 1;) {
      int oi = 0;
      while (oi == yi || oi == nbi) ++oi;
      ap.r = r_of(k);
      ap.Y = yi >= 0 ? L.rb[yi] : nullptr;
      ap.yc = yc;
      ap.rbn = nbi >= 0 ? L.rb[nbi] : nullptr;
      ap.rc = (float)(1.0 + beta[(size_t)k]);
      ap.rb_out = L.rb[oi];
      if (CTV_ADJ_PAIR && k - 1 >= k0 + 1) {
        // steps k and k-1 in one pass; the carries of step k-2 are rbar_k and rbar_{k-1}
        int oj = 0;
        while (oj == yi || oj == nbi || oj == oi) ++oj;
        ap.r_lo = r_of(k - 1);
        ap.yc_lo = (float)(-beta[(size_t)k]);
        ap.rc_lo = (float)(1.0 + beta[(size_t)k - 1]);
        ap.rb_out_lo = L.rb[oj];
        if (launch_adj_pair(tv_type, ap, batch, s) != cudaSuccess) return CTV_ECUDA;
        count_launch();
        yi = oi;
        yc = (float)(-beta[(size_t)k - 1]);
        nbi = oj;
        k -= 2;
        continue;
      }
      if (launch_adj_step(tv_type, ap, batch, s) != cudaSuccess) return CTV_ECUDA;
      count_launch();
      // next step k-1: carry = -beta_k rbar_{k+1}, and rbar_k just written
      yi = nbi;
      yc = (float)(-beta[(size_t)k]);
      nbi = oi;
      --k;
    }
  }
  lambar_finish_kernel<<<(batch + 127) / 128, 128, 0, s>>>(L.lamacc, lambdabar, batch);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? CTV_OK : CTV_ECUDA;
}

}  // extern "C"
