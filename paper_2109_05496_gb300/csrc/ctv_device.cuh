// Device building blocks of the fused FGP kernels (Algorithm 2 of Gao & Cao).
//
// Notation follows the paper: L maps an image to its finite differences
// (Eq. (5)/(6)), L^T is its adjoint, P_C projects onto the per-pixel set C
// (Eq. (26) plus a support), P_S projects the dual onto S (Eq. (20), (33),
// (35), (37)). A dual pixel is a float4 (r1, s1, r2, s2) = (Re p1, Im p1,
// Re p2, Im p2); p1 is zero on the last row and p2 on the last column, so the
// paper's edge cases of Eq. (7)-(10), (17), (20), (34) follow from the
// interior formulas.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ctv {

enum { TV1_ISO = 0, TV1_ANISO = 1, TV2_ISO = 2, TV2_ANISO = 3 };

// The per-pixel closed convex set C (a product set, so P_C is pointwise).
struct ConsDev {
  int amp;          // nonzero: |x| <= amax (Eq. (25))
  float amax;
  int sup;          // 0 none, 1 rectangle, 2 mask
  int j0, k0, j1, k1;
  const uint8_t* mask;
  int mask_ld;
  int box;          // nonzero: re_lo <= Re x <= re_hi, im_lo <= Im x <= im_hi
  float re_lo, re_hi, im_lo, im_hi;
};

// Per-image solver record, kept in the caller's workspace.
struct DevStats {
  double acc[4];            // running sums of the gap reduction (fidelity, TV, dual part)
  unsigned int blocks_done; // blocks of the current reduction that have finished
  int stop;                 // set once the gap test has passed
  int stop_set;             // dual buffer set holding q at the stop
  int stop_iter;            // iteration at which the run stopped
  int iters;                // iterations represented by the last evaluation
  int status;               // ctv_status of the image (CTV_ENONFINITE, CTV_EINVAL for a bad lambda)
  unsigned int nonfinite;   // nonzero once an evaluation met a NaN or infinity in b
  double primal, dual, gap; // last evaluation
};

__device__ __forceinline__ float4 f4(float a, float b, float c, float d) { return make_float4(a, b, c, d); }

// Packed FP32x2 arithmetic on (re, im) pairs (one instruction for both halves;
// each half rounds as the scalar operation would).
__device__ __forceinline__ float2 p2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float dot2(float2 a, float2 b) {
  const float2 t = mul2(a, b);
  return t.x + t.y;
}

// Non-finite test of one complex input value (NaN or an infinity in either part).
__device__ __forceinline__ bool nonfinite2(float2 v) { return !(isfinite(v.x) && isfinite(v.y)); }

// FP32 sums that stay accurate without FP64 arithmetic (whose rate on this GPU
// is a small fraction of FP32's). A running sum is a pair (s, c) updated by
// Kahan's compensated addition: s - c is the sum to within an FP32 rounding of
// the result, however many terms were added.
__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// Error-free sum of two floats (Knuth's TwoSum): a + b = s + e exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Warp-wide sum of a value held as an unevaluated pair hi + lo per lane, as a
// pair again (hi the rounded sum, lo its error estimate); valid in lane 0.
__device__ __forceinline__ void warp_sum_pair(float& hi, float& lo) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float oh = __shfl_down_sync(0xffffffffu, hi, off);
    const float ol = __shfl_down_sync(0xffffffffu, lo, off);
    float s, e;
    two_sum(hi, oh, s, e);
    e += lo + ol;
    hi = s + e;              // renormalise: hi + lo = s + e
    lo = e - (hi - s);
  }
}


// (hi, lo) += (h2, l2) for unevaluated FP32 pairs, without rounding loss beyond
// FP32^2 relative.
__device__ __forceinline__ void pair_add(float& hi, float& lo, float h2, float l2) {
  float s, e;
  two_sum(hi, h2, s, e);
  e += lo + l2;
  hi = s + e;
  lo = e - (hi - s);
}

// Block-wide sum of NV values held as FP32 pairs (hi, lo) per thread; the result
// is valid in thread 0. red: shared memory of NV * NT / 32 float2.
template <int NT, int NV>
__device__ __forceinline__ void block_sum_pairs(float (&hi)[NV], float (&lo)[NV], float2* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < NV; ++a) {
    warp_sum_pair(hi[a], lo[a]);
    if (lane == 0) red[a * (NT / 32) + warp] = make_float2(hi[a], lo[a]);
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      const float2 v = lane < NT / 32 ? red[a * (NT / 32) + lane] : make_float2(0.f, 0.f);
      hi[a] = v.x;
      lo[a] = v.y;
      warp_sum_pair(hi[a], lo[a]);
    }
  }
}

// One thread's share of the duality-gap terms of problem (1) at a dual point q
// (App. A): ||x - b||^2, TV(x) and ||b||^2 - ||w||^2 + ||w - P_C(w)||^2 with
// w = b - lam L^T q and x = P_C(w), as FP32 sums s (minus the compensation c of
// the bodies that add many terms per thread), and whether a value of b was a
// NaN or an infinity.
struct GapSums {
  float s[3], c[3];
  bool nf;
};


// P_C: support first (x = 0 outside), then the amplitude bound of Eq. (26),
// x * amax / max{amax, |x|}, or the box on the real and imaginary parts.
__device__ __forceinline__ float2 proj_C(float2 w, int gj, int gk, const ConsDev& c) {
  if (c.sup == 1) {
    if (gj < c.j0 || gj >= c.j1 || gk < c.k0 || gk >= c.k1) return make_float2(0.f, 0.f);
  } else if (c.sup == 2) {
    if (c.mask[(long long)gj * c.mask_ld + gk] == 0) return make_float2(0.f, 0.f);
  }
  if (c.amp) {
    const float a2 = w.x * w.x + w.y * w.y;
    if (a2 > c.amax * c.amax) {
      const float s = c.amax * rsqrtf(a2);
      w.x *= s;
      w.y *= s;
    }
  } else if (c.box) {
    w.x = fminf(fmaxf(w.x, c.re_lo), c.re_hi);
    w.y = fminf(fmaxf(w.y, c.im_lo), c.im_hi);
  }
  return w;
}

// P_S for the four TV types. g = (r1, s1, r2, s2).
#ifndef CTV_BRANCHLESS_PS
#define CTV_BRANCHLESS_PS 1
#endif
#ifndef CTV_PACK8
#define CTV_PACK8 1         // packed FP32x2 arithmetic in the 8-rows-per-thread strip body
#endif


template <int TV>
__device__ __forceinline__ float4 proj_S(float4 g, float alpha) {
#if CTV_BRANCHLESS_PS
  // Same values as below: min{1, radius / |g|} is exactly 1 inside the ball.
  if (TV == TV1_ISO) {
    const float s = fminf(1.f, rsqrtf(g.x * g.x + g.y * g.y + g.z * g.z + g.w * g.w));
    return f4(g.x * s, g.y * s, g.z * s, g.w * s);
  } else if (TV == TV1_ANISO) {
    const float s1 = fminf(1.f, rsqrtf(g.x * g.x + g.y * g.y));
    const float s2 = fminf(1.f, rsqrtf(g.z * g.z + g.w * g.w));
    return f4(g.x * s1, g.y * s1, g.z * s2, g.w * s2);
  } else if (TV == TV2_ISO) {
    const float sr = fminf(1.f, alpha * rsqrtf(g.x * g.x + g.z * g.z));
    const float si = fminf(1.f, (1.f - alpha) * rsqrtf(g.y * g.y + g.w * g.w));
    return f4(g.x * sr, g.y * si, g.z * sr, g.w * si);
  }
#endif
  if (TV == TV1_ISO) {            // Eq. (20): joint 4-vector into the unit ball
    const float nn = g.x * g.x + g.y * g.y + g.z * g.z + g.w * g.w;
    if (nn > 1.f) {
      const float s = rsqrtf(nn);
      g.x *= s; g.y *= s; g.z *= s; g.w *= s;
    }
  } else if (TV == TV1_ANISO) {   // Eq. (33): p1 and p2 into the unit disk separately
    const float n1 = g.x * g.x + g.y * g.y;
    if (n1 > 1.f) { const float s = rsqrtf(n1); g.x *= s; g.y *= s; }
    const float n2 = g.z * g.z + g.w * g.w;
    if (n2 > 1.f) { const float s = rsqrtf(n2); g.z *= s; g.w *= s; }
  } else if (TV == TV2_ISO) {     // Eq. (35): (r1, r2) into radius alpha, (s1, s2) into 1 - alpha
    const float a = alpha, c = 1.f - alpha;
    const float nr = g.x * g.x + g.z * g.z;
    if (nr > a * a) { const float s = a * rsqrtf(nr); g.x *= s; g.z *= s; }
    const float ns = g.y * g.y + g.w * g.w;
    if (ns > c * c) { const float s = c * rsqrtf(ns); g.y *= s; g.w *= s; }
  } else {                        // Eq. (37): componentwise clamps
    const float a = alpha, c = 1.f - alpha;
    g.x = fminf(fmaxf(g.x, -a), a);
    g.z = fminf(fmaxf(g.z, -a), a);
    g.y = fminf(fmaxf(g.y, -c), c);
    g.w = fminf(fmaxf(g.w, -c), c);
  }
  return g;
}

// One pixel's share of TV(x) given its two differences d1 = x[j,k] - x[j+1,k]
// and d2 = x[j,k] - x[j,k+1] (zero where the paper has no such difference):
// the summand of Eq. (7), (8), (9) or (10).
template <int TV>
__device__ __forceinline__ float tv_term(float d1r, float d1i, float d2r, float d2i, float alpha) {
  if (TV == TV1_ISO) return sqrtf(d1r * d1r + d1i * d1i + d2r * d2r + d2i * d2i);
  if (TV == TV1_ANISO) return sqrtf(d1r * d1r + d1i * d1i) + sqrtf(d2r * d2r + d2i * d2i);
  if (TV == TV2_ISO) return alpha * sqrtf(d1r * d1r + d2r * d2r) + (1.f - alpha) * sqrtf(d1i * d1i + d2i * d2i);
  return alpha * (fabsf(d1r) + fabsf(d2r)) + (1.f - alpha) * (fabsf(d1i) + fabsf(d2i));
}

// Everything one pass over one image needs.
struct Img {
  const float2* b;      // complex64, row stride ld
  int ld;
  const float4* q_in;   // q_{k-1}, dense m x n
  const float4* r_in;   // r_k
  float4* q_out;        // q_{k+T-1}
  float4* r_out;        // r_{k+T}
  int m, n;
  float lam, alpha;
  ConsDev C;
  float4* r_hist;         // HIST variants: r after inner step it goes to r_hist + it * hist_plane
  long long hist_plane;
};

// T iterations of Algorithm 2 on one tile, temporally blocked in shared memory.
//
// The block loads the dual state and b for an RW x RH region whose interior
// ((RW - 2T) x (RH - 2T) pixels starting at image pixel (j0, k0)) it owns, and
// then runs nsteps <= T iterations of
//     phase 1:  x = P_C(b - lam L^T r)                 (reads r at self, up, left)
//     phase 2:  q = P_S(r + L x / (8 lam))             (reads x at self, down, right)
//               r' = q + beta_k (q - q_prev)            (Alg. 2, steps 3-5)
// Each iteration invalidates one more ring of the region, so after T steps
// exactly the interior is correct, and only the interior is written back.
// Pixels outside the image hold r = x = 0, which is the boundary condition of
// Eq. (5)/(6). q and b live in registers (each thread owns PPT pixels), r and
// x in shared memory for the neighbours.
template <int TV, int T, int RW, int RH, int NT, bool HIST = false>
__device__ __forceinline__ void fgp_tile(const Img& I, int j0, int k0, const float* beta,
                                         int nsteps, bool first) {
  constexpr int R = RW * RH;
  constexpr int PPT = R / NT;
  static_assert(R % NT == 0, "region must split evenly over the threads");
  extern __shared__ float4 smem4[];
  float4* rs = smem4;
  float2* xs = reinterpret_cast<float2*>(smem4 + R);
  const int tid = threadIdx.x;
  const int gj0 = j0 - T, gk0 = k0 - T;
  const float4 z4 = f4(0.f, 0.f, 0.f, 0.f);

  float4 qreg[PPT];
  float2 breg[PPT];
#pragma unroll
  for (int s = 0; s < PPT; ++s) {
    const int i = tid + s * NT;
    const int lj = i / RW, lk = i % RW;
    const int gj = gj0 + lj, gk = gk0 + lk;
    float4 q = z4, r = z4;
    float2 bb = make_float2(0.f, 0.f);
    if ((unsigned)gj < (unsigned)I.m && (unsigned)gk < (unsigned)I.n) {
      bb = __ldg(I.b + (long long)gj * I.ld + gk);
      if (!first) {
        const long long o = (long long)gj * I.n + gk;
        q = __ldg(I.q_in + o);
        r = __ldg(I.r_in + o);
      }
    }
    qreg[s] = q;
    breg[s] = bb;
    rs[i] = r;
  }
  __syncthreads();

  const float lam = I.lam;
  // 1/(16 lam^2) times the 2 lam of Eq. (19); lam = 0 leaves q = 0 and x = P_C(b)
  const float c8 = lam > 0.f ? 1.f / (8.f * lam) : 0.f;
  for (int it = 0; it < nsteps; ++it) {
#pragma unroll
    for (int s = 0; s < PPT; ++s) {
      const int i = tid + s * NT;
      const int lj = i / RW, lk = i % RW;
      const int gj = gj0 + lj, gk = gk0 + lk;
      float2 xv = make_float2(0.f, 0.f);
      if ((unsigned)gj < (unsigned)I.m && (unsigned)gk < (unsigned)I.n) {
        const float4 rc = rs[i];
        const float4 ru = lj > 0 ? rs[i - RW] : z4;
        const float4 rl = lk > 0 ? rs[i - 1] : z4;
        // (L^T p)[j,k] = p1[j,k] - p1[j-1,k] + p2[j,k] - p2[j,k-1]
        const float dre = rc.x - ru.x + rc.z - rl.z;
        const float dim = rc.y - ru.y + rc.w - rl.w;
        xv = proj_C(make_float2(breg[s].x - lam * dre, breg[s].y - lam * dim), gj, gk, I.C);
      }
      xs[i] = xv;
    }
    __syncthreads();
    const float bt = beta[it];
#pragma unroll
    for (int s = 0; s < PPT; ++s) {
      const int i = tid + s * NT;
      const int lj = i / RW, lk = i % RW;
      const int gj = gj0 + lj, gk = gk0 + lk;
      if ((unsigned)gj < (unsigned)I.m && (unsigned)gk < (unsigned)I.n) {
        const float2 xc = xs[i];
        float d1r = 0.f, d1i = 0.f, d2r = 0.f, d2i = 0.f;
        if (gj < I.m - 1 && lj < RH - 1) { const float2 xd = xs[i + RW]; d1r = xc.x - xd.x; d1i = xc.y - xd.y; }
        if (gk < I.n - 1 && lk < RW - 1) { const float2 xr = xs[i + 1]; d2r = xc.x - xr.x; d2i = xc.y - xr.y; }
        const float4 rc = rs[i];
        const float4 qn = proj_S<TV>(f4(rc.x + c8 * d1r, rc.y + c8 * d1i, rc.z + c8 * d2r, rc.w + c8 * d2i), I.alpha);
        const float4 qo = qreg[s];
        const float4 rn = f4(qn.x + bt * (qn.x - qo.x), qn.y + bt * (qn.y - qo.y),
                             qn.z + bt * (qn.z - qo.z), qn.w + bt * (qn.w - qo.w));
        rs[i] = rn;
        qreg[s] = qn;
        if (HIST && lj >= T && lj < RH - T && lk >= T && lk < RW - T)
          I.r_hist[it * I.hist_plane + (long long)gj * I.n + gk] = rn;
      }
    }
    __syncthreads();
  }

#pragma unroll
  for (int s = 0; s < PPT; ++s) {
    const int i = tid + s * NT;
    const int lj = i / RW, lk = i % RW;
    const int gj = gj0 + lj, gk = gk0 + lk;
    if ((!HIST || I.q_out != nullptr) && lj >= T && lj < RH - T && lk >= T && lk < RW - T &&
        (unsigned)gj < (unsigned)I.m && (unsigned)gk < (unsigned)I.n) {
      const long long o = (long long)gj * I.n + gk;
      I.q_out[o] = qreg[s];
      I.r_out[o] = rs[i];
    }
  }
}

// Constraint specialisations of P_C for the column-strip kernel.
enum { CONS_NONE = 0, CONS_AMP = 1, CONS_RECT = 2, CONS_GEN = 3 };

__device__ __forceinline__ float2 proj_amp(float2 w, float amax) {
  const float a2 = w.x * w.x + w.y * w.y;
  if (a2 > amax * amax) {
    const float s = amax * rsqrtf(a2);
    w.x *= s;
    w.y *= s;
  }
  return w;
}

// CONS_RECT: amplitude bound (if any) plus a support rectangle; kin says whether
// the pixel's column lies inside the rectangle.
template <int CONS>
__device__ __forceinline__ float2 proj_C_t(float2 w, int gj, int gk, bool kin, const ConsDev& c) {
  if (CONS == CONS_NONE) return w;
  if (CONS == CONS_AMP) return proj_amp(w, c.amax);
  if (CONS == CONS_RECT) {
    if (!kin || gj < c.j0 || gj >= c.j1) return make_float2(0.f, 0.f);
    return c.amp ? proj_amp(w, c.amax) : w;
  }
  return proj_C(w, gj, gk, c);
}

// T iterations of Algorithm 2 on one tile, with column-strip ownership.
//
// Same contract as fgp_tile (an RW x RH region with a T-pixel halo, only the
// interior written back), but each thread owns PPT vertically consecutive pixels
// of one column: a warp covers 32 adjacent columns, WX warps side by side and WY
// warps stacked give RW = 32 WX and RH = PPT WY. q, r and the transient x of the
// owned pixels stay in registers, so the vertical neighbours of the stencil
// (r above for L^T, x below for L) come from registers except at the ends of
// a strip. Shared memory holds what other threads need - p2 = (r2, s2) of every
// pixel (left neighbour of L^T), x of every pixel (right and, at strip ends,
// lower neighbour of L), p1 = (r1, s1) of each strip's last row (upper
// neighbour of the next strip) - and b.
// EDGE = false is the fast path for regions that lie inside the image away
// from its last row and column: no per-pixel bounds or edge tests.
// GAPEV: the pass ends a check interval (nsteps <= T - 1) and also adds the
// block's share of the duality-gap terms at the final q into gs (see below).
template <int TV, int T, int WX, int WY, int PPT, bool HIST, bool EDGE, int CONS, bool GAPEV = false>
__device__ __forceinline__ void fgp_strip_body(const Img& I, int j0, int k0, const float* beta, int nsteps,
                                               bool first, GapSums* gs = nullptr) {
  constexpr int RW = 32 * WX, RH = PPT * WY, R = RW * RH;
  extern __shared__ float4 smem4[];
  float2* P2 = reinterpret_cast<float2*>(smem4);      // R
  float2* X = P2 + R;                                  // R
  float2* Bs = X + R;                                  // R
  float2* P1B = Bs + R;                                // WY * RW
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int wx = warp % WX, wy = warp / WX;
  const int lk = wx * 32 + lane;
  const int lj0 = wy * PPT;
  const int gk = k0 - T + lk;
  const int gj0 = j0 - T + lj0;
  const bool colin = !EDGE || (unsigned)gk < (unsigned)I.n;
  const bool kin = gk >= I.C.k0 && gk < I.C.k1;
  const float4 z4 = f4(0.f, 0.f, 0.f, 0.f);
  const float2 z2 = make_float2(0.f, 0.f);

  float4 q[PPT], r[PPT];
  float2 x[PPT];
#pragma unroll
  for (int s = 0; s < PPT; ++s) {
    const int gj = gj0 + s;
    q[s] = z4;
    r[s] = z4;
    float2 bb = z2;
    if (colin && (!EDGE || (unsigned)gj < (unsigned)I.m)) {
      const long long o = (long long)gj * I.n + gk;
      if (!first) {
        q[s] = __ldg(I.q_in + o);
        r[s] = __ldg(I.r_in + o);
      }
      bb = __ldg(I.b + (long long)gj * I.ld + gk);
    }
    P2[(lj0 + s) * RW + lk] = make_float2(r[s].z, r[s].w);
    Bs[(lj0 + s) * RW + lk] = bb;
  }
  P1B[wy * RW + lk] = make_float2(r[PPT - 1].x, r[PPT - 1].y);
  __syncthreads();

  const float lam = I.lam;
  const float c8 = lam > 0.f ? 1.f / (8.f * lam) : 0.f;
  const bool has_right = lk < RW - 1 && (!EDGE || (gk >= 0 && gk < I.n - 1));
  const bool strip_bottom_in = lj0 + PPT < RH;
  // Pixels outside the image start at b = q = r = 0 and stay there when their
  // forward differences are masked (rows j < 0 or j >= m - 1 have no d1,
  // columns k < 0 or k >= n - 1 no d2) and P_C(0) = 0: then L^T r and hence x
  // vanish there. That holds for no constraint, the amplitude bound and the
  // support rectangle, so their edge path needs no per-pixel image test in
  // the iterations; the general constraint (mask, box) keeps the tests.
  constexpr bool TESTS = EDGE && CONS == CONS_GEN;
  // Eight rows per thread (a 128-register budget) take the complex halves
  // through packed FP32x2 instructions, associated as the scalar form so the
  // results are the same bits. Measured against the scalar form: T = 6 (config
  // 5) +1.0% at 2048^2, +2.4% at 1024^2, +5.4% on a plan of 512 images; T = 8
  // (config 6) -1.7% at 2048^2; recompute tiles spilled. Under the 64-register
  // budgets of the other configurations the register pairs cost more than they
  // save (config 11 and 14: 167 / 164 -> 144 / 139 Gpixel-iter/s).
  constexpr bool PACK = CTV_PACK8 && PPT == 8 && T <= 6 && !HIST;
  // Rows whose values can still reach the interior after the remaining steps:
  // step it must produce q, r on rows [lo, RH - lo) and x on one more row, with
  // lo = T - (nsteps - 1 - it). With few rows per thread the rows outside are
  // skipped (a warp-uniform test, since a warp's rows share lj0); with PPT = 8
  // the per-row branches cost more instruction-level parallelism than the
  // skipped rows save. (Running the tests only in the warps whose rows reach
  // the top or bottom T rows of the region, with a test-free copy of the row
  // loop for the others, raised the register count past the 64 that two
  // blocks per SM allow.)
  constexpr bool SKIP_ROWS = PPT <= 4;
  // The row tests are the same in every lane of a warp (its rows share lj0);
  // taking them through a warp vote lets the compiler branch on them as uniform
  // (control instructions per pixel-iteration 7.5 -> 1.3, +1% at 2048^2).
#define CTV_ROW_SKIP(cond) __all_sync(0xffffffffu, (cond))

  // With two or four rows per thread the step loop is unrolled (nsteps <= T):
  // the loop-carried registers need no copies between steps. With eight rows
  // the unrolled steps need more than the 128 registers a thread may have
  // (spills), and with one row (1024-thread blocks of small images) it was
  // measured slower, so those keep the loop; so do recompute tiles (HIST),
  // whose per-step history stores made the unrolled loop spill at 64 registers.
  constexpr int STEP_UNROLL = (!HIST && (PPT == 2 || PPT == 4)) ? T : 1;
#pragma unroll STEP_UNROLL
  for (int it = 0; it < T; ++it) {
    if (it >= nsteps) break;
    // (a pass that evaluates the gap afterwards keeps one more ring of rows exact)
    const int lo = SKIP_ROWS ? T - (GAPEV ? 1 : 0) - (nsteps - 1 - it) : 0;
    const int hi = SKIP_ROWS ? RH - lo : RH;
    // phase 1: x = P_C(b - lam L^T r)
#pragma unroll
    for (int s = 0; s < PPT; ++s) {
      const int gj = gj0 + s;
      if (SKIP_ROWS && CTV_ROW_SKIP(lj0 + s < lo || lj0 + s > hi)) continue;
      x[s] = z2;
      if (!TESTS || (colin && (unsigned)gj < (unsigned)I.m)) {
        float2 up;
        if (s > 0) up = make_float2(r[s - 1].x, r[s - 1].y);
        else up = wy > 0 ? P1B[(wy - 1) * RW + lk] : z2;
        const float2 left = lk > 0 ? P2[(lj0 + s) * RW + lk - 1] : z2;
        const float2 bb = Bs[(lj0 + s) * RW + lk];
        // (L^T p)[j,k] = p1[j,k] - p1[j-1,k] + p2[j,k] - p2[j,k-1]
        if constexpr (PACK) {
          const float2 d = sub2(add2(sub2(lo2(r[s]), up), hi2(r[s])), left);
          x[s] = proj_C_t<CONS>(fma2(p2(-lam), d, bb), gj, gk, kin, I.C);
        } else {
          const float dre = r[s].x - up.x + r[s].z - left.x;
          const float dim = r[s].y - up.y + r[s].w - left.y;
          x[s] = proj_C_t<CONS>(make_float2(bb.x - lam * dre, bb.y - lam * dim), gj, gk, kin, I.C);
        }
      }
      X[(lj0 + s) * RW + lk] = x[s];
    }
    __syncthreads();
    // phase 2: q = P_S(r + L x / (8 lam)), r' = q + beta (q - q_prev)
    const float bt = beta[it];
#pragma unroll
    for (int s = 0; s < PPT; ++s) {
      const int gj = gj0 + s;
      if (SKIP_ROWS && CTV_ROW_SKIP(lj0 + s < lo || lj0 + s >= hi)) continue;
      if (!TESTS || (colin && (unsigned)gj < (unsigned)I.m)) {
        float2 e1 = z2, e2 = z2;   // (L x)[j,k]: x[j,k] - x[j+1,k] and x[j,k] - x[j,k+1]
        if (!EDGE || (gj >= 0 && gj < I.m - 1)) {
          float2 xd;
          if (s < PPT - 1) xd = x[s + 1];
          else xd = strip_bottom_in ? X[(lj0 + s + 1) * RW + lk] : x[s];
          e1 = PACK ? sub2(x[s], xd) : make_float2(x[s].x - xd.x, x[s].y - xd.y);
        }
        if (has_right) {
          const float2 xr = X[(lj0 + s) * RW + lk + 1];
          e2 = PACK ? sub2(x[s], xr) : make_float2(x[s].x - xr.x, x[s].y - xr.y);
        }
        if constexpr (PACK) {
          const float2 g1 = fma2(p2(c8), e1, lo2(r[s]));
          const float2 g2 = fma2(p2(c8), e2, hi2(r[s]));
          const float4 qn = proj_S<TV>(f4(g1.x, g1.y, g2.x, g2.y), I.alpha);
          const float2 n1 = fma2(p2(bt), sub2(lo2(qn), lo2(q[s])), lo2(qn));
          const float2 n2 = fma2(p2(bt), sub2(hi2(qn), hi2(q[s])), hi2(qn));
          r[s] = f4(n1.x, n1.y, n2.x, n2.y);
          q[s] = qn;
        } else {
          const float4 qn = proj_S<TV>(
              f4(r[s].x + c8 * e1.x, r[s].y + c8 * e1.y, r[s].z + c8 * e2.x, r[s].w + c8 * e2.y), I.alpha);
          r[s] = f4(qn.x + bt * (qn.x - q[s].x), qn.y + bt * (qn.y - q[s].y),
                    qn.z + bt * (qn.z - q[s].z), qn.w + bt * (qn.w - q[s].w));
          q[s] = qn;
        }
        if (HIST && lk >= T && lk < RW - T && lj0 + s >= T && lj0 + s < RH - T &&
            (!EDGE || (colin && (unsigned)gj < (unsigned)I.m)))
          I.r_hist[it * I.hist_plane + (long long)gj * I.n + gk] = r[s];
      }
      P2[(lj0 + s) * RW + lk] = make_float2(r[s].z, r[s].w);
    }
    P1B[wy * RW + lk] = make_float2(r[PPT - 1].x, r[PPT - 1].y);
    __syncthreads();
  }
#undef CTV_ROW_SKIP

  // (a recompute pass whose final state nobody reads passes q_out = nullptr)
  if ((!HIST || I.q_out != nullptr) && lk >= T && lk < RW - T && colin) {
#pragma unroll
    for (int s = 0; s < PPT; ++s) {
      const int lj = lj0 + s, gj = gj0 + s;
      if (lj >= T && lj < RH - T && (!EDGE || (unsigned)gj < (unsigned)I.m)) {
        const long long o = (long long)gj * I.n + gk;
        I.q_out[o] = q[s];
        I.r_out[o] = r[s];
      }
    }
  }

  if constexpr (GAPEV) {
    // The duality-gap terms at q_k (the final q of this pass) on the interior,
    // from the state the block holds. After nsteps <= T - 1 steps q_k is exact on
    // the interior and one ring around it, which is all that x = P_C(b - lam L^T
    // q_k) (Eq. (18)) on the interior and on its lower and right neighbours needs.
    // The last step ended with a barrier, so p2 and p1 of q_k may replace r's.
#pragma unroll
    for (int s = 0; s < PPT; ++s) P2[(lj0 + s) * RW + lk] = make_float2(q[s].z, q[s].w);
    P1B[wy * RW + lk] = make_float2(q[PPT - 1].x, q[PPT - 1].y);
    __syncthreads();
    const bool colint = lk >= T && lk < RW - T && colin;
#pragma unroll
    for (int s = 0; s < PPT; ++s) {
      const int lj = lj0 + s, gj = gj0 + s;
      // the terms read x on the interior rows and the row below them
      if (SKIP_ROWS && (lj < T || lj > RH - T)) continue;
      x[s] = z2;
      if (!TESTS || (colin && (unsigned)gj < (unsigned)I.m)) {
        float2 up;
        if (s > 0) up = make_float2(q[s - 1].x, q[s - 1].y);
        else up = wy > 0 ? P1B[(wy - 1) * RW + lk] : z2;
        const float2 left = lk > 0 ? P2[(lj0 + s) * RW + lk - 1] : z2;
        const float tr = q[s].x - up.x + q[s].z - left.x, ti = q[s].y - up.y + q[s].w - left.y;
        const float2 bb = Bs[(lj0 + s) * RW + lk];
        x[s] = proj_C_t<CONS>(make_float2(fmaf(-lam, tr, bb.x), fmaf(-lam, ti, bb.y)), gj, gk, kin, I.C);
        if (colint && lj >= T && lj < RH - T && (!EDGE || (unsigned)gj < (unsigned)I.m)) {
          gs->nf |= nonfinite2(bb);
          const float er = x[s].x - bb.x, ei = x[s].y - bb.y;
          gs->s[0] += er * er + ei * ei;
          // ||b||^2 - ||w||^2 = 2 <b, lam L^T q> - ||lam L^T q||^2, plus ||w - P_C(w)||^2
          const float dlr = lam * tr, dli = lam * ti;
          const float hr = (bb.x - dlr) - x[s].x, hi = (bb.y - dli) - x[s].y;
          gs->s[2] += (2.f * (bb.x * dlr + bb.y * dli) - (dlr * dlr + dli * dli)) + (hr * hr + hi * hi);
        }
      }
      X[(lj0 + s) * RW + lk] = x[s];
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < PPT; ++s) {
      const int lj = lj0 + s, gj = gj0 + s;
      if (colint && lj >= T && lj < RH - T && (!EDGE || (unsigned)gj < (unsigned)I.m)) {
        // interior rows end T rows above the region's last row, so the lower
        // neighbour is in the region
        const float2 xd = s < PPT - 1 ? x[s + 1] : X[(lj0 + s + 1) * RW + lk];
        const float2 xr = X[(lj0 + s) * RW + lk + 1];
        const bool d1 = !EDGE || gj < I.m - 1, d2 = !EDGE || gk < I.n - 1;
        gs->s[1] += tv_term<TV>(d1 ? x[s].x - xd.x : 0.f, d1 ? x[s].y - xd.y : 0.f, d2 ? x[s].x - xr.x : 0.f,
                                d2 ? x[s].y - xr.y : 0.f, I.alpha);
      }
    }
  }
}

// T iterations on a tile whose whole region lies outside the support of C, so
// that x = P_C(.) = 0 on every pixel of the region: L x vanishes and each step
// reduces to q = P_S(r), r' = q + beta (q - q_prev) pixel by pixel (the same
// values the general body computes there). No neighbour is read, so the block
// needs neither shared memory nor barriers, reads no b, and updates only the
// interior pixels it owns.
template <int TV, int T, int WX, int WY, int PPT, bool HIST, bool GAPEV = false>
__device__ __forceinline__ void fgp_strip_zero(const Img& I, int j0, int k0, const float* beta, int nsteps,
                                               bool first, GapSums* gs = nullptr) {
  constexpr int RW = 32 * WX, RH = PPT * WY;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int wx = warp % WX, wy = warp / WX;
  const int lk = wx * 32 + lane;
  const int lj0 = wy * PPT;
  const int gk = k0 - T + lk;
  const int gj0 = j0 - T + lj0;
  if (lk < T || lk >= RW - T || (unsigned)gk >= (unsigned)I.n) return;
  const float4 z4 = f4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int s = 0; s < PPT; ++s) {
    const int lj = lj0 + s, gj = gj0 + s;
    if (lj < T || lj >= RH - T || (unsigned)gj >= (unsigned)I.m) continue;
    const long long o = (long long)gj * I.n + gk;
    float4 q = z4, r = z4;
    if (!first) {
      q = __ldg(I.q_in + o);
      r = __ldg(I.r_in + o);
    }
    for (int it = 0; it < nsteps; ++it) {
      const float bt = beta[it];
      const float4 qn = proj_S<TV>(r, I.alpha);
      r = f4(qn.x + bt * (qn.x - q.x), qn.y + bt * (qn.y - q.y), qn.z + bt * (qn.z - q.z), qn.w + bt * (qn.w - q.w));
      q = qn;
      if (HIST) I.r_hist[it * I.hist_plane + o] = r;
    }
    if (!HIST || I.q_out != nullptr) {
      I.q_out[o] = q;
      I.r_out[o] = r;
    }
    if constexpr (GAPEV) {
      // x = 0 here and at every neighbour: TV(x) adds nothing, ||x - b||^2 = ||b||^2,
      // and w - P_C(w) = w turns the dual part into ||b||^2 as well
      const float2 bb = __ldg(I.b + (long long)gj * I.ld + gk);
      gs->nf |= nonfinite2(bb);
      const float b2 = bb.x * bb.x + bb.y * bb.y;
      gs->s[0] += b2;
      gs->s[2] += b2;
    }
  }
}

// Block-level choice between the bodies: for a support rectangle, a region
// entirely outside it takes the neighbour-free body and a region entirely inside
// it (and inside the image) the amplitude-only (or unconstrained) fast path; a
// region inside the image away from its last row and column takes the body
// without edge tests.
template <int TV, int T, int WX, int WY, int PPT, bool HIST, int CONS, bool GAPEV = false>
__device__ __forceinline__ void fgp_strip_tile(const Img& I, int j0, int k0, const float* beta, int nsteps,
                                               bool first, GapSums* gs = nullptr) {
  constexpr int RW = 32 * WX, RH = PPT * WY;
  const int gj0 = j0 - T, gk0 = k0 - T;
  const bool inside = gj0 >= 0 && gk0 >= 0 && gj0 + RH <= I.m - 1 && gk0 + RW <= I.n - 1;
  if constexpr (CONS == CONS_RECT) {
    const ConsDev& c = I.C;
    if (gj0 + RH <= c.j0 || gj0 >= c.j1 || gk0 + RW <= c.k0 || gk0 >= c.k1) {
      fgp_strip_zero<TV, T, WX, WY, PPT, HIST, GAPEV>(I, j0, k0, beta, nsteps, first, gs);
      return;
    }
    if (inside && gj0 >= c.j0 && gj0 + RH <= c.j1 && gk0 >= c.k0 && gk0 + RW <= c.k1) {
      if (c.amp) fgp_strip_body<TV, T, WX, WY, PPT, HIST, false, CONS_AMP, GAPEV>(I, j0, k0, beta, nsteps, first, gs);
      else fgp_strip_body<TV, T, WX, WY, PPT, HIST, false, CONS_NONE, GAPEV>(I, j0, k0, beta, nsteps, first, gs);
      return;
    }
  }
  if (inside) fgp_strip_body<TV, T, WX, WY, PPT, HIST, false, CONS, GAPEV>(I, j0, k0, beta, nsteps, first, gs);
  else fgp_strip_body<TV, T, WX, WY, PPT, HIST, true, CONS, GAPEV>(I, j0, k0, beta, nsteps, first, gs);
}

// Block-wide FP64 sum of NV values; the result is valid in thread 0.
template <int NT, int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* red /* smem, NV * NT/32 */) {
#pragma unroll
  for (int a = 0; a < NV; ++a) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[a] += __shfl_down_sync(0xffffffffu, v[a], off);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) red[a * (NT / 32) + warp] = v[a];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      double t = lane < NT / 32 ? red[a * (NT / 32) + lane] : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
      v[a] = t;
    }
  }
}

}  // namespace ctv
