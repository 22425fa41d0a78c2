// Phase retrieval, problem (24), by FISTA (Algorithm 1) with the FGP prox.
//
// Forward operator (Sec. V-A, Eq. (23)) on a zero-padded M x N grid:
//     A = crop o IFFT2 o (H *) o FFT2 o pad,      A^* = crop o IFFT2 o (conj(H) *) o FFT2 o pad
// with the object in the top-left m x n corner. cuFFT does the transforms
// (unnormalised; the 1/(MN) of the inverse is folded into the kernels that
// read its output). Hand-written kernels:
//   pr_mul_h      F *= H or conj(H), two complex values per 16-byte access
//   pr_residual   xi = A z (cropped, scaled); g = (xi/|xi|)(|xi| - sqrt(y)) written into
//                 the zero-padded buffer for the adjoint, and 1/2 sum (|xi| - sqrt(y))^2
//                 reduced in FP64 (Eq. (24), (27); xi/|xi| := 1 at xi = 0)
//   pr_form_v     v = z - gamma grad F(z)           (Alg. 1, step 3, gradient at z_k)
//   pr_fista      z_{k+1} = x_k + ((t_k - 1)/t_{k+1})(x_k - x_{k-1})   (Alg. 1, steps 4-5),
//                 written straight into the padded buffer; when the inner solve ends
//                 with the x-only finalize (no gap checks), that kernel forms z_{k+1}
//                 in the same pass over x instead (same arithmetic, one launch less)
// The prox of gamma (tau TV + I_C) is problem (15) with lam = tau gamma, solved by
// the fused FGP path, warm-started from the previous outer iteration's dual.
#include <cuda_runtime.h>
#include <cufft.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "async_status.cuh"
#include "ctv_device.cuh"
#include "ctv_host.h"

namespace ctv {

__global__ void pr_mul_h(float4* __restrict__ F, const float4* __restrict__ H, long long n2, int conj_h) {
  // n2 = number of complex pairs (M*N/2)
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
    const float4 f = F[i];
    float4 h = __ldg(H + i);
    if (conj_h) { h.y = -h.y; h.w = -h.w; }
    F[i] = make_float4(f.x * h.x - f.y * h.y, f.x * h.y + f.y * h.x,
                       f.z * h.z - f.w * h.w, f.z * h.w + f.w * h.z);
  }
}

__global__ void pr_mul_h_scalar(float2* __restrict__ F, const float2* __restrict__ H, long long n1, int conj_h) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n1; i += (long long)gridDim.x * blockDim.x) {
    const float2 f = F[i];
    float2 h = __ldg(H + i);
    if (conj_h) h.y = -h.y;
    F[i] = make_float2(f.x * h.x - f.y * h.y, f.x * h.y + f.y * h.x);
  }
}

constexpr int PR_NT = 256;

// grid: (ceil(n / PR_NT), m); one thread per pixel of the m x n crop.
__global__ void __launch_bounds__(PR_NT) pr_residual(const float2* __restrict__ F, int ldF, int m, int n, float inv_mn,
                                                     const float* __restrict__ sqrt_y, int ldy,
                                                     float2* __restrict__ Q, int ldQ, double* loss) {
  __shared__ double red[PR_NT / 32];
  const int j = blockIdx.y, k = blockIdx.x * PR_NT + threadIdx.x;
  double l = 0.0;
  bool nf = false;
  if (k < n) {
    const float2 f = F[(long long)j * ldF + k];
    const float xr = f.x * inv_mn, xi = f.y * inv_mn;
    const float a = sqrtf(xr * xr + xi * xi);
    const float sy = __ldg(sqrt_y + (long long)j * ldy + k);
    // a NaN or infinity in z, H or sqrt(y) reaches this point as a non-finite field or amplitude
    nf = !(isfinite(a) && isfinite(sy));
    const float d = a - sy;
    float ur = 1.f, ui = 0.f;
    if (a > 0.f) { ur = xr / a; ui = xi / a; }
    Q[(long long)j * ldQ + k] = make_float2(ur * d, ui * d);
    l = 0.5 * (double)d * (double)d;
  }
  if (__any_sync(0xffffffffu, nf) && (threadIdx.x & 31) == 0) raise_async(CTV_ENONFINITE);
  if (loss == nullptr) return;
  double v[1] = {l};
  __syncthreads();
  block_sum<PR_NT, 1>(v, red);
  if (threadIdx.x == 0) atomicAdd(loss, v[0]);
}

// v = z - gamma * inv_mn * F (crop); z in the padded buffer P.
__global__ void pr_form_v(const float2* __restrict__ P, int ldP, const float2* __restrict__ F, int ldF, float scale,
                          float2* __restrict__ V, int ldV, int m, int n) {
  const int j = blockIdx.y, k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float2 z = P[(long long)j * ldP + k];
  const float2 g = F[(long long)j * ldF + k];
  V[(long long)j * ldV + k] = make_float2(z.x - scale * g.x, z.y - scale * g.y);
}

// gradient output: grad = inv_mn * F (crop)
__global__ void pr_crop_scale(const float2* __restrict__ F, int ldF, float scale, float2* __restrict__ G, int ldG, int m, int n) {
  const int j = blockIdx.y, k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float2 g = F[(long long)j * ldF + k];
  G[(long long)j * ldG + k] = make_float2(scale * g.x, scale * g.y);
}

// dst (crop) = src
__global__ void pr_copy(const float2* __restrict__ S, int ldS, float2* __restrict__ D, int ldD, int m, int n) {
  const int j = blockIdx.y, k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  D[(long long)j * ldD + k] = S[(long long)j * ldS + k];
}

// z = x + beta (x - x_prev), written into the padded buffer (Alg. 1, step 5).
__global__ void pr_fista(const float2* __restrict__ X, const float2* __restrict__ Xp, int ldX, float beta,
                         float2* __restrict__ Z, int ldZ, int m, int n) {
  const int j = blockIdx.y, k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float2 x = X[(long long)j * ldX + k];
  const float2 xp = Xp[(long long)j * ldX + k];
  Z[(long long)j * ldZ + k] = make_float2(fmaf(beta, x.x - xp.x, x.x), fmaf(beta, x.y - xp.y, x.y));
}

// Sufficient-decrease terms of the backtracking line search:
// acc[0] += <x - z, g> (real-pair inner product), acc[1] += ||x - z||^2.
__global__ void __launch_bounds__(PR_NT) pr_ls_terms(const float2* __restrict__ X, int ldX, const float2* __restrict__ Z,
                                                     int ldZ, const float2* __restrict__ G, int ldG, int m, int n,
                                                     double* acc) {
  __shared__ double red[2 * (PR_NT / 32)];
  const int j = blockIdx.y, k = blockIdx.x * PR_NT + threadIdx.x;
  double v[2] = {0.0, 0.0};
  if (k < n) {
    const float2 x = X[(long long)j * ldX + k];
    const float2 z = Z[(long long)j * ldZ + k];
    const float2 g = G[(long long)j * ldG + k];
    const float dx = x.x - z.x, dy = x.y - z.y;
    v[0] = (double)(dx * g.x + dy * g.y);
    v[1] = (double)(dx * dx + dy * dy);
  }
  block_sum<PR_NT, 2>(v, red);
  if (threadIdx.x == 0) {
    atomicAdd(acc, v[0]);
    atomicAdd(acc + 1, v[1]);
  }
}

static size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

int take_async_status_pr() { return take_unit_async_status(); }

}  // namespace ctv

struct ctv_pr_plan {
  int m, n, M, N;
  // The 2-D transforms of the M x N field run as 1-D passes: row transforms
  // of only the m rows that hold the object (the others are zero on input,
  // or not needed on output), and column transforms of every column.
  cufftHandle fft_rows;   // m rows of length N, contiguous
  cufftHandle fft_cols;   // N columns of length M, stride N
  char* base;        // one device allocation holding every buffer below
  size_t bytes;
  float2* P;         // M x N, zero outside the m x n corner, holds z
  float2* F;         // M x N transform buffer
  float2* Q;         // M x N, zero outside the corner, holds the residual field
  float2* X[2];      // m x n: x_k and x_{k-1}
  float2* V;         // m x n: prox input
  float4* dual;      // m x n: FGP dual, warm start across outer iterations
  void* fgp_ws;
  size_t fgp_ws_bytes;
  double* loss;      // scratch FP64 accumulators (4)
  float2* Gz;        // m x n: grad F(z_k), kept across line-search trials
  float4* dual_keep; // m x n: warm-start dual restored before every trial
};

namespace ctv {

static ctv_status pr_set_stream(ctv_pr_plan* p, cudaStream_t s) {
  if (cufftSetStream(p->fft_rows, s) != CUFFT_SUCCESS || cufftSetStream(p->fft_cols, s) != CUFFT_SUCCESS)
    return CTV_ECUDA;
  return CTV_OK;
}

// F = FFT2(src) for a field that is zero outside its first m rows.
static ctv_status pr_fft_padded(ctv_pr_plan* p, const float2* src, cudaStream_t s) {
  if (p->M > p->m &&
      cudaMemsetAsync(p->F + (size_t)p->m * p->N, 0, (size_t)(p->M - p->m) * p->N * sizeof(float2), s) != cudaSuccess)
    return CTV_ECUDA;
  if (cufftExecC2C(p->fft_rows, (cufftComplex*)src, (cufftComplex*)p->F, CUFFT_FORWARD) != CUFFT_SUCCESS)
    return CTV_ECUDA;
  if (cufftExecC2C(p->fft_cols, (cufftComplex*)p->F, (cufftComplex*)p->F, CUFFT_FORWARD) != CUFFT_SUCCESS)
    return CTV_ECUDA;
  return CTV_OK;
}

// F = IFFT2(F) (unnormalised) on its first m rows; the other rows are left undefined.
static ctv_status pr_ifft_rows(ctv_pr_plan* p) {
  if (cufftExecC2C(p->fft_cols, (cufftComplex*)p->F, (cufftComplex*)p->F, CUFFT_INVERSE) != CUFFT_SUCCESS)
    return CTV_ECUDA;
  if (cufftExecC2C(p->fft_rows, (cufftComplex*)p->F, (cufftComplex*)p->F, CUFFT_INVERSE) != CUFFT_SUCCESS)
    return CTV_ECUDA;
  return CTV_OK;
}

// F(z) for the padded field src (object in its corner): FFT, H, IFFT, then the
// residual g = (xi/|xi|)(|xi| - sqrt(y)) into Q's corner and 1/2 sum (|xi| - sqrt(y))^2.
static ctv_status pr_forward_loss(ctv_pr_plan* p, const float2* src, const float* sqrt_y, const float2* H,
                                  double* loss_acc, cudaStream_t s) {
  const long long MN = (long long)p->M * p->N;
  const float inv = 1.0f / (float)MN;
  if (pr_fft_padded(p, src, s) != CTV_OK) return CTV_ECUDA;
  if ((MN & 1) == 0) {
    pr_mul_h<<<152 * 8, 256, 0, s>>>((float4*)p->F, (const float4*)H, MN / 2, 0);
  } else {
    pr_mul_h_scalar<<<152 * 8, 256, 0, s>>>(p->F, H, MN, 0);
  }
  count_launch();
  if (pr_ifft_rows(p) != CTV_OK) return CTV_ECUDA;
  dim3 g((p->n + PR_NT - 1) / PR_NT, p->m);
  pr_residual<<<g, PR_NT, 0, s>>>(p->F, p->N, p->m, p->n, inv, sqrt_y, p->n, p->Q, p->N, loss_acc);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? CTV_OK : CTV_ECUDA;
}

// A^* of the residual held in Q: FFT, conj(H), IFFT; grad F = (1/(MN)) F's corner.
static ctv_status pr_adjoint(ctv_pr_plan* p, const float2* H, cudaStream_t s) {
  const long long MN = (long long)p->M * p->N;
  if (pr_fft_padded(p, p->Q, s) != CTV_OK) return CTV_ECUDA;
  if ((MN & 1) == 0) {
    pr_mul_h<<<152 * 8, 256, 0, s>>>((float4*)p->F, (const float4*)H, MN / 2, 1);
  } else {
    pr_mul_h_scalar<<<152 * 8, 256, 0, s>>>(p->F, H, MN, 1);
  }
  count_launch();
  if (pr_ifft_rows(p) != CTV_OK) return CTV_ECUDA;
  return cudaGetLastError() == cudaSuccess ? CTV_OK : CTV_ECUDA;
}

static ctv_status pr_forward_residual(ctv_pr_plan* p, const float* sqrt_y, const float2* H, double* loss_acc,
                                      cudaStream_t s) {
  ctv_status st = pr_forward_loss(p, p->P, sqrt_y, H, loss_acc, s);
  if (st != CTV_OK) return st;
  return pr_adjoint(p, H, s);
}

}  // namespace ctv

extern "C" {

int ctv_pr_plan_create(int m, int n, int M, int N, ctv_pr_plan** out) {
  using namespace ctv;
  if (out == nullptr) return CTV_EINVAL;
  *out = nullptr;
  if (m <= 0 || n <= 0 || M < m || N < n) return CTV_EINVAL;
  if ((long long)M * N > (1LL << 31)) return CTV_EINVAL;
  ctv_pr_plan* p = new ctv_pr_plan();
  memset(p, 0, sizeof(*p));
  p->m = m; p->n = n; p->M = M; p->N = N;
  const size_t big = al256((size_t)M * N * sizeof(float2));
  const size_t small = al256((size_t)m * n * sizeof(float2));
  const size_t dual = al256((size_t)m * n * sizeof(float4));
  p->fgp_ws_bytes = denoise_workspace_bytes(1, m, n);
  p->bytes = 3 * big + 4 * small + 2 * dual + al256(p->fgp_ws_bytes) + 256;
  if (cudaMalloc(&p->base, p->bytes) != cudaSuccess) { delete p; return CTV_ENOMEM; }
  char* c = p->base;
  p->P = (float2*)c; c += big;
  p->F = (float2*)c; c += big;
  p->Q = (float2*)c; c += big;
  p->X[0] = (float2*)c; c += small;
  p->X[1] = (float2*)c; c += small;
  p->V = (float2*)c; c += small;
  p->dual = (float4*)c; c += dual;
  p->fgp_ws = c; c += al256(p->fgp_ws_bytes);
  p->Gz = (float2*)c; c += small;
  p->dual_keep = (float4*)c; c += dual;
  p->loss = (double*)c;
  if (cudaMemset(p->base, 0, p->bytes) != cudaSuccess) { cudaFree(p->base); delete p; return CTV_ECUDA; }
  int nr = N, nc = M;
  if (cufftPlanMany(&p->fft_rows, 1, &nr, nullptr, 1, N, nullptr, 1, N, CUFFT_C2C, m) != CUFFT_SUCCESS) {
    cudaFree(p->base);
    delete p;
    return CTV_ENOMEM;
  }
  if (cufftPlanMany(&p->fft_cols, 1, &nc, &nc, N, 1, &nc, N, 1, CUFFT_C2C, N) != CUFFT_SUCCESS) {
    cufftDestroy(p->fft_rows);
    cudaFree(p->base);
    delete p;
    return CTV_ENOMEM;
  }
  *out = p;
  return CTV_OK;
}

void ctv_pr_plan_destroy(ctv_pr_plan* p) {
  if (p == nullptr) return;
  cufftDestroy(p->fft_rows);
  cufftDestroy(p->fft_cols);
  cudaFree(p->base);
  delete p;
}

int ctv_pr_gradient(ctv_pr_plan* p, const void* z, const float* sqrt_y, const void* H, void* grad, double* loss,
                    ctv_stream stream) {
  using namespace ctv;
  if (p == nullptr || z == nullptr || sqrt_y == nullptr || H == nullptr || grad == nullptr) return CTV_EINVAL;
  if (((uintptr_t)H & 15) || ((uintptr_t)z & 7) || ((uintptr_t)grad & 7)) return CTV_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (pr_set_stream(p, s) != CTV_OK) return CTV_ECUDA;
  dim3 g((p->n + 255) / 256, p->m);
  pr_copy<<<g, 256, 0, s>>>((const float2*)z, p->n, p->P, p->N, p->m, p->n);
  count_launch();
  if (loss != nullptr && cudaMemsetAsync(loss, 0, sizeof(double), s) != cudaSuccess) return CTV_ECUDA;
  ctv_status st = pr_forward_residual(p, sqrt_y, (const float2*)H, loss, s);
  if (st != CTV_OK) return st;
  const float inv = 1.0f / ((float)p->M * (float)p->N);
  pr_crop_scale<<<g, 256, 0, s>>>(p->F, p->N, inv, (float2*)grad, p->n, p->m, p->n);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? CTV_OK : CTV_ECUDA;
}

int ctv_pr_solve(ctv_pr_plan* p, const float* sqrt_y, const void* H, float tau, float gamma,
                 const ctv_constraint* C, int tv_type, const ctv_opts* inner, int outer_iters, int accelerate,
                 void* x_io, double* loss_hist, ctv_stream stream) {
  using namespace ctv;
  if (p == nullptr || sqrt_y == nullptr || H == nullptr || x_io == nullptr || inner == nullptr) return CTV_EINVAL;
  if (((uintptr_t)H & 15) || ((uintptr_t)x_io & 7)) return CTV_EINVAL;
  if (!(tau >= 0.f) || !(gamma > 0.f) || isinf(tau) || isinf(gamma) || outer_iters < 0) return CTV_EINVAL;
  if (tv_type < 0 || tv_type > 3) return CTV_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (pr_set_stream(p, s) != CTV_OK) return CTV_ECUDA;
  const int m = p->m, n = p->n;
  dim3 g((n + 255) / 256, m);
  // z_1 = x_0 (into the padded buffer), x_{0} kept as the first "previous" iterate
  pr_copy<<<g, 256, 0, s>>>((const float2*)x_io, n, p->P, p->N, m, n);
  pr_copy<<<g, 256, 0, s>>>((const float2*)x_io, n, p->X[1], n, m, n);
  count_launch();
  count_launch();
  if (loss_hist != nullptr && outer_iters > 0 &&
      cudaMemsetAsync(loss_hist, 0, sizeof(double) * (size_t)outer_iters, s) != cudaSuccess)
    return CTV_ECUDA;
  const float lam = tau * gamma;
  const float inv = 1.0f / ((float)p->M * (float)p->N);
  double t = 1.0;
  int cur = 0;   // X[cur] receives x_k, X[cur ^ 1] holds x_{k-1}
  ctv_opts o = *inner;
  for (int k = 0; k < outer_iters; ++k) {
    ctv_status st = pr_forward_residual(p, sqrt_y, (const float2*)H, loss_hist ? loss_hist + k : nullptr, s);
    if (st != CTV_OK) return st;
    pr_form_v<<<g, 256, 0, s>>>(p->P, p->N, p->F, p->N, gamma * inv, p->V, n, m, n);
    count_launch();
    o.warm_start = k > 0 ? 1 : 0;
    float beta = 0.f;
    if (accelerate) {
      const double tn = (1.0 + sqrt(1.0 + 4.0 * t * t)) / 2.0;
      beta = (float)((t - 1.0) / tn);
      t = tn;
    }
    // the inner solve's finalize also forms z_{k+1} when it is the x-only one
    int fused = 0;
    DenoiseCall c;
    memset(&c, 0, sizeof(c));
    c.b = p->V; c.x = p->X[cur]; c.batch = 1; c.m = m; c.n = n; c.ld = n;
    c.lam = lam; c.C = C; c.tv = tv_type; c.opts = &o; c.dual_state = p->dual;
    c.workspace = p->fgp_ws; c.workspace_bytes = p->fgp_ws_bytes; c.stats = nullptr; c.stream = stream;
    c.mom_z = p->P; c.mom_ld = p->N; c.mom_xprev = p->X[cur ^ 1]; c.mom_beta = beta; c.mom_written = &fused;
    st = run_denoise(c);
    if (st != CTV_OK) return st;
    if (!fused) {
      pr_fista<<<g, 256, 0, s>>>(p->X[cur], p->X[cur ^ 1], n, beta, p->P, p->N, m, n);
      count_launch();
    }
    cur ^= 1;
  }
  // the last x_k sits in X[cur ^ 1]
  pr_copy<<<g, 256, 0, s>>>(p->X[cur ^ 1], n, (float2*)x_io, n, m, n);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? CTV_OK : CTV_ECUDA;
}

int ctv_pr_solve_ls(ctv_pr_plan* p, const float* sqrt_y, const void* H, float tau, float gamma0, float eta,
                    const ctv_constraint* C, int tv_type, const ctv_opts* inner, int outer_iters, int accelerate,
                    void* x_io, double* loss_hist, float* gamma_hist, ctv_stream stream) {
  using namespace ctv;
  if (p == nullptr || sqrt_y == nullptr || H == nullptr || x_io == nullptr || inner == nullptr) return CTV_EINVAL;
  if (((uintptr_t)H & 15) || ((uintptr_t)x_io & 7)) return CTV_EINVAL;
  if (!(tau >= 0.f) || !(gamma0 > 0.f) || isinf(tau) || isinf(gamma0) || !(eta > 0.f && eta < 1.f) || outer_iters < 0)
    return CTV_EINVAL;
  if (tv_type < 0 || tv_type > 3) return CTV_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (pr_set_stream(p, s) != CTV_OK) return CTV_ECUDA;
  const int m = p->m, n = p->n;
  dim3 g((n + 255) / 256, m);
  dim3 gr((n + PR_NT - 1) / PR_NT, m);
  const float inv = 1.0f / ((float)p->M * (float)p->N);
  pr_copy<<<g, 256, 0, s>>>((const float2*)x_io, n, p->P, p->N, m, n);
  pr_copy<<<g, 256, 0, s>>>((const float2*)x_io, n, p->X[1], n, m, n);
  count_launch();
  count_launch();
  if (loss_hist != nullptr && outer_iters > 0 &&
      cudaMemsetAsync(loss_hist, 0, sizeof(double) * (size_t)outer_iters, s) != cudaSuccess)
    return CTV_ECUDA;
  double t = 1.0;
  float gamma = gamma0;
  int cur = 0;
  ctv_opts o = *inner;
  for (int k = 0; k < outer_iters; ++k) {
    // F(z_k) and grad F(z_k)
    if (cudaMemsetAsync(p->loss, 0, 4 * sizeof(double), s) != cudaSuccess) return CTV_ECUDA;
    ctv_status st = pr_forward_loss(p, p->P, sqrt_y, (const float2*)H, p->loss, s);
    if (st != CTV_OK) return st;
    st = pr_adjoint(p, (const float2*)H, s);
    if (st != CTV_OK) return st;
    pr_crop_scale<<<g, 256, 0, s>>>(p->F, p->N, inv, p->Gz, n, m, n);
    count_launch();
    if (loss_hist != nullptr && cudaMemcpyAsync(loss_hist + k, p->loss, sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return CTV_ECUDA;
    if (k > 0 && cudaMemcpyAsync(p->dual_keep, p->dual, (size_t)m * n * sizeof(float4), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return CTV_ECUDA;
    bool accepted = false;
    for (int trial = 0; trial < 60 && !accepted; ++trial) {
      if (trial > 0 && k > 0 &&
          cudaMemcpyAsync(p->dual, p->dual_keep, (size_t)m * n * sizeof(float4), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return CTV_ECUDA;
      pr_form_v<<<g, 256, 0, s>>>(p->P, p->N, p->Gz, n, gamma, p->V, n, m, n);
      count_launch();
      o.warm_start = k > 0 ? 1 : 0;
      DenoiseCall c;
      memset(&c, 0, sizeof(c));
      c.b = p->V; c.x = p->X[cur]; c.batch = 1; c.m = m; c.n = n; c.ld = n;
      c.lam = tau * gamma; c.C = C; c.tv = tv_type; c.opts = &o; c.dual_state = p->dual;
      c.workspace = p->fgp_ws; c.workspace_bytes = p->fgp_ws_bytes; c.stats = nullptr; c.stream = stream;
      st = run_denoise(c);
      if (st != CTV_OK) return st;
      // F at the candidate, through Q's zero-padded corner
      pr_copy<<<g, 256, 0, s>>>(p->X[cur], n, p->Q, p->N, m, n);
      count_launch();
      st = pr_forward_loss(p, p->Q, sqrt_y, (const float2*)H, p->loss + 1, s);
      if (st != CTV_OK) return st;
      pr_ls_terms<<<gr, PR_NT, 0, s>>>(p->X[cur], n, p->P, p->N, p->Gz, n, m, n, p->loss + 2);
      count_launch();
      double h[4];
      if (cudaMemcpyAsync(h, p->loss, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CTV_ECUDA;
      if (cudaStreamSynchronize(s) != cudaSuccess) return CTV_ECUDA;
      // F(x) <= F(z) + <x - z, grad F(z)> + ||x - z||^2 / (2 gamma)
      if (h[1] <= h[0] + h[2] + h[3] / (2.0 * (double)gamma)) {
        accepted = true;
      } else {
        gamma *= eta;
        if (cudaMemsetAsync(p->loss + 1, 0, 3 * sizeof(double), s) != cudaSuccess) return CTV_ECUDA;
      }
    }
    if (gamma_hist != nullptr) gamma_hist[k] = gamma;
    float beta = 0.f;
    if (accelerate) {
      const double tn = (1.0 + sqrt(1.0 + 4.0 * t * t)) / 2.0;
      beta = (float)((t - 1.0) / tn);
      t = tn;
    }
    pr_fista<<<g, 256, 0, s>>>(p->X[cur], p->X[cur ^ 1], n, beta, p->P, p->N, m, n);
    count_launch();
    cur ^= 1;
  }
  pr_copy<<<g, 256, 0, s>>>(p->X[cur ^ 1], n, (float2*)x_io, n, m, n);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? CTV_OK : CTV_ECUDA;
}

int ctv_prox_grad_step(const void* z, const void* grad, float gamma, float tau, const ctv_constraint* C, int tv_type,
                       const ctv_opts* inner, void* dual_state, const void* x_prev, void* x_out, void* z_next,
                       float beta, int m, int n, void* workspace, size_t workspace_bytes, ctv_stream stream) {
  using namespace ctv;
  if (z == nullptr || grad == nullptr || inner == nullptr || x_prev == nullptr || x_out == nullptr ||
      z_next == nullptr || workspace == nullptr)
    return CTV_EINVAL;
  if (m <= 0 || n <= 0 || !(gamma > 0.f) || !(tau >= 0.f) || isinf(gamma) || isinf(tau)) return CTV_EINVAL;
  const size_t need = al256((size_t)m * n * sizeof(float2)) + denoise_workspace_bytes(1, m, n);
  if (workspace_bytes < need || ((uintptr_t)workspace & 255)) return CTV_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  float2* V = (float2*)workspace;
  void* fws = (char*)workspace + al256((size_t)m * n * sizeof(float2));
  dim3 g((n + 255) / 256, m);
  pr_form_v<<<g, 256, 0, s>>>((const float2*)z, n, (const float2*)grad, n, gamma, V, n, m, n);
  count_launch();
  DenoiseCall c;
  memset(&c, 0, sizeof(c));
  c.b = V; c.x = x_out; c.batch = 1; c.m = m; c.n = n; c.ld = n;
  c.lam = tau * gamma; c.C = C; c.tv = tv_type; c.opts = inner; c.dual_state = dual_state;
  c.workspace = fws; c.workspace_bytes = denoise_workspace_bytes(1, m, n); c.stats = nullptr; c.stream = stream;
  int fused = 0;
  c.mom_z = (float2*)z_next; c.mom_ld = n; c.mom_xprev = (const float2*)x_prev; c.mom_beta = beta;
  c.mom_written = &fused;
  ctv_status st = run_denoise(c);
  if (st != CTV_OK) return st;
  if (!fused) {
    pr_fista<<<g, 256, 0, s>>>((const float2*)x_out, (const float2*)x_prev, n, beta, (float2*)z_next, n, m, n);
    count_launch();
  }
  return cudaGetLastError() == cudaSuccess ? CTV_OK : CTV_ECUDA;
}

size_t ctv_prox_grad_workspace_size(int m, int n) {
  if (m <= 0 || n <= 0) return 0;
  return ctv::al256((size_t)m * n * sizeof(float2)) + ctv::denoise_workspace_bytes(1, m, n);
}

}  // extern "C"
