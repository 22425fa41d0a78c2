// Complex constrained TV denoising, problem (1), by Algorithm 2 (FGP).
//
// Kernels
//   fgp_pass_kernel        T fused FGP iterations per launch on shared-memory tiles
//                          (pass_tv.cuh; fgp_tile / fgp_strip_tile in ctv_device.cuh);
//                          a pass that ends a check interval with fewer than T
//                          iterations also adds up the duality-gap terms at its
//                          final q (the gap-evaluating variant, pass_gap_tv*.cu).
//   fgp_gap_kernel         x = P_C(b - lam L^T q) (Eq. (18)) together with the sums
//                          of the primal value of problem (1) and of the dual value
//                          of App. A (Eq. (30) times lam), per block into a slot.
//   fgp_gap_finish_kernel  adds the slots of a check or of the final evaluation,
//                          forms primal, dual and gap, applies the stopping test
//                          and, for the final call, writes the statistics. Later
//                          passes read the stop flag and return.
//   fgp_finalize_kernel    x (and the exported q) only, for solves whose statistics
//                          nobody reads.
// Host entry points: ctv_denoise, ctv_denoise_batched (declared in ctv.h).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "async_status.cuh"
#include "ctv.h"
#include "ctv_configs.cuh"
#include "ctv_device.cuh"
#include "gap_device.cuh"
#include "ctv_host.h"
#include "ctv_kernels.h"

namespace ctv {

// Duality gap / finalize evaluation (Eq. (18), problem (1), App. A Eq. (30)) on
// 64 x 16 tiles with a one-pixel halo (gap_tile_add): persistent blocks walk the
// tiles of an image, keep the three sums in compensated FP32 and store the
// block's sums, as FP32 pairs, in its slot; fgp_gap_finish_kernel evaluates
// them. No FP64 arithmetic per block (this GPU's FP64 rate is a small fraction of
// its FP32 rate) and no fence or atomic per block.
template <int TV>
__global__ void __launch_bounds__(GAP_NT, 4) fgp_gap_kernel(GapParams p) {
  __shared__ float4 qs[GAP_RW * GAP_RH];
  __shared__ float2 xs[GAP_RW * GAP_RH];
  __shared__ float2 red[3 * (GAP_NT / 32)];
  const int z = blockIdx.z;
  DevStats* st = p.st + z;
  const int stopped = *(volatile int*)&st->stop;
  if (!p.final_call && stopped) return;
  const int set = stopped ? st->stop_set : p.default_set;
  GapImg g;
  g.b = p.b + z * p.b_stride;
  g.ld = p.ld;
  const bool zq = p.zero_q != 0 && !stopped;
  const float4* q = set == 0 ? p.qA : (set == 1 ? p.qB : p.dual_in);
  g.q = zq ? nullptr : q + z * p.d_stride;
  g.x = p.x != nullptr ? p.x + z * p.x_stride : nullptr;
  g.q_export = p.q_export != nullptr ? p.q_export + z * p.d_stride : nullptr;
  g.m = p.m;
  g.n = p.n;
  const float lv = p.lam_dev != nullptr ? p.lam_dev[z] : p.lam;
  g.lam = lv >= 0.f ? lv : 0.f;
  g.alpha = p.alpha;
  g.C = p.C;
  GapSums acc = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, false};
  bool nf = false;
  const int tx = (p.n + GAP_RW - 3) / (GAP_RW - 2), ty = (p.m + GAP_RH - 3) / (GAP_RH - 2);
  for (int t = blockIdx.x; t < tx * ty; t += gridDim.x) {
    const int by = t / tx, bx = t - by * tx;
    gap_tile_add<TV>(g, by * (GAP_RH - 2), bx * (GAP_RW - 2), qs, xs, acc, nf);
    __syncthreads();
  }
  float hs[3], ls[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    hs[a] = acc.s[a];
    ls[a] = -acc.c[a];
  }
  block_sum_pairs<GAP_NT, 3>(hs, ls, red);
  const bool block_nf = __syncthreads_or(nf) != 0;
  if (block_nf && threadIdx.x == 0) raise_async(CTV_ENONFINITE);
  gap_store_slot(st, p.slots + z * p.slot_stride, blockIdx.x, hs, ls, block_nf);
}

// Evaluation of a slot reduction, one block per image (see GapFinishParams).
constexpr int GF_NT = 1024;
__global__ void __launch_bounds__(GF_NT) fgp_gap_finish_kernel(GapFinishParams f) {
  __shared__ float2 red[3 * (GF_NT / 32)];
  const int z = blockIdx.x;
  DevStats* st = f.st + z;
  const int stopped = *(volatile int*)&st->stop;
  if (!f.final_call && stopped) return;   // an earlier check stopped the solve; this one did not run
  const float* slots = f.slots + z * f.slot_stride;
  float h[3] = {0.f, 0.f, 0.f}, l[3] = {0.f, 0.f, 0.f};
#pragma unroll 4
  for (unsigned i = threadIdx.x; i < f.nblk; i += GF_NT) {
    const float4* sl = reinterpret_cast<const float4*>(slots + 8 * (size_t)i);
    const float4 a = sl[0], b = sl[1];
    pair_add(h[0], l[0], a.x, a.y);
    pair_add(h[1], l[1], a.z, a.w);
    pair_add(h[2], l[2], b.x, b.y);
  }
  block_sum_pairs<GF_NT, 3>(h, l, red);
  if (threadIdx.x == 0) {
    const float lv = f.lam_dev != nullptr ? f.lam_dev[z] : f.lam;
    const bool bad_lam = !(lv >= 0.f);
    gap_finish(st, (double)h[0] + (double)l[0], (double)h[1] + (double)l[1], (double)h[2] + (double)l[2],
               bad_lam ? 0.f : lv, bad_lam, f.set, stopped, f.iter, f.gap_tol, f.final_call);
    // inside a stop graph, the check that stops the solve skips the remaining intervals
    if (f.n_cond > 0 && st->stop) {
#pragma unroll
      for (int i = 0; i < CTV_MAX_STOP_INTERVALS; ++i)
        if (i < f.n_cond) cudaGraphSetConditional(f.cond[i], 0u);
    }
  }
}

cudaError_t launch_gap_finish(const GapFinishParams& f, int batch, cudaStream_t s) {
  fgp_gap_finish_kernel<<<batch, GF_NT, 0, s>>>(f);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Configurations of the fused pass (table in ctv_configs.cuh)
// ----------------------------------------------------------------------------
struct Cfg {
  int T, RW, RH, NT;
};
#define CTV_CFG_ROW(id, kind, T, A, B, C) \
  {T, CfgGeom<kind, A, B, C>::RW, CfgGeom<kind, A, B, C>::RH, CfgGeom<kind, A, B, C>::NT},
static const Cfg kCfgs[] = {CTV_PASS_CONFIGS(CTV_CFG_ROW)};
#undef CTV_CFG_ROW
static const int kNumCfgs = (int)(sizeof(kCfgs) / sizeof(kCfgs[0]));

cudaError_t launch_pass(int tv, int cfg, const PassParams& p, dim3 grid, cudaStream_t s) {
  if (cfg < 0 || cfg >= kNumCfgs) return cudaErrorInvalidValue;
  const int cons = cons_mode(p.C);
  if (p.gap_eval) {
    if (!pass_gap_eval_ok(cfg)) return cudaErrorInvalidValue;
    switch (tv) {
      case TV1_ISO: return launch_pass_gap_tv<TV1_ISO>(cfg, cons, p, grid, s);
      case TV1_ANISO: return launch_pass_gap_tv<TV1_ANISO>(cfg, cons, p, grid, s);
      case TV2_ISO: return launch_pass_gap_tv<TV2_ISO>(cfg, cons, p, grid, s);
      case TV2_ANISO: return launch_pass_gap_tv<TV2_ANISO>(cfg, cons, p, grid, s);
    }
    return cudaErrorInvalidValue;
  }
  switch (tv) {
    case TV1_ISO: return launch_pass_tv<TV1_ISO>(cfg, cons, p, grid, s);
    case TV1_ANISO: return launch_pass_tv<TV1_ANISO>(cfg, cons, p, grid, s);
    case TV2_ISO: return launch_pass_tv<TV2_ISO>(cfg, cons, p, grid, s);
    case TV2_ANISO: return launch_pass_tv<TV2_ANISO>(cfg, cons, p, grid, s);
  }
  return cudaErrorInvalidValue;
}

bool pass_gap_eval_ok(int cfg) {
  switch (cfg) {
#define CTV_GAP_OK(id, kind, T, A, B, C) \
  case id: return GapEvalOk<kind, C>::value;
    CTV_PASS_CONFIGS(CTV_GAP_OK)
#undef CTV_GAP_OK
  }
  return false;
}

// x = P_C(b - lam L^T q) (Eq. (18)) and the optional export of q, without the
// objective terms: the finalize of a solve without gap checks whose statistics
// nobody reads. One thread per pixel; the same arithmetic as gap_tile, so the
// same x.
constexpr int FIN_NT = 128;
__global__ void __launch_bounds__(FIN_NT) fgp_finalize_kernel(GapParams p) {
  const int z = blockIdx.z;
  const int k = blockIdx.x * FIN_NT + threadIdx.x;
  const int m = p.m, n = p.n;
  if (k >= n) return;
  const float4 z4 = f4(0.f, 0.f, 0.f, 0.f);
  const float4* q = p.default_set == 0 ? p.qA : (p.default_set == 1 ? p.qB : p.dual_in);
  if (p.zero_q) q = nullptr;
  else q += z * p.d_stride;
  const float2* b = p.b + z * p.b_stride;
  float2* x = p.x + z * p.x_stride;
  float4* qe = p.q_export != nullptr ? p.q_export + z * p.d_stride : nullptr;
  const float lv = p.lam_dev != nullptr ? p.lam_dev[z] : p.lam;
  const float lam = lv >= 0.f ? lv : 0.f;
  bool nf = false;
  for (int j = blockIdx.y; j < m; j += gridDim.y) {
    const long long o = (long long)j * n + k;
    float4 qc = z4, qu = z4, ql = z4;
    if (q != nullptr) {
      qc = __ldg(q + o);
      if (j > 0) qu = __ldg(q + o - n);
      if (k > 0) ql = __ldg(q + o - 1);
    }
    const float2 bb = __ldg(b + (long long)j * p.ld + k);
    nf |= nonfinite2(bb);
    const float2 xv =
        proj_C(make_float2(fmaf(-lam, qc.x - qu.x + qc.z - ql.z, bb.x), fmaf(-lam, qc.y - qu.y + qc.w - ql.w, bb.y)), j, k,
               p.C);
    x[(long long)j * p.ld + k] = xv;
    if (qe != nullptr) qe[o] = qc;
    if (p.mom_z != nullptr) {   // Alg. 1, step 5, as pr_fista forms it
      const float2 xp = __ldg(p.mom_xprev + (long long)j * p.ld + k);
      p.mom_z[(long long)j * p.mom_ld + k] =
          make_float2(fmaf(p.mom_beta, xv.x - xp.x, xv.x), fmaf(p.mom_beta, xv.y - xp.y, xv.y));
    }
  }
  // a NaN or infinity in b: one report per warp (the threads past column n have returned)
  const unsigned am = __activemask();
  if (__any_sync(am, nf) && (int)(threadIdx.x & 31) == __ffs(am) - 1) {
    raise_async(CTV_ENONFINITE);
    if (p.st != nullptr) {
      atomicOr(&p.st[z].nonfinite, 1u);
      atomicExch(&p.st[z].status, (int)CTV_ENONFINITE);
    }
  }
}

cudaError_t launch_finalize(const GapParams& p, int batch, cudaStream_t s) {
  dim3 grid((p.n + FIN_NT - 1) / FIN_NT, p.m < 65535 ? p.m : 65535, batch);
  fgp_finalize_kernel<<<grid, FIN_NT, 0, s>>>(p);
  return cudaGetLastError();
}

int take_async_status_denoise() { return take_unit_async_status(); }

int sm_count() {
  static int cached[kMaxDevices] = {};
  const int d = device_slot();
  if (d >= 0 && cached[d] > 0) return cached[d];
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    n = 0;
  if (n <= 0) n = 1;
  if (d >= 0) cached[d] = n;
  return n;
}

// Resident blocks per SM of a kernel at `threads` threads (and no dynamic shared
// memory), once per device and kernel.
int occupancy_once(const void* kernel, int threads, int (&cached)[kMaxDevices]) {
  const int d = device_slot();
  if (d >= 0 && cached[d] > 0) return cached[d];
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm <= 0)
    per_sm = 1;
  if (d >= 0) cached[d] = per_sm;
  return per_sm;
}

template <int TV>
static long long launch_gap_tv(const GapParams& p, int batch, cudaStream_t s) {
  static int per_sm_cache[kMaxDevices] = {};
  const int per_sm = occupancy_once((const void*)fgp_gap_kernel<TV>, GAP_NT, per_sm_cache);
  const long long tiles = (long long)((p.n + GAP_RW - 3) / (GAP_RW - 2)) * ((p.m + GAP_RH - 3) / (GAP_RH - 2));
  const long long cap = (long long)per_sm * sm_count();
  const long long blocks = tiles < cap ? tiles : cap;
  fgp_gap_kernel<TV><<<dim3((unsigned)blocks, 1, batch), GAP_NT, 0, s>>>(p);
  return blocks;
}

cudaError_t launch_gap(int tv, const GapParams& p, int batch, cudaStream_t s) {
  long long blocks = 0;
  switch (tv) {
    case TV1_ISO: blocks = launch_gap_tv<TV1_ISO>(p, batch, s); break;
    case TV1_ANISO: blocks = launch_gap_tv<TV1_ANISO>(p, batch, s); break;
    case TV2_ISO: blocks = launch_gap_tv<TV2_ISO>(p, batch, s); break;
    case TV2_ANISO: blocks = launch_gap_tv<TV2_ANISO>(p, batch, s); break;
    default: return cudaErrorInvalidValue;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  GapFinishParams f;
  memset(&f, 0, sizeof(f));
  f.st = p.st;
  f.slots = p.slots;
  f.slot_stride = p.slot_stride;
  f.nblk = (unsigned)blocks;
  f.lam = p.lam;
  f.lam_dev = p.lam_dev;
  f.set = p.default_set;
  f.iter = p.iter;
  f.gap_tol = p.gap_tol;
  f.final_call = p.final_call;
  f.n_cond = p.n_cond;
  for (int i = 0; i < p.n_cond; ++i) f.cond[i] = p.cond[i];
  return launch_gap_finish(f, batch, s);
}

dim3 pass_grid(int cfg, int m, int n, int batch) {
  const Cfg& cf = kCfgs[cfg];
  return dim3((n + (cf.RW - 2 * cf.T) - 1) / (cf.RW - 2 * cf.T), (m + (cf.RH - 2 * cf.T) - 1) / (cf.RH - 2 * cf.T),
              batch);
}

int default_config(int m, int n, int iters, int tv, int cons, int check_every) {
  // plans of many images (plan_list.cuh lists the configurations they support):
  // 64 x 64 regions with 8 rows per thread, 6 iterations per pass (on 512 images
  // of sides 64 to 1024, two GPUs: 150.7 and 153.3 Gpixel-iter/s, against 151.6
  // and 151.0 for 8 iterations and 143.1 and 142.4 for 4 rows per thread)
  if (m <= 0 || n <= 0) return 5;
  if (iters < 2) return 0;
  if (m > 0 && n > 0) {
    const int t = tuned_config(m, n, tv);
    if (t >= 0) return t;
  }
  // measured on GB300 (phantoms of 256^2 to 2048^2, all four TV types, 200
  // iterations, |x| <= 1 with and without a support rectangle; Gpixel-iter/s of
  // the best configuration): column-strip kernels throughout. Small images fill
  // too few SMs with 64-row regions, so 32 x 32 regions with one row per thread
  // (8 iterations per pass below about 320^2: 61.9; 4 up to about 448^2: 96.1).
  // From there 64 x 64 regions of 8 iterations: 8 rows per thread with a support
  // rectangle (122.2 at 512^2, 158.0 at 768^2), 4 without (132.8, 159.0); 6
  // iterations and 8 rows per thread around 1024^2 (209.5 with the rectangle,
  // 172.9 without); above about 1280^2, 8 iterations and 4 rows per thread with
  // the rectangle (223.6 at 1536^2, 245.0 at 2048^2: the rectangle's outside
  // tiles take the neighbour-free body, so long passes cost little there), and
  // without it 8 rows per thread (181.3 at 1536^2 for 8 iterations, 188.9 at
  // 2048^2 for 6).
  const double px = (double)m * (double)n;
  const bool rect = cons == CONS_RECT;
  int cfg;
  if (px < 320.0 * 320.0) cfg = 17;
  else if (px < 448.0 * 448.0) cfg = 16;
  else if (px < 896.0 * 896.0) cfg = rect ? 6 : 18;
  else if (px < 1280.0 * 1280.0) cfg = 5;
  else if (px < 1792.0 * 1792.0) cfg = rect ? 18 : 6;
  else cfg = rect ? 18 : 5;
  // A stopping test ends a pass at every check, so checks every `check_every`
  // iterations cost ceil(check_every / T) passes per interval. Where 6 iterations
  // per pass need no more passes than 8, the same region with T = 6 recomputes a
  // narrower halo (2.75 against 2.90 ms per 2048^2 solve with checks every 10).
  if (check_every > 0 && (check_every + 5) / 6 <= (check_every + 7) / 8) {
    if (cfg == 18) cfg = 14;
    else if (cfg == 6) cfg = 5;
  }
  return cfg;
}

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

static_assert(sizeof(DevStats) <= 256, "statistics record must fit its 256-byte slot");
size_t denoise_workspace_bytes(int batch, int m, int n) { return denoise_workspace_bytes_c(batch, m, n); }

bool convert_constraint(const ctv_constraint* C, int m, int n, ConsDev* out) {
  memset(out, 0, sizeof(*out));
  if (C == nullptr) return true;
  if (C->amp_bound) {
    if (!(C->amp_max >= 0.f) || isinf(C->amp_max)) return false;
    out->amp = 1;
    out->amax = C->amp_max;
  }
  if (C->box) {
    if (C->amp_bound) return false;
    if (!(C->box_re[0] <= C->box_re[1]) || !(C->box_im[0] <= C->box_im[1])) return false;
    out->box = 1;
    out->re_lo = C->box_re[0];
    out->re_hi = C->box_re[1];
    out->im_lo = C->box_im[0];
    out->im_hi = C->box_im[1];
  }
  if (C->support_kind == 1) {
    out->sup = 1;
    out->j0 = C->rect[0];
    out->k0 = C->rect[1];
    out->j1 = C->rect[2];
    out->k1 = C->rect[3];
  } else if (C->support_kind == 2) {
    if (C->mask == nullptr || C->mask_ld < n) return false;
    out->sup = 2;
    out->mask = C->mask;
    out->mask_ld = C->mask_ld;
  } else if (C->support_kind != 0) {
    return false;
  }
  (void)m;
  return true;
}

void nesterov_betas(int K, std::vector<double>* beta) {
  // t_1 = 1, t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2, beta_k = (t_k - 1) / t_{k+1} (Alg. 2, steps 4-5)
  beta->assign((size_t)K + 1, 0.0);
  double t = 1.0;
  for (int k = 1; k <= K; ++k) {
    const double tn = (1.0 + sqrt(1.0 + 4.0 * t * t)) / 2.0;
    (*beta)[k] = (t - 1.0) / tn;
    t = tn;
  }
}

// ----------------------------------------------------------------------------
// Stop graphs. A solve with gap checks and a tolerance launches every pass up
// front; once the test passes, the device flag turns the remaining passes into
// launches that return at once, but each still costs its block launches (about
// 15 us per pass at 2048^2). On large images such a solve instead runs as a CUDA
// graph in which each check interval (its passes and its check) is the body of
// a conditional IF node with its own handle (a handle belongs to one node): the
// check whose test passes clears the handles of all later intervals
// (cudaGraphSetConditional) and the graph skips them. The handles' default value
// (1) is restored at every launch, so an instantiated graph is reused by later
// calls with identical arguments; it is built on the second such call, since
// building it costs more host time than one solve saves.
// ----------------------------------------------------------------------------
constexpr double kStopGraphMinPixels = 512.0 * 512.0;

struct StopGraph {
  cudaGraph_t G = nullptr;
  std::vector<cudaGraphConditionalHandle> h;   // one per check interval
  int next = 0;                                 // interval opened next
  cudaStream_t cs = nullptr;          // private stream the bodies are captured on
  cudaGraphNode_t prev = nullptr;     // last node of the chain
  cudaGraph_t fin = nullptr;          // the finalize, added as a child graph
  bool have_prev = false, open = false;
  int kernels = 0;

  bool begin(int intervals) {
    if (cudaGraphCreate(&G, 0) != cudaSuccess) return false;
    h.assign((size_t)intervals, 0);
    for (int i = 0; i < intervals; ++i)
      if (cudaGraphConditionalHandleCreate(&h[(size_t)i], G, 1u, cudaGraphCondAssignDefault) != cudaSuccess)
        return false;
    return cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess;
  }
  // the handles a check at the end of the interval just opened must clear
  void later_handles(GapParams* g) const {
    g->n_cond = 0;
    for (size_t i = (size_t)next; i < h.size(); ++i) g->cond[g->n_cond++] = h[i];
  }
  // appends an IF node after the chain and starts capturing its body
  cudaStream_t open_interval() {
    if (next >= (int)h.size()) return nullptr;
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    memset(&np.conditional, 0, sizeof(np.conditional));
    np.conditional.handle = h[(size_t)next++];
    np.conditional.type = cudaGraphCondTypeIf;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, G, have_prev ? &prev : nullptr, nullptr, have_prev ? 1 : 0, &np) != cudaSuccess)
      return nullptr;
    if (cudaStreamBeginCaptureToGraph(cs, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed) != cudaSuccess)
      return nullptr;
    prev = node;
    have_prev = true;
    open = true;
    return cs;
  }
  bool close_interval() {
    cudaGraph_t body;
    open = false;
    return cudaStreamEndCapture(cs, &body) == cudaSuccess;
  }
  cudaStream_t open_final() {
    if (cudaGraphCreate(&fin, 0) != cudaSuccess) return nullptr;
    if (cudaStreamBeginCaptureToGraph(cs, fin, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
      return nullptr;
    open = true;
    return cs;
  }
  bool close_final() {
    cudaGraph_t g2;
    open = false;
    if (cudaStreamEndCapture(cs, &g2) != cudaSuccess) return false;
    cudaGraphNode_t node;
    return cudaGraphAddChildGraphNode(&node, G, have_prev ? &prev : nullptr, have_prev ? 1 : 0, fin) == cudaSuccess;
  }
  cudaGraphExec_t instantiate() {
    cudaGraphExec_t ex = nullptr;
    if (cudaGraphInstantiate(&ex, G, 0) != cudaSuccess) return nullptr;
    return ex;
  }
  ~StopGraph() {
    if (open && cs != nullptr) {
      cudaGraph_t g2 = nullptr;
      cudaStreamEndCapture(cs, &g2);
    }
    if (fin != nullptr) cudaGraphDestroy(fin);
    if (G != nullptr) cudaGraphDestroy(G);
    if (cs != nullptr) cudaStreamDestroy(cs);
  }
};

static bool stream_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cst) != cudaSuccess) return true;
  return cst != cudaStreamCaptureStatusNone;
}

// every argument that shapes the launches, as bytes
static std::string stop_graph_key(const DenoiseCall& c, const ConsDev& C, int cfg) {
  std::string k;
  auto add = [&k](const void* p, size_t n) { k.append((const char*)p, n); };
  int dev = -1;
  cudaGetDevice(&dev);
  add(&dev, sizeof(dev));
  add(&c.b, sizeof(c.b));
  add(&c.x, sizeof(c.x));
  add(&c.batch, sizeof(c.batch));
  add(&c.batch_stride, sizeof(c.batch_stride));
  add(&c.m, sizeof(c.m));
  add(&c.n, sizeof(c.n));
  add(&c.ld, sizeof(c.ld));
  add(&c.lam, sizeof(c.lam));
  add(&c.lam_dev, sizeof(c.lam_dev));
  add(&c.tv, sizeof(c.tv));
  add(&c.dual_state, sizeof(c.dual_state));
  add(&c.workspace, sizeof(c.workspace));
  add(c.opts, sizeof(ctv_opts));
  add(&C, sizeof(C));
  add(&cfg, sizeof(cfg));
  return k;
}

static std::mutex g_sg_mu;
static std::vector<std::pair<std::string, std::pair<cudaGraphExec_t, int>>> g_sg_cache;   // most recent last
constexpr size_t kStopGraphCache = 16;

// Keys of solves seen once: instantiating a stop graph costs more host time than
// one solve saves, so a graph is built on the second call with the same arguments.
static std::vector<std::string> g_sg_seen;

static bool stop_graph_seen_before(const std::string& key) {
  std::lock_guard<std::mutex> lk(g_sg_mu);
  for (size_t i = 0; i < g_sg_seen.size(); ++i)
    if (g_sg_seen[i] == key) return true;
  if (g_sg_seen.size() >= 4 * kStopGraphCache) g_sg_seen.erase(g_sg_seen.begin());
  g_sg_seen.push_back(key);
  return false;
}

static cudaGraphExec_t stop_graph_lookup(const std::string& key, int* kernels) {
  std::lock_guard<std::mutex> lk(g_sg_mu);
  for (size_t i = 0; i < g_sg_cache.size(); ++i) {
    if (g_sg_cache[i].first == key) {
      auto e = g_sg_cache[i];
      g_sg_cache.erase(g_sg_cache.begin() + (long)i);
      g_sg_cache.push_back(e);
      *kernels = e.second.second;
      return e.second.first;
    }
  }
  return nullptr;
}

static void stop_graph_store(const std::string& key, cudaGraphExec_t ex, int kernels) {
  std::lock_guard<std::mutex> lk(g_sg_mu);
  if (g_sg_cache.size() >= kStopGraphCache) {
    cudaGraphExecDestroy(g_sg_cache.front().second.first);   // freed once any launch of it completes
    g_sg_cache.erase(g_sg_cache.begin());
  }
  g_sg_cache.push_back({key, {ex, kernels}});
}

ctv_status run_denoise(const DenoiseCall& c) {
  if (c.b == nullptr || c.x == nullptr || c.workspace == nullptr) return CTV_EINVAL;
  if (c.batch <= 0 || c.m <= 0 || c.n <= 0 || c.ld < c.n) return CTV_EINVAL;
  if (c.batch > 65535) return CTV_EINVAL;
  if (c.lam_dev == nullptr && (!(c.lam >= 0.f) || isinf(c.lam))) return CTV_EINVAL;
  if (c.tv < 0 || c.tv > 3) return CTV_EINVAL;
  if (((uintptr_t)c.b & 7) || ((uintptr_t)c.x & 7) || ((uintptr_t)c.workspace & 255)) return CTV_EINVAL;
  if (c.dual_state != nullptr && ((uintptr_t)c.dual_state & 15)) return CTV_EINVAL;
  const ctv_opts* o = c.opts;
  const int K = o ? o->max_iters : 0;
  const int check_every = o ? o->check_every : 0;
  const double gap_tol = o ? o->gap_tol : 0.0;
  const float alpha = o ? o->alpha : 0.5f;
  const int warm = o ? o->warm_start : 0;
  int cfg = o ? o->config : -1;
  if (K < 0 || check_every < 0 || !(gap_tol >= 0.0) || !(alpha >= 0.f && alpha <= 1.f)) return CTV_EINVAL;
  if (warm && c.dual_state == nullptr) return CTV_EINVAL;
  if (cfg >= kNumCfgs || cfg < -1) return CTV_EINVAL;
  ConsDev C;
  if (!convert_constraint(c.C, c.m, c.n, &C)) return CTV_EINVAL;
  if (cfg < 0) cfg = default_config(c.m, c.n, K, c.tv, cons_mode(C), check_every);
  if (c.workspace_bytes < denoise_workspace_bytes(c.batch, c.m, c.n)) return CTV_EINVAL;

  cudaStream_t s = (cudaStream_t)c.stream;
  const size_t px = (size_t)c.m * c.n;
  char* ws = (char*)c.workspace;
  DevStats* st = (DevStats*)ws;
  size_t off = align256((size_t)c.batch * 256);
  float* slots = (float*)(ws + off);
  const long long slot_stride = 8 * (long long)gap_slots_per_image(c.m, c.n);
  off += align256((size_t)c.batch * gap_slots_per_image(c.m, c.n) * 32);
  float4* set_q[2];
  float4* set_r[2];
  const size_t dbytes = align256((size_t)c.batch * px * sizeof(float4));
  set_q[0] = (float4*)(ws + off); off += dbytes;
  set_r[0] = (float4*)(ws + off); off += dbytes;
  set_q[1] = (float4*)(ws + off); off += dbytes;
  set_r[1] = (float4*)(ws + off); off += dbytes;

  if (cudaMemsetAsync(st, 0, (size_t)c.batch * sizeof(DevStats), s) != cudaSuccess) return CTV_ECUDA;

  const bool lam_zero = c.lam_dev == nullptr && c.lam == 0.f;
  const Cfg& cf = kCfgs[cfg];
  GapParams g;
  memset(&g, 0, sizeof(g));
  g.b = (const float2*)c.b;
  g.b_stride = c.batch_stride;
  g.ld = c.ld;
  g.qA = set_q[0];
  g.qB = set_q[1];
  g.d_stride = (long long)px;
  g.dual_in = (const float4*)c.dual_state;
  g.m = c.m;
  g.n = c.n;
  g.lam = c.lam;
  g.lam_dev = c.lam_dev;
  g.alpha = alpha;
  g.C = C;
  g.st = st;
  g.slots = slots;
  g.slot_stride = slot_stride;
  g.gap_tol = gap_tol;

  // the passes, checks and finalize of the solve, onto stream es, or (sg != nullptr) into a
  // stop graph whose check intervals are conditional nodes
  auto enqueue = [&](cudaStream_t es, StopGraph* sg) -> ctv_status {
    GapParams gg = g;
    int last_set = -1;   // -1: no pass has run
    if (K > 0 && !lam_zero) {
      std::vector<double> beta;
      nesterov_betas(K, &beta);
      if (o != nullptr && o->plain_gp) std::fill(beta.begin(), beta.end(), 0.0);   // Eq. (21): r_{k+1} = q_k
      PassParams p;
      memset(&p, 0, sizeof(p));
      p.b = (const float2*)c.b;
      p.b_stride = c.batch_stride;
      p.ld = c.ld;
      p.d_stride = (long long)px;
      p.m = c.m;
      p.n = c.n;
      p.lam = c.lam;
      p.lam_dev = c.lam_dev;
      p.alpha = alpha;
      p.C = C;
      // the stop flag is read by every block before its loads; without a stopping test
      // nobody sets it, so the passes skip that read
      p.st = check_every > 0 && gap_tol > 0.0 ? st : nullptr;
      const dim3 grid = pass_grid(cfg, c.m, c.n, c.batch);
      if (grid.y > 65535) return CTV_EINVAL;
      int k = 1;
      int out = 0;
      const float4* q_in = (const float4*)c.dual_state;
      const float4* r_in = (const float4*)c.dual_state;
      bool first = !warm;
      // measurement: mode 1 times every pass, mode 2 each run of passes up to a check
      const int pmode = sg == nullptr ? prof_mode() : 0;
      int run_slot = -1, run_n = 0;
      double run_units = 0.0;
      auto close_run = [&](cudaStream_t rs) {
        if (run_slot >= 0) prof_end(run_slot, rs, run_units, run_n);
        run_slot = -1;
        run_n = 0;
        run_units = 0.0;
      };
      while (k <= K) {
        if (sg != nullptr && !sg->open) {
          es = sg->open_interval();
          if (es == nullptr) return CTV_ECUDA;
        }
        int steps = K - k + 1;
        if (steps > cf.T) steps = cf.T;
        if (check_every > 0) {
          const int to_check = check_every - ((k - 1) % check_every);
          if (steps > to_check) steps = to_check;
        }
        for (int i = 0; i < 8; ++i) p.beta[i] = i < steps ? (float)beta[(size_t)k + i] : 0.f;
        p.nsteps = steps;
        p.first = first ? 1 : 0;
        // every other pass walks the tiles in reverse order, so that it starts on
        // the tiles the previous pass wrote last, whose q and r are still in L2
        p.reverse = out;
        p.q_in = q_in;
        p.r_in = r_in;
        p.q_out = set_q[out];
        p.r_out = set_r[out];
        const double units = (double)c.batch * (double)px * (double)steps;
        // A check after this pass is evaluated inside it when it runs fewer than T steps
        // (then q_k is exact one ring beyond the tile interiors, all the gap terms need).
        const bool check_after = check_every > 0 && (k + steps - 1) % check_every == 0 && k + steps - 1 < K;
        const bool fused_check = check_after && steps < cf.T && pass_gap_eval_ok(cfg) &&
                                 (size_t)grid.x * grid.y <= gap_slots_per_image(c.m, c.n);
        p.gap_eval = fused_check ? 1 : 0;
        if (fused_check) {
          p.gst = st;
          p.slots = slots;
          p.slot_stride = slot_stride;
          close_run(es);   // (timing runs cover plain passes only)
        }
        const int slot = pmode == 1 && !fused_check ? prof_begin(es) : -1;
        if (pmode == 2 && run_slot < 0 && !fused_check) run_slot = prof_begin(es);
        if (launch_pass(c.tv, cfg, p, grid, es) != cudaSuccess) return CTV_ECUDA;
        count_launch();
        if (sg != nullptr) sg->kernels++;
        prof_end(slot, es, units, 1);
        if (!fused_check) {
          run_units += units;
          ++run_n;
        }
        first = false;
        k += steps;
        last_set = out;
        q_in = set_q[out];
        r_in = set_r[out];
        out ^= 1;
        if (fused_check) {
          // the passes' block sums, evaluated and tested by one block per image
          GapFinishParams f;
          memset(&f, 0, sizeof(f));
          f.st = st;
          f.slots = slots;
          f.slot_stride = slot_stride;
          f.nblk = grid.x * grid.y;
          f.lam = c.lam;
          f.lam_dev = c.lam_dev;
          f.set = last_set;
          f.iter = k - 1;
          f.gap_tol = gap_tol;
          f.final_call = 0;
          if (sg != nullptr) {
            sg->later_handles(&gg);
            f.n_cond = gg.n_cond;
            for (int i = 0; i < gg.n_cond; ++i) f.cond[i] = gg.cond[i];
          }
          if (launch_gap_finish(f, c.batch, es) != cudaSuccess) return CTV_ECUDA;
          count_launch();
          if (sg != nullptr) {
            sg->kernels++;
            if (!sg->close_interval()) return CTV_ECUDA;
          }
        } else if (check_after) {
          close_run(es);
          gg.default_set = last_set;
          gg.zero_q = 0;
          gg.x = nullptr;
          gg.q_export = nullptr;
          gg.iter = k - 1;
          gg.final_call = 0;
          if (sg != nullptr) sg->later_handles(&gg);
          else gg.n_cond = 0;
          if (launch_gap(c.tv, gg, c.batch, es) != cudaSuccess) return CTV_ECUDA;
          count_launches(2);
          if (sg != nullptr) {
            sg->kernels += 2;
            if (!sg->close_interval()) return CTV_ECUDA;
          }
        }
      }
      close_run(es);
      if (sg != nullptr && sg->open && !sg->close_interval()) return CTV_ECUDA;
    }
    // finalize: x = P_C(b - lam L^T q_K), final statistics, optional export of q_K
    if (sg != nullptr) {
      es = sg->open_final();
      if (es == nullptr) return CTV_ECUDA;
    }
    gg.x = (float2*)c.x;
    gg.x_stride = c.batch_stride;
    gg.q_export = (float4*)c.dual_state;
    gg.final_call = 1;
    gg.n_cond = 0;
    gg.iter = (K > 0 && !lam_zero) ? K : 0;
    if (last_set >= 0) {
      gg.default_set = last_set;
      gg.zero_q = 0;
    } else if (warm) {
      gg.default_set = 2;   // the warm-start dual itself
      gg.zero_q = lam_zero ? 1 : 0;
    } else {
      gg.default_set = 0;
      gg.zero_q = 1;
    }
    if (warm && last_set < 0 && gg.q_export == gg.dual_in) gg.q_export = nullptr;  // unchanged
    // without gap checks and with nobody reading the statistics, only x (and q) are written
    const bool light = c.stats == nullptr && check_every == 0;
    if (light && c.mom_z != nullptr && c.batch == 1) {
      gg.mom_z = c.mom_z;
      gg.mom_ld = c.mom_ld;
      gg.mom_xprev = c.mom_xprev;
      gg.mom_beta = c.mom_beta;
      if (c.mom_written != nullptr) *c.mom_written = 1;
    }
    if ((light ? launch_finalize(gg, c.batch, es) : launch_gap(c.tv, gg, c.batch, es)) != cudaSuccess)
      return CTV_ECUDA;
    count_launches(light ? 1 : 2);
    if (sg != nullptr) {
      sg->kernels += light ? 1 : 2;
      if (!sg->close_final()) return CTV_ECUDA;
    }
    return CTV_OK;
  };

  // Solves that can stop early run, on large images, as a cached CUDA graph whose
  // check intervals are conditional nodes (see StopGraph); otherwise, and if the
  // graph cannot be built, the launches go straight onto the stream.
  bool done = false;
  // (one image only: in a batch each image stops on its own, and a check clears the
  // graph's handles for the whole launch)
  if (!c.plain_launches && c.batch == 1 && K > check_every && check_every > 0 && gap_tol > 0.0 && !lam_zero &&
      (K + check_every - 1) / check_every <= CTV_MAX_STOP_INTERVALS && (double)px >= kStopGraphMinPixels &&
      !prof_active() && !stream_capturing(s)) {
    std::string key = stop_graph_key(c, C, cfg);
    int kernels = 0;
    cudaGraphExec_t ex = stop_graph_lookup(key, &kernels);
    const bool hit = ex != nullptr;
    if (ex == nullptr && stop_graph_seen_before(key)) {
      StopGraph sg;
      if (sg.begin((K + check_every - 1) / check_every)) {
        const ctv_status est = enqueue(nullptr, &sg);
        if (est == CTV_OK) ex = sg.instantiate();
        kernels = sg.kernels;
        if (ex != nullptr) stop_graph_store(key, ex, kernels);
      }
      cudaGetLastError();   // a failed build falls back to plain launches
    }
    if (ex != nullptr) {
      if (cudaGraphLaunch(ex, s) != cudaSuccess) return CTV_ECUDA;
      if (hit) count_launches(kernels);   // a new graph counted its kernels as it was built
      done = true;
    }
  }
  if (!done) {
    const ctv_status est = enqueue(s, nullptr);
    if (est != CTV_OK) return est;
  }

  if (c.stats != nullptr) {
    std::vector<DevStats> hs((size_t)c.batch);
    if (cudaMemcpyAsync(hs.data(), st, (size_t)c.batch * sizeof(DevStats), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return CTV_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CTV_ECUDA;
    for (int i = 0; i < c.batch; ++i) {
      c.stats[i].iters = hs[i].iters;
      c.stats[i].stopped = hs[i].stop;
      c.stats[i].primal = hs[i].primal;
      c.stats[i].dual = hs[i].dual;
      c.stats[i].gap = hs[i].gap;
      c.stats[i].status = hs[i].status;
    }
  }
  return CTV_OK;
}

int num_configs() { return kNumCfgs; }
bool config_info(int i, int* T, int* RW, int* RH, int* NT) {
  if (i < 0 || i >= kNumCfgs) return false;
  if (T) *T = kCfgs[i].T;
  if (RW) *RW = kCfgs[i].RW;
  if (RH) *RH = kCfgs[i].RH;
  if (NT) *NT = kCfgs[i].NT;
  return true;
}

}  // namespace ctv

// ----------------------------------------------------------------------------
// C ABI
// ----------------------------------------------------------------------------
extern "C" {

size_t ctv_denoise_workspace_size(int batch, int m, int n) { return ctv::denoise_workspace_bytes(batch, m, n); }

int ctv_denoise(const void* b, void* x, int m, int n, int ld, float lambda, const ctv_constraint* C,
                int tv_type, const ctv_opts* opts, void* dual_state, void* workspace, size_t workspace_bytes,
                ctv_stats* stats, ctv_stream stream) {
  ctv::DenoiseCall c;
  memset(&c, 0, sizeof(c));
  c.b = b;
  c.x = x;
  c.batch = 1;
  c.m = m;
  c.n = n;
  c.ld = ld;
  c.batch_stride = 0;
  c.lam = lambda;
  c.lam_dev = nullptr;
  c.C = C;
  c.tv = tv_type;
  c.opts = opts;
  c.dual_state = dual_state;
  c.workspace = workspace;
  c.workspace_bytes = workspace_bytes;
  c.stats = stats;
  c.stream = stream;
  return ctv::run_denoise(c);
}

int ctv_denoise_batched(const void* b, void* x, int batch, int m, int n, int ld, long long batch_stride,
                        const float* lambdas, const ctv_constraint* C, int tv_type, const ctv_opts* opts,
                        void* dual_state, void* workspace, size_t workspace_bytes, ctv_stats* stats,
                        ctv_stream stream) {
  if (lambdas == nullptr || ((uintptr_t)lambdas & 3)) return CTV_EINVAL;
  if (batch > 1 && batch_stride < (long long)m * ld) return CTV_EINVAL;
  ctv::DenoiseCall c;
  memset(&c, 0, sizeof(c));
  c.b = b;
  c.x = x;
  c.batch = batch;
  c.m = m;
  c.n = n;
  c.ld = ld;
  c.batch_stride = batch_stride;
  c.lam = 0.f;
  c.lam_dev = lambdas;
  c.C = C;
  c.tv = tv_type;
  c.opts = opts;
  c.dual_state = dual_state;
  c.workspace = workspace;
  c.workspace_bytes = workspace_bytes;
  c.stats = stats;
  c.stream = stream;
  return ctv::run_denoise(c);
}

int ctv_num_configs(void) { return ctv::num_configs(); }

int ctv_default_config(int m, int n, int iters, int tv_type, const ctv_constraint* C) {
  ctv::ConsDev cd;
  if (!ctv::convert_constraint(C, m, n, &cd)) return -1;
  return ctv::default_config(m, n, iters, tv_type, ctv::cons_mode(cd));
}

int ctv_config_info(int config, int* iters_per_pass, int* region_w, int* region_h, int* threads) {
  return ctv::config_info(config, iters_per_pass, region_w, region_h, threads) ? CTV_OK : CTV_EINVAL;
}

}  // extern "C"
