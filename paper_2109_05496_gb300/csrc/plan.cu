// Batched denoising of many images of uneven sizes in one launch per pass.
//
// A plan holds, in one device allocation, a descriptor per image (its own m, n,
// lambda, alpha, TV type, C and dual buffers) and two work lists of tiles over
// all images: one for the fused FGP pass, one for the gap / finalize
// evaluation. Each pass of Algorithm 2 is then one launch per TV type present,
// whose blocks each take one tile of one image of that type, so small images no
// longer pay a launch each and each launch keeps the register budget of its type. The whole schedule (zeroing of the per-image
// records, the passes, the optional gap checks and the finalize) is captured
// once into a CUDA graph on a private stream and replayed on the caller's stream
// by ctv_plan_execute. Every image keeps its own stopping test.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "async_status.cuh"
#include "ctv.h"
#include "ctv_configs.cuh"
#include "ctv_device.cuh"
#include "gap_device.cuh"
#include "ctv_host.h"
#include "ctv_kernels.h"
#include "plan_list.cuh"

namespace ctv {

struct ListGapParams {
  const PlanImg* imgs;
  const WorkItem* items;
  int n_items;
  int default_set;
  int zero_q;
  int iter;
  double gap_tol;
  int final_call;
};

__device__ __forceinline__ void list_gap_commit(const PlanImg* d, GapSums& gsum, float2* red, unsigned units,
                                                int set, int stopped, int iter, double gap_tol, int final_call,
                                                int* last, bool& nf) {
  const bool block_nf = __syncthreads_or(nf) != 0;
  if (block_nf && threadIdx.x == 0) raise_async(CTV_ENONFINITE);
  float hs[3], ls[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    hs[a] = gsum.s[a];
    ls[a] = -gsum.c[a];
    gsum.s[a] = gsum.c[a] = 0.f;
  }
  block_sum_pairs<GAP_NT, 3>(hs, ls, red);
  const double acc[3] = {(double)hs[0] + (double)ls[0], (double)hs[1] + (double)ls[1], (double)hs[2] + (double)ls[2]};
  gap_commit(d->st, acc, d->gnblk, units, d->lam, false, set, stopped, iter, gap_tol, final_call, last, block_nf);
  nf = false;
}

// Persistent: each block walks a contiguous run of gap tiles (items are in
// image order, so a run covers one image or a few), keeps per-thread FP64 sums
// while the image stays the same and commits them - one block reduction and one
// set of atomics - when the image changes or the run ends. A commit counts the
// tiles it covers, so an image's reduction completes with its last tile.
__global__ void __launch_bounds__(GAP_NT, 4) fgp_gap_list_kernel(ListGapParams p) {
  __shared__ float4 qs[GAP_RW * GAP_RH];
  __shared__ float2 xs[GAP_RW * GAP_RH];
  __shared__ float2 red[3 * (GAP_NT / 32)];
  __shared__ int last;
  const int per = (p.n_items + (int)gridDim.x - 1) / (int)gridDim.x;
  const int i0 = (int)blockIdx.x * per, i1 = min(i0 + per, p.n_items);
  GapSums acc = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, false};
  bool nf = false;
  int cur = -1, cur_set = 0, cur_stopped = 0;
  unsigned units = 0;
  for (int i = i0; i < i1; ++i) {
    const WorkItem w = p.items[i];
    if (w.img != cur && units > 0) {
      list_gap_commit(p.imgs + cur, acc, red, units, cur_set, cur_stopped, p.iter, p.gap_tol, p.final_call, &last,
                      nf);
      units = 0;
    }
    cur = w.img;
    const PlanImg& d = p.imgs[w.img];
    // (an image's stop flag cannot change while its tiles are being evaluated:
    // it is set only by the commit that completes the image)
    const int stopped = *(volatile int*)&d.st->stop;
    if (!p.final_call && stopped) continue;
    const int set = stopped ? d.st->stop_set : p.default_set;
    cur_set = set;
    cur_stopped = stopped;
    GapImg g;
    g.b = d.b;
    g.ld = d.ld;
    g.q = (p.zero_q && !stopped) ? nullptr : d.q[set];
    g.x = p.final_call ? d.x : nullptr;
    g.q_export = nullptr;
    g.m = d.m;
    g.n = d.n;
    g.lam = d.lam;
    g.alpha = d.alpha;
    g.C = d.C;
    const int j0 = (w.tile / d.gtiles_x) * (GAP_RH - 2), k0 = (w.tile % d.gtiles_x) * (GAP_RW - 2);
    switch (d.tv) {
      case TV1_ISO: gap_tile_add<TV1_ISO>(g, j0, k0, qs, xs, acc, nf); break;
      case TV1_ANISO: gap_tile_add<TV1_ANISO>(g, j0, k0, qs, xs, acc, nf); break;
      case TV2_ISO: gap_tile_add<TV2_ISO>(g, j0, k0, qs, xs, acc, nf); break;
      default: gap_tile_add<TV2_ANISO>(g, j0, k0, qs, xs, acc, nf); break;
    }
    __syncthreads();   // qs and xs are reused by the next tile
    ++units;
  }
  if (units > 0)
    list_gap_commit(p.imgs + cur, acc, red, units, cur_set, cur_stopped, p.iter, p.gap_tol, p.final_call, &last,
                      nf);
}

int take_async_status_plan() { return take_unit_async_status(); }

// Blocks of a gap / finalize launch: resident blocks, at most one per item.
static int gap_list_blocks(int n_items) {
  static int per_sm_cache[kMaxDevices] = {};
  const int per_sm = occupancy_once((const void*)fgp_gap_list_kernel, GAP_NT, per_sm_cache);
  const long long cap = (long long)per_sm * sm_count();
  return (int)(n_items < cap ? n_items : cap);
}

static bool plan_config_ok(int cfg) {
#define CTV_PLAN_ID(id, kind, T, A, B, C) if (cfg == id) return true;
  CTV_PLAN_CONFIGS(CTV_PLAN_ID)
#undef CTV_PLAN_ID
  return false;
}

// One launch over the work items of the images of one TV type (items sorted by
// type), so that every launch uses the register budget of that type alone.
static cudaError_t launch_list(int tv, int cfg, int cons, const ListPassParams& p, int nblocks, cudaStream_t s,
                               bool set_attr) {
  switch (tv) {
    case TV1_ISO: return launch_plan_list_tv<TV1_ISO>(cfg, cons, p, nblocks, s, set_attr);
    case TV1_ANISO: return launch_plan_list_tv<TV1_ANISO>(cfg, cons, p, nblocks, s, set_attr);
    case TV2_ISO: return launch_plan_list_tv<TV2_ISO>(cfg, cons, p, nblocks, s, set_attr);
    default: return launch_plan_list_tv<TV2_ANISO>(cfg, cons, p, nblocks, s, set_attr);
  }
}

static size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace ctv

struct ctv_plan {
  int count;
  int K, check_every;
  double gap_tol;
  int cfg;
  char* dev;
  size_t bytes;
  ctv::PlanImg* d_imgs;
  ctv::WorkItem* d_pass;
  int n_pass;
  int tv_begin[5];   // pass items of TV type t are [tv_begin[t], tv_begin[t + 1])
  int cons;          // constraint specialisation shared by every image (CONS_GEN if they differ)
  ctv::WorkItem* d_gap;
  int n_gap;
  ctv::DevStats* d_st;
  std::vector<double> beta;
  cudaStream_t cap;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  int launches_per_execute;
  double pixel_iters;
};

namespace ctv {

// The schedule of one execution, captured on s. The passes of different TV types
// touch different images, so each type's passes form their own chain (streams
// aux[t], forked from s and joined back at every gap launch): in the graph the
// four chains run concurrently and fill each other's launch tails.
static ctv_status plan_enqueue(ctv_plan* P, cudaStream_t s, const cudaStream_t* aux, cudaEvent_t* ev) {
  if (cudaMemsetAsync(P->d_st, 0, sizeof(DevStats) * (size_t)P->count, s) != cudaSuccess) return CTV_ECUDA;
  auto fork = [&]() -> bool {
    if (cudaEventRecord(ev[4], s) != cudaSuccess) return false;
    for (int t = 0; t < 4; ++t)
      if (cudaStreamWaitEvent(aux[t], ev[4], 0) != cudaSuccess) return false;
    return true;
  };
  auto join = [&]() -> bool {
    for (int t = 0; t < 4; ++t)
      if (cudaEventRecord(ev[t], aux[t]) != cudaSuccess || cudaStreamWaitEvent(s, ev[t], 0) != cudaSuccess)
        return false;
    return true;
  };
  if (!fork()) return CTV_ECUDA;
  int launches = 0;
  int last_set = -1;
  int T = 1;
  config_info(P->cfg, &T, nullptr, nullptr, nullptr);
  const int K = P->K, every = P->check_every;
  ListGapParams g;
  memset(&g, 0, sizeof(g));
  g.imgs = P->d_imgs;
  g.items = P->d_gap;
  g.n_items = P->n_gap;
  const int gap_grid = gap_list_blocks(P->n_gap);
  g.gap_tol = P->gap_tol;
  if (K > 0) {
    ListPassParams p;
    memset(&p, 0, sizeof(p));
    p.imgs = P->d_imgs;
    p.items = P->d_pass;
    int k = 1, out = 0;
    bool first = true;
    while (k <= K) {
      int steps = std::min(T, K - k + 1);
      if (every > 0) steps = std::min(steps, every - ((k - 1) % every));
      for (int i = 0; i < 8; ++i) p.beta[i] = i < steps ? (float)P->beta[(size_t)k + i] : 0.f;
      p.nsteps = steps;
      p.first = first ? 1 : 0;
      p.can_stop = every > 0 ? 1 : 0;
      p.in_set = out ^ 1;
      p.out_set = out;
      for (int t = 0; t < 4; ++t) {
        const int nb = P->tv_begin[t + 1] - P->tv_begin[t];
        if (nb == 0) continue;
        p.items = P->d_pass + P->tv_begin[t];
        if (launch_list(t, P->cfg, P->cons, p, nb, aux[t], false) != cudaSuccess) return CTV_ECUDA;
        ++launches;
      }
      first = false;
      k += steps;
      last_set = out;
      out ^= 1;
      if (every > 0 && (k - 1) % every == 0 && k - 1 < K) {
        g.default_set = last_set;
        g.zero_q = 0;
        g.iter = k - 1;
        g.final_call = 0;
        if (!join()) return CTV_ECUDA;
        fgp_gap_list_kernel<<<gap_grid, GAP_NT, 0, s>>>(g);
        if (cudaGetLastError() != cudaSuccess) return CTV_ECUDA;
        ++launches;
        if (!fork()) return CTV_ECUDA;
      }
    }
  }
  g.default_set = last_set >= 0 ? last_set : 0;
  g.zero_q = last_set < 0 ? 1 : 0;
  g.iter = K;
  g.final_call = 1;
  if (!join()) return CTV_ECUDA;
  fgp_gap_list_kernel<<<gap_grid, GAP_NT, 0, s>>>(g);
  if (cudaGetLastError() != cudaSuccess) return CTV_ECUDA;
  ++launches;
  P->launches_per_execute = launches;
  return CTV_OK;
}

}  // namespace ctv

extern "C" {

int ctv_plan_create(const ctv_image_desc* descs, int count, const ctv_opts* opts, ctv_plan** out) {
  using namespace ctv;
  if (out == nullptr) return CTV_EINVAL;
  *out = nullptr;
  if (descs == nullptr || count <= 0 || opts == nullptr) return CTV_EINVAL;
  if (opts->max_iters < 0 || opts->check_every < 0 || !(opts->gap_tol >= 0.0) || opts->warm_start) return CTV_EINVAL;
  if (opts->plain_gp) return CTV_EUNSUPPORTED;
  if (opts->config == CTV_CONFIG_AUTOTUNE) {
    // time one execution of a plan in each supported configuration on these images
    // (one candidate's memory at a time) and build the fastest
    cudaStream_t ts;
    if (cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking) != cudaSuccess) return CTV_ECUDA;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) { cudaStreamDestroy(ts); return CTV_ECUDA; }
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); cudaStreamDestroy(ts); return CTV_ECUDA; }
    int best = -1;
    float best_ms = 0.f;
    ctv_status st = CTV_OK;
    ctv_opts o = *opts;
#define CTV_PLAN_TRY(id, kind, T, A, B, C)                                                    \
    if (st == CTV_OK) {                                                                       \
      o.config = id;                                                                          \
      ctv_plan* cand = nullptr;                                                               \
      st = (ctv_status)ctv_plan_create(descs, count, &o, &cand);                              \
      if (st == CTV_OK) {                                                                     \
        float ms = 0.f;                                                                       \
        if (ctv_plan_execute(cand, (ctv_stream)ts) != CTV_OK || cudaEventRecord(e0, ts) != cudaSuccess || \
            ctv_plan_execute(cand, (ctv_stream)ts) != CTV_OK || cudaEventRecord(e1, ts) != cudaSuccess || \
            cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) \
          st = CTV_ECUDA;                                                                     \
        else if (best < 0 || ms < best_ms) {                                                  \
          best = id;                                                                          \
          best_ms = ms;                                                                       \
        }                                                                                     \
        ctv_plan_destroy(cand);                                                               \
      }                                                                                       \
    }
    CTV_PLAN_CONFIGS(CTV_PLAN_TRY)
#undef CTV_PLAN_TRY
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(ts);
    if (st != CTV_OK) return st;
    o.config = best;
    return ctv_plan_create(descs, count, &o, out);
  }
  int cfg = opts->config;
  if (cfg < -1 || cfg >= num_configs()) return CTV_EINVAL;
  if (cfg < 0) cfg = default_config(0, 0, opts->max_iters, -1, CONS_AMP);
  if (!plan_config_ok(cfg)) return CTV_EUNSUPPORTED;
  int T = 1, RW = 0, RH = 0, NT = 0;
  config_info(cfg, &T, &RW, &RH, &NT);
  const int TW = RW - 2 * T, TH = RH - 2 * T;
  const int GW = GAP_RW - 2, GH = GAP_RH - 2;

  std::vector<PlanImg> imgs((size_t)count);
  std::vector<WorkItem> pass_items, gap_items;
  size_t state_bytes = 0;
  double px_total = 0.0;
  for (int i = 0; i < count; ++i) {
    const ctv_image_desc& d = descs[i];
    if (d.b == nullptr || d.x == nullptr || d.m <= 0 || d.n <= 0 || d.ld < d.n) return CTV_EINVAL;
    if (((uintptr_t)d.b & 7) || ((uintptr_t)d.x & 7)) return CTV_EINVAL;
    if (!(d.lambda >= 0.f) || isinf(d.lambda) || d.tv_type < 0 || d.tv_type > 3) return CTV_EINVAL;
    if (!(d.alpha >= 0.f && d.alpha <= 1.f)) return CTV_EINVAL;
    PlanImg& p = imgs[(size_t)i];
    memset(&p, 0, sizeof(p));
    if (!convert_constraint(&d.C, d.m, d.n, &p.C)) return CTV_EINVAL;
    p.b = (const float2*)d.b;
    p.x = (float2*)d.x;
    p.ld = d.ld;
    p.m = d.m;
    p.n = d.n;
    p.lam = d.lambda;
    p.alpha = d.alpha;
    p.tv = d.tv_type;
    p.tiles_x = (d.n + TW - 1) / TW;
    const int tiles_y = (d.m + TH - 1) / TH;
    p.gtiles_x = (d.n + GW - 1) / GW;
    const int gtiles_y = (d.m + GH - 1) / GH;
    p.gnblk = (unsigned)(p.gtiles_x * gtiles_y);
    for (int t = 0; t < p.tiles_x * tiles_y; ++t) pass_items.push_back({i, t});
    for (int t = 0; t < (int)p.gnblk; ++t) gap_items.push_back({i, t});
    state_bytes += 4 * a256((size_t)d.m * d.n * sizeof(float4));
    px_total += (double)d.m * d.n;
  }
  if (pass_items.size() > 0x7fffffffu || gap_items.size() > 0x7fffffffu) return CTV_EINVAL;
  std::stable_sort(pass_items.begin(), pass_items.end(),
                   [&](const WorkItem& a, const WorkItem& b) { return imgs[(size_t)a.img].tv < imgs[(size_t)b.img].tv; });
  int tv_begin[5] = {0, 0, 0, 0, 0};
  for (const WorkItem& w : pass_items) tv_begin[imgs[(size_t)w.img].tv + 1]++;
  for (int t = 0; t < 4; ++t) tv_begin[t + 1] += tv_begin[t];
  int cons = cons_mode(imgs[0].C);
  for (int i = 1; i < count; ++i)
    if (cons_mode(imgs[(size_t)i].C) != cons) cons = CONS_GEN;

  ctv_plan* P = new ctv_plan();
  P->count = count;
  P->K = opts->max_iters;
  P->check_every = opts->check_every;
  P->gap_tol = opts->gap_tol;
  P->cfg = cfg;
  P->n_pass = (int)pass_items.size();
  for (int t = 0; t < 5; ++t) P->tv_begin[t] = tv_begin[t];
  P->cons = cons;
  P->n_gap = (int)gap_items.size();
  P->pixel_iters = px_total * P->K;
  nesterov_betas(P->K, &P->beta);
  const size_t b_imgs = a256(sizeof(PlanImg) * (size_t)count);
  const size_t b_pass = a256(sizeof(WorkItem) * pass_items.size());
  const size_t b_gap = a256(sizeof(WorkItem) * gap_items.size());
  const size_t b_st = a256(sizeof(DevStats) * (size_t)count);
  P->bytes = b_imgs + b_pass + b_gap + b_st + state_bytes;
  if (cudaMalloc(&P->dev, P->bytes) != cudaSuccess) {
    delete P;
    return CTV_ENOMEM;
  }
  char* c = P->dev;
  P->d_imgs = (PlanImg*)c; c += b_imgs;
  P->d_pass = (WorkItem*)c; c += b_pass;
  P->d_gap = (WorkItem*)c; c += b_gap;
  P->d_st = (DevStats*)c; c += b_st;
  for (int i = 0; i < count; ++i) {
    PlanImg& p = imgs[(size_t)i];
    const size_t db = a256((size_t)p.m * p.n * sizeof(float4));
    p.q[0] = (float4*)c; c += db;
    p.r[0] = (float4*)c; c += db;
    p.q[1] = (float4*)c; c += db;
    p.r[1] = (float4*)c; c += db;
    p.st = P->d_st + i;
  }
  bool ok = cudaMemcpy(P->d_imgs, imgs.data(), sizeof(PlanImg) * (size_t)count, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(P->d_pass, pass_items.data(), sizeof(WorkItem) * pass_items.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(P->d_gap, gap_items.data(), sizeof(WorkItem) * gap_items.size(), cudaMemcpyHostToDevice) == cudaSuccess;
  ListPassParams dummy;
  memset(&dummy, 0, sizeof(dummy));
  for (int t = 0; t < 4; ++t) ok = ok && launch_list(t, cfg, cons, dummy, 0, nullptr, true) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking) == cudaSuccess;
  cudaStream_t aux[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  for (int t = 0; t < 4; ++t) ok = ok && cudaStreamCreateWithFlags(&aux[t], cudaStreamNonBlocking) == cudaSuccess;
  for (int t = 0; t < 5; ++t) ok = ok && cudaEventCreateWithFlags(&ev[t], cudaEventDisableTiming) == cudaSuccess;
  auto drop_aux = [&]() {
    for (int t = 0; t < 4; ++t)
      if (aux[t] != nullptr) cudaStreamDestroy(aux[t]);
    for (int t = 0; t < 5; ++t)
      if (ev[t] != nullptr) cudaEventDestroy(ev[t]);
  };
  if (!ok) {
    drop_aux();
    if (P->cap != nullptr) cudaStreamDestroy(P->cap);
    cudaFree(P->dev);
    delete P;
    return CTV_ECUDA;
  }
  // capture the schedule once
  if (cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    drop_aux();
    cudaStreamDestroy(P->cap);
    cudaFree(P->dev);
    delete P;
    return CTV_ECUDA;
  }
  ctv_status st = plan_enqueue(P, P->cap, aux, ev);
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(P->cap, &graph);
  drop_aux();
  if (st != CTV_OK || ce != cudaSuccess || graph == nullptr ||
      cudaGraphInstantiate(&P->exec, graph, 0) != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(P->cap);
    cudaFree(P->dev);
    delete P;
    return CTV_ECUDA;
  }
  P->graph = graph;
  *out = P;
  return CTV_OK;
}

int ctv_plan_execute(ctv_plan* P, ctv_stream stream) {
  if (P == nullptr) return CTV_EINVAL;
  if (cudaGraphLaunch(P->exec, (cudaStream_t)stream) != cudaSuccess) return CTV_ECUDA;
  for (int i = 0; i < P->launches_per_execute; ++i) ctv::count_launch();
  return CTV_OK;
}

int ctv_plan_stats(const ctv_plan* P, ctv_stats* out, ctv_stream stream) {
  if (P == nullptr || out == nullptr) return CTV_EINVAL;
  std::vector<ctv::DevStats> hs((size_t)P->count);
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(hs.data(), P->d_st, sizeof(ctv::DevStats) * hs.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return CTV_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CTV_ECUDA;
  for (int i = 0; i < P->count; ++i) {
    out[i].iters = hs[(size_t)i].iters;
    out[i].stopped = hs[(size_t)i].stop;
    out[i].primal = hs[(size_t)i].primal;
    out[i].dual = hs[(size_t)i].dual;
    out[i].gap = hs[(size_t)i].gap;
    out[i].status = hs[(size_t)i].status;
  }
  return CTV_OK;
}

int ctv_plan_info(const ctv_plan* P, int* config, int* launches_per_execute, double* pixel_iters, size_t* device_bytes) {
  if (P == nullptr) return CTV_EINVAL;
  if (config) *config = P->cfg;
  if (launches_per_execute) *launches_per_execute = P->launches_per_execute;
  if (pixel_iters) *pixel_iters = P->pixel_iters;
  if (device_bytes) *device_bytes = P->bytes;
  return CTV_OK;
}

void ctv_plan_destroy(ctv_plan* P) {
  if (P == nullptr) return;
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  if (P->cap) cudaStreamDestroy(P->cap);
  cudaFree(P->dev);
  delete P;
}

}  // extern "C"
