// Autotuner for the fused FGP pass: picks the kernel configuration (temporal
// blocking depth and tile shape) by timing every configuration on the caller's
// own data, and remembers the winner per (size class, TV type) for the
// configuration-selecting default (opts->config = -1) of every entry point.
//
// The size class of an m x n image is floor(log2(m * n)); the table starts with
// the choices measured on GB300 and can be read and written so that a caller
// can persist it (the Python package keeps a JSON cache per GPU name).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "ctv.h"
#include "ctv_host.h"

namespace ctv {

namespace {
constexpr int kClasses = 40;
std::mutex g_mu;
// one table per device ordinal (tuned choices are facts about one GPU); the last
// slot serves devices with ordinals beyond the cached range
int g_table[kMaxDevices + 1][kClasses][4];   // -1: not tuned
bool g_init = false;

void init_locked() {
  if (g_init) return;
  for (int d = 0; d <= kMaxDevices; ++d)
    for (int c = 0; c < kClasses; ++c)
      for (int t = 0; t < 4; ++t) g_table[d][c][t] = -1;
  g_init = true;
}

int (&table_of_current_device())[kClasses][4] {
  const int d = device_slot();
  return g_table[d >= 0 ? d : kMaxDevices];
}
}  // namespace

int size_class(int m, int n) {
  const double px = (double)m * (double)n;
  int c = px >= 1.0 ? (int)floor(log2(px)) : 0;
  return c < 0 ? 0 : (c >= kClasses ? kClasses - 1 : c);
}

int tuned_config(int m, int n, int tv) {
  std::lock_guard<std::mutex> lk(g_mu);
  init_locked();
  if (tv < 0 || tv > 3) return -1;
  return table_of_current_device()[size_class(m, n)][tv];
}

}  // namespace ctv

extern "C" {

int ctv_tune_set(int size_class, int tv_type, int config) {
  using namespace ctv;
  if (size_class < 0 || size_class >= kClasses || tv_type < 0 || tv_type > 3) return CTV_EINVAL;
  if (config < -1 || config >= num_configs()) return CTV_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  init_locked();
  table_of_current_device()[size_class][tv_type] = config;
  return CTV_OK;
}

int ctv_tune_get(int size_class, int tv_type, int* config) {
  using namespace ctv;
  if (config == nullptr || size_class < 0 || size_class >= kClasses || tv_type < 0 || tv_type > 3) return CTV_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  init_locked();
  *config = table_of_current_device()[size_class][tv_type];
  return CTV_OK;
}

int ctv_size_class(int m, int n) { return (m <= 0 || n <= 0) ? -1 : ctv::size_class(m, n); }

int ctv_autotune_denoise(const void* b, void* x, int m, int n, int ld, float lambda, const ctv_constraint* C,
                         int tv_type, const ctv_opts* opts, void* workspace, size_t workspace_bytes, int repeats,
                         int* best_config, float* times_ms, ctv_stream stream) {
  using namespace ctv;
  if (opts == nullptr || best_config == nullptr || repeats < 1) return CTV_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return CTV_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return CTV_ECUDA;
  }
  int best = -1;
  float best_ms = 0.f;
  ctv_status status = CTV_OK;
  for (int cfg = 0; cfg < num_configs() && status == CTV_OK; ++cfg) {
    ctv_opts o = *opts;
    o.config = cfg;
    o.warm_start = 0;
    o.gap_tol = 0.0;
    o.check_every = 0;
    DenoiseCall c;
    memset(&c, 0, sizeof(c));
    c.b = b; c.x = x; c.batch = 1; c.m = m; c.n = n; c.ld = ld; c.lam = lambda; c.C = C; c.tv = tv_type;
    c.opts = &o; c.workspace = workspace; c.workspace_bytes = workspace_bytes; c.stream = stream;
    status = run_denoise(c);   // warm-up (also validates the arguments)
    if (status != CTV_OK) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < repeats && status == CTV_OK; ++r) status = run_denoise(c);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) { status = CTV_ECUDA; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= (float)repeats;
    if (times_ms != nullptr) times_ms[cfg] = ms;
    if (best < 0 || ms < best_ms) { best = cfg; best_ms = ms; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != CTV_OK) return status;
  *best_config = best;
  return ctv_tune_set(size_class(m, n), tv_type, best);
}

}  // extern "C"
