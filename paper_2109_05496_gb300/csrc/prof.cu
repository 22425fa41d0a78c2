// Kernel-level timing of the fused FGP pass with CUDA events, for measurement.
//
// Mode 1 brackets every launch of the fused pass kernel with two events recorded
// on the launching stream. Mode 2 brackets each run of consecutive pass launches
// of a solve instead (closed before a gap check or the finalize), so that the
// passes inside a run keep their back-to-back overlap (programmatic dependent
// launch) and the time is that of the pass sequence itself. ctv_profile_read
// sums the bracketed times. Every kernel launch of the library is counted
// whether or not timing is enabled.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "ctv.h"
#include "ctv_host.h"

namespace ctv {

namespace {
std::mutex g_mu;
int g_mode = 0;                  // 0 off, 1 per launch, 2 per run of consecutive passes
std::vector<cudaEvent_t> g_ev;   // pairs (start, stop)
size_t g_used = 0;               // pairs in use
double g_units = 0.0;            // pixel-iterations of the timed launches
long long g_timed = 0;           // pass launches inside the bracketed intervals
std::atomic<long long> g_launches{0};
long long g_launch_base = 0;
}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
bool prof_active() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_mode != 0;
}

int prof_mode() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_mode;
}

int prof_begin(cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_mode == 0) return -1;
  if (g_used * 2 + 2 > g_ev.size()) {
    for (int i = 0; i < 2; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      g_ev.push_back(e);
    }
  }
  const int slot = (int)g_used++;
  cudaEventRecord(g_ev[2 * slot], s);
  return slot;
}

void prof_end(int slot, cudaStream_t s, double units, int launches) {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEventRecord(g_ev[2 * slot + 1], s);
  g_units += units;
  g_timed += launches;
}

}  // namespace ctv

extern "C" {

int ctv_profile_enable(int on) {
  if (on < 0 || on > 2) return CTV_EINVAL;
  std::lock_guard<std::mutex> lk(ctv::g_mu);
  ctv::g_mode = on;
  ctv::g_used = 0;
  ctv::g_units = 0.0;
  ctv::g_timed = 0;
  ctv::g_launch_base = ctv::g_launches.load();
  return CTV_OK;
}

int ctv_profile_read(double* pass_ms, long long* pass_launches, double* pass_pixel_iters, long long* all_launches) {
  std::lock_guard<std::mutex> lk(ctv::g_mu);
  double total = 0.0;
  for (size_t i = 0; i < ctv::g_used; ++i) {
    if (cudaEventSynchronize(ctv::g_ev[2 * i + 1]) != cudaSuccess) return CTV_ECUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctv::g_ev[2 * i], ctv::g_ev[2 * i + 1]) != cudaSuccess) return CTV_ECUDA;
    total += ms;
  }
  if (pass_ms) *pass_ms = total;
  if (pass_launches) *pass_launches = ctv::g_timed;
  if (pass_pixel_iters) *pass_pixel_iters = ctv::g_units;
  if (all_launches) *all_launches = ctv::g_launches.load() - ctv::g_launch_base;
  return CTV_OK;
}

}  // extern "C"
