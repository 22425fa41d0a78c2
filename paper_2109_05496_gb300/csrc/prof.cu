// Kernel-level timing of the fused FGP pass with CUDA events, for measurement.
//
// While enabled, every launch of the fused pass kernel is bracketed by two
// events recorded on the launching stream; ctv_profile_read sums their elapsed
// times. Every kernel launch of the library is counted whether or not timing
// is enabled.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "ctv.h"
#include "ctv_host.h"

namespace ctv {

namespace {
std::mutex g_mu;
bool g_on = false;
std::vector<cudaEvent_t> g_ev;   // pairs (start, stop)
size_t g_used = 0;               // pairs in use
double g_units = 0.0;            // pixel-iterations of the timed launches
std::atomic<long long> g_launches{0};
long long g_launch_base = 0;
}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
bool prof_active() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_on;
}

int prof_begin(cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return -1;
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

void prof_end(int slot, cudaStream_t s, double units) {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEventRecord(g_ev[2 * slot + 1], s);
  g_units += units;
}

}  // namespace ctv

extern "C" {

int ctv_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(ctv::g_mu);
  ctv::g_on = on != 0;
  ctv::g_used = 0;
  ctv::g_units = 0.0;
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
  if (pass_launches) *pass_launches = (long long)ctv::g_used;
  if (pass_pixel_iters) *pass_pixel_iters = ctv::g_units;
  if (all_launches) *all_launches = ctv::g_launches.load() - ctv::g_launch_base;
  return CTV_OK;
}

}  // extern "C"
