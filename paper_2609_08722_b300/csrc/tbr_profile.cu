// Per-kernel device timing: when enabled, every launch of the library's
// kernels is bracketed by a pair of CUDA events recorded on the launch stream,
// so a caller can read each kernel's launch count and summed duration without
// a profiler (the events do not change what the kernels compute).
#include <mutex>
#include <vector>

#include "tbr_host.h"

namespace tbr {
namespace {

struct Pending {
  int kernel;
  cudaEvent_t start, stop;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free;
int64_t g_launches[TBR_K_COUNT] = {0};
double g_ms[TBR_K_COUNT] = {0};

cudaEvent_t take_event() {
  if (!g_free.empty()) {
    cudaEvent_t e = g_free.back();
    g_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void drain_locked() {
  for (const Pending& p : g_pending) {
    float ms = 0.0f;
    if (cudaEventSynchronize(p.stop) == cudaSuccess && cudaEventElapsedTime(&ms, p.start, p.stop) == cudaSuccess) {
      g_launches[p.kernel] += 1;
      g_ms[p.kernel] += ms;
    }
    g_free.push_back(p.start);
    g_free.push_back(p.stop);
  }
  g_pending.clear();
}

}  // namespace

KernelTimer::KernelTimer(int kernel, cudaStream_t st) : kernel_(kernel), st_(st) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return;
  start_ = take_event();
  stop_ = take_event();
  if (start_ && stop_) cudaEventRecord(start_, st_);
  active_ = start_ && stop_;
}

KernelTimer::~KernelTimer() {
  if (!active_) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEventRecord(stop_, st_);
  g_pending.push_back({kernel_, start_, stop_});
}

}  // namespace tbr

using namespace tbr;

extern "C" {

tbr_status tbr_profile_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = on != 0;
  return TBR_OK;
}

tbr_status tbr_profile_read(int32_t kernel, tbr_kernel_time* out) {
  if (kernel < 0 || kernel >= TBR_K_COUNT || !out) return fail(TBR_ERR_INVALID_ARG, "bad kernel id or NULL");
  std::lock_guard<std::mutex> lk(g_mu);
  drain_locked();
  out->launches = g_launches[kernel];
  out->total_ms = g_ms[kernel];
  return TBR_OK;
}

void tbr_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain_locked();
  for (int k = 0; k < TBR_K_COUNT; ++k) {
    g_launches[k] = 0;
    g_ms[k] = 0.0;
  }
}

}  // extern "C"
