// Per-kernel launch statistics: when enabled, every kernel launch of the
// library is bracketed by two CUDA events recorded on the launching stream;
// inolf_stats_read waits for them and accumulates launches and device time
// per kernel name.
#include <cuda_runtime.h>

#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "inolf_internal.h"

namespace inolf {
namespace {

struct Pending {
  std::string name;
  cudaEvent_t a, b;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Pending> g_pending;
std::map<std::string, std::pair<int64_t, double>> g_totals;

}  // namespace

LaunchTimer::LaunchTimer(const char* name, cudaStream_t st) : name_(name), st_(st) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return;
  if (cudaEventCreate((cudaEvent_t*)&a_) != cudaSuccess || cudaEventCreate((cudaEvent_t*)&b_) != cudaSuccess) return;
  cudaEventRecord((cudaEvent_t)a_, st_);
  active_ = true;
}

LaunchTimer::~LaunchTimer() {
  if (!active_) return;
  cudaEventRecord((cudaEvent_t)b_, st_);
  std::lock_guard<std::mutex> lk(g_mu);
  g_pending.push_back({name_, (cudaEvent_t)a_, (cudaEvent_t)b_});
}

}  // namespace inolf

using namespace inolf;

extern "C" inolf_status inolf_stats_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = on != 0;
  return INOLF_OK;
}

extern "C" inolf_status inolf_stats_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& p : g_pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  g_pending.clear();
  g_totals.clear();
  return INOLF_OK;
}

extern "C" inolf_status inolf_stats_read(inolf_kernel_stat* out, int32_t max, int32_t* n) {
  if (!n || max < 0 || (max > 0 && !out)) return fail(INOLF_E_INVALID, "inolf_stats_read: bad argument");
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& p : g_pending) {
    float ms = 0.0f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      auto& t = g_totals[p.name];
      t.first += 1;
      t.second += ms;
    }
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  g_pending.clear();
  int32_t k = 0;
  for (auto& kv : g_totals) {
    if (k < max) {
      std::memset(&out[k], 0, sizeof(inolf_kernel_stat));
      std::strncpy(out[k].name, kv.first.c_str(), sizeof(out[k].name) - 1);
      out[k].launches = kv.second.first;
      out[k].ms = kv.second.second;
    }
    ++k;
  }
  *n = k;
  return INOLF_OK;
}
