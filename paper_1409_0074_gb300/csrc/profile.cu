// profile.cu -- opt-in per-kernel timing with CUDA events recorded on the
// stream each kernel is launched on (laGP_profile / laGP_profile_read).
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/lagp.h"
#include "lagp_internal.h"

namespace lagp {
namespace {
struct Rec {
  const char* name;
  cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
bool g_suspend = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void recycle_all() {
  for (auto& r : g_recs) {
    if (r.a) g_pool.push_back(r.a);
    if (r.b) g_pool.push_back(r.b);
  }
  g_recs.clear();
}
}  // namespace

void prof_suspend(bool on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_suspend = on;
}

void prof_begin(const char* name, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on || g_suspend) return;
  Rec r{name, take_event(), nullptr};
  if (r.a) cudaEventRecord(r.a, s);
  g_recs.push_back(r);
}

void prof_end(cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on || g_suspend || g_recs.empty() || g_recs.back().b) return;
  g_recs.back().b = take_event();
  if (g_recs.back().b) cudaEventRecord(g_recs.back().b, s);
}

}  // namespace lagp

using namespace lagp;

extern "C" int laGP_profile(int enable) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (enable) {
    for (auto& r : g_recs) {
      if (r.b) cudaEventSynchronize(r.b);
    }
    recycle_all();
  }
  g_on = enable != 0;
  return LAGP_OK;
}

extern "C" int laGP_profile_read(int max_kernels, char* names, double* total_ms,
                                 int32_t* launches) {
  if (max_kernels < 0 || (max_kernels > 0 && (!names || !total_ms || !launches)))
    return LAGP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(g_mu);
  int k = 0;
  for (auto& r : g_recs) {
    if (!r.a || !r.b) continue;
    if (cudaEventSynchronize(r.b) != cudaSuccess) return LAGP_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return LAGP_ERR_CUDA;
    int slot = -1;
    for (int i = 0; i < k; ++i)
      if (std::strncmp(names + 32 * i, r.name, 31) == 0) slot = i;
    if (slot < 0) {
      if (k >= max_kernels) continue;
      slot = k++;
      std::strncpy(names + 32 * slot, r.name, 31);
      names[32 * slot + 31] = 0;
      total_ms[slot] = 0.0;
      launches[slot] = 0;
    }
    total_ms[slot] += ms;
    launches[slot] += 1;
  }
  return k;
}
