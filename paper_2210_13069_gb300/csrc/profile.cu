// profile.cu -- opt-in kernel timing with CUDA events on the launching stream.
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "lrtei_internal.h"

namespace lrtei {
namespace {
struct Rec {
  std::string name;
  cudaEvent_t a, b;
};
std::mutex g_mu;
std::atomic<long long> g_launches{0};
std::atomic<long long> g_allocs{0};  // device allocations the library has requested (never reset)
std::vector<Rec> g_recs;
bool g_on = false;
}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(); }
void set_launch_count(long long n) { g_launches.store(n); }
void count_alloc() { g_allocs.fetch_add(1, std::memory_order_relaxed); }

ProfScope::ProfScope(const char* n, cudaStream_t s) : name(n), st(s) {
  if (!g_on) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    cudaGetLastError();
    a = b = nullptr;
    return;
  }
  cudaEventRecord(a, st);
}

ProfScope::~ProfScope() {
  if (!a) return;
  cudaEventRecord(b, st);
  std::lock_guard<std::mutex> lk(g_mu);
  g_recs.push_back({name, a, b});
}
}  // namespace lrtei

extern "C" {
lrtei_status lrtei_profile_enable(int on) {
  lrtei::g_on = on != 0;
  return LRTEI_OK;
}

void lrtei_profile_reset(void) {
  std::lock_guard<std::mutex> lk(lrtei::g_mu);
  for (auto& r : lrtei::g_recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  lrtei::g_recs.clear();
  lrtei::g_launches.store(0);
}

lrtei_status lrtei_profile_get(const char* kernel, double* total_ms, int64_t* launches) {
  if (!kernel || !total_ms || !launches) {
    lrtei::set_error("NULL argument");
    return LRTEI_ERR_ARG;
  }
  if (kernel[0] == '*' && kernel[1] == 0) {  // all launches since the last reset
    *total_ms = 0.0;
    *launches = lrtei::g_launches.load();
    return LRTEI_OK;
  }
  if (std::string(kernel) == "alloc") {  // device allocations requested since the library was loaded
    *total_ms = 0.0;
    *launches = lrtei::g_allocs.load();
    return LRTEI_OK;
  }
  std::lock_guard<std::mutex> lk(lrtei::g_mu);
  double tot = 0.0;
  int64_t cnt = 0;
  for (auto& r : lrtei::g_recs) {
    if (r.name != kernel) continue;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e != cudaSuccess) return lrtei::cuda_fail(e, "profile event");
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess) return lrtei::cuda_fail(e, "profile elapsed");
    tot += ms;
    ++cnt;
  }
  *total_ms = tot;
  *launches = cnt;
  return LRTEI_OK;
}
}
