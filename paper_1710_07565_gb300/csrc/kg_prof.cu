// Launch accounting and optional per-kernel CUDA-event timing.  When enabled,
// every launch site records an event pair on the stream it launches on; the
// totals per kernel class are read back after the caller's timed region.
#include <mutex>
#include <vector>

#include "kg.h"
#include "kg_prof.h"

namespace kg {

namespace {
std::mutex g_mu;
bool g_enabled = false;
unsigned long long g_launches = 0;
struct Pair {
  int cls;
  cudaEvent_t a, b;
};
std::vector<Pair> g_pairs;
std::vector<cudaEvent_t> g_free;

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
}  // namespace

ProfScope::ProfScope(int cls, cudaStream_t s) : cls_(cls), s_(s), a_(nullptr) {
  std::lock_guard<std::mutex> lock(g_mu);
  ++g_launches;
  if (!g_enabled) return;
  a_ = take_event();
  cudaEventRecord(static_cast<cudaEvent_t>(a_), s_);
}

ProfScope::~ProfScope() {
  if (!a_) return;
  std::lock_guard<std::mutex> lock(g_mu);
  cudaEvent_t b = take_event();
  cudaEventRecord(b, s_);
  g_pairs.push_back(Pair{cls_, static_cast<cudaEvent_t>(a_), b});
}

}  // namespace kg

using namespace kg;

extern "C" {

unsigned long long kg_launch_count(void) {
  std::lock_guard<std::mutex> lock(g_mu);
  return g_launches;
}

kg_status kg_profile_begin(void) {
  std::lock_guard<std::mutex> lock(g_mu);
  for (auto& p : g_pairs) {
    g_free.push_back(p.a);
    g_free.push_back(p.b);
  }
  g_pairs.clear();
  g_enabled = true;
  return KG_OK;
}

// ms[c] / launches[c] for c < KG_PROF_CLASSES; synchronises the recorded events.
kg_status kg_profile_end(double* ms, unsigned long long* launches) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_enabled = false;
  for (int c = 0; c < KG_PROF_CLASSES; ++c) {
    if (ms) ms[c] = 0.0;
    if (launches) launches[c] = 0;
  }
  kg_status st = KG_OK;
  for (auto& p : g_pairs) {
    float t = 0.f;
    if (cudaEventSynchronize(p.b) != cudaSuccess || cudaEventElapsedTime(&t, p.a, p.b) != cudaSuccess)
      st = KG_ERR_CUDA;
    if (ms) ms[p.cls] += t;
    if (launches) launches[p.cls] += 1;
    g_free.push_back(p.a);
    g_free.push_back(p.b);
  }
  g_pairs.clear();
  return st;
}

}  // extern "C"
