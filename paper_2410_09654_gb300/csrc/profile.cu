// Optional per-kernel timing (CUDA events on the launching stream) and a launch counter.
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace ps {

namespace {
struct Pending {
  const char* name;
  cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_enabled = false;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;
std::map<std::string, std::pair<long long, double>> g_totals;  // name -> (launches, ms)
std::atomic<long long> g_launches{0};

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

void drain_locked() {
  for (Pending& p : g_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      auto& t = g_totals[p.name];
      t.first += 1;
      t.second += ms;
    }
    g_pool.push_back(p.a);
    g_pool.push_back(p.b);
  }
  g_pending.clear();
}
}  // namespace

KTimer::KTimer(const char* name, cudaStream_t s) : name_(name), s_(s), a_(nullptr) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_enabled) return;
  a_ = take_event();
  if (a_) cudaEventRecord((cudaEvent_t)a_, s_);
}

KTimer::~KTimer() {
  if (!a_) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = take_event();
  if (!b) return;
  cudaEventRecord(b, s_);
  g_pending.push_back({name_, (cudaEvent_t)a_, b});
  if (g_pending.size() > 3800) drain_locked();
}

}  // namespace ps

extern "C" {

int pauli_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(ps::g_mu);
  ps::drain_locked();
  ps::g_enabled = on != 0;
  if (on) {
    ps::g_totals.clear();
    // pre-create events so that timing does not create them inside the measured region
    while (ps::g_pool.size() < 8192) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreate(&e) != cudaSuccess) break;
      ps::g_pool.push_back(e);
    }
  }
  return PS_OK;
}

int pauli_profile_report(char* buf, int64_t len, int64_t* needed) {
  std::lock_guard<std::mutex> lk(ps::g_mu);
  ps::drain_locked();
  std::string s = "{";
  bool first = true;
  for (auto& kv : ps::g_totals) {
    char line[256];
    snprintf(line, sizeof(line), "%s\"%s\": [%lld, %.6f]", first ? "" : ", ", kv.first.c_str(), kv.second.first,
             kv.second.second);
    s += line;
    first = false;
  }
  s += "}";
  if (needed) *needed = (int64_t)s.size() + 1;
  if (!buf || len < (int64_t)s.size() + 1) return PS_ERR_CAPACITY;
  memcpy(buf, s.c_str(), s.size() + 1);
  return PS_OK;
}

int64_t pauli_launch_count(void) { return ps::g_launches.load(); }

}  // extern "C"
