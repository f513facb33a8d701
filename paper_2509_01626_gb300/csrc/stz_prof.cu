// stz_prof.cu -- the launch counter and per-kernel event timing behind
// stz_profile_* and stz_launch_count (include/stz.h).
#include <string.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "stz.h"
#include "stz_prof.cuh"

namespace stz {

namespace {
std::atomic<unsigned long long> g_launches{0};
std::atomic<int> g_enabled{0};
std::mutex g_mu;
struct Rec {
  std::string name;
  cudaEvent_t a, b;
  bool done;
  double bytes;
};
std::vector<Rec> g_recs;           // pending event pairs
std::vector<cudaEvent_t> g_pool;   // reusable events
struct Acc {
  std::string name;
  unsigned long long launches;
  double ms, bytes;
};
std::vector<Acc> g_acc;

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void resolve_locked() {
  for (auto& r : g_recs) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess) cudaEventElapsedTime(&ms, r.a, r.b);
    bool found = false;
    for (auto& a : g_acc)
      if (a.name == r.name) {
        a.launches++;
        a.ms += ms;
        a.bytes += r.bytes;
        found = true;
        break;
      }
    if (!found) g_acc.push_back({r.name, 1ull, (double)ms, r.bytes});
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
}
}  // namespace

void prof_begin(const char* name, cudaStream_t s, int* slot, double bytes) {
  *slot = -1;
  // a launch into a graph being captured runs when the graph does: it is
  // counted at each graph launch (prof_count_launches), and never timed
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) return;
  g_launches.fetch_add(1);
  if (!g_enabled.load()) return;
  std::lock_guard<std::mutex> lk(g_mu);
  Rec r;
  r.name = name;
  r.a = get_event();
  r.b = get_event();
  r.done = false;
  r.bytes = bytes;
  cudaEventRecord(r.a, s);
  g_recs.push_back(r);
  *slot = (int)g_recs.size() - 1;
}

void prof_count_launches(unsigned long long n) { g_launches.fetch_add(n); }

bool prof_enabled() { return g_enabled.load() != 0; }

void prof_end(int slot, cudaStream_t s) {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (slot < (int)g_recs.size()) {
    cudaEventRecord(g_recs[slot].b, s);
    g_recs[slot].done = true;
  }
}

void prof_add_bytes(const char* name, double bytes) {
  if (!g_enabled.load()) return;
  std::lock_guard<std::mutex> lk(g_mu);
  for (size_t i = g_recs.size(); i-- > 0;)
    if (g_recs[i].name == name) {
      g_recs[i].bytes += bytes;
      return;
    }
}

}  // namespace stz

using namespace stz;

extern "C" {

unsigned long long stz_launch_count(void) { return g_launches.load(); }

void stz_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_enabled.store(on ? 1 : 0);
}

void stz_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  resolve_locked();
  g_acc.clear();
}

int stz_profile_read(stz_kernel_time* out, int max_entries) {
  std::lock_guard<std::mutex> lk(g_mu);
  resolve_locked();
  int n = (int)g_acc.size();
  for (int i = 0; i < n && i < max_entries; i++) {
    memset(out[i].name, 0, sizeof(out[i].name));
    strncpy(out[i].name, g_acc[i].name.c_str(), sizeof(out[i].name) - 1);
    out[i].launches = g_acc[i].launches;
    out[i].total_ms = g_acc[i].ms;
    out[i].algo_bytes = g_acc[i].bytes;
  }
  return n;
}

}  // extern "C"
