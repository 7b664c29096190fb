// profiling.cpp - launch counter and CUDA-event timing per kernel class.
//
// mlsgd_profile_start(cls) enables timing of every later launch whose class
// name equals cls ("*" = every class); mlsgd_profile_stop() waits for the
// recorded events and reports launches, summed device time and summed
// algorithmic bytes / flops per class.  Events are recorded on the stream the
// kernel is launched on.  Process-wide, not thread-safe by design: the bench
// drives one stream from one thread.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "mlsgd.h"

namespace mlsgd {

namespace {
struct Rec {
  std::string cls;
  int ev0, ev1;
  double bytes, flops;
};
struct Prof {
  bool on = false;
  std::string target;
  std::vector<cudaEvent_t> pool;
  size_t next = 0;
  std::vector<Rec> recs;
  int pending = -1;
  std::string pending_cls;
};
Prof g_prof;
std::atomic<long long> g_launches{0};
const size_t kMaxEvents = 1 << 20;

int take_event() {
  if (g_prof.next >= kMaxEvents) return -1;
  if (g_prof.next == g_prof.pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    g_prof.pool.push_back(e);
  }
  return (int)g_prof.next++;
}
}  // namespace

void prof_begin(const char* cls, cudaStream_t st) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  g_prof.pending = -1;
  if (!g_prof.on || (g_prof.target != "*" && g_prof.target != cls)) return;
  const int e = take_event();
  if (e < 0) return;
  cudaEventRecord(g_prof.pool[e], st);
  g_prof.pending = e;
  g_prof.pending_cls = cls;
}

void prof_end(const char* cls, cudaStream_t st, double bytes, double flops) {
  if (g_prof.pending < 0) return;
  const int e = take_event();
  if (e < 0) { g_prof.pending = -1; return; }
  cudaEventRecord(g_prof.pool[e], st);
  g_prof.recs.push_back(Rec{g_prof.pending_cls, g_prof.pending, e, bytes, flops});
  g_prof.pending = -1;
}

}  // namespace mlsgd

using namespace mlsgd;

extern "C" {

int64_t mlsgd_launch_count(void) { return g_launches.load(); }

int mlsgd_profile_start(const char* cls) {
  g_prof.on = cls != nullptr;
  g_prof.target = cls ? cls : "";
  g_prof.next = 0;
  g_prof.recs.clear();
  g_prof.pending = -1;
  return 0;
}

int mlsgd_profile_stop(mlsgd_profile_entry* out, int max_entries) {
  g_prof.on = false;
  std::map<std::string, mlsgd_profile_entry> agg;
  for (const Rec& r : g_prof.recs) {
    float ms = 0.f;
    if (cudaEventSynchronize(g_prof.pool[r.ev1]) != cudaSuccess) return -1;
    if (cudaEventElapsedTime(&ms, g_prof.pool[r.ev0], g_prof.pool[r.ev1]) != cudaSuccess) return -1;
    mlsgd_profile_entry& a = agg[r.cls];
    std::strncpy(a.cls, r.cls.c_str(), sizeof(a.cls) - 1);
    a.launches += 1;
    a.total_ms += ms;
    a.bytes += r.bytes;
    a.flops += r.flops;
  }
  int n = 0;
  for (auto& kv : agg) {
    if (n < max_entries && out) out[n] = kv.second;
    ++n;
  }
  g_prof.recs.clear();
  g_prof.next = 0;
  return n;
}

}  // extern "C"
