// Launch counting and CUDA-event timing per kernel class (ld_profile_* entry points).
#include <string.h>

#include <algorithm>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "profile.cuh"
#include "record.cuh"

namespace ld {

namespace {

struct Slot {
  std::string name;
  cudaEvent_t start, stop;
};

struct Profiler {
  std::mutex mu;
  bool on = false;
  std::string filter;  // empty: time every class
  std::vector<cudaEvent_t> pool;
  std::vector<Slot> slots;
  std::map<std::string, long long> launches;
  std::map<std::string, double> ms;
  std::map<std::string, long long> timed;
  std::map<std::string, double> bytes;
  std::map<std::string, double> flops;
};

Profiler& prof() {
  static Profiler p;
  return p;
}

cudaEvent_t take_event(Profiler& p, size_t idx) {
  while (p.pool.size() <= idx) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    p.pool.push_back(e);
  }
  return p.pool[idx];
}

}  // namespace

ProfScope::ProfScope(const char* name, cudaStream_t stream, double bytes, double flops)
    : slot_(-1), stream_(stream) {
  Profiler& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  if (!p.on) return;
  p.launches[name] += 1;
  p.bytes[name] += bytes;
  p.flops[name] += flops;
  if (!p.filter.empty() && p.filter != name) return;
  const size_t k = p.slots.size();
  cudaEvent_t a = take_event(p, 2 * k), b = take_event(p, 2 * k + 1);
  if (!a || !b) return;
  p.slots.push_back(Slot{name, a, b});
  cudaEventRecord(a, stream);
  slot_ = (int)k;
}

ProfScope::~ProfScope() {
  if (slot_ < 0) return;
  Profiler& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  if (slot_ < (int)p.slots.size()) cudaEventRecord(p.slots[slot_].stop, stream_);
}

}  // namespace ld

extern "C" {

// Starts counting launches per kernel class and timing the class `kernel`
// (NULL or "" = every class) with CUDA events. Clears earlier results.
ld_status ld_profile_start(const char* kernel) {
  ld::Profiler& p = ld::prof();
  std::lock_guard<std::mutex> g(p.mu);
  p.on = true;
  p.filter = kernel ? kernel : "";
  p.slots.clear();
  p.launches.clear();
  p.ms.clear();
  p.timed.clear();
  p.bytes.clear();
  p.flops.clear();
  return LD_OK;
}

// Stops profiling; waits for the recorded events and sums their intervals.
ld_status ld_profile_stop(void) {
  ld::Profiler& p = ld::prof();
  std::lock_guard<std::mutex> g(p.mu);
  p.on = false;
  ld_status st = LD_OK;
  for (auto& s : p.slots) {
    if (cudaEventSynchronize(s.stop) != cudaSuccess) {
      st = LD_ERR_CUDA;
      continue;
    }
    float t = 0.f;
    if (cudaEventElapsedTime(&t, s.start, s.stop) != cudaSuccess) {
      st = LD_ERR_CUDA;
      continue;
    }
    p.ms[s.name] += t;
    p.timed[s.name] += 1;
  }
  p.slots.clear();
  return st;
}

// Launches of kernel class `kernel` (NULL = all classes) since ld_profile_start,
// and the summed event time of its timed launches (0 if it was not timed).
ld_status ld_profile_query(const char* kernel, int64_t* launches, double* total_ms) {
  if (!launches || !total_ms) return LD_ERR_INVALID_ARG;
  ld::Profiler& p = ld::prof();
  std::lock_guard<std::mutex> g(p.mu);
  long long n = 0;
  double t = 0.0;
  for (auto& kv : p.launches)
    if (!kernel || kv.first == kernel) n += kv.second;
  for (auto& kv : p.ms)
    if (!kernel || kv.first == kernel) t += kv.second;
  *launches = n;
  *total_ms = t;
  return LD_OK;
}

// Algorithmic bytes and flops summed over the launches of class `kernel` (NULL =
// all classes) since ld_profile_start.
ld_status ld_profile_work(const char* kernel, double* bytes, double* flops) {
  if (!bytes || !flops) return LD_ERR_INVALID_ARG;
  ld::Profiler& p = ld::prof();
  std::lock_guard<std::mutex> g(p.mu);
  double b = 0.0, f = 0.0;
  for (auto& kv : p.bytes)
    if (!kernel || kv.first == kernel) b += kv.second;
  for (auto& kv : p.flops)
    if (!kernel || kv.first == kernel) f += kv.second;
  *bytes = b;
  *flops = f;
  return LD_OK;
}

// Names of the kernel classes seen since ld_profile_start, comma-separated, into
// buf (truncated to cap bytes including the terminator).
ld_status ld_profile_classes(char* buf, int64_t cap) {
  if (!buf || cap <= 0) return LD_ERR_INVALID_ARG;
  ld::Profiler& p = ld::prof();
  std::lock_guard<std::mutex> g(p.mu);
  std::string out;
  for (auto& kv : p.launches) {
    if (!out.empty()) out += ",";
    out += kv.first;
  }
  const size_t k = std::min<size_t>(out.size(), (size_t)cap - 1);
  memcpy(buf, out.data(), k);
  buf[k] = 0;
  return LD_OK;
}

}  // extern "C"
