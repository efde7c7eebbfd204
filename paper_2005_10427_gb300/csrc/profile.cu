// Launch profiler behind qsd_profile_*: CUDA events around every kernel
// launch of the library (on the launching stream) and the entries the launch
// processed, so that callers can compute per-kernel throughput against the
// minimum-traffic roofline. Off by default; costs two event records per
// launch when on.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <vector>

#include "kernels.cuh"

namespace qsd {

namespace {

struct Rec {
  ProfTag tag;
  cudaEvent_t a = nullptr, b = nullptr;
  int slot = -1;  // pinned host slot for a device-side entry count
};

std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_free_events;
int* g_slots = nullptr;  // pinned
int g_nslots = 0, g_used_slots = 0;
constexpr int kSlots = 1 << 16;

cudaEvent_t get_event() {
  if (!g_free_events.empty()) {
    cudaEvent_t e = g_free_events.back();
    g_free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

}  // namespace

bool prof_enabled() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_on;
}

int prof_begin(const ProfTag& tag, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return -1;
  Rec r;
  r.tag = tag;
  if (tag.entries < 0 && tag.dev_entries) {
    if (!g_slots) {
      if (cudaMallocHost(&g_slots, sizeof(int) * kSlots) != cudaSuccess) {
        g_slots = nullptr;
        return -1;
      }
      g_nslots = kSlots;
    }
    if (g_used_slots < g_nslots) {
      r.slot = g_used_slots++;
      cudaMemcpyAsync(g_slots + r.slot, tag.dev_entries, sizeof(int), cudaMemcpyDeviceToHost, st);
    }
  }
  r.a = get_event();
  r.b = get_event();
  cudaEventRecord(r.a, st);
  g_recs.push_back(r);
  return (int)g_recs.size() - 1;
}

void prof_end(int rec, cudaStream_t st) {
  if (rec < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (rec < (int)g_recs.size()) cudaEventRecord(g_recs[rec].b, st);
}

}  // namespace qsd

extern "C" {

qsd_status qsd_profile_enable(int enable) {
  std::lock_guard<std::mutex> lk(qsd::g_mu);
  qsd::g_on = enable != 0;
  return QSD_OK;
}

qsd_status qsd_profile_reset(void) {
  std::lock_guard<std::mutex> lk(qsd::g_mu);
  for (auto& r : qsd::g_recs) {
    cudaEventSynchronize(r.b);
    qsd::g_free_events.push_back(r.a);
    qsd::g_free_events.push_back(r.b);
  }
  qsd::g_recs.clear();
  qsd::g_used_slots = 0;
  return QSD_OK;
}

qsd_status qsd_profile_read(qsd_profile_record* out, int max_records, int* n_records) {
  if (!n_records || (max_records > 0 && !out)) return QSD_ERR_INVALID_ARGUMENT;
  std::lock_guard<std::mutex> lk(qsd::g_mu);
  *n_records = (int)qsd::g_recs.size();
  for (int i = 0; i < (int)qsd::g_recs.size() && i < max_records; ++i) {
    qsd::Rec& r = qsd::g_recs[i];
    if (cudaEventSynchronize(r.b) != cudaSuccess) return QSD_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return QSD_ERR_CUDA;
    int64_t entries = r.tag.entries;
    if (entries < 0) {
      entries = r.slot >= 0 ? (int64_t)qsd::g_slots[r.slot] : -1;
      if (entries >= 0 && r.tag.complement) entries = r.tag.total - entries;
    }
    qsd_profile_record& o = out[i];
    std::memset(&o, 0, sizeof(o));
    std::strncpy(o.kernel, r.tag.kernel, sizeof(o.kernel) - 1);
    o.group = r.tag.group;
    o.pass = r.tag.pass;
    o.entries = entries;
    o.algo_bytes = entries >= 0 ? entries * r.tag.bytes_per_entry : -1;
    o.ms = ms;
  }
  return QSD_OK;
}

}  // extern "C"
