// Implementation of the event-based kernel profiler (see prof.h) and the C entry points
// bandred_profile_begin / bandred_profile_end / bandred_launch_count.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/bandred.h"
#include "prof.h"

namespace bandred {
namespace prof {

namespace {

struct Record {
  int kind;
  double flops, bytes;
  cudaEvent_t e0, e1;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Record> g_records;
std::vector<cudaEvent_t> g_pool;
size_t g_pool_used = 0;
std::atomic<long long> g_launches{0};

cudaEvent_t take_event() {
  if (g_pool_used == g_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    g_pool.push_back(e);
  }
  return g_pool[g_pool_used++];
}

const char* const kNames[kNumKinds] = {"panel_qr_f64", "symm", "syr2k", "gemm", "splitk_reduce", "convert", "other",
                                           "stream_gemm", "rank_update"};

}  // namespace

const char* kind_name(int k) { return (k >= 0 && k < kNumKinds) ? kNames[k] : "?"; }
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches() { return g_launches.load(std::memory_order_relaxed); }

Scope::Scope(Kind kind, cudaStream_t s, double flops, double bytes) : s_(s) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_on) return;
  Record r{kind, flops, bytes, take_event(), take_event()};
  if (!r.e0 || !r.e1) return;
  cudaEventRecord(r.e0, s);
  slot_ = (int)g_records.size();
  g_records.push_back(r);
}

Scope::~Scope() {
  if (slot_ < 0) return;
  std::lock_guard<std::mutex> lock(g_mu);
  if (slot_ < (int)g_records.size()) cudaEventRecord(g_records[slot_].e1, s_);
}

// ---------------------------------------------------------------- device trace
namespace {

struct TraceMeta {
  int kind;
  long long iteration;
};

std::mutex g_tmu;
unsigned long long* g_tbuf = nullptr;  // device: 2 words per record (min start, min of ~end)
size_t g_tcap = 0;
std::vector<TraceMeta> g_tmeta;
thread_local int t_pending_kind = -1;
thread_local long long t_pending_iter = 0;

}  // namespace

TraceScope::TraceScope(int kind, long long iteration) {
  t_pending_kind = kind;
  t_pending_iter = iteration;
}

TraceScope::~TraceScope() { t_pending_kind = -1; }

unsigned long long* trace_take() {
  if (t_pending_kind < 0) return nullptr;
  std::lock_guard<std::mutex> lock(g_tmu);
  const int kind = t_pending_kind;
  t_pending_kind = -1;
  if (!g_tbuf || g_tmeta.size() >= g_tcap) return nullptr;
  g_tmeta.push_back(TraceMeta{kind, t_pending_iter});
  return g_tbuf + 2 * (g_tmeta.size() - 1);
}

namespace {
std::mutex g_pmu;
long long* g_phase_buf = nullptr;
int g_phase_steps = 0;
}  // namespace

long long* phase_take(int* steps) {
  std::lock_guard<std::mutex> lock(g_pmu);
  long long* p = g_phase_buf;
  *steps = g_phase_steps;
  g_phase_buf = nullptr;
  g_phase_steps = 0;
  return p;
}

namespace {
long long* g_chase_buf = nullptr;
int g_chase_steps = 0;
}  // namespace

long long* chase_phase_take(int* steps) {
  std::lock_guard<std::mutex> lock(g_pmu);
  long long* p = g_chase_buf;
  *steps = g_chase_steps;
  g_chase_buf = nullptr;
  g_chase_steps = 0;
  return p;
}

}  // namespace prof
}  // namespace bandred

using namespace bandred::prof;

extern "C" {

int bandred_profile_begin(void) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_records.clear();
  g_pool_used = 0;
  g_on = true;
  return 0;
}

int bandred_profile_end(bandred_kernel_stat* out, int max_entries) {
  std::vector<Record> recs;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    g_on = false;
    recs.swap(g_records);
  }
  bandred_kernel_stat agg[kNumKinds];
  std::memset(agg, 0, sizeof(agg));
  for (int k = 0; k < kNumKinds; ++k) std::strncpy(agg[k].name, kind_name(k), sizeof(agg[k].name) - 1);
  for (const Record& r : recs) {
    if (cudaEventSynchronize(r.e1) != cudaSuccess) return BANDRED_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.e0, r.e1) != cudaSuccess) return BANDRED_ERR_CUDA;
    bandred_kernel_stat& a = agg[r.kind];
    a.launches += 1;
    a.ms += ms;
    a.flops += r.flops;
    a.bytes += r.bytes;
  }
  int n = 0;
  for (int k = 0; k < kNumKinds && n < max_entries; ++k)
    if (agg[k].launches) out[n++] = agg[k];
  return n;
}

long long bandred_launch_count(void) { return launches(); }

int bandred_trace_begin(void* dev_buf, size_t bytes) {
  if (!dev_buf || (reinterpret_cast<uintptr_t>(dev_buf) & 255u)) return -1;
  if (bytes < 16) return -2;
  std::lock_guard<std::mutex> lock(g_tmu);
  // every word all ones: the start stamps and the complemented end stamps both take the minimum
  if (cudaMemset(dev_buf, 0xFF, bytes / 16 * 16) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
    return BANDRED_ERR_CUDA;
  g_tbuf = static_cast<unsigned long long*>(dev_buf);
  g_tcap = bytes / 16;
  g_tmeta.clear();
  return 0;
}

int bandred_panel_phase_trace(void* buf, int max_steps) {
  if (max_steps < 0 || (max_steps > 0 && !buf)) return -2;
  std::lock_guard<std::mutex> lock(g_pmu);
  g_phase_buf = static_cast<long long*>(buf);
  g_phase_steps = max_steps;
  return 0;
}

int bandred_sb2st_phase_trace(void* buf, int max_steps) {
  if (max_steps < 0 || (max_steps > 0 && !buf)) return -2;
  std::lock_guard<std::mutex> lock(bandred::prof::g_pmu);
  bandred::prof::g_chase_buf = static_cast<long long*>(buf);
  bandred::prof::g_chase_steps = max_steps;
  return 0;
}

int bandred_trace_end(bandred_trace_record* out, int max_records) {
  if (max_records < 0 || (max_records > 0 && !out)) return -2;
  std::vector<TraceMeta> meta;
  unsigned long long* buf;
  {
    std::lock_guard<std::mutex> lock(g_tmu);
    meta.swap(g_tmeta);
    buf = g_tbuf;
    g_tbuf = nullptr;
    g_tcap = 0;
  }
  if (!buf) return 0;
  const int n = (int)std::min<size_t>(meta.size(), (size_t)max_records);
  std::vector<unsigned long long> host(2 * (size_t)n);
  if (cudaDeviceSynchronize() != cudaSuccess) return BANDRED_ERR_CUDA;
  if (n && cudaMemcpy(host.data(), buf, host.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost) != cudaSuccess)
    return BANDRED_ERR_CUDA;
  for (int i = 0; i < n; ++i) {
    out[i].kind = meta[i].kind;
    out[i].iteration = meta[i].iteration;
    out[i].t0_ns = host[2 * i];
    out[i].t1_ns = ~host[2 * i + 1];  // ~0 when the kernel never ran
  }
  return n;
}

}  // extern "C"
