// Implementation of the event-based kernel profiler (see prof.h) and the C entry points
// bandred_profile_begin / bandred_profile_end / bandred_launch_count.
#include <atomic>
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

}  // extern "C"
