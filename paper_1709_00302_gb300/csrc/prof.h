// Per-kernel-class timing with CUDA events (enabled between bandred_profile_begin and
// bandred_profile_end) and a count of every kernel launch the library issues.
#pragma once
#include <cuda_runtime.h>

namespace bandred {
namespace prof {

// kStream / kRank: the general split-precision products of ge2gb (C = op(A) B streaming A
// once; C += A B^T reading and writing C once); kGemm: FP64 products and the small
// split-precision products of sy2sb.
enum Kind { kPanel = 0, kSymm, kSyr2k, kGemm, kSplitReduce, kConvert, kOther, kStream, kRank, kNumKinds };

const char* kind_name(int k);
void count_launch(int n = 1);
long long launches();

// Records an event pair around the launches issued while it lives (when profiling is on)
// and attributes the given algorithmic flops and HBM bytes to `kind`.
class Scope {
 public:
  Scope(Kind kind, cudaStream_t s, double flops, double bytes);
  ~Scope();
  Scope(const Scope&) = delete;
  Scope& operator=(const Scope&) = delete;

 private:
  int slot_ = -1;
  cudaStream_t s_;
};

// Device trace (bandred_trace_begin / bandred_trace_end).  A TraceScope names the next
// traced launch on this host thread (its kind and panel column); the launcher of that
// kernel takes the record with trace_take() (nullptr when tracing is off or the buffer is
// full) and passes it to the kernel, whose CTAs stamp their start and end into it
// (trace_start / trace_end in common.cuh).
enum TraceKind { kTracePanel = 0, kTraceRankL, kTraceRankR, kTraceSymm, kTracePanelRow, kTraceLeft, kTraceRight, kTraceW };

class TraceScope {
 public:
  TraceScope(int kind, long long iteration);
  ~TraceScope();
  TraceScope(const TraceScope&) = delete;
  TraceScope& operator=(const TraceScope&) = delete;
};
unsigned long long* trace_take();
// The armed phase buffer of bandred_panel_phase_trace (taken by the next grid panel), or nullptr.
long long* phase_take(int* steps);
// The armed buffer of bandred_sb2st_phase_trace (taken by the next bulge chase), or nullptr.
long long* chase_phase_take(int* steps);

}  // namespace prof
}  // namespace bandred
