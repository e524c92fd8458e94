// Definitions of the opaque C-ABI handles (include/pk.h), shared by the translation
// units that implement entry points.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "pk_internal.h"

#include "tuned_table.h"

struct pk_ctx {
  pk_tuning tuning = kTunedDefault;
  int32_t debug = 0;               // PK_DEBUG_* bits
  uint64_t hbm_budget = 0;         // plans' workspaces must fit (0: no limit)
  int32_t device = -1;
  cudaStream_t stream = nullptr;
  cudaStream_t capture = nullptr;  // private stream on which launch sequences are recorded
  std::string err;
  void* own_ws = nullptr;
  uint64_t own_ws_bytes = 0;
  pk::SliceResult* pinned_result = nullptr;
};
struct pk_knot {
  pk::Knot k;
};
// A plan's launch sequence recorded as a CUDA graph for one (state, arena, precision).
struct PlanGraph {
  void* ws = nullptr;
  void* arena = nullptr;
  int32_t precision = -1;
  cudaGraphExec_t exec = nullptr;
};
struct pk_plan {
  pk::Plan p;
  uint8_t* pinned_program = nullptr;
  uint8_t* pinned_grad = nullptr;  // the reverse-pass program and its downloaded results
  PlanGraph graph;
  PlanGraph grad_graph;            // the reverse-pass launch sequence (arena = null)
};

namespace pk {
// Kernel classes of the launch-sequence timing: build, rows (row / thread-per-output /
// sequence kernels), split-K, results, GEMM on the CUDA cores, tensor-core GEMM, digit
// conversion for the tensor-core GEMM.
constexpr int kNumClasses = 7;
// Per-launch CUDA events of one recorded launch sequence (launch.cu).
struct Prof;
Prof* prof_new();
void prof_free(Prof* p);
// Per class c: out[c] summed milliseconds, out[7+c] launches, out[14+c] complex
// multiply-adds, out[21+c] algorithmic bytes, out[28+c] milliseconds weighted by the share
// of the GPU's CTA slots each launch fills, over n recorded sequences whose events have
// completed.
cudaError_t prof_read(Prof* const* profs, int n, double* out);
// Per launch of n recorded sequences: (sequence, class, start ms, end ms, complex
// multiply-adds, algorithmic bytes), times relative to the first sequence's first event.
cudaError_t prof_timeline(Prof* const* profs, int n, double* out, int64_t cap, int64_t* count);
// launch_plan with an event pair around every launch, recorded into `prof` (which must
// outlive any graph the launches are captured into).
cudaError_t launch_plan_prof(const Plan& p, int32_t precision, void* ws, void* arena,
                             cudaStream_t stream, Prof* prof);
// Z(q) of `p` modulo `prime` into the 8 bytes at d_sum (exact.cu); program uploaded in
// `ws`, tensors in `arena` (complex64 layout).
cudaError_t launch_exact(const Plan& p, uint32_t prime, void* ws, void* arena, void* d_sum,
                         cudaStream_t stream);
// Enqueue every kernel of every slice of `p` at `precision` on `stream` (launch.cu);
// `ws` holds the plan state (bytes [0, off_arena)), `arena` the tensors.
cudaError_t launch_plan(const Plan& p, int32_t precision, void* ws, void* arena,
                        cudaStream_t stream);
// Options of a launch sequence enqueued directly (not replayed from a graph).
struct LaunchOpts {
  int64_t slice_first = 0;   // slices [slice_first, slice_first + slice_count); the first
  int64_t slice_count = -1;  // one clears every slice record, so records outside the range
                             // read 0; slice_count -1: every slice
  bool check_finite = false; // scan the initial tensors and every step's result for NaN /
                             // Inf (steps launched one at a time); the first hit is written
                             // into the error word (status_nonfinite)
  bool nvtx = false;         // an NVTX range around every launch, named by step and class
};
cudaError_t launch_plan_opts(const Plan& p, int32_t precision, void* ws, void* arena,
                             cudaStream_t stream, const LaunchOpts& opts);
// Same, with CUDA-event timing per kernel class; waits for the stream (launch.cu).
cudaError_t profile_plan(const Plan& p, int32_t precision, void* ws, void* arena,
                         cudaStream_t stream, double* out);
// The reverse-pass program of a PK_FLAG_GRAD plan on `ws` (layout GradProgram::off_*).
cudaError_t launch_grad(const Plan& p, int32_t precision, void* ws, cudaStream_t stream);
// Sets the kernel attributes launch_plan relies on (shared-memory limits), once per
// device; call before recording a launch sequence into a graph (launch.cu).
cudaError_t prepare_kernels();
}  // namespace pk
