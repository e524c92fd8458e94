// Enqueueing a plan's kernels (Sec. III contraction sequence) for one precision.
//
//  complex128: every kernel in FP64 on complex128 tensors;
//  complex64 : every kernel in FP32 on complex64 tensors, except (when the plan has a
//              tail) the last steps, which run in complex128 on a separate tail region
//              whose complex64 inputs are widened first;
//  split     : every kernel on float-float ("split FP32") tensors.
//  The slice scalar and the sum over slices are always formed in FP64.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <string>
#include <type_traits>
#include <vector>

#include "handles.h"
#include "kernels.cuh"
#include "gemm_tc.cuh"

namespace pk {

namespace {

// Widens the listed complex64 tensors into complex128 copies (one grid row each) and
// carries their bookkeeping over (the max-abs bits re-encoded as a double).
__global__ void __launch_bounds__(256) k_widen(const ConvRec* __restrict__ conv,
                                               const Cx<float>* arena, Cx<double>* tail,
                                               Meta* meta) {
  const ConvRec c = conv[blockIdx.y];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < c.elems;
       e += (long long)gridDim.x * blockDim.x) {
    Cx<float> v = arena[c.src_off + e];
    tail[c.dst_off + e] = {(double)v.re, (double)v.im};
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    float m = __uint_as_float((unsigned)meta[c.src_meta].maxbits);
    meta[c.dst_meta].maxbits = (unsigned long long)__double_as_longlong((double)m);
    meta[c.dst_meta].exp = meta[c.src_meta].exp;
  }
}

// ---- finite check (debug): NaN / Inf in a tensor just written sets the error word
template <typename R>
__device__ __forceinline__ bool finite_cx(const Cx<R>& v) {
  return isfinite(v.re) && isfinite(v.im);
}
template <>
__device__ __forceinline__ bool finite_cx<ff>(const Cx<ff>& v) {
  return isfinite(v.re.hi) && isfinite(v.re.lo) && isfinite(v.im.hi) && isfinite(v.im.lo);
}

// Writes `code` into bits 1 and up of the error word unless a code is there already (the
// checks run in stream order, so the first tensor found non-finite is the one reported);
// bit 0 (wait expiry) is kept.  A failed exchange means another writer changed the word,
// so the loop ends after a few rounds; it is bounded all the same.
__device__ void set_nonfinite(unsigned long long* word, unsigned long long code) {
  unsigned long long old = *(volatile unsigned long long*)word;
  for (int i = 0; i < 64 && (old >> 1) == 0ull; ++i) {
    const unsigned long long seen = atomicCAS(word, old, old | code);
    if (seen == old) return;
    old = seen;
  }
}

// Entries [0, n) at x, or with `rec` the initial tensor rec[blockIdx.y].
template <typename R>
__global__ void __launch_bounds__(256) k_check_finite(const Cx<R>* x, long long n,
                                                      const Recipe* rec,
                                                      unsigned long long* word,
                                                      unsigned long long code) {
  if (rec) {
    x += rec[blockIdx.y].offset;
    n = rec[blockIdx.y].elems;
  }
  bool bad = false;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    bad |= !finite_cx(x[e]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) set_nonfinite(word, code);
}

template <typename R>
cudaError_t check_tensor(const Cx<R>* x, long long n, unsigned long long* word,
                         unsigned long long code, cudaStream_t st) {
  const unsigned bx = (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 1216));
  k_check_finite<R><<<bx, 256, 0, st>>>(x, n, nullptr, word, code);
  return cudaGetLastError();
}

}  // namespace

// Optional per-launch timing: an event pair around every launch, summed per class.  When
// the launches are recorded into a graph, the events become event-record nodes and each
// replay re-records them.
struct Prof {
  double ms[kNumClasses] = {}, n[kNumClasses] = {}, cmacs[kNumClasses] = {},
         bytes[kNumClasses] = {};
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  std::vector<int> cls;
  std::vector<double> ev_cmacs, ev_bytes;   // per launch
  std::vector<double> ev_fill;              // per launch: share of the GPU's CTA slots it fills
  ~Prof() {
    for (auto& e : ev) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
  }
};

namespace {

int g_sms = 152;   // multiprocessors of the current device (set by prepare_kernels)

// Share of the GPU a launch of `grid` CTAs occupies when `per_sm` of them fit on one
// multiprocessor: 1 for a grid that fills every slot, less for smaller grids.
double gpu_fill(long long grid, int per_sm) {
  return std::min(1.0, (double)grid / ((double)g_sms * (double)per_sm));
}

constexpr const char* kClassName[kNumClasses] = {"build", "rows", "splitk", "results",
                                                  "gemm", "gemm_tc", "digits"};

struct Marker {
  Prof* prof;
  cudaStream_t st;
  bool nvtx = false;   // NVTX range per launch: "step <i> <class>" (i = -1: not a step)
  int step = -1;
  // During stream capture a plain event record only marks a dependency; the external
  // flag makes it an event-record node of the graph, re-recorded by every replay.
  void record(cudaEvent_t e) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs == cudaStreamCaptureStatusActive)
      cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else
      cudaEventRecord(e, st);
  }
  void begin(int c, double cm, double by, double fill) {
    if (nvtx) nvtxRangePushA(("step " + std::to_string(step) + " " + kClassName[c]).c_str());
    if (!prof) return;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    prof->ev.push_back({a, b});
    prof->cls.push_back(c);
    prof->ev_cmacs.push_back(cm);
    prof->ev_bytes.push_back(by);
    prof->ev_fill.push_back(fill);
    prof->n[c] += 1;
    prof->cmacs[c] += cm;
    prof->bytes[c] += by;
    record(a);
  }
  void end() {
    if (prof) record(prof->ev.back().second);
    if (nvtx) nvtxRangePop();
  }
};

// Rows below which one thread per row leaves the GPU short of threads (152 SMs x 2048
// resident threads); such steps with several outputs per row run thread per output.
constexpr long long kFewRows = 152LL * 2048;

template <typename R>
cudaError_t launch_rows(const Step& s, Cx<R>* arena, Meta* meta, cudaStream_t st, Marker& mk,
                        double cm, double by) {
  const size_t sm = sizeof(long long) * (size_t)(2 * s.K + s.N);
  const int kmax = sizeof(R) == 8 ? 16 : 32;   // K held in registers by the row kernel
  // few rows, several columns: the row kernel over (row, chunk of columns) work items
  // when A's row fits the registers, else one thread per output
  const bool chunked = s.R < kFewRows && s.N > 1 && s.K <= kmax && sm <= 200 * 1024;
  int nc = (int)s.N;
  if (chunked) {
    const long long want = std::min<long long>(s.N, (kFewRows + s.R - 1) / s.R);  // chunks
    nc = (int)((s.N + want - 1) / want);
  }
  if (!chunked && s.R < kFewRows && s.N > 1 && sizeof(long long) * 2 * (size_t)s.K <= 200 * 1024) {
    const long long outs = s.R * s.N;
    const long long blocks = std::max<long long>(1, std::min<long long>((outs + 255) / 256, 152 * 16));
    mk.begin(1, cm, by, gpu_fill(blocks, 8));
    k_outs<R><<<(unsigned)blocks, 256, sizeof(long long) * 2 * (size_t)s.K, st>>>(s, arena, meta);
    mk.end();
    return cudaGetLastError();
  }
  const long long items = s.R * ((s.N + nc - 1) / nc);
  long long blocks = (items + 255) / 256;
  blocks = std::max<long long>(1, std::min<long long>(blocks, 152 * 8));
  mk.begin(1, cm, by, gpu_fill(blocks, 8));
  if (sm > 200 * 1024) {
    k_rows_big<R><<<(unsigned)blocks, 256, 0, st>>>(s, arena, meta);
    mk.end();
    return cudaGetLastError();
  }
  const int K = (int)s.K;
  void (*fn)(const Step, Cx<R>*, Meta*, int);
  if (K <= 1)
    fn = k_rows<R, 1>;
  else if (K <= 2)
    fn = k_rows<R, 2>;
  else if (K <= 4)
    fn = k_rows<R, 4>;
  else if (K <= 8)
    fn = k_rows<R, 8>;
  else if (K <= 16)
    fn = k_rows<R, 16>;
  else if (K <= kmax)
    fn = k_rows<R, 32>;
  else
    fn = k_rows<R, 0>;
  fn<<<(unsigned)blocks, 256, sm, st>>>(s, arena, meta, nc);  // limit raised by prepare_kernels
  mk.end();
  return cudaGetLastError();
}

// One contraction step; `counter` is its split-K ticket or its tensor-core tile counter
// (zeroed with the bookkeeping before every slice), `by` its algorithmic bytes
// (for the optional timing only).
// Digit conversion of both operands, then the tensor-core GEMM, for S digits.
template <int S>
cudaError_t launch_tc(const Step& s, Cx<ff>* arena, Meta* meta, unsigned char* tcs,
                      unsigned* ticket, unsigned long long* err, cudaStream_t stream, Marker& mk,
                      double cm, double by, int64_t db_groups) {
  const TcScratch L = tc_scratch(s.Bsz, s.M, s.N, s.K, S);
  // class 6 (digit conversion): its bytes are the operands it reads, |A| + |B|
  const long long nA = (tc::kMc / 32) * s.Bsz * L.tiles_m * L.groups,
                  nB = s.Bsz * L.tiles_n * L.groups;
  mk.begin(6, 0.0, (double)sizeof(Cx<ff>) * (double)(s.R * s.K + s.Bsz * s.K * s.N),
           gpu_fill(nA + nB, 4));   // 4 CTAs per SM (64 registers x 256 threads)
  k_digits<S><<<(unsigned)(nA + nB), tc::kConvThreads, tc::Cfg<S>::kConvSmem, stream>>>(s, arena, tcs, nA);
  mk.end();
  // persistent: at most one CTA per tile slot of the GPU, each looping over its tiles;
  // tiles of steps with at most two flush groups come from the tile counter
  const long long tc_tiles = L.tiles_m * L.tiles_n * s.Bsz;
  const bool q = L.groups <= 2;
  if (db_groups > 0 && L.groups >= db_groups) {   // one CTA per SM, two accumulator sets
    const long long grid = std::min<long long>(tc_tiles, (long long)g_sms);
    mk.begin(5, cm, by, gpu_fill(grid, 1));
    if (q)
      k_gemm_tc<S, true, true><<<(unsigned)grid, tc::kThreads, tc::Cfg<S>::kSmemDB, stream>>>(
          s, arena, meta, tcs, ticket, err);
    else
      k_gemm_tc<S, true, false><<<(unsigned)grid, tc::kThreads, tc::Cfg<S>::kSmemDB, stream>>>(
          s, arena, meta, tcs, ticket, err);
  } else {
    const long long grid = std::min<long long>(tc_tiles, 2LL * g_sms);
    mk.begin(5, cm, by, gpu_fill(grid, 2));
    if (q)
      k_gemm_tc<S, false, true><<<(unsigned)grid, tc::kThreads, tc::Cfg<S>::kSmem, stream>>>(
          s, arena, meta, tcs, ticket, err);
    else
      k_gemm_tc<S, false, false><<<(unsigned)grid, tc::kThreads, tc::Cfg<S>::kSmem, stream>>>(
          s, arena, meta, tcs, ticket, err);
  }
  mk.end();
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_step(const Step& s, Cx<R>* arena, Meta* meta, Cx<double>* partial,
                        unsigned* counter, cudaStream_t stream, Marker& mk, double by,
                        unsigned char* tc_scratch = nullptr, unsigned long long* err = nullptr,
                        int64_t db_groups = 0) {
  const double cm = (double)s.R * (double)s.K * (double)s.N;
  const long long gemm_tiles = ((s.M + 63) / 64) * ((s.N + 63) / 64) * s.Bsz;
  cudaError_t e;
  if constexpr (std::is_same<R, ff>::value) {
    if (s.tc && tc_scratch && err)  // digits of A and B, then the tensor-core GEMM
      return s.tc == 4
                 ? launch_tc<4>(s, arena, meta, tc_scratch, counter, err, stream, mk, cm, by, db_groups)
                 : launch_tc<5>(s, arena, meta, tc_scratch, counter, err, stream, mk, cm, by, db_groups);
  }
  if (s.kernel == KGEMM && gemm_tiles < (1LL << 31)) {
    mk.begin(4, cm, by, gpu_fill(gemm_tiles, 8));
    k_gemm<R><<<(unsigned)gemm_tiles, 256, 0, stream>>>(s, arena, meta);
    mk.end();
    e = cudaGetLastError();
  } else if (s.kernel == KSPLITK) {
    mk.begin(2, cm, by, gpu_fill((long long)s.chunks * s.R * s.N, 8));
    k_splitk<R><<<dim3((unsigned)s.chunks, (unsigned)(s.R * s.N)), 256, 0, stream>>>(
        s, arena, meta, partial, counter);
    mk.end();
    e = cudaGetLastError();
  } else {
    e = launch_rows<R>(s, arena, meta, stream, mk, cm, by);
  }
  return e;
}

double step_bytes(const Plan& p, const Step& s, double elem_bytes) {
  return elem_bytes * (double)(p.tensors[s.a].elems + (s.b >= 0 ? p.tensors[s.b].elems : 0) +
                               p.tensors[s.c].elems);
}

// Steps [first, last) of the plan, all in storage type R.
template <typename R>
cudaError_t launch_bulk(const Plan& p, char* base, char* arena_base, int32_t first, int32_t last,
                        cudaStream_t stream, Marker& mk, const LaunchOpts& o, long long sl) {
  Cx<R>* arena = (Cx<R>*)arena_base;
  Meta* meta = (Meta*)(base + p.off_meta);
  Cx<double>* partial = (Cx<double>*)(base + p.off_scratch);
  unsigned* counters = (unsigned*)(base + p.off_counter);
  unsigned char* tcs = (std::is_same<R, ff>::value && p.tc_bytes > 0)
                           ? (unsigned char*)arena_base + p.tc_offset() : nullptr;
  const TinyStep* tiny = (const TinyStep*)(base + p.off_tiny);
  unsigned long long* err = &((SliceResult*)(base + p.off_result))[p.n_slices].status;
  size_t sg = 0;
  for (int32_t i = first; i < last;) {
    while (sg < p.segments.size() && p.segments[sg].first < i) ++sg;
    if (!o.check_finite && sg < p.segments.size() && p.segments[sg].first == i &&
        i + p.segments[sg].count <= last) {  // a run of small steps: one sequence launch
      const Segment& g = p.segments[sg];
      double cm = 0, by = 0;
      for (int32_t j = i; j < i + g.count; ++j) {
        cm += (double)p.steps[j].R * (double)p.steps[j].K * (double)p.steps[j].N;
        by += step_bytes(p, p.steps[j], (double)sizeof(Cx<R>));
      }
      mk.step = i;
      mk.begin(1, cm, by, gpu_fill(1, 8));
      k_seg<R><<<1, 256, 0, stream>>>(tiny + g.tiny0, g.count, arena, meta);
      mk.end();
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      i += g.count;
      continue;
    }
    mk.step = i;
    cudaError_t e = launch_step<R>(p.steps[i], arena, meta, partial, counters + i, stream, mk,
                                   step_bytes(p, p.steps[i], (double)sizeof(Cx<R>)), tcs, err,
                                   p.tuning.tc_db_groups);
    if (e == cudaSuccess && o.check_finite)
      e = check_tensor<R>(arena + p.steps[i].off_c, p.tensors[p.steps[i].c].elems, err,
                          status_nonfinite(sl, i), stream);
    if (e != cudaSuccess) return e;
    ++i;
  }
  return cudaSuccess;
}

template <typename R>
cudaError_t launch_build(const Plan& p, char* base, char* arena_base, long long sl, cudaStream_t stream,
                         Marker& mk, const LaunchOpts& o) {
  if (p.n_init <= 0) return cudaSuccess;
  if (p.n_init > 65535) return cudaErrorInvalidValue;
  int64_t maxel = 1, initel = 0;
  for (const auto& r : p.recipes) {
    maxel = std::max<int64_t>(maxel, r.elems);
    initel += r.elems;
  }
  const unsigned bx = (unsigned)std::min<int64_t>((maxel + 255) / 256, 64);
  mk.step = -1;
  mk.begin(0, 0, (double)sizeof(Cx<R>) * (double)initel, gpu_fill((long long)bx * p.n_init, 8));
  k_build<R><<<dim3(bx, (unsigned)p.n_init), 256, 0, stream>>>(
      (const Recipe*)(base + p.off_recipe), (const Slot*)(base + p.off_slots),
      (Cx<R>*)arena_base, (Meta*)(base + p.off_meta), p.q, sl, (int)p.sliced.size());
  mk.end();
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && o.check_finite) {
    k_check_finite<R><<<dim3(bx, (unsigned)p.n_init), 256, 0, stream>>>(
        (const Cx<R>*)arena_base, 0, (const Recipe*)(base + p.off_recipe),
        &((SliceResult*)(base + p.off_result))[p.n_slices].status, status_nonfinite(sl, -1));
    e = cudaGetLastError();
  }
  return e;
}

// `ws` holds the plan's state (program, bookkeeping, results, scratch: the bytes before
// off_arena); `arena` holds its tensors (and the complex128 tail region, if any).
cudaError_t launch_impl(const Plan& p, int32_t precision, void* ws, void* arena, cudaStream_t stream,
                        Prof* prof, const LaunchOpts& o) {
  char* base = (char*)ws;
  char* arena_base = (char*)arena;
  Marker mk{prof, stream, o.nvtx};
  SliceResult* res = (SliceResult*)(base + p.off_result);
  const int32_t n_steps = (int32_t)p.steps.size();
  const long long first = o.slice_first;
  const long long stop = o.slice_count < 0 ? p.n_slices : first + o.slice_count;
  if (first < 0 || stop > p.n_slices || stop <= first) return cudaErrorInvalidValue;
  unsigned long long* errw = &res[p.n_slices].status;
  cudaError_t e;
  for (long long sl = first; sl < stop; ++sl) {
    // bookkeeping and split-K tickets; the first slice also clears the slice results and
    // the total record (its status word is the evaluation's error word)
    const uint64_t clear = sl == first ? p.off_result - p.off_meta + sizeof(SliceResult) * (p.n_slices + 1)
                                       : p.off_result - p.off_meta;
    e = cudaMemsetAsync(base + p.off_meta, 0, clear, stream);
    if (e != cudaSuccess) return e;
    if (precision == PK_C128) {
      if ((e = launch_build<double>(p, base, arena_base, sl, stream, mk, o)) != cudaSuccess) return e;
      if ((e = launch_bulk<double>(p, base, arena_base, 0, n_steps, stream, mk, o, sl)) != cudaSuccess) return e;
      mk.step = -1;
      mk.begin(3, 0, 0, gpu_fill(1, 8));
      k_slice_result<double><<<1, 32, 0, stream>>>((Cx<double>*)arena_base,
                                                   p.tensors[p.final_tensor].offset,
                                                   (Meta*)(base + p.off_meta), p.final_tensor, res, sl);
      mk.end();
    } else if (precision == PK_SPLIT) {
      if ((e = launch_build<ff>(p, base, arena_base, sl, stream, mk, o)) != cudaSuccess) return e;
      if ((e = launch_bulk<ff>(p, base, arena_base, 0, n_steps, stream, mk, o, sl)) != cudaSuccess) return e;
      mk.step = -1;
      mk.begin(3, 0, 0, gpu_fill(1, 8));
      k_slice_result<ff><<<1, 32, 0, stream>>>((Cx<ff>*)arena_base,
                                               p.tensors[p.final_tensor].offset,
                                               (Meta*)(base + p.off_meta), p.final_tensor, res, sl);
      mk.end();
    } else if (p.tail.empty() && p.conv.empty()) {  // complex64
      if ((e = launch_build<float>(p, base, arena_base, sl, stream, mk, o)) != cudaSuccess) return e;
      if ((e = launch_bulk<float>(p, base, arena_base, 0, n_steps, stream, mk, o, sl)) != cudaSuccess) return e;
      mk.step = -1;
      mk.begin(3, 0, 0, gpu_fill(1, 8));
      k_slice_result<float><<<1, 32, 0, stream>>>((Cx<float>*)arena_base,
                                                  p.tensors[p.final_tensor].offset,
                                                  (Meta*)(base + p.off_meta), p.final_tensor, res, sl);
      mk.end();
    } else {  // complex64 with a complex128 tail
      if ((e = launch_build<float>(p, base, arena_base, sl, stream, mk, o)) != cudaSuccess) return e;
      if ((e = launch_bulk<float>(p, base, arena_base, 0, p.tail_first, stream, mk, o, sl)) != cudaSuccess) return e;
      Cx<double>* tail = (Cx<double>*)(arena_base + (p.off_tail - p.off_arena));
      Meta* meta = (Meta*)(base + p.off_meta);
      if (!p.conv.empty()) {
        int64_t maxel = 1;
        for (const auto& c : p.conv) maxel = std::max<int64_t>(maxel, c.elems);
        const unsigned bx = (unsigned)std::min<int64_t>((maxel + 255) / 256, 256);
        mk.begin(0, 0, 24.0 * (double)maxel, gpu_fill((long long)bx * p.conv.size(), 8));
        k_widen<<<dim3(bx, (unsigned)p.conv.size()), 256, 0, stream>>>(
            (const ConvRec*)(base + p.off_conv), (const Cx<float>*)arena_base, tail, meta);
        mk.end();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
      }
      for (const TailStep& ts : p.tail) {
        Step s = p.steps[ts.step];
        s.a = ts.meta_a;
        s.b = ts.meta_b;
        s.off_a = ts.off_a;
        s.off_b = ts.off_b;
        s.off_c = ts.off_c;
        mk.step = ts.step;
        e = launch_step<double>(s, tail, meta, (Cx<double>*)(base + p.off_scratch),
                                (unsigned*)(base + p.off_counter) + ts.step, stream, mk,
                                step_bytes(p, p.steps[ts.step], 16.0));
        if (e == cudaSuccess && o.check_finite)
          e = check_tensor<double>(tail + ts.off_c, p.tensors[p.steps[ts.step].c].elems, errw,
                                   status_nonfinite(sl, ts.step), stream);
        if (e != cudaSuccess) return e;
      }
      mk.step = -1;
      mk.begin(3, 0, 0, gpu_fill(1, 8));
      k_slice_result<double><<<1, 32, 0, stream>>>(tail, p.final_tail_off, meta, p.final_tensor,
                                                   res, sl);
      mk.end();
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  mk.step = -1;
  mk.begin(3, 0, 0, gpu_fill(1, 8));
  k_sum_slices<<<1, 256, 0, stream>>>(res, p.n_slices);
  mk.end();
  return cudaGetLastError();
}

// The reverse-pass program of a PK_FLAG_GRAD plan (forward, recompute and adjoint
// steps on one arena), per slice followed by the slice scalar and the accumulation of
// the clause tensors' adjoints; then the sum over slices.
template <typename R>
cudaError_t launch_grad_impl(const Plan& p, char* base, cudaStream_t stream) {
  const GradProgram& G = p.grad;
  Marker mk{nullptr, stream};
  Cx<R>* arena = (Cx<R>*)(base + G.off_arena);
  Meta* meta = (Meta*)(base + G.off_meta);
  SliceResult* res = (SliceResult*)(base + G.off_result);
  Cx<double>* partial = (Cx<double>*)(base + G.off_scratch);
  unsigned* counters = (unsigned*)(base + G.off_counter);
  const uint64_t nl = std::max<size_t>(1, G.leaves.size());
  Cx<double>* acc = (Cx<double>*)(base + G.off_acc);
  long long* acc_exp = (long long*)(base + G.off_acc + 16ull * (uint64_t)p.q * p.q * nl);
  if (p.n_init > 65535) return cudaErrorInvalidValue;
  int64_t maxel = 1;
  for (const auto& r : G.recipes) maxel = std::max<int64_t>(maxel, r.elems);
  const unsigned bx = (unsigned)std::min<int64_t>((maxel + 255) / 256, 64);
  cudaError_t e = cudaMemsetAsync(base + G.off_acc, 0, G.off_arena - G.off_acc, stream);
  if (e != cudaSuccess) return e;
  for (long long sl = 0; sl < p.n_slices; ++sl) {
    e = cudaMemsetAsync(base + G.off_meta, 0, G.off_result - G.off_meta, stream);
    if (e != cudaSuccess) return e;
    if (p.n_init > 0) {
      k_build<R><<<dim3(bx, (unsigned)p.n_init), 256, 0, stream>>>(
          (const Recipe*)(base + G.off_recipe), (const Slot*)(base + G.off_slots), arena, meta,
          p.q, sl, (int)p.sliced.size());
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const TinyStep* tiny = (const TinyStep*)(base + G.off_tiny);
    size_t sg = 0;
    for (size_t i = 0; i < G.steps.size();) {
      while (sg < G.segments.size() && (size_t)G.segments[sg].first < i) ++sg;
      if (sg < G.segments.size() && (size_t)G.segments[sg].first == i) {  // one sequence launch
        const Segment& g = G.segments[sg];
        k_seg<R><<<1, 256, 0, stream>>>(tiny + g.tiny0, g.count, arena, meta);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        i += g.count;
        continue;
      }
      e = launch_step<R>(G.steps[i], arena, meta, partial, counters + i, stream, mk, 0.0);
      if (e != cudaSuccess) return e;
      ++i;
    }
    k_slice_result<R><<<1, 32, 0, stream>>>(arena, G.root_offset, meta, G.root_meta, res, sl);
    if (!G.leaves.empty())
      k_grad_accum<R><<<(unsigned)G.leaves.size(), 256, 0, stream>>>(
          (const GradLeaf*)(base + G.off_leaves), arena, meta, acc, acc_exp, p.q, sl);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  k_sum_slices<<<1, 256, 0, stream>>>(res, p.n_slices);
  return cudaGetLastError();
}

}  // namespace

namespace {
template <typename R>
cudaError_t raise_rows_smem() {
  const int lim = 200 * 1024;
  void (*fns[])(const Step, Cx<R>*, Meta*, int) = {k_rows<R, 1>,  k_rows<R, 2>,  k_rows<R, 4>,
                                                   k_rows<R, 8>,  k_rows<R, 16>, k_rows<R, 32>,
                                                   k_rows<R, 0>};
  for (auto f : fns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e != cudaSuccess) return e;
  }
  return cudaFuncSetAttribute(k_outs<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

template <int S, bool DB, bool Q>
cudaError_t prepare_gemm_tc() {
  cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<S, DB, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       DB ? tc::Cfg<S>::kSmemDB : tc::Cfg<S>::kSmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_gemm_tc<S, DB, Q>, cudaFuncAttributePreferredSharedMemoryCarveout,
                              cudaSharedmemCarveoutMaxShared);
}

template <int S>
cudaError_t prepare_tc() {
  cudaError_t e;
  if ((e = prepare_gemm_tc<S, false, false>()) != cudaSuccess) return e;
  if ((e = prepare_gemm_tc<S, false, true>()) != cudaSuccess) return e;
  if ((e = prepare_gemm_tc<S, true, false>()) != cudaSuccess) return e;
  if ((e = prepare_gemm_tc<S, true, true>()) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_digits<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              tc::Cfg<S>::kConvSmem);
}
}  // namespace

cudaError_t prepare_kernels() {
  static bool done[256] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
    g_sms = sms;
  if (dev >= 0 && dev < 256 && done[dev]) return cudaSuccess;
  if ((e = raise_rows_smem<double>()) != cudaSuccess) return e;
  if ((e = raise_rows_smem<float>()) != cudaSuccess) return e;
  if ((e = raise_rows_smem<ff>()) != cudaSuccess) return e;
  if ((e = prepare_tc<4>()) != cudaSuccess) return e;
  if ((e = prepare_tc<5>()) != cudaSuccess) return e;
  if (dev >= 0 && dev < 256) done[dev] = true;
  return cudaSuccess;
}

cudaError_t launch_plan(const Plan& p, int32_t precision, void* ws, void* arena,
                        cudaStream_t stream) {
  cudaError_t e = prepare_kernels();
  if (e != cudaSuccess) return e;
  return launch_impl(p, precision, ws, arena, stream, nullptr, LaunchOpts{});
}

cudaError_t launch_plan_opts(const Plan& p, int32_t precision, void* ws, void* arena,
                             cudaStream_t stream, const LaunchOpts& opts) {
  cudaError_t e = prepare_kernels();
  if (e != cudaSuccess) return e;
  return launch_impl(p, precision, ws, arena, stream, nullptr, opts);
}

cudaError_t launch_grad(const Plan& p, int32_t precision, void* ws, cudaStream_t stream) {
  cudaError_t e = prepare_kernels();
  if (e != cudaSuccess) return e;
  if (!p.grad.built) return cudaErrorInvalidValue;
  if (precision == PK_C128) return launch_grad_impl<double>(p, (char*)ws, stream);
  if (precision == PK_SPLIT) return launch_grad_impl<ff>(p, (char*)ws, stream);
  return launch_grad_impl<float>(p, (char*)ws, stream);
}

cudaError_t launch_plan_prof(const Plan& p, int32_t precision, void* ws, void* arena,
                             cudaStream_t stream, Prof* prof) {
  cudaError_t e = prepare_kernels();
  if (e != cudaSuccess) return e;
  return launch_impl(p, precision, ws, arena, stream, prof, LaunchOpts{});
}

Prof* prof_new() { return new Prof(); }
void prof_free(Prof* p) { delete p; }

// Per class: summed event durations of the recorded launches (after they completed),
// launches, complex multiply-adds, algorithmic bytes.
cudaError_t prof_read(Prof* const* profs, int n, double* out) {
  double ms[kNumClasses] = {}, cnt[kNumClasses] = {}, cm[kNumClasses] = {}, by[kNumClasses] = {},
         fm[kNumClasses] = {};
  cudaError_t err = cudaSuccess;
  for (int j = 0; j < n; ++j) {
    const Prof& prof = *profs[j];
    for (size_t i = 0; i < prof.ev.size(); ++i) {
      float t = 0;
      cudaError_t e = cudaEventElapsedTime(&t, prof.ev[i].first, prof.ev[i].second);
      if (e != cudaSuccess && err == cudaSuccess) err = e;
      ms[prof.cls[i]] += t;
      fm[prof.cls[i]] += t * prof.ev_fill[i];
    }
    for (int c = 0; c < kNumClasses; ++c) {
      cnt[c] += prof.n[c];
      cm[c] += prof.cmacs[c];
      by[c] += prof.bytes[c];
    }
  }
  for (int c = 0; c < kNumClasses; ++c) {
    out[c] = ms[c];
    out[kNumClasses + c] = cnt[c];
    out[2 * kNumClasses + c] = cm[c];
    out[3 * kNumClasses + c] = by[c];
    out[4 * kNumClasses + c] = fm[c];
  }
  return err;
}

// Every recorded launch of n sequences (events completed) as 6 doubles: sequence index,
// class, start and end in milliseconds after the first sequence's first event (negative
// when earlier), complex multiply-adds, algorithmic bytes.  Writes at most cap records;
// *count = the number of launches.
cudaError_t prof_timeline(Prof* const* profs, int n, double* out, int64_t cap, int64_t* count) {
  int64_t k = 0;
  cudaEvent_t ref = nullptr;
  for (int j = 0; j < n && !ref; ++j)
    if (!profs[j]->ev.empty()) ref = profs[j]->ev[0].first;
  for (int j = 0; j < n; ++j) {
    const Prof& prof = *profs[j];
    for (size_t i = 0; i < prof.ev.size(); ++i, ++k) {
      if (k >= cap) continue;
      float t0 = 0, t1 = 0;
      cudaError_t e = cudaEventElapsedTime(&t0, ref, prof.ev[i].first);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t1, ref, prof.ev[i].second);
      if (e != cudaSuccess) return e;
      double* r = out + 6 * k;
      r[0] = j;
      r[1] = prof.cls[i];
      r[2] = t0;
      r[3] = t1;
      r[4] = prof.ev_cmacs[i];
      r[5] = prof.ev_bytes[i];
    }
  }
  *count = k;
  return cudaSuccess;
}

cudaError_t profile_plan(const Plan& p, int32_t precision, void* ws, void* arena,
                         cudaStream_t stream, double* out) {
  cudaError_t pe = prepare_kernels();
  if (pe != cudaSuccess) return pe;
  Prof prof;
  cudaError_t e = launch_impl(p, precision, ws, arena, stream, &prof, LaunchOpts{});
  cudaError_t e2 = cudaStreamSynchronize(stream);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return e;
  Prof* one = &prof;
  return prof_read(&one, 1, out);
}

}  // namespace pk
