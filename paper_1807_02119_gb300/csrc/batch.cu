// Batched evaluation: many knots (each with its own plan) in one persistent launch.
//
// Every CTA repeatedly takes the next knot from an atomic work counter and performs
// that knot's whole contraction itself -- initial tensors (one warp per tensor), then
// every pairwise step with the CTA's threads spread over the outputs and a block
// barrier between steps, then the slice scalar -- so knots of very different sizes
// balance across the SMs and no CTA ever waits for another one.  The launch (preceded
// by a reset of the counter) is recorded once into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "handles.h"
#include "kernels.cuh"

namespace pk {

// Per-knot header of the batch image (all offsets relative to the batch arrays).
struct BatchKnot {
  int64_t recipe0, n_recipe;   // recipes of the knot
  int64_t slot_base;           // added to Recipe::slot0
  int64_t step0, n_steps;      // steps of the knot
  int64_t arena_off;           // first arena element of the knot
  int64_t meta_off;            // first bookkeeping slot of the knot
  int64_t n_slices;
  int64_t final_offset;        // final tensor (arena elements, relative)
  int32_t n_sliced, q, final_tensor, pad;
};

// A step of the batch image: the contraction's extents and operand offsets, with its
// stride runs packed into the batch's run array (rows, then contracted, then columns)
// instead of the fixed-size run tables of a Step, so the image is about ten times smaller.
struct BatchStep {
  int32_t a, b, c;           // bookkeeping slots relative to the knot (b = -1: constant 1)
  int16_t nrow, nk, nn, pad;
  int64_t off_a, off_b, off_c;
  int64_t R, K, N;
  int64_t run0;              // first run of this step in the run array
};

namespace {


template <typename S>
__device__ __forceinline__ S block_max(S v, S* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  v = lane < (int)(blockDim.x >> 5) ? red[lane] : S(0);
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;  // every thread holds the block maximum
}

// One pairwise step of one knot by the whole CTA (outputs spread over the threads); the
// step's runs are staged in shared memory first.
template <typename R>
__device__ void cta_step(const BatchStep& s, const Run* __restrict__ runs, Run* srun,
                         Cx<R>* arena, Meta* meta, long long* tbl, int ktab,
                         typename Traits<R>::S* red) {
  using S = typename Traits<R>::S;
  const int nruns = s.nrow + s.nk + s.nn;
  for (int i = threadIdx.x; i < nruns; i += blockDim.x) srun[i] = runs[s.run0 + i];
  __syncthreads();
  const Run* row = srun;
  const Run* kr = srun + s.nrow;
  const Run* nr = srun + s.nrow + s.nk;
  const int ea = bin_exp(bits_to_val<S>(meta[s.a].maxbits));
  int eb = 0;
  long long xb = 0;
  const bool hasB = s.b >= 0;
  if (hasB) {
    eb = bin_exp(bits_to_val<S>(meta[s.b].maxbits));
    xb = meta[s.b].exp;
  }
  const long long exp_c = meta[s.a].exp + xb + ea + eb;
  const S scale = (S)ldexp(1.0, -(ea + eb));
  const bool tab = s.K <= ktab;
  if (tab)
    for (long long k = threadIdx.x; k < s.K; k += blockDim.x)
      split_runs((unsigned long long)k, kr, s.nk, tbl[k], tbl[ktab + k]);
  __syncthreads();
  const Cx<R>* A = arena + s.off_a;
  const Cx<R>* B = arena + s.off_b;
  Cx<R>* C = arena + s.off_c;
  const long long outs = s.R * s.N;
  S vmax = 0;
  for (long long o = threadIdx.x; o < outs; o += blockDim.x) {
    const long long r = o % s.R, n = o / s.R;
    long long oa, ob, d, nb = 0;
    split_runs((unsigned long long)r, row, s.nrow, oa, ob);
    if (hasB) split_runs((unsigned long long)n, nr, s.nn, d, nb);
    Acc<R> acc;
    for (long long k = 0; k < s.K; ++k) {
      long long ka, kb;
      if (tab) {
        ka = tbl[k];
        kb = tbl[ktab + k];
      } else {
        split_runs((unsigned long long)k, kr, s.nk, ka, kb);
      }
      const Cx<R> av = ldc(A + oa + ka);
      if (hasB)
        acc.mac(av, ldc(B + ob + nb + kb));
      else
        acc.add(av);
    }
    const Cx<R> v = acc.get(scale);
    st(C + o, v);  // C is [n, r] with r innermost: entry o = r + n R
    vmax = fmax(vmax, mag(v));
  }
  vmax = block_max(vmax, red);
  if (threadIdx.x == 0) {
    meta[s.c].maxbits = max_bits(vmax);
    meta[s.c].exp = exp_c;
  }
  __syncthreads();
}

// T threads per CTA; ktab offsets of the contracted index per step in shared memory.
template <typename R, int T>
__global__ void __launch_bounds__(T) k_batch(const BatchKnot* __restrict__ knots, int n_knots,
                                             const Recipe* recs, const Slot* slots,
                                             const BatchStep* steps, const Run* runs, Cx<R>* arena,
                                             Meta* meta_all, SliceResult* out, unsigned* next,
                                             int ktab) {
  using S = typename Traits<R>::S;
  extern __shared__ long long tbl[];
  __shared__ S red[32];
  __shared__ Run srun[3 * kMaxRuns];
  __shared__ int kn_s;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) kn_s = (int)atomicAdd(next, 1u);
    __syncthreads();
    const int kn = kn_s;
    if (kn >= n_knots) return;
    const BatchKnot K = knots[kn];
    Cx<R>* A0 = arena + K.arena_off;
    Meta* meta = meta_all + K.meta_off;
    double tre = 0, tim = 0;
    long long texp = LLONG_MIN;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (long long sl = 0; sl < K.n_slices; ++sl) {
      int sdig[64];
      {
        long long t = sl;
        for (int i = 0; i < K.n_sliced && i < 64; ++i) {
          sdig[i] = (int)(t % K.q);
          t /= K.q;
        }
      }
      // initial tensors: one warp per tensor
      for (long long j = warp; j < K.n_recipe; j += nwarps) {
        const Recipe r = recs[K.recipe0 + j];
        S vmax = 0;
        for (long long e = lane; e < r.elems; e += 32) {
          double re, im;
          recipe_value(r, slots + K.slot_base, e, K.q, sdig, re, im);
          const Cx<R> v{from_double<R>(re), from_double<R>(im)};
          st(A0 + r.offset + e, v);
          vmax = fmax(vmax, mag(v));
        }
        for (int o = 16; o > 0; o >>= 1) vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        if (lane == 0) {
          meta[r.meta].maxbits = max_bits(vmax);
          meta[r.meta].exp = r.exp2;
        }
      }
      __syncthreads();
      for (long long i = 0; i < K.n_steps; ++i)
        cta_step<R>(steps[K.step0 + i], runs, srun, A0, meta, tbl, ktab, red);
      if (threadIdx.x == 0) {  // add this slice's scalar at a common exponent
        const Cx<R> v = ldc(A0 + K.final_offset);
        double vr = to_double(v.re), vi = to_double(v.im);
        long long ve = meta[K.final_tensor].exp;
        double m = fmax(fabs(vr), fabs(vi));
        if (m > 0) {
          int k;
          frexp(m, &k);
          vr = ldexp(vr, -k);
          vi = ldexp(vi, -k);
          ve += k;
          if (texp == LLONG_MIN) {
            tre = vr;
            tim = vi;
            texp = ve;
          } else {
            const long long e = max(texp, ve);
            const long long da = max(texp - e, -2000LL), db = max(ve - e, -2000LL);
            tre = ldexp(tre, (int)da) + ldexp(vr, (int)db);
            tim = ldexp(tim, (int)da) + ldexp(vi, (int)db);
            texp = e;
          }
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      out[kn].re = tre;
      out[kn].im = tim;
      out[kn].exp = texp == LLONG_MIN ? 0 : texp;
    }
  }
}

uint64_t a256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

}  // namespace
}  // namespace pk

struct pk_batch {
  int32_t precision = 0;
  int32_t n = 0;
  std::vector<pk::BatchKnot> knots;
  std::vector<pk::Recipe> recipes;
  std::vector<pk::Slot> slots;
  std::vector<pk::BatchStep> steps;
  std::vector<pk::Run> runs;
  std::vector<pk::Knot> kinfo;
  std::vector<pk::Scaled> factor;
  std::vector<int32_t> qs;
  uint64_t off_knots = 0, off_recipes = 0, off_slots = 0, off_steps = 0, off_runs = 0, off_meta = 0,
           off_results = 0, off_counter = 0, off_arena = 0, total = 0, image_bytes = 0;
  std::vector<uint8_t> image;
  uint8_t* pinned = nullptr;
  pk::SliceResult* pinned_results = nullptr;
  void* graph_ws = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int32_t device = -1;
  int32_t threads = 256, ktab = 2048;   // launch shape (the context's tuning at creation)
};

namespace {

pk_status bfail(pk_ctx* c, pk_status s, const std::string& m) {
  if (c) c->err = m;
  return s;
}

template <typename R>
void* batch_kernel(int threads) {
  if (threads == 128) return (void*)pk::k_batch<R, 128>;
  if (threads == 512) return (void*)pk::k_batch<R, 512>;
  return (void*)pk::k_batch<R, 256>;
}

cudaError_t build_graph(pk_batch* b, void* ws, cudaStream_t stream) {
  (void)stream;
  if (b->exec && b->graph_ws == ws) return cudaSuccess;
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (b->graph) {
    cudaGraphDestroy(b->graph);
    b->graph = nullptr;
  }
  char* base = (char*)ws;
  cudaError_t e = cudaGraphCreate(&b->graph, 0);
  if (e != cudaSuccess) return e;
  cudaMemsetParams mp;
  std::memset(&mp, 0, sizeof(mp));
  mp.dst = base + b->off_counter;
  mp.value = 0;
  mp.elementSize = 4;
  mp.width = 1;
  mp.height = 1;
  cudaGraphNode_t memset_node, kernel_node;
  e = cudaGraphAddMemsetNode(&memset_node, b->graph, nullptr, 0, &mp);
  if (e != cudaSuccess) return e;
  void* func;
  if (b->precision == PK_C128)
    func = batch_kernel<double>(b->threads);
  else if (b->precision == PK_C64)
    func = batch_kernel<float>(b->threads);
  else
    func = batch_kernel<pk::ff>(b->threads);
  const size_t smem = sizeof(long long) * 2 * (size_t)b->ktab;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const pk::BatchKnot* knots = (const pk::BatchKnot*)(base + b->off_knots);
  int n = b->n;
  const pk::Recipe* recs = (const pk::Recipe*)(base + b->off_recipes);
  const pk::Slot* slots = (const pk::Slot*)(base + b->off_slots);
  const pk::BatchStep* steps = (const pk::BatchStep*)(base + b->off_steps);
  const pk::Run* runs = (const pk::Run*)(base + b->off_runs);
  void* arena = base + b->off_arena;
  pk::Meta* meta = (pk::Meta*)(base + b->off_meta);
  pk::SliceResult* res = (pk::SliceResult*)(base + b->off_results);
  unsigned* counter = (unsigned*)(base + b->off_counter);
  int ktab = b->ktab;
  void* args[] = {&knots, &n, &recs, &slots, &steps, &runs, &arena, &meta, &res, &counter, &ktab};
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, b->threads, smem);
  if (e != cudaSuccess) return e;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  const int grid = std::max(1, std::min(per_sm * sms, n));
  cudaKernelNodeParams kp;
  std::memset(&kp, 0, sizeof(kp));
  kp.func = func;
  kp.gridDim = dim3((unsigned)grid);
  kp.blockDim = dim3((unsigned)b->threads);
  kp.sharedMemBytes = (unsigned)smem;
  kp.kernelParams = args;
  e = cudaGraphAddKernelNode(&kernel_node, b->graph, &memset_node, 1, &kp);
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) return e;
  b->graph_ws = ws;
  return cudaSuccess;
}

}  // namespace

extern "C" {

pk_status pk_batch_create(pk_ctx* ctx, const pk_plan* const* plans, int32_t n, int32_t precision,
                          pk_batch** out) {
  if (!out || (n > 0 && !plans) || n < 0) return bfail(ctx, PK_EINVAL, "bad argument");
  if (precision != PK_C128 && precision != PK_C64 && precision != PK_SPLIT)
    return bfail(ctx, PK_EINVAL, "bad precision");
  *out = nullptr;
  pk_batch* b = new (std::nothrow) pk_batch();
  if (!b) return bfail(ctx, PK_ENOMEM, "out of host memory");
  b->precision = precision;
  b->n = n;
  b->device = ctx ? ctx->device : -1;
  b->threads = ctx ? ctx->tuning.batch_threads : kTunedDefault.batch_threads;
  b->ktab = ctx ? ctx->tuning.batch_ktab : kTunedDefault.batch_ktab;
  int64_t arena = 0, meta = 0;
  for (int32_t i = 0; i < n; ++i) {
    if (!plans[i]) {
      delete b;
      return bfail(ctx, PK_EINVAL, "null plan");
    }
    const pk::Plan& P = plans[i]->p;
    pk::BatchKnot k;
    std::memset(&k, 0, sizeof(k));
    k.recipe0 = (int64_t)b->recipes.size();
    k.n_recipe = (int64_t)P.recipes.size();
    k.slot_base = (int64_t)b->slots.size();
    k.step0 = (int64_t)b->steps.size();
    k.n_steps = (int64_t)P.steps.size();
    k.arena_off = arena;
    k.meta_off = meta;
    k.n_slices = P.n_slices;
    k.final_offset = P.tensors[P.final_tensor].offset;
    k.n_sliced = (int32_t)P.sliced.size();
    k.q = P.q;
    k.final_tensor = P.final_tensor;
    b->knots.push_back(k);
    b->recipes.insert(b->recipes.end(), P.recipes.begin(), P.recipes.end());
    b->slots.insert(b->slots.end(), P.slots.begin(), P.slots.end());
    for (const pk::Step& st : P.steps) {
      pk::BatchStep bs;
      std::memset(&bs, 0, sizeof(bs));
      bs.a = st.a;
      bs.b = st.b;
      bs.c = st.c;
      bs.nrow = (int16_t)st.nrow;
      bs.nk = (int16_t)st.nk;
      bs.nn = (int16_t)st.nn;
      bs.off_a = st.off_a;
      bs.off_b = st.off_b;
      bs.off_c = st.off_c;
      bs.R = st.R;
      bs.K = st.K;
      bs.N = st.N;
      bs.run0 = (int64_t)b->runs.size();
      b->runs.insert(b->runs.end(), st.row, st.row + st.nrow);
      b->runs.insert(b->runs.end(), st.kr, st.kr + st.nk);
      b->runs.insert(b->runs.end(), st.nr, st.nr + st.nn);
      b->steps.push_back(bs);
    }
    b->kinfo.push_back(P.knot);
    b->factor.push_back(P.factor);
    b->qs.push_back(P.q);
    arena += (P.arena_elems + 63) / 64 * 64;
    meta += (int64_t)P.tensors.size();
  }
  const uint64_t eb = precision == PK_C64 ? 8 : 16;
  uint64_t off = 0;
  b->off_knots = off;
  off = pk::a256(off + sizeof(pk::BatchKnot) * std::max<size_t>(1, b->knots.size()));
  b->off_recipes = off;
  off = pk::a256(off + sizeof(pk::Recipe) * std::max<size_t>(1, b->recipes.size()));
  b->off_slots = off;
  off = pk::a256(off + sizeof(pk::Slot) * std::max<size_t>(1, b->slots.size()));
  b->off_steps = off;
  off = pk::a256(off + sizeof(pk::BatchStep) * std::max<size_t>(1, b->steps.size()));
  b->off_runs = off;
  off = pk::a256(off + sizeof(pk::Run) * std::max<size_t>(1, b->runs.size()));
  b->image_bytes = off;
  b->off_meta = off;
  off = pk::a256(off + 16ull * (uint64_t)std::max<int64_t>(1, meta));
  b->off_results = off;
  off = pk::a256(off + sizeof(pk::SliceResult) * (uint64_t)std::max(1, n));
  b->off_counter = off;
  off = pk::a256(off + 256);
  b->off_arena = off;
  b->total = off + eb * (uint64_t)std::max<int64_t>(1, arena);
  b->image.assign(b->image_bytes, 0);
  if (!b->knots.empty())
    std::memcpy(b->image.data() + b->off_knots, b->knots.data(), sizeof(pk::BatchKnot) * b->knots.size());
  if (!b->recipes.empty())
    std::memcpy(b->image.data() + b->off_recipes, b->recipes.data(),
                sizeof(pk::Recipe) * b->recipes.size());
  if (!b->slots.empty())
    std::memcpy(b->image.data() + b->off_slots, b->slots.data(), sizeof(pk::Slot) * b->slots.size());
  if (!b->steps.empty())
    std::memcpy(b->image.data() + b->off_steps, b->steps.data(), sizeof(pk::BatchStep) * b->steps.size());
  if (!b->runs.empty())
    std::memcpy(b->image.data() + b->off_runs, b->runs.data(), sizeof(pk::Run) * b->runs.size());
  *out = b;
  return PK_OK;
}

pk_status pk_batch_workspace_bytes(const pk_batch* b, uint64_t* bytes, uint64_t* upload_bytes) {
  if (!b || !bytes) return PK_EINVAL;
  *bytes = b->total;
  if (upload_bytes) *upload_bytes = b->image_bytes;
  return PK_OK;
}

pk_status pk_batch_upload(pk_ctx* ctx, pk_batch* b, void* d_ws, uint64_t bytes) {
  if (!ctx || !b || !d_ws) return bfail(ctx, PK_EINVAL, "bad argument");
  if (ctx->device < 0) return bfail(ctx, PK_ENODEVICE, "host-only context");
  if (bytes < b->total) return bfail(ctx, PK_ENOMEM, "workspace smaller than pk_batch_workspace_bytes");
  if ((uintptr_t)d_ws & 255u) return bfail(ctx, PK_EINVAL, "workspace must be 256-byte aligned");
  if (!b->pinned) {
    if (cudaMallocHost((void**)&b->pinned, std::max<uint64_t>(1, b->image_bytes)) != cudaSuccess)
      return bfail(ctx, PK_ENOMEM, "pinned host allocation failed");
    std::memcpy(b->pinned, b->image.data(), b->image_bytes);
  }
  cudaError_t e = cudaMemcpyAsync(d_ws, b->pinned, b->image_bytes, cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) return bfail(ctx, PK_ECUDA, std::string("batch upload: ") + cudaGetErrorString(e));
  return PK_OK;
}

pk_status pk_batch_upload_inputs(pk_ctx* ctx, pk_batch* b, void* d_ws, uint64_t bytes,
                                 uint64_t* copied) {
  if (!ctx || !b || !d_ws) return bfail(ctx, PK_EINVAL, "bad argument");
  if (ctx->device < 0) return bfail(ctx, PK_ENODEVICE, "host-only context");
  if (bytes < b->total) return bfail(ctx, PK_ENOMEM, "workspace smaller than pk_batch_workspace_bytes");
  if ((uintptr_t)d_ws & 255u) return bfail(ctx, PK_EINVAL, "workspace must be 256-byte aligned");
  if (!b->pinned) {
    if (cudaMallocHost((void**)&b->pinned, std::max<uint64_t>(1, b->image_bytes)) != cudaSuccess)
      return bfail(ctx, PK_ENOMEM, "pinned host allocation failed");
    std::memcpy(b->pinned, b->image.data(), b->image_bytes);
  }
  // knots, recipes and slots lie first in the image, the steps and runs after them
  const uint64_t n = b->off_steps - b->off_knots;
  cudaError_t e = cudaMemcpyAsync((char*)d_ws + b->off_knots, b->pinned + b->off_knots, n,
                                  cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) return bfail(ctx, PK_ECUDA, std::string("batch upload: ") + cudaGetErrorString(e));
  if (copied) *copied = n;
  return PK_OK;
}

pk_status pk_batch_launch(pk_ctx* ctx, pk_batch* b, void* d_ws, uint64_t bytes) {
  if (!ctx || !b || !d_ws) return bfail(ctx, PK_EINVAL, "bad argument");
  if (ctx->device < 0) return bfail(ctx, PK_ENODEVICE, "host-only context");
  if (bytes < b->total) return bfail(ctx, PK_ENOMEM, "workspace smaller than pk_batch_workspace_bytes");
  if (b->n == 0) return PK_OK;
  cudaError_t e = build_graph(b, d_ws, ctx->stream);
  if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, ctx->stream);
  if (e != cudaSuccess) return bfail(ctx, PK_ECUDA, std::string("batch launch: ") + cudaGetErrorString(e));
  return PK_OK;
}

pk_status pk_batch_download(pk_ctx* ctx, pk_batch* b, const void* d_ws, pk_scaled* Z, pk_scaled* V) {
  if (!ctx || !b || !d_ws || (!Z && b->n > 0)) return bfail(ctx, PK_EINVAL, "bad argument");
  if (b->n == 0) return PK_OK;
  if (!b->pinned_results &&
      cudaMallocHost((void**)&b->pinned_results, sizeof(pk::SliceResult) * b->n) != cudaSuccess)
    return bfail(ctx, PK_ENOMEM, "pinned host allocation failed");
  cudaError_t e = cudaMemcpyAsync(b->pinned_results, (const char*)d_ws + b->off_results,
                                  sizeof(pk::SliceResult) * b->n, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return bfail(ctx, PK_ECUDA, std::string("batch download: ") + cudaGetErrorString(e));
  pk_status status = PK_OK;
  for (int32_t i = 0; i < b->n; ++i) {
    pk::Scaled z;
    z.re = b->pinned_results[i].re;
    z.im = b->pinned_results[i].im;
    z.e = b->pinned_results[i].exp;
    z.norm();
    z = pk::s_mul(z, b->factor[i]);
    Z[i].re = z.re;
    Z[i].im = z.im;
    Z[i].exp2 = z.e;
    if (V) {
      const pk::Knot& k = b->kinfo[i];
      if (!pk::jones_defined(k)) {
        V[i].re = V[i].im = 0;
        V[i].exp2 = 0;
        status = PK_EINVAL;
        continue;
      }
      pk::Scaled v = pk::s_mul(pk::jones_prefactor(k, b->qs[i]), z);
      V[i].re = v.re;
      V[i].im = v.im;
      V[i].exp2 = v.e;
    }
  }
  if (status != PK_OK) ctx->err = "some batch entries violate the A(q) exponent condition: V left 0";
  return status;
}

pk_status pk_eval_batch(pk_ctx* ctx, const pk_plan* const* plans, int32_t n, int32_t precision,
                        void* d_ws, uint64_t bytes, pk_scaled* Z, pk_scaled* V) {
  pk_batch* b = nullptr;
  pk_status s = pk_batch_create(ctx, plans, n, precision, &b);
  if (s != PK_OK) return s;
  s = pk_batch_upload(ctx, b, d_ws, bytes);
  if (s == PK_OK) s = pk_batch_launch(ctx, b, d_ws, bytes);
  if (s == PK_OK) s = pk_batch_download(ctx, b, d_ws, Z, V);
  pk_batch_destroy(b);
  return s;
}

void pk_batch_destroy(pk_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->pinned) cudaFreeHost(b->pinned);
  if (b->pinned_results) cudaFreeHost(b->pinned_results);
  delete b;
}

}  // extern "C"
