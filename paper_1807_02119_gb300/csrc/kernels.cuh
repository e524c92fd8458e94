// Device kernels of the contraction (Sec. III), included by launch.cu: initial tensors
// of G_T, one pairwise contraction step, and the per-slice / all-slice results.
//
// A step computes C[b, m, n] = sum_k A[b, m, k] B[b, k, n] where b (batch) are indices
// kept in both operands, m kept only in A, n kept only in B, and k summed.  The
// operands stay in the layout their producer wrote; every class of indices is a short
// list of merged stride runs, so the index permutation is folded into the loads and
// the store (no separate transpose pass).  C is written as [n-part, row-part] with the
// row part (b and m, in A's order) innermost and contiguous.
//
// Storage types R: double (complex128), float (complex64) and ff (complex "split FP32":
// each real number is an unevaluated float pair hi + lo, |lo| <= ulp(hi)/2, computed
// with exact FMA two-products and TwoSum additions -- about 48 significant bits on the
// FP32 units).
//
// Scaling: a stored tensor x stands for x * 2^exp.  A step multiplies its products by
// 2^-(eA+eB), eX being the binary exponent of max|X| (so operands enter at magnitude
// below 1), and records exp(C) = exp(A) + exp(B) + eA + eB.  Powers of two are exact.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <climits>
#include <type_traits>

#include "pk_internal.h"

namespace pk {

struct ff {
  float hi, lo;
};

template <typename R>
struct Cx {
  R re, im;
};

// S: the scalar type of magnitudes and scale factors for a storage type
template <typename R>
struct Traits {
  using S = R;
};
template <>
struct Traits<ff> {
  using S = float;
};

// ---- float-float arithmetic (Dekker / Knuth error-free transformations)
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = fmaf(a, b, -p);
}
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ ff ff_norm(float hi, float lo) {
  float s = __fadd_rn(hi, lo);
  return {s, __fsub_rn(lo, __fsub_rn(s, hi))};
}
// a * b for float-float a, b: the exact product of the high parts plus the cross terms
__device__ __forceinline__ void ff_mul(const ff& a, const ff& b, float& p, float& e) {
  two_prod(a.hi, b.hi, p, e);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
}
// (hi, lo) += (p, e)
__device__ __forceinline__ void ff_acc(float& hi, float& lo, float p, float e) {
  float s, err;
  two_sum(hi, p, s, err);
  lo = __fadd_rn(lo, __fadd_rn(err, e));
  hi = s;
}

// ---- loads, stores, conversions
template <typename R>
__device__ __forceinline__ Cx<R> ld(const Cx<R>* p);
template <>
__device__ __forceinline__ Cx<double> ld(const Cx<double>* p) {
  double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}
template <>
__device__ __forceinline__ Cx<float> ld(const Cx<float>* p) {
  float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return {v.x, v.y};
}
template <>
__device__ __forceinline__ Cx<ff> ld(const Cx<ff>* p) {
  float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return {{v.x, v.y}, {v.z, v.w}};
}
// Coherent loads (plain ld.global): for data the same kernel wrote earlier, which the
// read-only path of __ldg does not guarantee to see.
__device__ __forceinline__ Cx<double> ldc(const Cx<double>* p) {
  double2 v = *reinterpret_cast<const double2*>(p);
  return {v.x, v.y};
}
__device__ __forceinline__ Cx<float> ldc(const Cx<float>* p) {
  float2 v = *reinterpret_cast<const float2*>(p);
  return {v.x, v.y};
}
__device__ __forceinline__ Cx<ff> ldc(const Cx<ff>* p) {
  float4 v = *reinterpret_cast<const float4*>(p);
  return {{v.x, v.y}, {v.z, v.w}};
}
__device__ __forceinline__ void st(Cx<double>* p, Cx<double> x) {
  *reinterpret_cast<double2*>(p) = make_double2(x.re, x.im);
}
__device__ __forceinline__ void st(Cx<float>* p, Cx<float> x) {
  *reinterpret_cast<float2*>(p) = make_float2(x.re, x.im);
}
__device__ __forceinline__ void st(Cx<ff>* p, Cx<ff> x) {
  *reinterpret_cast<float4*>(p) = make_float4(x.re.hi, x.re.lo, x.im.hi, x.im.lo);
}

template <typename R>
__device__ __forceinline__ R from_double(double x) {
  return (R)x;
}
template <>
__device__ __forceinline__ ff from_double<ff>(double x) {
  float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double to_double(double x) { return x; }
__device__ __forceinline__ double to_double(float x) { return (double)x; }
__device__ __forceinline__ double to_double(ff x) { return (double)x.hi + (double)x.lo; }

template <typename R>
__device__ __forceinline__ Cx<R> czero() {
  return {from_double<R>(0.0), from_double<R>(0.0)};
}
// max(|re|, |im|) in the scalar type (the high part for float-float)
__device__ __forceinline__ double mag(const Cx<double>& v) { return fmax(fabs(v.re), fabs(v.im)); }
__device__ __forceinline__ float mag(const Cx<float>& v) { return fmaxf(fabsf(v.re), fabsf(v.im)); }
__device__ __forceinline__ float mag(const Cx<ff>& v) { return fmaxf(fabsf(v.re.hi), fabsf(v.im.hi)); }

__device__ __forceinline__ void cmac(Cx<double>& acc, const Cx<double>& a, const Cx<double>& b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
__device__ __forceinline__ void cmac(Cx<float>& acc, const Cx<float>& a, const Cx<float>& b) {
  acc.re = fmaf(a.re, b.re, acc.re);
  acc.re = fmaf(-a.im, b.im, acc.re);
  acc.im = fmaf(a.re, b.im, acc.im);
  acc.im = fmaf(a.im, b.re, acc.im);
}

// ---- accumulators: plain in the storage precision, or float-float
template <typename R>
struct Acc {
  Cx<R> v{0, 0};
  __device__ __forceinline__ void mac(const Cx<R>& a, const Cx<R>& b) { cmac(v, a, b); }
  __device__ __forceinline__ void add(const Cx<R>& a) {
    v.re += a.re;
    v.im += a.im;
  }
  __device__ __forceinline__ Cx<R> get(R scale) const { return {v.re * scale, v.im * scale}; }
};
template <>
struct Acc<ff> {
  float rh = 0, rl = 0, ih = 0, il = 0;
  __device__ __forceinline__ void mac(const Cx<ff>& a, const Cx<ff>& b) {
    float p, e;
    ff_mul(a.re, b.re, p, e);
    ff_acc(rh, rl, p, e);
    ff_mul(a.im, b.im, p, e);
    ff_acc(rh, rl, -p, -e);
    ff_mul(a.re, b.im, p, e);
    ff_acc(ih, il, p, e);
    ff_mul(a.im, b.re, p, e);
    ff_acc(ih, il, p, e);
  }
  __device__ __forceinline__ void add(const Cx<ff>& a) {
    ff_acc(rh, rl, a.re.hi, a.re.lo);
    ff_acc(ih, il, a.im.hi, a.im.lo);
  }
  __device__ __forceinline__ Cx<ff> get(float scale) const {  // scale: a power of two
    ff r = ff_norm(rh, rl), i = ff_norm(ih, il);
    return {{r.hi * scale, r.lo * scale}, {i.hi * scale, i.lo * scale}};
  }
};

// ---- bookkeeping
__device__ __forceinline__ unsigned long long max_bits(double m) {
  return (unsigned long long)__double_as_longlong(m);
}
__device__ __forceinline__ unsigned long long max_bits(float m) {
  return (unsigned long long)__float_as_uint(m);
}
template <typename S>
__device__ __forceinline__ S bits_to_val(unsigned long long b);
template <>
__device__ __forceinline__ double bits_to_val<double>(unsigned long long b) {
  return __longlong_as_double((long long)b);
}
template <>
__device__ __forceinline__ float bits_to_val<float>(unsigned long long b) {
  return __uint_as_float((unsigned)b);
}

// binary exponent e with m * 2^-e in [0.5, 1); 0 for m == 0
template <typename S>
__device__ __forceinline__ int bin_exp(S m) {
  if (!(m > S(0))) return 0;
  int e;
  frexp(m, &e);
  return e;
}

template <typename S>
__device__ __forceinline__ void block_max_to_meta(S v, Meta* meta) {
  __shared__ S red[32];
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    int nw = (blockDim.x + 31) >> 5;
    v = lane < nw ? red[lane] : S(0);
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0 && v > S(0)) atomicMax(&meta->maxbits, max_bits(v));
  }
}

// ------------------------------------------------------------------ initial tensors
// Entry e of an initial tensor: sum_{s<q} prod_j f_j(s, x_j) in double (x_j = the
// digit of e at slot j's position, or the fixed value of a sliced index); an absorbed
// slot contributes its clause matrix entry M(s, x_j) (diagonal or off-diagonal weight).
__device__ __forceinline__ void recipe_value(const Recipe& r, const Slot* slots, long long e, int q,
                                             const int* sdig, double& sre, double& sim) {
  sre = 0;
  sim = 0;
  if (r.kind == 1) {
    sre = 1;
    return;
  }
  for (int s = 0; s < q; ++s) {
    double pre = 1, pim = 0;
    bool zero = false;
    for (int j = 0; j < r.nslot; ++j) {
      const Slot sl = slots[r.slot0 + j];
      int x;
      if (sl.dimpos >= 0) {
        long long t = e;
        for (int d = 0; d < sl.dimpos; ++d) t /= q;
        x = (int)(t % q);
      } else {
        x = sdig[sl.slice_ord];
      }
      if (sl.absorbed) {
        const double fre = s == x ? sl.dre : sl.ore, fim = s == x ? sl.dim : sl.oim;
        const double nre = pre * fre - pim * fim;
        const double nim = pre * fim + pim * fre;
        pre = nre;
        pim = nim;
      } else if (s != x) {
        zero = true;
        break;
      }
    }
    if (!zero) {
      sre += pre;
      sim += pim;
    }
  }
}

// One grid row (blockIdx.y) per initial tensor, formed in double and rounded once to
// the storage type.
template <typename R>
__global__ void __launch_bounds__(256) k_build(const Recipe* __restrict__ rec,
                                               const Slot* __restrict__ slots, Cx<R>* arena,
                                               Meta* meta, int q, long long slice, int n_sliced) {
  using S = typename Traits<R>::S;
  const Recipe r = rec[blockIdx.y];
  S vmax = 0;
  int sdig[64];
  {
    long long s = slice;
    for (int i = 0; i < n_sliced && i < 64; ++i) {
      sdig[i] = (int)(s % q);
      s /= q;
    }
  }
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < r.elems;
       e += (long long)gridDim.x * blockDim.x) {
    double sre, sim;
    recipe_value(r, slots, e, q, sdig, sre, sim);
    const Cx<R> v{from_double<R>(sre), from_double<R>(sim)};
    st(arena + r.offset + e, v);
    vmax = fmax(vmax, mag(v));
  }
  block_max_to_meta(vmax, meta + r.meta);
  if (blockIdx.x == 0 && threadIdx.x == 0) meta[r.meta].exp = r.exp2;
}

// ------------------------------------------------------------------ contraction step
// Offsets of index x of a run class (x below the class's extent, which -- like every
// tensor -- is at most 2^31, so the digits are taken with 32-bit division).
__device__ __forceinline__ void split_runs(unsigned long long x, const Run* runs, int n,
                                           long long& oa, long long& ob) {
  unsigned y = (unsigned)x;
  oa = 0;
  ob = 0;
  for (int i = 0; i < n; ++i) {
    const unsigned sz = (unsigned)runs[i].size;
    const unsigned qd = y / sz, d = y - qd * sz;
    y = qd;
    oa += (long long)d * runs[i].sa;
    ob += (long long)d * runs[i].sb;
  }
}
__device__ __forceinline__ void split_runs32(unsigned x, const Run* runs, int n, long long& oa,
                                             long long& ob) {
  oa = 0;
  ob = 0;
  for (int i = 0; i < n; ++i) {
    unsigned sz = (unsigned)runs[i].size;
    unsigned qd = x / sz;
    unsigned d = x - qd * sz;
    x = qd;
    oa += (long long)d * runs[i].sa;
    ob += (long long)d * runs[i].sb;
  }
}

// scale = 2^-(eA+eB); when write_exp, also records exp(C) = exp(A) + exp(B) + eA + eB
template <typename S>
__device__ __forceinline__ S step_scale(const Step& s, Meta* meta, bool write_exp) {
  int ea = bin_exp(bits_to_val<S>(meta[s.a].maxbits));
  int eb = 0;
  long long xb = 0;
  if (s.b >= 0) {
    eb = bin_exp(bits_to_val<S>(meta[s.b].maxbits));
    xb = meta[s.b].exp;
  }
  if (write_exp) meta[s.c].exp = meta[s.a].exp + xb + ea + eb;
  return (S)ldexp(1.0, -(ea + eb));
}

// Thread per (output row r, chunk of nc columns): the row's offsets are decoded once and
// its K values A[r, :] loaded once (registers when K <= KREG), then each output C[n, r] of
// the chunk is formed against B (read through the L1/texture path: it is small or shared
// across the warp).  nc = N gives one thread per row; smaller chunks give steps with few
// rows enough threads to fill the GPU while the decoding stays amortised over nc outputs.
// Consecutive threads take consecutive rows, so the C stores of a warp are contiguous.
template <typename R, int KREG>
__global__ void __launch_bounds__(256) k_rows(const Step s, Cx<R>* arena, Meta* meta, int nc) {
  using S = typename Traits<R>::S;
  extern __shared__ long long sm[];
  long long* kA = sm;
  long long* kB = sm + s.K;
  long long* nB = sm + 2 * s.K;
  for (long long k = threadIdx.x; k < s.K; k += blockDim.x) split_runs32((unsigned)k, s.kr, s.nk, kA[k], kB[k]);
  for (long long n = threadIdx.x; n < s.N; n += blockDim.x) {
    long long dummy;
    split_runs32((unsigned)n, s.nr, s.nn, dummy, nB[n]);
  }
  const S scale = step_scale<S>(s, meta, blockIdx.x == 0 && threadIdx.x == 0);
  __syncthreads();
  const Cx<R>* A = arena + s.off_a;
  const Cx<R>* B = arena + s.off_b;
  Cx<R>* C = arena + s.off_c;
  const bool hasB = s.b >= 0;
  const int K = (int)s.K, N = (int)s.N;
  const unsigned R_ = (unsigned)s.R;
  const unsigned chunks = (unsigned)((N + nc - 1) / nc);   // R chunks <= R N <= 2^31
  S vmax = 0;
  for (unsigned w = blockIdx.x * blockDim.x + threadIdx.x; w < R_ * chunks; w += gridDim.x * blockDim.x) {
    const unsigned c = w / R_, r = w - c * R_;
    const int n0 = (int)c * nc, n1 = min(N, n0 + nc);
    long long oa, ob;
    split_runs32(r, s.row, s.nrow, oa, ob);
    if (KREG > 0) {
      Cx<R> a[KREG > 0 ? KREG : 1];
#pragma unroll
      for (int k = 0; k < KREG; ++k)
        if (k < K) a[k] = ld(A + oa + kA[k]);
      for (int n = n0; n < n1; ++n) {
        Acc<R> acc;
        if (hasB) {
          const Cx<R>* Bn = B + ob + nB[n];
#pragma unroll
          for (int k = 0; k < KREG; ++k)
            if (k < K) acc.mac(a[k], ld(Bn + kB[k]));
        } else {
#pragma unroll
          for (int k = 0; k < KREG; ++k)
            if (k < K) acc.add(a[k]);
        }
        const Cx<R> v = acc.get(scale);
        st(C + (long long)n * R_ + r, v);
        vmax = fmax(vmax, mag(v));
      }
    } else {
      for (int n = n0; n < n1; ++n) {
        Acc<R> acc;
        const Cx<R>* Bn = B + ob + (hasB ? nB[n] : 0);
        for (int k = 0; k < K; ++k) {
          Cx<R> av = ld(A + oa + kA[k]);
          if (hasB)
            acc.mac(av, ld(Bn + kB[k]));
          else
            acc.add(av);
        }
        const Cx<R> v = acc.get(scale);
        st(C + (long long)n * R_ + r, v);
        vmax = fmax(vmax, mag(v));
      }
    }
  }
  block_max_to_meta(vmax, meta + s.c);
}

// Thread per output C[n, r] for steps with too few rows to fill the GPU one thread per
// row: each thread forms one output's K-term sum, reading the contracted index's offsets
// from shared memory; consecutive threads write consecutive C entries (C index
// n * R + r is the thread's linear index).
template <typename R>
__global__ void __launch_bounds__(256) k_outs(const Step s, Cx<R>* arena, Meta* meta) {
  using S = typename Traits<R>::S;
  extern __shared__ long long sm[];
  long long* kA = sm;
  long long* kB = sm + s.K;
  for (long long k = threadIdx.x; k < s.K; k += blockDim.x) split_runs32((unsigned)k, s.kr, s.nk, kA[k], kB[k]);
  const S scale = step_scale<S>(s, meta, blockIdx.x == 0 && threadIdx.x == 0);
  __syncthreads();
  const Cx<R>* A = arena + s.off_a;
  const Cx<R>* B = arena + s.off_b;
  Cx<R>* C = arena + s.off_c;
  const bool hasB = s.b >= 0;
  const int K = (int)s.K;
  // R N <= 2^31 (the tensor size limit): 32-bit index arithmetic
  const unsigned R_ = (unsigned)s.R;
  const unsigned total = (unsigned)(s.R * s.N);
  S vmax = 0;
  for (unsigned o = blockIdx.x * blockDim.x + threadIdx.x; o < total; o += gridDim.x * blockDim.x) {
    const unsigned n = o / R_, r = o - n * R_;
    long long oa, ob, nb, dummy;
    split_runs32(r, s.row, s.nrow, oa, ob);
    split_runs32(n, s.nr, s.nn, dummy, nb);
    const Cx<R>* Ar = A + oa;
    const Cx<R>* Bn = B + ob + nb;
    Acc<R> acc;
    if (hasB) {
      for (int k = 0; k < K; ++k) acc.mac(ld(Ar + kA[k]), ld(Bn + kB[k]));
    } else {
      for (int k = 0; k < K; ++k) acc.add(ld(Ar + kA[k]));
    }
    const Cx<R> v = acc.get(scale);
    st(C + o, v);
    vmax = fmax(vmax, mag(v));
  }
  block_max_to_meta(vmax, meta + s.c);
}

// Consecutive small steps of one plan in one CTA: each step's outputs spread over the
// threads, a block barrier between steps, its max-abs formed by a block reduction.
// Operands written by earlier steps of the same launch are read with coherent loads
// (the writes are visible to the CTA after the barrier).
template <typename R>
__global__ void __launch_bounds__(256) k_seg(const TinyStep* __restrict__ steps, int n,
                                             Cx<R>* arena, Meta* meta) {
  using S = typename Traits<R>::S;
  __shared__ long long kA[kTinyK], kB[kTinyK];
  __shared__ S red[32];
  for (int i = 0; i < n; ++i) {
    const TinyStep& s = steps[i];
    const int ea = bin_exp(bits_to_val<S>(meta[s.a].maxbits));
    const bool hasB = s.b >= 0;
    const int eb = hasB ? bin_exp(bits_to_val<S>(meta[s.b].maxbits)) : 0;
    const long long exp_c = meta[s.a].exp + (hasB ? meta[s.b].exp : 0) + ea + eb;
    const S scale = (S)ldexp(1.0, -(ea + eb));
    for (long long k = threadIdx.x; k < s.K; k += blockDim.x) split_runs32((unsigned)k, s.kr, s.nk, kA[k], kB[k]);
    __syncthreads();
    const Cx<R>* A = arena + s.off_a;
    const Cx<R>* B = arena + s.off_b;
    Cx<R>* C = arena + s.off_c;
    const unsigned outs = (unsigned)(s.R * s.N), R_ = (unsigned)s.R;
    const int K = (int)s.K;
    S vmax = 0;
    for (unsigned o = threadIdx.x; o < outs; o += blockDim.x) {
      const unsigned nn = o / R_, r = o - nn * R_;
      long long oa, ob, d, nb = 0;
      split_runs32(r, s.row, s.nrow, oa, ob);
      if (hasB) split_runs32(nn, s.nr, s.nn, d, nb);
      Acc<R> acc;
      if (hasB) {
        for (int k = 0; k < K; ++k) acc.mac(ldc(A + oa + kA[k]), ldc(B + ob + nb + kB[k]));
      } else {
        for (int k = 0; k < K; ++k) acc.add(ldc(A + oa + kA[k]));
      }
      const Cx<R> v = acc.get(scale);
      st(C + o, v);
      vmax = fmax(vmax, mag(v));
    }
    for (int off = 16; off > 0; off >>= 1) vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = vmax;
    __syncthreads();
    if (threadIdx.x == 0) {
      S m = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
      meta[s.c].maxbits = m > S(0) ? max_bits(m) : 0ull;
      meta[s.c].exp = exp_c;
    }
    __syncthreads();
  }
}

// Same contraction without offset tables (K too long for shared memory): every k
// offset is recomputed from the stride runs.
template <typename R>
__global__ void __launch_bounds__(256) k_rows_big(const Step s, Cx<R>* arena, Meta* meta) {
  using S = typename Traits<R>::S;
  const S scale = step_scale<S>(s, meta, blockIdx.x == 0 && threadIdx.x == 0);
  const Cx<R>* A = arena + s.off_a;
  const Cx<R>* B = arena + s.off_b;
  Cx<R>* C = arena + s.off_c;
  const bool hasB = s.b >= 0;
  const unsigned R_ = (unsigned)s.R;
  S vmax = 0;
  for (unsigned r = blockIdx.x * blockDim.x + threadIdx.x; r < R_; r += gridDim.x * blockDim.x) {
    long long oa, ob;
    split_runs32(r, s.row, s.nrow, oa, ob);
    for (long long n = 0; n < s.N; ++n) {
      long long dummy, nb = 0;
      if (hasB) split_runs((unsigned long long)n, s.nr, s.nn, dummy, nb);
      Acc<R> acc;
      for (long long k = 0; k < s.K; ++k) {
        long long ka, kb;
        split_runs((unsigned long long)k, s.kr, s.nk, ka, kb);
        Cx<R> av = ld(A + oa + ka);
        if (hasB)
          acc.mac(av, ld(B + ob + nb + kb));
        else
          acc.add(av);
      }
      const Cx<R> v = acc.get(scale);
      st(C + n * (long long)R_ + r, v);
      vmax = fmax(vmax, mag(v));
    }
  }
  block_max_to_meta(vmax, meta + s.c);
}

// ------------------------------------------------------------------ GEMM-shaped steps
// Per batch index b: C_b[m, n] = sum_k A_b[m, k] B_b[k, n] on 64 x 64 output tiles,
// K in chunks of 16.  Operand tiles are gathered through the stride runs (the index
// permutation) into shared memory, coalesced along whichever of m/k (A) or k/n (B) is
// unit-stride in memory; each of the 256 threads accumulates a 4 x 4 block of complex
// outputs in registers.
// Offsets in A, B and C of index x of a GEMM-view run class (x below the class's extent,
// at most 2^31: 32-bit division).
__device__ __forceinline__ void runs4(long long x, const Run4* r, int n, long long& oa,
                                      long long& ob, long long& oc) {
  unsigned y = (unsigned)x;
  oa = ob = oc = 0;
  for (int i = 0; i < n; ++i) {
    const unsigned sz = (unsigned)r[i].size;
    const unsigned qd = y / sz, d = y - qd * sz;
    y = qd;
    oa += (long long)d * r[i].sa;
    ob += (long long)d * r[i].sb;
    oc += (long long)d * r[i].sc;
  }
}

template <typename R>
__global__ void __launch_bounds__(256) k_gemm(const Step s, Cx<R>* arena, Meta* meta) {
  using S = typename Traits<R>::S;
  constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4, LDA = BM + 1, LDB = BN + 1;
  __shared__ Cx<R> As[BK * LDA];
  __shared__ Cx<R> Bs[BK * LDB];
  __shared__ long long am[BM], cm[BM], bn[BN], cn[BN], ak[BK], bk[BK];
  __shared__ long long base[3];
  const int tid = threadIdx.x;
  const long long tiles_m = (s.M + BM - 1) / BM, tiles_n = (s.N + BN - 1) / BN;
  long long t = blockIdx.x;
  const long long tm = t % tiles_m;
  t /= tiles_m;
  const long long tn = t % tiles_n;
  const long long bb = t / tiles_n;
  if (tid == 0) runs4(bb, s.gb, s.ngb, base[0], base[1], base[2]);
  if (tid < BM) {
    long long m = tm * BM + tid;
    if (m < s.M) {
      long long d;
      runs4(m, s.gm, s.ngm, am[tid], d, cm[tid]);
    } else {
      am[tid] = -1;
      cm[tid] = -1;
    }
  } else if (tid < BM + BN) {
    int j = tid - BM;
    long long n = tn * BN + j;
    if (n < s.N) {
      long long d;
      runs4(n, s.gn, s.ngn, d, bn[j], cn[j]);
    } else {
      bn[j] = -1;
      cn[j] = -1;
    }
  }
  const S scale = step_scale<S>(s, meta, blockIdx.x == 0 && tid == 0);
  __syncthreads();
  const Cx<R>* A = arena + s.off_a + base[0];
  const Cx<R>* B = arena + s.off_b + base[1];
  Acc<R> acc[TM][TN];
  const int tx = tid & 15, ty = tid >> 4;
  for (long long k0 = 0; k0 < s.K; k0 += BK) {
    if (tid < BK) {
      long long k = k0 + tid;
      if (k < s.K) {
        long long ka, kb;
        split_runs((unsigned long long)k, s.kr, s.nk, ka, kb);
        ak[tid] = ka;
        bk[tid] = kb;
      } else {
        ak[tid] = -1;
        bk[tid] = -1;
      }
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < (BM * BK) / 256; ++p) {
      int idx = tid + p * 256, i, j;
      if (s.a_kinner) {
        i = idx / BK;
        j = idx % BK;
      } else {
        i = idx % BM;
        j = idx / BM;
      }
      Cx<R> v = czero<R>();
      if (am[i] >= 0 && ak[j] >= 0) v = ld(A + am[i] + ak[j]);
      As[j * LDA + i] = v;
    }
#pragma unroll
    for (int p = 0; p < (BN * BK) / 256; ++p) {
      int idx = tid + p * 256, j, kk;
      if (s.b_kinner) {
        j = idx / BK;
        kk = idx % BK;
      } else {
        j = idx % BN;
        kk = idx / BN;
      }
      Cx<R> v = czero<R>();
      if (bn[j] >= 0 && bk[kk] >= 0) v = ld(B + bk[kk] + bn[j]);
      Bs[kk * LDB + j] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      Cx<R> a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk * LDA + tx * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk * LDB + ty * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j].mac(a[i], b[j]);
    }
    __syncthreads();
  }
  Cx<R>* C = arena + s.off_c + base[2];
  S vmax = 0;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int mi = tx * TM + i;
    if (cm[mi] < 0) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int nj = ty * TN + j;
      if (cn[nj] < 0) continue;
      const Cx<R> v = acc[i][j].get(scale);
      st(C + cm[mi] + cn[nj], v);
      vmax = fmax(vmax, mag(v));
    }
  }
  block_max_to_meta(vmax, meta + s.c);
}

// Few outputs, long K: block (chunk, output) sums its slice of K in double; the last
// block to finish (ticket counter) adds the partials of every output in chunk order,
// so the result does not depend on scheduling.
template <typename R>
__global__ void __launch_bounds__(256) k_splitk(const Step s, Cx<R>* arena, Meta* meta,
                                                Cx<double>* partial, unsigned* counter) {
  using S = typename Traits<R>::S;
  const int chunks = s.chunks;
  const long long o = blockIdx.y;
  const long long r = o % s.R, n = o / s.R;
  long long oa, ob, dummy, nb = 0;
  split_runs((unsigned long long)r, s.row, s.nrow, oa, ob);
  if (s.b >= 0) split_runs((unsigned long long)n, s.nr, s.nn, dummy, nb);
  const long long per = (s.K + chunks - 1) / chunks;
  const long long k0 = (long long)blockIdx.x * per, k1 = min((long long)s.K, k0 + per);
  const Cx<R>* A = arena + s.off_a;
  const Cx<R>* B = arena + s.off_b + ob + nb;
  double are = 0, aim = 0;
  if constexpr (std::is_same<R, ff>::value) {
    // float-float products and sums on the FP32 units (FP64 runs at a small fraction of
    // their rate on this GPU); each thread's partial goes to double for the reduction
    Acc<ff> acc;
    for (long long k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
      long long ka, kb;
      split_runs32((unsigned)k, s.kr, s.nk, ka, kb);  // K <= 2^31: 32-bit digits
      const Cx<ff> av = ld(A + oa + ka);
      if (s.b >= 0)
        acc.mac(av, ld(B + kb));
      else
        acc.add(av);
    }
    const Cx<ff> t = acc.get(1.0f);
    are = to_double(t.re);
    aim = to_double(t.im);
  } else {
    for (long long k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
      long long ka, kb;
      split_runs32((unsigned)k, s.kr, s.nk, ka, kb);  // K <= 2^31: 32-bit digits
      const Cx<R> av = ld(A + oa + ka);
      const double xr = to_double(av.re), xi = to_double(av.im);
      if (s.b >= 0) {
        const Cx<R> bv = ld(B + kb);
        const double yr = to_double(bv.re), yi = to_double(bv.im);
        are += xr * yr - xi * yi;
        aim += xr * yi + xi * yr;
      } else {
        are += xr;
        aim += xi;
      }
    }
  }
  __shared__ double rr[32], ri[32];
  for (int off = 16; off > 0; off >>= 1) {
    are += __shfl_xor_sync(0xffffffffu, are, off);
    aim += __shfl_xor_sync(0xffffffffu, aim, off);
  }
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    rr[w] = are;
    ri[w] = aim;
  }
  __syncthreads();
  __shared__ bool last;
  if (threadIdx.x == 0) {
    double tre = 0, tim = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      tre += rr[i];
      tim += ri[i];
    }
    partial[o * chunks + blockIdx.x] = {tre, tim};
    __threadfence();
    unsigned tk = atomicAdd(counter, 1u);
    last = (tk == gridDim.x * gridDim.y - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const S scale = step_scale<S>(s, meta, threadIdx.x == 0);
  Cx<R>* C = arena + s.off_c;
  const long long outs = s.R * s.N;
  S vmax = 0;
  for (long long oo = threadIdx.x; oo < outs; oo += blockDim.x) {
    double tre = 0, tim = 0;
    const volatile double* pp = (const volatile double*)partial;
    for (int c = 0; c < chunks; ++c) {
      tre += pp[2 * (oo * chunks + c)];
      tim += pp[2 * (oo * chunks + c) + 1];
    }
    // C is laid out [n, r] with r innermost: output o = r + n * R, the same linear index
    const Cx<R> v{from_double<R>(tre * (double)scale), from_double<R>(tim * (double)scale)};
    st(C + oo, v);
    vmax = fmax(vmax, mag(v));
  }
  block_max_to_meta(vmax, meta + s.c);
  if (threadIdx.x == 0) *counter = 0u;
}

// ------------------------------------------------------------------ results
template <typename R>
__global__ void k_slice_result(const Cx<R>* arena, long long off, const Meta* meta, int tensor,
                               SliceResult* out, long long slice) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const Cx<R> v = arena[off];
  out[slice].re = to_double(v.re);
  out[slice].im = to_double(v.im);
  out[slice].exp = meta[tensor].exp;
}

// Reverse pass: adds this slice's adjoint of every clause tensor (true value: stored x
// 2^exp) into its complex128 accumulator (true value: acc x 2^acc_exp), one block per
// tensor.  Entries whose sliced coordinates differ from this slice's values get nothing
// from it.  Both terms are brought to the larger of their binary exponents before the
// sum, so neither can overflow; the block's order of work is fixed (deterministic).
template <typename R>
__global__ void __launch_bounds__(256) k_grad_accum(const GradLeaf* __restrict__ leaves,
                                                    const Cx<R>* arena, const Meta* meta,
                                                    Cx<double>* acc, long long* acc_exp, int q,
                                                    long long slice) {
  const GradLeaf L = leaves[blockIdx.x];
  int sdig[2] = {0, 0};
  for (int j = 0; j < 2; ++j)
    if (L.slice_ord[j] >= 0) {
      long long s = slice;
      for (int i = 0; i < L.slice_ord[j]; ++i) s /= q;
      sdig[j] = (int)(s % q);
    }
  const int n = L.rank == 2 ? q * q : (L.rank == 1 ? q : 1);
  Cx<double>* A = acc + (long long)blockIdx.x * q * q;
  const long long ev = L.meta >= 0 ? meta[L.meta].exp : 0;
  auto incoming = [&](int e) -> Cx<double> {
    const int d[2] = {L.rank == 2 ? e / q : e, L.rank == 2 ? e % q : 0};
    long long off = 0;
    for (int j = 0; j < L.rank && j < 2; ++j) {
      if (L.slice_ord[j] >= 0) {
        if (d[j] != sdig[j]) return {0.0, 0.0};
      } else {
        off += (long long)d[j] * L.stride[j];
      }
    }
    if (L.meta < 0) return {1.0, 0.0};
    const Cx<R> v = arena[L.offset + off];
    return {to_double(v.re), to_double(v.im)};
  };
  __shared__ double red_i[256], red_a[256];
  double mi = 0, ma = 0;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const Cx<double> v = incoming(e);
    mi = fmax(mi, fmax(fabs(v.re), fabs(v.im)));
    ma = fmax(ma, fmax(fabs(A[e].re), fabs(A[e].im)));
  }
  red_i[threadIdx.x] = mi;
  red_a[threadIdx.x] = ma;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      red_i[threadIdx.x] = fmax(red_i[threadIdx.x], red_i[threadIdx.x + o]);
      red_a[threadIdx.x] = fmax(red_a[threadIdx.x], red_a[threadIdx.x + o]);
    }
    __syncthreads();
  }
  mi = red_i[0];
  ma = red_a[0];
  if (!(mi > 0)) return;  // nothing from this slice (uniform across the block)
  const long long eo = acc_exp[blockIdx.x];
  long long enew = ev + bin_exp(mi);
  if (ma > 0) enew = max(enew, eo + (long long)bin_exp(ma));
  auto pow2 = [](long long d) { return ldexp(1.0, (int)max(-1100LL, min(1000LL, d))); };
  const double so = ma > 0 ? pow2(eo - enew) : 0.0, si = pow2(ev - enew);
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const Cx<double> v = incoming(e);
    A[e] = {A[e].re * so + v.re * si, A[e].im * so + v.im * si};
  }
  if (threadIdx.x == 0) acc_exp[blockIdx.x] = enew;
}

// Sum over slices in double with a common exponent; fixed assignment and tree order.
static __global__ void k_sum_slices(SliceResult* res, long long n) {
  __shared__ long long emax_s[256];
  __shared__ double sre[256], sim[256];
  long long emax = LLONG_MIN;
  bool bad = false;   // a non-finite slice value makes the total NaN, never a silent 0
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    if (!isfinite(res[i].re) || !isfinite(res[i].im)) bad = true;
    double m = fmax(fabs(res[i].re), fabs(res[i].im));
    if (m > 0) {
      int e;
      frexp(m, &e);
      emax = max(emax, res[i].exp + e);
    }
  }
  emax_s[threadIdx.x] = emax;
  if (__syncthreads_or(bad)) {
    if (threadIdx.x == 0) {
      res[n].re = res[n].im = __longlong_as_double(0x7FF8000000000000LL);
      res[n].exp = 0;
    }
    return;
  }
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) emax_s[threadIdx.x] = max(emax_s[threadIdx.x], emax_s[threadIdx.x + o]);
    __syncthreads();
  }
  emax = emax_s[0];
  double are = 0, aim = 0, cre = 0, cim = 0;  // Kahan-compensated
  if (emax != LLONG_MIN) {
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
      long long d = res[i].exp - emax;
      double f = d < -2000 ? 0.0 : ldexp(1.0, (int)max(d, -2000LL));
      double yr = res[i].re * f - cre, tr = are + yr;
      cre = (tr - are) - yr;
      are = tr;
      double yi = res[i].im * f - cim, ti = aim + yi;
      cim = (ti - aim) - yi;
      aim = ti;
    }
  }
  sre[threadIdx.x] = are;
  sim[threadIdx.x] = aim;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sre[threadIdx.x] += sre[threadIdx.x + o];
      sim[threadIdx.x] += sim[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    res[n].re = sre[0];
    res[n].im = sim[0];
    res[n].exp = emax == LLONG_MIN ? 0 : emax;
  }
}

}  // namespace pk
