// Device kernels of the contraction (Sec. III): building the initial tensors of G_T,
// one pairwise contraction step, and the per-slice / all-slice results.
//
// A step computes C[b, m, n] = sum_k A[b, m, k] B[b, k, n] where b (batch) are indices
// kept in both operands, m kept only in A, n kept only in B, and k summed.  The
// operands stay in the layout their producer wrote; every class of indices is a short
// list of merged stride runs, so the index permutation is folded into the loads and
// the store (no separate transpose pass).  C is written as [n-part, row-part] with the
// row part (b and m, in A's order) innermost and contiguous.
//
// Scaling: a stored tensor x stands for x * 2^exp.  A step multiplies its products by
// 2^-(eA+eB), eX being the binary exponent of max|X| (so operands enter at magnitude
// below 1), and records exp(C) = exp(A) + exp(B) + eA + eB.  Powers of two are exact.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <climits>

#include "pk_internal.h"

namespace pk {

template <typename R>
struct Cx {
  R re, im;
};
template <typename R>
struct VecOf;
template <>
struct VecOf<double> {
  using T = double2;
};
template <>
struct VecOf<float> {
  using T = float2;
};

template <typename R>
__device__ __forceinline__ Cx<R> ld(const Cx<R>* p) {
  typename VecOf<R>::T v = __ldg(reinterpret_cast<const typename VecOf<R>::T*>(p));
  return {v.x, v.y};
}
template <typename R>
__device__ __forceinline__ void st(Cx<R>* p, Cx<R> x) {
  typename VecOf<R>::T v;
  v.x = x.re;
  v.y = x.im;
  *reinterpret_cast<typename VecOf<R>::T*>(p) = v;
}
template <typename R>
__device__ __forceinline__ void cmac(Cx<R>& acc, const Cx<R>& a, const Cx<R>& b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}

__device__ __forceinline__ unsigned long long max_bits(double m) {
  return (unsigned long long)__double_as_longlong(m);
}
__device__ __forceinline__ unsigned long long max_bits(float m) {
  return (unsigned long long)__float_as_uint(m);
}
template <typename R>
__device__ __forceinline__ R bits_to_val(unsigned long long b);
template <>
__device__ __forceinline__ double bits_to_val<double>(unsigned long long b) {
  return __longlong_as_double((long long)b);
}
template <>
__device__ __forceinline__ float bits_to_val<float>(unsigned long long b) {
  return __uint_as_float((unsigned)b);
}

// binary exponent e with m * 2^-e in [0.5, 1); 0 for m == 0
template <typename R>
__device__ __forceinline__ int bin_exp(R m) {
  if (!(m > R(0))) return 0;
  int e;
  frexp(m, &e);
  return e;
}

template <typename R>
__device__ __forceinline__ void block_max_to_meta(R v, Meta* meta) {
  __shared__ R red[32];
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    int nw = (blockDim.x + 31) >> 5;
    v = lane < nw ? red[lane] : R(0);
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0 && v > R(0)) atomicMax(&meta->maxbits, max_bits(v));
  }
}

// ------------------------------------------------------------------ initial tensors
// One grid row (blockIdx.y) per initial tensor; entry = sum_{s<q} prod_j f_j(s, x_j).
template <typename R>
__global__ void __launch_bounds__(256) k_build(const Recipe* __restrict__ rec,
                                               const Slot* __restrict__ slots, Cx<R>* arena,
                                               Meta* meta, int q, long long slice, int n_sliced) {
  const Recipe r = rec[blockIdx.y];
  R vmax = 0;
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
    double sre = 0, sim = 0;
    if (r.kind == 1) {
      sre = 1;
    } else {
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
            if (s == x) {
              double nre = pre * sl.dre - pim * sl.dim;
              double nim = pre * sl.dim + pim * sl.dre;
              pre = nre;
              pim = nim;
            }
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
    Cx<R> v{(R)sre, (R)sim};
    st(arena + r.offset + e, v);
    vmax = fmax(vmax, fmax(fabs(v.re), fabs(v.im)));
  }
  block_max_to_meta(vmax, meta + r.meta);
}

// ------------------------------------------------------------------ contraction step
__device__ __forceinline__ void split_runs(unsigned long long x, const Run* runs, int n,
                                           long long& oa, long long& ob) {
  oa = 0;
  ob = 0;
  for (int i = 0; i < n; ++i) {
    unsigned long long sz = (unsigned long long)runs[i].size;
    unsigned long long d = x % sz;
    x /= sz;
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
template <typename R>
__device__ __forceinline__ R step_scale(const Step& s, Meta* meta, bool write_exp) {
  int ea = bin_exp(bits_to_val<R>(meta[s.a].maxbits));
  int eb = 0;
  long long xb = 0;
  if (s.b >= 0) {
    eb = bin_exp(bits_to_val<R>(meta[s.b].maxbits));
    xb = meta[s.b].exp;
  }
  if (write_exp) meta[s.c].exp = meta[s.a].exp + xb + ea + eb;
  return (R)ldexp(1.0, -(ea + eb));
}

// Thread per output row r (batch x free-of-A): the K values A[r, :] are loaded once
// (registers when K <= KREG), then each of the N outputs C[n, r] is formed against B
// (read through the L1/texture path: it is small or shared across the warp).
template <typename R, int KREG>
__global__ void __launch_bounds__(256) k_rows(const Step s, Cx<R>* arena, Meta* meta) {
  extern __shared__ long long sm[];
  long long* kA = sm;
  long long* kB = sm + s.K;
  long long* nB = sm + 2 * s.K;
  for (long long k = threadIdx.x; k < s.K; k += blockDim.x) split_runs(k, s.kr, s.nk, kA[k], kB[k]);
  for (long long n = threadIdx.x; n < s.N; n += blockDim.x) {
    long long dummy;
    split_runs(n, s.nr, s.nn, dummy, nB[n]);
  }
  const R scale = step_scale<R>(s, meta, blockIdx.x == 0 && threadIdx.x == 0);
  __syncthreads();
  const Cx<R>* A = arena + s.off_a;
  const Cx<R>* B = arena + s.off_b;
  Cx<R>* C = arena + s.off_c;
  const bool hasB = s.b >= 0;
  const int K = (int)s.K, N = (int)s.N;
  const unsigned R_ = (unsigned)s.R;
  R vmax = 0;
  for (unsigned r = blockIdx.x * blockDim.x + threadIdx.x; r < R_; r += gridDim.x * blockDim.x) {
    long long oa, ob;
    split_runs32(r, s.row, s.nrow, oa, ob);
    if (KREG > 0) {
      Cx<R> a[KREG > 0 ? KREG : 1];
#pragma unroll
      for (int k = 0; k < KREG; ++k)
        if (k < K) a[k] = ld(A + oa + kA[k]);
      for (int n = 0; n < N; ++n) {
        Cx<R> acc{0, 0};
        if (hasB) {
          const Cx<R>* Bn = B + ob + nB[n];
#pragma unroll
          for (int k = 0; k < KREG; ++k)
            if (k < K) cmac(acc, a[k], ld(Bn + kB[k]));
        } else {
#pragma unroll
          for (int k = 0; k < KREG; ++k)
            if (k < K) {
              acc.re += a[k].re;
              acc.im += a[k].im;
            }
        }
        acc.re *= scale;
        acc.im *= scale;
        st(C + (long long)n * R_ + r, acc);
        vmax = fmax(vmax, fmax(fabs(acc.re), fabs(acc.im)));
      }
    } else {
      for (int n = 0; n < N; ++n) {
        Cx<R> acc{0, 0};
        const Cx<R>* Bn = B + ob + (hasB ? nB[n] : 0);
        for (int k = 0; k < K; ++k) {
          Cx<R> av = ld(A + oa + kA[k]);
          if (hasB)
            cmac(acc, av, ld(Bn + kB[k]));
          else {
            acc.re += av.re;
            acc.im += av.im;
          }
        }
        acc.re *= scale;
        acc.im *= scale;
        st(C + (long long)n * R_ + r, acc);
        vmax = fmax(vmax, fmax(fabs(acc.re), fabs(acc.im)));
      }
    }
  }
  block_max_to_meta(vmax, meta + s.c);
}

// Same contraction without offset tables (K too long for shared memory): every k
// offset is recomputed from the stride runs.
template <typename R>
__global__ void __launch_bounds__(256) k_rows_big(const Step s, Cx<R>* arena, Meta* meta) {
  const R scale = step_scale<R>(s, meta, blockIdx.x == 0 && threadIdx.x == 0);
  const Cx<R>* A = arena + s.off_a;
  const Cx<R>* B = arena + s.off_b;
  Cx<R>* C = arena + s.off_c;
  const bool hasB = s.b >= 0;
  const unsigned R_ = (unsigned)s.R;
  R vmax = 0;
  for (unsigned r = blockIdx.x * blockDim.x + threadIdx.x; r < R_; r += gridDim.x * blockDim.x) {
    long long oa, ob;
    split_runs32(r, s.row, s.nrow, oa, ob);
    for (long long n = 0; n < s.N; ++n) {
      long long dummy, nb = 0;
      if (hasB) split_runs((unsigned long long)n, s.nr, s.nn, dummy, nb);
      Cx<R> acc{0, 0};
      for (long long k = 0; k < s.K; ++k) {
        long long ka, kb;
        split_runs((unsigned long long)k, s.kr, s.nk, ka, kb);
        Cx<R> av = ld(A + oa + ka);
        if (hasB) {
          cmac(acc, av, ld(B + ob + nb + kb));
        } else {
          acc.re += av.re;
          acc.im += av.im;
        }
      }
      acc.re *= scale;
      acc.im *= scale;
      st(C + n * (long long)R_ + r, acc);
      vmax = fmax(vmax, fmax(fabs(acc.re), fabs(acc.im)));
    }
  }
  block_max_to_meta(vmax, meta + s.c);
}

// ------------------------------------------------------------------ GEMM-shaped steps
// Per batch index b: C_b[m, n] = sum_k A_b[m, k] B_b[k, n] on 64 x 64 output tiles,
// K in chunks of 16.  Operand tiles are gathered through the stride runs (the index
// permutation) into shared memory, coalesced along whichever of m/k (A) or k/n (B) is
// unit-stride in memory; each of the 256 threads accumulates a 4 x 4 block of complex
// outputs in registers (4 real FMAs per complex multiply-add).
__device__ __forceinline__ void runs4(long long x, const Run4* r, int n, long long& oa,
                                      long long& ob, long long& oc) {
  oa = ob = oc = 0;
  for (int i = 0; i < n; ++i) {
    long long sz = r[i].size;
    long long d = x % sz;
    x /= sz;
    oa += d * r[i].sa;
    ob += d * r[i].sb;
    oc += d * r[i].sc;
  }
}

template <typename R>
__global__ void __launch_bounds__(256) k_gemm(const Step s, Cx<R>* arena, Meta* meta) {
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
  const R scale = step_scale<R>(s, meta, blockIdx.x == 0 && tid == 0);
  __syncthreads();
  const Cx<R>* A = arena + s.off_a + base[0];
  const Cx<R>* B = arena + s.off_b + base[1];
  Cx<R> acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = {0, 0};
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
      Cx<R> v{0, 0};
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
      Cx<R> v{0, 0};
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
        for (int j = 0; j < TN; ++j) cmac(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
  Cx<R>* C = arena + s.off_c + base[2];
  R vmax = 0;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int mi = tx * TM + i;
    if (cm[mi] < 0) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int nj = ty * TN + j;
      if (cn[nj] < 0) continue;
      Cx<R> v{acc[i][j].re * scale, acc[i][j].im * scale};
      st(C + cm[mi] + cn[nj], v);
      vmax = fmax(vmax, fmax(fabs(v.re), fabs(v.im)));
    }
  }
  block_max_to_meta(vmax, meta + s.c);
}

// Few outputs, long K: block (chunk, output) sums its slice of K; the last block to
// finish (ticket counter) adds the partials of every output in chunk order, so the
// result does not depend on scheduling.
template <typename R>
__global__ void __launch_bounds__(256) k_splitk(const Step s, Cx<R>* arena, Meta* meta,
                                                Cx<double>* partial, unsigned* counter) {
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
  Cx<double> acc{0, 0};
  for (long long k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    long long ka, kb;
    split_runs((unsigned long long)k, s.kr, s.nk, ka, kb);
    Cx<R> av = ld(A + oa + ka);
    if (s.b >= 0) {
      Cx<R> bv = ld(B + kb);
      acc.re += (double)av.re * bv.re - (double)av.im * bv.im;
      acc.im += (double)av.re * bv.im + (double)av.im * bv.re;
    } else {
      acc.re += av.re;
      acc.im += av.im;
    }
  }
  __shared__ double rr[32], ri[32];
  for (int off = 16; off > 0; off >>= 1) {
    acc.re += __shfl_xor_sync(0xffffffffu, acc.re, off);
    acc.im += __shfl_xor_sync(0xffffffffu, acc.im, off);
  }
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    rr[w] = acc.re;
    ri[w] = acc.im;
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
    unsigned t = atomicAdd(counter, 1u);
    last = (t == gridDim.x * gridDim.y - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const R scale = step_scale<R>(s, meta, threadIdx.x == 0);
  Cx<R>* C = arena + s.off_c;
  const long long outs = s.R * s.N;
  R vmax = 0;
  for (long long oo = threadIdx.x; oo < outs; oo += blockDim.x) {
    double tre = 0, tim = 0;
    const volatile double* pp = (const volatile double*)partial;
    for (int c = 0; c < chunks; ++c) {
      tre += pp[2 * (oo * chunks + c)];
      tim += pp[2 * (oo * chunks + c) + 1];
    }
    // C is laid out [n, r] with r innermost: output o = r + n * R, the same linear index
    Cx<R> v{(R)(tre * (double)scale), (R)(tim * (double)scale)};
    st(C + oo, v);
    vmax = fmax(vmax, fmax(fabs(v.re), fabs(v.im)));
  }
  block_max_to_meta(vmax, meta + s.c);
  if (threadIdx.x == 0) *counter = 0u;
}

// ------------------------------------------------------------------ results
template <typename R>
__global__ void k_slice_result(const Cx<R>* arena, long long off, const Meta* meta, int tensor,
                               SliceResult* out, long long slice) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Cx<R> v = arena[off];
  out[slice].re = (double)v.re;
  out[slice].im = (double)v.im;
  out[slice].exp = meta[tensor].exp;
}

// Sum over slices in double with a common exponent; fixed assignment and tree order.
__global__ void k_sum_slices(SliceResult* res, long long n) {
  __shared__ long long emax_s[256];
  __shared__ double sre[256], sim[256];
  long long emax = LLONG_MIN;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    double m = fmax(fabs(res[i].re), fabs(res[i].im));
    if (m > 0) {
      int e;
      frexp(m, &e);
      emax = max(emax, res[i].exp + e);
    }
  }
  emax_s[threadIdx.x] = emax;
  __syncthreads();
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

// ------------------------------------------------------------------ launchers
namespace {
template <typename R>
size_t rows_smem(const Step& s) {
  return sizeof(long long) * (size_t)(2 * s.K + s.N);
}

template <typename R>
cudaError_t launch_rows(const Step& s, Cx<R>* arena, Meta* meta, cudaStream_t st) {
  size_t sm = rows_smem<R>(s);
  long long blocks = (s.R + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  if (sm > 200 * 1024) {
    k_rows_big<R><<<(unsigned)blocks, 256, 0, st>>>(s, arena, meta);
    return cudaGetLastError();
  }
  int kmax = sizeof(R) == 8 ? 16 : 32;
  const int K = (int)s.K;
  void (*fn)(const Step, Cx<R>*, Meta*);
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
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  fn<<<(unsigned)blocks, 256, sm, st>>>(s, arena, meta);
  return cudaGetLastError();
}
}  // namespace

// Enqueues every kernel of every slice.  With `prof` set, an event pair brackets each
// launch and per-class milliseconds / counts / algorithmic work are accumulated.
constexpr int kNumClasses = 5;  // build, rows, split-K, results, GEMM
struct Prof {
  double ms[kNumClasses] = {}, n[kNumClasses] = {}, cmacs[kNumClasses] = {},
         bytes[kNumClasses] = {};
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  std::vector<int> cls;
};

template <typename R>
cudaError_t launch_plan_impl(const Plan& p, void* ws, cudaStream_t stream, Prof* prof) {
  char* base = (char*)ws;
  Cx<R>* arena = (Cx<R>*)(base + p.off_arena);
  Meta* meta = (Meta*)(base + p.off_meta);
  const Recipe* rec = (const Recipe*)(base + p.off_recipe);
  const Slot* slots = (const Slot*)(base + p.off_slots);
  SliceResult* res = (SliceResult*)(base + p.off_result);
  Cx<double>* partial = (Cx<double>*)(base + p.off_scratch);
  unsigned* counters = (unsigned*)(base + p.off_counter);
  if (p.n_init > 65535) return cudaErrorInvalidValue;
  int64_t maxel = 1, initel = 0;
  for (const auto& r : p.recipes) {
    maxel = std::max<int64_t>(maxel, r.elems);
    initel += r.elems;
  }
  unsigned bx = (unsigned)std::min<int64_t>((maxel + 255) / 256, 64);
  const double eb = (double)sizeof(Cx<R>);
  auto mark = [&](int c, double cm, double by, bool begin) -> cudaError_t {
    if (!prof) return cudaSuccess;
    if (begin) {
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      prof->ev.push_back({a, b});
      prof->cls.push_back(c);
      prof->n[c] += 1;
      prof->cmacs[c] += cm;
      prof->bytes[c] += by;
      return cudaEventRecord(a, stream);
    }
    return cudaEventRecord(prof->ev.back().second, stream);
  };
  cudaError_t e;
  for (long long sl = 0; sl < p.n_slices; ++sl) {
    e = cudaMemsetAsync(base + p.off_meta, 0, p.off_result - p.off_meta, stream);
    if (e != cudaSuccess) return e;
    if (p.n_init > 0) {
      mark(0, 0, eb * (double)initel, true);
      k_build<R><<<dim3(bx, (unsigned)p.n_init), 256, 0, stream>>>(
          rec, slots, arena, meta, p.q, sl, (int)p.sliced.size());
      mark(0, 0, 0, false);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    for (size_t i = 0; i < p.steps.size(); ++i) {
      const Step& s = p.steps[i];
      const double cm = (double)s.R * (double)s.K * (double)s.N;
      const double by = eb * (double)(p.tensors[s.a].elems + (s.b >= 0 ? p.tensors[s.b].elems : 0) +
                                      p.tensors[s.c].elems);
      const long long gemm_tiles = ((s.M + 63) / 64) * ((s.N + 63) / 64) * s.Bsz;
      if (s.kernel == KGEMM && gemm_tiles < (1LL << 31)) {
        mark(4, cm, by, true);
        k_gemm<R><<<(unsigned)gemm_tiles, 256, 0, stream>>>(s, arena, meta);
        mark(4, 0, 0, false);
        e = cudaGetLastError();
      } else if (s.kernel == KSPLITK) {
        mark(2, cm, by, true);
        k_splitk<R><<<dim3((unsigned)s.chunks, (unsigned)(s.R * s.N)), 256, 0, stream>>>(
            s, arena, meta, partial, counters + i);
        mark(2, 0, 0, false);
        e = cudaGetLastError();
      } else {
        mark(1, cm, by, true);
        e = launch_rows<R>(s, arena, meta, stream);
        mark(1, 0, 0, false);
      }
      if (e != cudaSuccess) return e;
    }
    mark(3, 0, 0, true);
    k_slice_result<R><<<1, 32, 0, stream>>>(arena, p.tensors[p.final_tensor].offset, meta,
                                            p.final_tensor, res, sl);
    mark(3, 0, 0, false);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  mark(3, 0, 0, true);
  k_sum_slices<<<1, 256, 0, stream>>>(res, p.n_slices);
  mark(3, 0, 0, false);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_plan(const Plan& p, void* ws, cudaStream_t stream) {
  return launch_plan_impl<R>(p, ws, stream, nullptr);
}

template <typename R>
cudaError_t profile_plan(const Plan& p, void* ws, cudaStream_t stream, double* out) {
  Prof prof;
  cudaError_t e = launch_plan_impl<R>(p, ws, stream, &prof);
  cudaError_t e2 = cudaStreamSynchronize(stream);
  if (e == cudaSuccess) e = e2;
  for (size_t i = 0; i < prof.ev.size(); ++i) {
    float ms = 0;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, prof.ev[i].first, prof.ev[i].second);
    prof.ms[prof.cls[i]] += ms;
    cudaEventDestroy(prof.ev[i].first);
    cudaEventDestroy(prof.ev[i].second);
  }
  for (int c = 0; c < kNumClasses; ++c) {
    out[c] = prof.ms[c];
    out[kNumClasses + c] = prof.n[c];
    out[2 * kNumClasses + c] = prof.cmacs[c];
    out[3 * kNumClasses + c] = prof.bytes[c];
  }
  return e;
}
template cudaError_t profile_plan<double>(const Plan&, void*, cudaStream_t, double*);
template cudaError_t profile_plan<float>(const Plan&, void*, cudaStream_t, double*);

template cudaError_t launch_plan<double>(const Plan&, void*, cudaStream_t);
template cudaError_t launch_plan<float>(const Plan&, void*, cudaStream_t);

}  // namespace pk
