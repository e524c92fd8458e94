// Complex GEMM step on the 5th-generation tensor cores (tcgen05: BF16 operands from
// shared memory, FP32 accumulators in tensor memory) for the split-FP32 precision.
//
// The float-float operands carry about 48 significant bits, far more than a BF16 product,
// so each operand is cut into S signed 8-bit digits (the splitting idea of Ozaki et al.,
// "Error-free transformations of matrix multiplication", Numer. Algorithms 2012):
// with e(m) the binary exponent of row m's largest entry (over all of K),
//     x 2^-e(m) = sum_i d_i 2^(-7-8i) + r,   d_i integers, |d_i| <= 128,  |r| <= 2^(-8S-7),
// and likewise for the columns of B.  A digit is exact in BF16 (8 significant bits), a
// digit product (|d_a d_b| <= 2^14) is exact, and a sum of such products stays exact in
// FP32 while it stays below 2^24: the S digit pairs (i, j) of one level L = i + j are
// accumulated together, and every level is flushed to float-float registers before
// (L + 1) K' 2^14 can reach 2^24.  Levels L >= S are dropped (their weight is at most
// 2^(-8S) of the leading term); the result is
//     C(m, n) = 2^(e(m) + e(n)) sum_{L < S} acc_L(m, n) 2^(-14-8L).
//
// Complex arithmetic as one real product: with the rows of C interleaved (re, im),
//     [re row m] = [Re A(m,:), -Im A(m,:)] . [Re B; Im B],
//     [im row m] = [Im A(m,:),  Re A(m,:)] . [Re B; Im B],
// so a CTA tile of 64 complex rows x 64 complex columns is one M=128, N=64 MMA per
// BF16 K-step of 16 (K' = 2 K).
//
// Data movement: the operands are gathered through the step's stride runs (arbitrary
// index permutations, which a TMA tensor map cannot express), converted to digits by all
// threads and written to shared memory in the canonical K-major layout without swizzle
// (8-row x 16-byte core matrices); one thread issues the MMAs and commits them to an
// mbarrier; every wait is bounded (on expiry the tile is poisoned with NaN and counted
// in pk_tc_timeouts, so a failure shows up as a wrong result, not a hang).
#pragma once

#include <cuda_bf16.h>

namespace pk {
namespace tc {

constexpr int kMc = 64;          // complex rows per tile
constexpr int kNc = 64;          // complex columns per tile
constexpr int kKc = 32;          // complex k per chunk
constexpr int kM = 2 * kMc;      // MMA M (re and im rows interleaved)
constexpr int kN = kNc;          // MMA N
constexpr int kKr = 2 * kKc;     // MMA K per chunk (real: re half, im half)
constexpr int kThreads = 256;
constexpr int kABytes = kM * kKr * 2;   // one digit slice of the A tile (BF16)
constexpr int kBBytes = kN * kKr * 2;   // one digit slice of the B tile

template <int S>
struct Cfg {
  static constexpr int kSmem = S * (kABytes + kBBytes) + 1024;  // + alignment slack
  static constexpr int kCols = S * kN <= 32 ? 32 : S * kN <= 64 ? 64 : S * kN <= 128 ? 128
                               : S * kN <= 256 ? 256 : 512;
  // chunks per flush: S pairs per level x (chunks x kKr) terms x 2^14 < 2^24
  static constexpr int kFlush = (1 << 10) / (S * kKr) > 0 ? ((1 << 10) - 1) / (S * kKr) : 1;
};

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17,
// M >> 4 at bit 24.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kN >> 3) << 17) |
                            ((uint32_t)(kM >> 4) << 24);

// Shared-memory matrix descriptor, K-major without swizzle: start address >> 4 (bits
// 0-13), leading byte offset >> 4 (bits 16-29: between the two 8-element K core columns
// of a K=16 step), stride byte offset >> 4 (bits 32-45: between 8-row groups), version 1
// (bits 46-47), layout type 0 (bits 61-63).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   mbar)
               : "memory");
}

}  // namespace tc

__device__ int pk_tc_timeouts;  // bounded waits that expired (poisoned tiles)

namespace tc {

// Bounded wait for an mbarrier phase; false if it did not complete, or if another CTA
// has already given up (then every later wait returns at once).
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  for (int i = 0; i < (1 << 20); ++i) {
    if ((i & 1023) == 1023 && *(volatile int*)&pk_tc_timeouts != 0) return false;
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row, k) in a K-major, unswizzled tile with `kcores` 8-element
// K core columns: 8-row groups of kcores x 128 bytes, core matrices of 8 rows x 16 bytes.
__device__ __forceinline__ uint32_t tile_off(int row, int k, int kcores) {
  return (uint32_t)((row >> 3) * kcores * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// S digits of the float-float value (h + l) 2^-e (|value| <= 1): d_i = nearest integer of
// the running remainder times 2^(7+8i); the remainder is carried exactly as a float pair.
template <int S>
__device__ __forceinline__ void digits(float h, float l, int e, __nv_bfloat16* d) {
  float yh = ldexpf(h, 7 - e), yl = ldexpf(l, 7 - e);
#pragma unroll
  for (int i = 0; i < S; ++i) {
    const float di = rintf(yh);
    d[i] = __float2bfloat16_rn(di);
    float s, err;
    two_sum(__fsub_rn(yh, di), yl, s, err);
    yh = s * 256.0f;
    yl = err * 256.0f;
  }
}

}  // namespace tc

// One CTA per (batch, 64-row, 64-column) tile of the step's GEMM view.
template <int S>
__global__ void __launch_bounds__(tc::kThreads, 1) k_gemm_tc(const Step s, Cx<ff>* arena, Meta* meta) {
  using namespace tc;
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ long long am[kMc], cm[kMc], bn[kNc], cn[kNc], ak[kKc], bk[kKc];
  __shared__ long long base[3];
  __shared__ int ea[kMc], eb[kNc];
  __shared__ float red[kThreads];
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int bad;

  unsigned char* sm = (unsigned char*)(((uintptr_t)dsm + 1023) & ~(uintptr_t)1023);
  unsigned char* As = sm;                     // S slices of kM x kKr
  unsigned char* Bs = sm + S * kABytes;       // S slices of kN x kKr
  const int tid = threadIdx.x, warp = tid >> 5;
  const long long tiles_m = (s.M + kMc - 1) / kMc, tiles_n = (s.N + kNc - 1) / kNc;
  long long t = blockIdx.x;
  const long long tm = t % tiles_m;
  t /= tiles_m;
  const long long tn = t % tiles_n;
  const long long bb = t / tiles_n;

  if (tid == 0) {
    runs4(bb, s.gb, s.ngb, base[0], base[1], base[2]);
    bad = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < kMc) {
    const long long m = tm * kMc + tid;
    long long d;
    if (m < s.M) {
      runs4(m, s.gm, s.ngm, am[tid], d, cm[tid]);
    } else {
      am[tid] = -1;
      cm[tid] = -1;
    }
  } else if (tid < kMc + kNc) {
    const int j = tid - kMc;
    const long long n = tn * kNc + j;
    long long d;
    if (n < s.N) {
      runs4(n, s.gn, s.ngn, d, bn[j], cn[j]);
    } else {
      bn[j] = -1;
      cn[j] = -1;
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(Cfg<S>::kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  const float scale = step_scale<float>(s, meta, blockIdx.x == 0 && tid == 0);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;
  const Cx<ff>* A = arena + s.off_a + base[0];
  const Cx<ff>* B = arena + s.off_b + base[1];
  const long long nchunks = (s.K + kKc - 1) / kKc;

  // ---- exponents: largest entry of every tile row of A and column of B over all K
  {
    float mx = 0;
    const int r = tid >> 2, sub = tid & 3;  // 4 threads per row (tid < 256: rows 0..63)
    for (long long c = 0; c < nchunks; ++c) {
      if (tid < kKc) {
        const long long k = c * kKc + tid;
        long long ka = -1, kb = -1;
        if (k < s.K) split_runs((unsigned long long)k, s.kr, s.nk, ka, kb);
        ak[tid] = ka;
        bk[tid] = kb;
      }
      __syncthreads();
      for (int k = sub; k < kKc; k += 4) {
        if (ak[k] >= 0 && am[r] >= 0) mx = fmaxf(mx, mag(ld(A + am[r] + ak[k])));
      }
      __syncthreads();
    }
    red[tid] = mx;
    __syncthreads();
    if (sub == 0) {
      const float v = fmaxf(fmaxf(red[tid], red[tid + 1]), fmaxf(red[tid + 2], red[tid + 3]));
      ea[r] = bin_exp(v);
    }
    __syncthreads();
    mx = 0;
    for (long long c = 0; c < nchunks; ++c) {
      if (tid < kKc) {
        const long long k = c * kKc + tid;
        long long ka = -1, kb = -1;
        if (k < s.K) split_runs((unsigned long long)k, s.kr, s.nk, ka, kb);
        ak[tid] = ka;
        bk[tid] = kb;
      }
      __syncthreads();
      for (int k = sub; k < kKc; k += 4) {
        if (bk[k] >= 0 && bn[r] >= 0) mx = fmaxf(mx, mag(ld(B + bk[k] + bn[r])));
      }
      __syncthreads();
    }
    red[tid] = mx;
    __syncthreads();
    if (sub == 0) {
      const float v = fmaxf(fmaxf(red[tid], red[tid + 1]), fmaxf(red[tid + 2], red[tid + 3]));
      eb[r] = bin_exp(v);
    }
    __syncthreads();
  }

  // ---- main loop: digits to shared memory, S(S+1)/2 digit-pair MMAs per K step
  const int lane_row = tid & 127;             // TMEM lane = row of the interleaved C
  const int col_half = tid >> 7;              // columns 32 * col_half .. + 31
  float acc_h[32], acc_l[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) acc_h[j] = acc_l[j] = 0.f;
  uint32_t phase = 0;
  bool first = true;
  const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
  for (long long c = 0; c < nchunks; ++c) {
    if (tid < kKc) {
      const long long k = c * kKc + tid;
      long long ka = -1, kb = -1;
      if (k < s.K) split_runs((unsigned long long)k, s.kr, s.nk, ka, kb);
      ak[tid] = ka;
      bk[tid] = kb;
    }
    __syncthreads();
    // A: 64 rows x 32 k complex; (m, k) -> rows 2m (re), 2m+1 (im), columns k and 32+k
    for (int idx = tid; idx < kMc * kKc; idx += kThreads) {
      int m, k;
      if (s.a_kinner) {
        m = idx / kKc;
        k = idx % kKc;
      } else {
        m = idx % kMc;
        k = idx / kMc;
      }
      Cx<ff> v{{0.f, 0.f}, {0.f, 0.f}};
      if (am[m] >= 0 && ak[k] >= 0) v = ld(A + am[m] + ak[k]);
      __nv_bfloat16 dr[S], di[S];
      digits<S>(v.re.hi, v.re.lo, ea[m], dr);
      digits<S>(v.im.hi, v.im.lo, ea[m], di);
#pragma unroll
      for (int i = 0; i < S; ++i) {
        unsigned char* sl = As + i * kABytes;
        *(__nv_bfloat16*)(sl + tile_off(2 * m, k, kKr / 8)) = dr[i];
        *(__nv_bfloat16*)(sl + tile_off(2 * m, kKc + k, kKr / 8)) = __hneg(di[i]);
        *(__nv_bfloat16*)(sl + tile_off(2 * m + 1, k, kKr / 8)) = di[i];
        *(__nv_bfloat16*)(sl + tile_off(2 * m + 1, kKc + k, kKr / 8)) = dr[i];
      }
    }
    // B: 32 k x 64 columns complex; (k, n) -> row n, columns k (re) and 32+k (im)
    for (int idx = tid; idx < kNc * kKc; idx += kThreads) {
      int n, k;
      if (s.b_kinner) {
        n = idx / kKc;
        k = idx % kKc;
      } else {
        n = idx % kNc;
        k = idx / kNc;
      }
      Cx<ff> v{{0.f, 0.f}, {0.f, 0.f}};
      if (bn[n] >= 0 && bk[k] >= 0) v = ld(B + bk[k] + bn[n]);
      __nv_bfloat16 dr[S], di[S];
      digits<S>(v.re.hi, v.re.lo, eb[n], dr);
      digits<S>(v.im.hi, v.im.lo, eb[n], di);
#pragma unroll
      for (int i = 0; i < S; ++i) {
        unsigned char* sl = Bs + i * kBBytes;
        *(__nv_bfloat16*)(sl + tile_off(n, k, kKr / 8)) = dr[i];
        *(__nv_bfloat16*)(sl + tile_off(n, kKc + k, kKr / 8)) = di[i];
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      fence_after();
#pragma unroll 1
      for (int L = 0; L < S; ++L)
        for (int i = 0; i <= L; ++i)
          for (int kk = 0; kk < kKr / 16; ++kk) {
            const uint64_t da = smem_desc(a0 + i * kABytes + kk * 256, 128, (kKr / 8) * 128);
            const uint64_t db = smem_desc(b0 + (L - i) * kBBytes + kk * 256, 128, (kKr / 8) * 128);
            mma_bf16(tmem + L * kN, da, db, (first && i == 0 && kk == 0) ? 0u : 1u);
          }
      commit(smem_u32(&mbar));
    }
    const bool ok = mbar_wait(smem_u32(&mbar), phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        bad = 1;
        atomicAdd(&pk_tc_timeouts, 1);
      }
      break;
    }
    fence_after();
    first = false;
    if ((c + 1) % Cfg<S>::kFlush == 0 || c + 1 == nchunks) {
      // levels -> float-float: sum_L acc_L 2^(-14-8L), each level an exact integer
#pragma unroll 1
      for (int L = 0; L < S; ++L) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + L * kN + col_half * 32, v);
        const float w = ldexpf(1.0f, -14 - 8 * L);
#pragma unroll
        for (int j = 0; j < 32; ++j) ff_acc(acc_h[j], acc_l[j], v[j] * w, 0.f);
      }
      fence_before();
      first = true;
    }
    __syncthreads();
  }

  // ---- epilogue: scale by 2^(e(m) + e(n)) and the step's normalisation, pair re / im
  const int m = lane_row >> 1, part = lane_row & 1;
  Cx<ff>* C = arena + s.off_c + base[2];
  float vmax = 0;
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const int n = col_half * 32 + j;
    const int e = ea[m] + eb[n];
    ff mine = ff_norm(acc_h[j], acc_l[j]);
    mine.hi = ldexpf(mine.hi, e) * scale;
    mine.lo = ldexpf(mine.lo, e) * scale;
    if (bad) mine.hi = mine.lo = __int_as_float(0x7fc00000);
    ff other;
    other.hi = __shfl_xor_sync(0xffffffffu, mine.hi, 1);
    other.lo = __shfl_xor_sync(0xffffffffu, mine.lo, 1);
    if ((j & 1) == part && cm[m] >= 0 && cn[n] >= 0) {
      const Cx<ff> out = part == 0 ? Cx<ff>{mine, other} : Cx<ff>{other, mine};
      st(C + cm[m] + cn[n], out);
      vmax = fmaxf(vmax, mag(out));
    }
  }
  block_max_to_meta(vmax, meta + s.c);
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(Cfg<S>::kCols)
                 : "memory");
}

}  // namespace pk
