// Complex GEMM step on the 5th-generation tensor cores (tcgen05: BF16 operands from
// shared memory, FP32 accumulators in tensor memory) for the split-FP32 precision.
//
// The float-float operands carry about 48 significant bits, far more than a BF16 product,
// so each operand is cut into S signed 8-bit digits (the splitting idea of Ozaki et al.,
// "Error-free transformations of matrix multiplication", Numer. Algorithms 2012):
// with e(m) the binary exponent of row m's largest entry (over one flush group of K),
//     x 2^-e(m) = sum_i d_i 2^(-7-8i) + r,   d_i integers, |d_i| <= 128,  |r| <= 2^(-8S-7),
// and likewise for the columns of B.  A digit is exact in BF16 (8 significant bits), a
// digit product (|d_a d_b| <= 2^14) is exact, and a sum of such products stays exact in
// FP32 while it stays below 2^24: the S digit pairs (i, j) of one level L = i + j are
// accumulated together, and every level is flushed to float-float registers before
// (L + 1) K' 2^14 can reach 2^24 (there levels 0 and 1 are combined exactly, levels 2 and
// up in FP32, whose rounding stays below the truncation).  Levels L >= S are dropped
// (their weight is at most 2^(-8S) of the leading term); the result is
//     C(m, n) = sum_groups 2^(e_g(m) + e_g(n)) sum_{L < S} acc_{g,L}(m, n) 2^(-14-8L),
// each group's exponents applied (exactly: powers of two) when its levels are flushed.
//
// Complex arithmetic as one real product: with the columns of C interleaved (re, im),
//     [re column n] = [Re A(m,:), Im A(m,:)] . [ Re B(:,n); -Im B(:,n)],
//     [im column n] = [Re A(m,:), Im A(m,:)] . [ Im B(:,n);  Re B(:,n)],
// so every complex row of A is one real row of K' = 2 K entries (stored once) and the
// doubling falls on the columns of B.  A CTA tile of 128 complex rows x 24 complex
// columns is one M=128, N=48 MMA per BF16 K-step of 16.
//
// Data movement, three kernels per step:
//  * k_digits<S>: one CTA per (32-row part of a 128-row block of A, or 24-column block of
//    B; flush group of kFlush chunks of K) gathers the block into shared memory, finds its
//    rows' exponents over the group, then converts it into S digit slices per chunk (16
//    complex k) laid out exactly as the MMA reads them from shared memory (the canonical
//    K-major layout without swizzle: 8-row x 16-byte core matrices) and stores each chunk
//    contiguously in the workspace.  The operands are gathered through the step's stride
//    runs (arbitrary index permutations, which a TMA tensor map cannot express); each
//    element is read from memory once.
//  * k_gemm_tc: warp 0 streams the chunks of its (batch, row block, column block) into a
//    2-stage shared-memory ring with bulk asynchronous copies (cp.async.bulk, completion by
//    mbarrier transaction count); warp 1 issues the S (S+1)/2 digit-pair products of a K
//    step as S MMAs (A digit i against B digits 0 .. S-1-i stacked along N: one issuing
//    thread cannot keep the tensor pipe busy with N = 48 MMAs) and releases each stage
//    with tcgen05.commit; eight epilogue warps flush the S level
//    accumulators from TMEM into float-float registers every kFlush chunks and finally
//    store C.  Every wait is bounded: on expiry the CTA sets the evaluation's error word
//    (the status of its total result record, which the host turns into PK_ETIMEOUT),
//    waits -- again bounded -- for its own bulk copies and MMAs still in flight, writes
//    its tile as NaN, frees its tensor memory and exits; the other CTAs of the same
//    evaluation see the error word and give up at once, so a failure is reported, not hung.
#pragma once

#include <cuda_bf16.h>

namespace pk {
namespace tc {

constexpr int kMc = kTcMc;       // complex rows per tile
constexpr int kNc = kTcNc;       // complex columns per tile
constexpr int kKc = kTcKc;       // complex k per chunk
constexpr int kM = kMc;          // MMA M (one real row per complex row of A)
constexpr int kN = 2 * kNc;      // MMA N (re and im columns interleaved)
constexpr int kKr = 2 * kKc;     // MMA K per chunk (real: re half, im half)
constexpr int kKcores = kKr / 8; // 16-byte K core columns per row
constexpr int kABytes = kM * kKr * 2;   // one digit slice of an A chunk (BF16): 8 KB
constexpr int kBBytes = kN * kKr * 2;   // one digit slice of a B chunk: 3 KB
constexpr int kStages = 2;     // stage ring, two CTAs per SM
constexpr int kStagesDB = 4;   // stage ring of the double-buffered variant (one CTA per SM)
constexpr int kEpiWarps = 8;
constexpr int kThreads = 32 * (2 + kEpiWarps);   // producer, MMA issuer, epilogue
constexpr int kConvThreads = 256;
// the GEMM's tile order takes row blocks in groups whose A digits fill about this much of L2
constexpr long long kRowGroupBytes = 48ll << 20;

template <int S>
struct Cfg {
  static constexpr int kAChunk = S * kABytes;     // one chunk of A digits (all slices)
  static constexpr int kBChunk = S * kBBytes;
  static constexpr int kStage = kAChunk + kBChunk;
  static constexpr int kSmem = kStages * kStage;   // two CTAs per SM (16-byte alignment suffices)
  static constexpr int kSmemDB = kStagesDB * kStage;   // the double-buffered variant: one CTA per SM
  static_assert(kSmemDB <= 220 * 1024, "stage ring of the double-buffered variant");
  // the digit kernel's staging tile: 32 rows x (flush group + 1) complex entries
  static constexpr int kConvSmem = 32 * (tc_flush(S) * kKc + 1) * 16;
  // one MMA spans the stacked B digits: M = 128 allows N in multiples of 16 up to 256
  static_assert(kN % 16 == 0 && S * kN <= 256, "stacked B digits exceed one MMA");
  static_assert(kAChunk == tc_a_chunk(S) && kBChunk == tc_b_chunk(S),
                "chunk sizes must match the host's scratch layout");
  static constexpr int kCols = S * kN <= 32 ? 32 : S * kN <= 64 ? 64 : S * kN <= 128 ? 128
                               : S * kN <= 256 ? 256 : 512;
  // chunks per flush: S pairs per level x (chunks x kKr) terms x 2^14 < 2^24
  static constexpr int kFlush = tc_flush(S);
  static_assert(kFlush >= 1, "flush group");
};

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17,
// M >> 4 at bit 24.
constexpr uint32_t idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(kM >> 4) << 24);
}

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

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   mbar)
               : "memory");
}

// Bounded wait for an mbarrier phase; false if it did not complete within 2^20 polls.
// `err` is the evaluation's error word: when it is given and another role or CTA of the
// same evaluation has already given up (err != 0), the wait returns false at once.  The
// drain waits of the give-up path pass nullptr: they run out their own bound only.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase,
                                          const unsigned long long* err) {
  for (int i = 0; i < (1 << 20); ++i) {
    if (err && (i & 1023) == 1023 && *(const volatile unsigned long long*)err != 0ull) return false;
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

// 16 and 8 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
// Two loads of 8 columns each, one wait.
__device__ __forceinline__ void tmem_ld8x2(uint32_t ta, uint32_t tb, float* a, float* b) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%16];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%17];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(ta), "r"(tb));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    a[i] = __uint_as_float(r[i]);
    b[i] = __uint_as_float(r[8 + i]);
  }
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row, k) in a K-major, unswizzled tile with `kcores` 8-element
// K core columns: 8-row groups of kcores x 128 bytes, core matrices of 8 rows x 16 bytes.
__device__ __forceinline__ uint32_t tile_off(int row, int k, int kcores) {
  return (uint32_t)((row >> 3) * kcores * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// 2^x as a product of two exact floats (each exponent within [-126, 127]).
__device__ __forceinline__ void pow2_pair(int x, float& f1, float& f2) {
  const int x1 = x / 2, x2 = x - x1;
  f1 = __int_as_float((max(-126, min(127, x1)) + 127) << 23);
  f2 = __int_as_float((max(-126, min(127, x2)) + 127) << 23);
}


}  // namespace tc


namespace tc {

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes)
               : "memory");
}
// Contiguous global -> shared copy by the bulk-copy (TMA) engine; completes on `mbar` as
// transaction bytes.  Addresses 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}

// 16-byte asynchronous global -> shared copy (both addresses 16-byte aligned), cached in
// L2 only; completed by cp_async_wait.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// The S digit slices of one real component of 8 consecutive k of one tile row: x[u] =
// (hi, lo) of k = 8 o + u, scaled by f1 f2 = 2^(7 - e) (e the row's exponent over the
// group, |hi| < 2^e; two exact powers of two, so that any exponent the stored values can
// have is covered), giving float-float values y = (yh + yl) with |y| < 2^7.  Digit i is
// the nearest integer d_i of the running remainder times 2^(8i): rounding by adding and
// subtracting 1.5 * 2^23 (exact round-to-nearest-even on the FP32 adder for |yh| < 2^22,
// no conversion instruction); the remainder r = yh - d_i is exact and a multiple of
// ulp(yh), while |yl| <= ulp(yh) / 2, so |r| >= |yl| unless r = 0 and the fast two-sum
// (Dekker) that renormalises (r + yl) is exact.  An integer d_i with |d_i| <= 256 keeps
// only the top 16 bits of its FP32 pattern, which are its BF16 pattern.  Digit i of the 8
// values, packed into 16 bytes (one core-matrix row), goes to out + i * slice and, when
// out2 is given, also to out2 + i * slice, negated if `neg2`.
template <int S>
__device__ __forceinline__ void digit_rows8(const float* xh, const float* xl, float f1, float f2,
                                            unsigned char* out, unsigned char* out2, bool neg2,
                                            int slice) {
  constexpr float kRound = 12582912.0f;   // 1.5 * 2^23
  float yh[8], yl[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    yh[u] = (xh[u] * f1) * f2;
    yl[u] = (xl[u] * f1) * f2;
  }
  const uint32_t flip = neg2 ? 0x80008000u : 0u;   // negate the BF16 digits (exact)
#pragma unroll
  for (int i = 0; i < S; ++i) {
    uint32_t w[4];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float di = __fsub_rn(__fadd_rn(yh[u], kRound), kRound);
      if (u & 1)   // BF16 of value u - 1 in the low half, of u in the high half
        w[u >> 1] = __byte_perm(w[u >> 1], __float_as_uint(di), 0x7632);
      else
        w[u >> 1] = __float_as_uint(di);
      if (i + 1 < S) {
        const float r = __fsub_rn(yh[u], di);
        const float sum = __fadd_rn(r, yl[u]);
        const float err = __fsub_rn(yl[u], __fsub_rn(sum, r));
        yh[u] = sum * 256.0f;
        yl[u] = err * 256.0f;
      }
    }
    *(uint4*)(out + i * slice) = make_uint4(w[0], w[1], w[2], w[3]);
    if (out2)
      *(uint4*)(out2 + i * slice) = make_uint4(w[0] ^ flip, w[1] ^ flip, w[2] ^ flip, w[3] ^ flip);
  }
}

}  // namespace tc

// Digits of one block of the A operand (IS_A: 32 of a tile's 128 rows) or the B operand
// (24 columns) of a GEMM step over one flush group of K (kFlush chunks of 16 complex k).
// The block's entries are gathered once into shared memory (16-byte asynchronous copies;
// consecutive threads follow the operand's unit stride: along K, or along the rows), then
// each row's exponent over the group is taken from there, and the S digit slices of the
// group's chunks are written in whole 16-byte core-matrix rows, consecutive threads taking
// consecutive tile rows (full 32-byte sectors).  Row stride in shared memory kG + 1
// entries: rows 16 bytes apart modulo 128 keep the conversion's reads free of conflicts.
template <int S, bool IS_A>
__device__ __forceinline__ void digits_block(const Step& s, const Cx<ff>* arena, unsigned char* scratch,
                                             long long blk, long long* ro, long long* kt,
                                             long long& base, int* ex, float4* tile) {
  using namespace tc;
  constexpr int kParts = IS_A ? kMc / 32 : 1;     // CTAs per tile block
  constexpr int kRows = IS_A ? 32 : kNc;          // rows this CTA converts
  constexpr int kG = Cfg<S>::kFlush * kKc;        // complex k of one flush group
  constexpr int kLd = kG + 1;                     // shared-memory row stride (entries)
  constexpr int kPer = kConvThreads / 32;         // threads per row in the exponent pass
  static_assert(kRows <= 32 && kG <= kConvThreads && kG % 8 == 0, "block geometry");
  const TcScratch L = tc_scratch(s.Bsz, s.M, s.N, s.K, S);
  const long long tiles = IS_A ? L.tiles_m : L.tiles_n;
  const int part = (int)(blk % kParts);
  blk /= kParts;
  const long long g = blk % L.groups, t = blk / L.groups;
  const long long tile_i = t % tiles, bb = t / tiles;
  const int r0 = part * kRows;                    // first tile row of this CTA
  const int tid = threadIdx.x;
  const bool kin = IS_A ? s.a_kinner != 0 : s.b_kinner != 0;
  const long long k0 = g * kG;
  const long long kpad = L.chunks * kKc;               // K rounded up to whole chunks
  const int kgn = (int)min((long long)kG, kpad - k0);  // this group's k (whole chunks)
  if (tid == 0) {
    long long a, b, c;
    runs4(bb, s.gb, s.ngb, a, b, c);
    base = IS_A ? a : b;
  }
  if (tid < kRows) {
    const long long r = tile_i * (IS_A ? kMc : kNc) + r0 + tid;
    long long a, b, c, cc = -1;
    if (r < (IS_A ? s.M : s.N)) {
      if (IS_A)
        runs4(r, s.gm, s.ngm, a, b, c);
      else
        runs4(r, s.gn, s.ngn, a, b, c);
      ro[tid] = IS_A ? a : b;
      cc = c;
    } else {
      ro[tid] = -1;
    }
    // the row's (column's) C offset for the GEMM's epilogue: once per row, by the first
    // flush group (columns: by batch index 0, their offsets do not depend on it)
    if (g == 0 && (IS_A || bb == 0)) {
      if (IS_A && cc >= 0) {
        long long a2, b2, cb;
        runs4(bb, s.gb, s.ngb, a2, b2, cb);
        cc += cb;
      }
      ((long long*)(scratch + (IS_A ? L.cr_off : L.cc_off)))
          [IS_A ? (bb * tiles + tile_i) * kMc + r0 + tid : tile_i * kNc + tid] = cc;
    }
  }
  if (tid < kG) {
    const long long k = k0 + tid;
    long long ka = -1, kb = -1;
    if (k < s.K) split_runs((unsigned long long)k, s.kr, s.nk, ka, kb);
    kt[tid] = IS_A ? ka : kb;
  }
  __syncthreads();
  const Cx<ff>* src = arena + (IS_A ? s.off_a : s.off_b) + base;

  // ---- gather the block: entry (r, k) -> tile[r * kLd + k]; missing entries are 0
  for (int idx = tid; idx < kRows * kgn; idx += kConvThreads) {
    const int r = kin ? idx / kgn : idx % kRows;
    const int k = kin ? idx % kgn : idx / kRows;
    float4* d = tile + r * kLd + k;
    if (ro[r] >= 0 && kt[k] >= 0)
      cp_async16(smem_u32(d), src + ro[r] + kt[k]);
    else
      *d = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  cp_async_wait();
  __syncthreads();

  // ---- exponents over the group: kPer consecutive threads per row
  {
    const int r = tid / kPer, j = tid % kPer;
    float mx = 0.f;
    if (r < kRows)
      for (int k = j; k < kgn; k += kPer) {
        const float4 v = tile[r * kLd + k];
        mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.z)));
      }
#pragma unroll
    for (int o = kPer / 2; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (r < kRows && j == 0) {
      ex[r] = bin_exp(mx);
      ((int*)(scratch + (IS_A ? L.ea_off : L.eb_off)))[((bb * tiles + tile_i) * L.groups + g) *
                                                           (IS_A ? kMc : kNc) + r0 + r] = ex[r];
    }
  }
  __syncthreads();

  // ---- digits: items (row, 8 consecutive k), consecutive threads on consecutive rows
  constexpr int kChunkBytes = IS_A ? Cfg<S>::kAChunk : Cfg<S>::kBChunk;
  constexpr int kSlice = IS_A ? kABytes : kBBytes;
  unsigned char* dst0 = scratch + (IS_A ? L.a_off : L.b_off) +
                        (bb * tiles + tile_i) * L.chunks * (long long)kChunkBytes;
  const int octs = kgn / 8;
  for (int idx = tid; idx < kRows * octs; idx += kConvThreads) {
    const int r = idx % kRows, o = idx / kRows;
    float sc1, sc2;   // 2^(7 - e): the row's largest entry below 2^7
    pow2_pair(7 - ex[r], sc1, sc2);
    const long long k = k0 + 8 * o;
    const int kl = (int)(k % kKc);   // 0 or 8
    unsigned char* ch = dst0 + (k / kKc) * (long long)kChunkBytes;
    const float4* row = tile + r * kLd + 8 * o;
#pragma unroll
    for (int part = 0; part < 2; ++part) {   // the real, then the imaginary components
      float xh[8], xl[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float4 v = row[u];
        xh[u] = part ? v.z : v.x;
        xl[u] = part ? v.w : v.y;
      }
      if (IS_A)   // row [Re | Im]
        digit_rows8<S>(xh, xl, sc1, sc2, ch + tile_off(r0 + r, part * kKc + kl, kKcores), nullptr,
                       false, kSlice);
      else if (part == 0)   // Re: row 2r first half, row 2r + 1 second half
        digit_rows8<S>(xh, xl, sc1, sc2, ch + tile_off(2 * r, kl, kKcores),
                       ch + tile_off(2 * r + 1, kKc + kl, kKcores), false, kSlice);
      else                  // Im: row 2r + 1 first half, -Im: row 2r second half
        digit_rows8<S>(xh, xl, sc1, sc2, ch + tile_off(2 * r + 1, kl, kKcores),
                       ch + tile_off(2 * r, kKc + kl, kKcores), true, kSlice);
    }
  }
}

// Digits of both operands of a GEMM step in one launch: blocks [0, nA) convert A (four
// per batch index, 128-row block and flush group), the rest convert B.
template <int S>
__global__ void __launch_bounds__(tc::kConvThreads, 4) k_digits(const Step s, const Cx<ff>* arena,
                                                             unsigned char* scratch, long long nA) {
  __shared__ long long ro[32], kt[tc::kConvThreads];
  __shared__ long long base;
  __shared__ int ex[32];
  extern __shared__ float4 tile[];
  const long long blk = blockIdx.x;
  if (blk < nA)
    digits_block<S, true>(s, arena, scratch, blk, ro, kt, base, ex, tile);
  else
    digits_block<S, false>(s, arena, scratch, blk - nA, ro, kt, base, ex, tile);
}

// C tiles (128 complex rows x 24 complex columns of one batch index) from the digit
// chunks, persistently (grouped tile order: tiles in flight together share the A row
// blocks of a group and a run of B column blocks in L2).  Q = true: the producer of each CTA takes its next tile from the step's
// tile counter (`ticket`, zero at launch) and passes it to the MMA issuer and the epilogue
// through a small queue in shared memory, so the tiles in flight on the GPU stay a window
// of consecutive tiles however unevenly the CTAs progress (best for short tiles).
// Q = false: CTA b takes tiles b, b + gridDim.x, ..., each role computing them itself (no
// hand-over between the roles; measured faster for tiles with many flush groups).  Warp 0 streams the chunks of its tiles into the stage ring, warp 1 issues the MMAs,
// warps 2..9 flush the level accumulators and store C.  The ring's and the accumulators' barrier phases run on across
// tiles: the producer loads the next tile's chunks while the current one is multiplied and
// flushed, and the epilogue stores a tile from its registers after releasing the
// accumulators, while the next tile's MMAs run; barriers and tensor memory are set up once.
// DB = false: two CTAs per SM, a 2-stage ring and one set of level accumulators (the other
// CTA's MMAs fill in while one CTA flushes).
// DB = true: one CTA per SM, a 4-stage ring and two accumulator sets in TMEM (columns 0
// and 256), used by alternate flush groups, so the flush of group g overlaps the MMAs of
// group g + 1.
template <int S, bool DB, bool Q>
__global__ void __launch_bounds__(tc::kThreads, DB ? 1 : 2) k_gemm_tc(const Step s, Cx<ff>* arena,
                                                                      Meta* meta,
                                                                      const unsigned char* scratch,
                                                                      unsigned* ticket,
                                                                      unsigned long long* err) {
  using namespace tc;
  constexpr int kSt = DB ? kStagesDB : kStages;     // stages of the ring
  constexpr int kTq = 4;                            // tile queue: tiles handed out ahead
  constexpr int kSets = DB ? 2 : 1;                 // accumulator sets
  constexpr uint32_t kCols = DB ? 512u : (uint32_t)Cfg<S>::kCols;
  constexpr int kFlush = Cfg<S>::kFlush;
  static_assert(!DB || S * kN <= 256, "two accumulator sets must fit 512 TMEM columns");
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ long long cn_s[kEpiWarps][kNc / 2];   // per epilogue warp: its columns' C offsets
  __shared__ int eb_s[kEpiWarps][kNc / 2];         // ... and their group exponents
  __shared__ __align__(8) unsigned long long full[kSt], empty[kSt], acc_full[kSets],
      acc_empty[kSets], drain, tq_full[kTq], tq_empty[kTq];
  __shared__ int tq[kTq];   // tile indices handed out (-1: no tiles left)
  __shared__ uint32_t tmem_slot;
  __shared__ int bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const TcScratch L = tc_scratch(s.Bsz, s.M, s.N, s.K, S);
  const long long ntiles = L.tiles_m * L.tiles_n * s.Bsz;

  if (tid == 0) {
    bad = 0;
    for (int i = 0; i < kSt; ++i) {
      mbar_init(smem_u32(&full[i]), 1);
      mbar_init(smem_u32(&empty[i]), 1);
    }
    for (int i = 0; i < kSets; ++i) {
      mbar_init(smem_u32(&acc_full[i]), 1);
      mbar_init(smem_u32(&acc_empty[i]), kEpiWarps);
    }
    mbar_init(smem_u32(&drain), 1);
    for (int i = 0; i < kTq; ++i) {
      mbar_init(smem_u32(&tq_full[i]), 1);
      mbar_init(smem_u32(&tq_empty[i]), 1 + kEpiWarps);   // the MMA issuer and 8 epilogue warps
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  const float scale = step_scale<float>(s, meta, blockIdx.x == 0 && tid == 0);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;
  const long long nchunks = L.chunks;
  const int ngroups = (int)((nchunks + kFlush - 1) / kFlush);
  const uint32_t sm0 = smem_u32(dsm);
  // (batch, row block, column block) of a tile.  Within a batch index the row blocks go
  // in groups of rg; inside a group the tiles run down the group's row blocks of one
  // column block, then on to the next column block.  With rg = 1 (column blocks fastest)
  // the tiles in flight together (one per CTA) cover gridDim.x / tiles_n row blocks and
  // every column block, so B's digits are read from memory once per such wave.  A group of
  // rg row blocks (as many as hold about kRowGroupBytes of A digits) whose A digits stay in
  // L2 while its column blocks are swept reads B once per group instead, fewer times when
  // rg exceeds the rows of a wave (wide N and long K).  Steps of at most two flush groups
  // keep column blocks fastest (measured faster).
  long long rg = max(1ll, min(L.tiles_m, kRowGroupBytes / (L.chunks * (long long)Cfg<S>::kAChunk)));
  if (Q || rg * L.tiles_n <= (long long)gridDim.x) rg = 1;
  auto tile_coords = [&](long long t, long long& bb, long long& tm, long long& tn) {
    const long long per_b = L.tiles_m * L.tiles_n;
    bb = t / per_b;
    const long long u = t - bb * per_b;
    const long long r0 = (u / (rg * L.tiles_n)) * rg;
    const long long gm = min(rg, L.tiles_m - r0);
    const long long v = u - r0 * L.tiles_n;
    tn = v / gm;
    tm = r0 + v % gm;
  };

  constexpr int kCw = kN / 2;  // columns per epilogue thread (two warps per lane quarter)
  int issued = 0;   // producer: chunks of this CTA whose bulk copies were started
  int mmas = 0;     // MMA issuer: chunks of this CTA whose MMAs were issued
  float vmax = 0;

  if (warp == 0) {
    if (lane == 0) {  // producer
      long long gc = 0;   // chunks of this CTA so far (all its tiles)
      for (int i = 0;; ++i) {
        long long t;
        if constexpr (Q) {   // hand out the next tile (or the end) through queue slot i mod kTq
          const int slot = i % kTq;
          if (i >= kTq &&
              !mbar_wait(smem_u32(&tq_empty[slot]), (uint32_t)(((i / kTq) - 1) & 1), err)) {
            bad = 1;
            atomicOr(err, 1ull);
            goto producer_done;
          }
          t = (long long)atomicAdd(ticket, 1u);
          tq[slot] = t < ntiles ? (int)t : -1;
          mbar_arrive(smem_u32(&tq_full[slot]));
        } else {
          t = (long long)blockIdx.x + (long long)i * gridDim.x;
        }
        if (t >= ntiles) break;
        long long bb, tm, tn;
        tile_coords(t, bb, tm, tn);
        const unsigned char* asrc =
            scratch + L.a_off + (bb * L.tiles_m + tm) * nchunks * (long long)Cfg<S>::kAChunk;
        const unsigned char* bsrc =
            scratch + L.b_off + (bb * L.tiles_n + tn) * nchunks * (long long)Cfg<S>::kBChunk;
        for (long long c = 0; c < nchunks; ++c, ++gc) {
          const int st = (int)(gc % kSt);
          if (gc >= kSt &&
              !mbar_wait(smem_u32(&empty[st]), (uint32_t)(((gc / kSt) - 1) & 1), err)) {
            bad = 1;
            atomicOr(err, 1ull);
            goto producer_done;
          }
          const uint32_t dst = sm0 + st * Cfg<S>::kStage;
          mbar_expect_tx(smem_u32(&full[st]), Cfg<S>::kStage);
          bulk_g2s(dst, asrc + c * Cfg<S>::kAChunk, Cfg<S>::kAChunk, smem_u32(&full[st]));
          bulk_g2s(dst + Cfg<S>::kAChunk, bsrc + c * Cfg<S>::kBChunk, Cfg<S>::kBChunk,
                   smem_u32(&full[st]));
          issued = (int)(gc + 1);
        }
      }
    producer_done:;
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      long long gc = 0, gg = 0;   // chunks and flush groups of this CTA so far
      for (int i = 0;; ++i) {
        if constexpr (Q) {
          const int slot = i % kTq;
          if (!mbar_wait(smem_u32(&tq_full[slot]), (uint32_t)((i / kTq) & 1), err)) {
            bad = 1;
            atomicOr(err, 1ull);
            goto mma_done;
          }
          const int t = tq[slot];
          mbar_arrive(smem_u32(&tq_empty[slot]));
          if (t < 0) break;
        } else {
          if ((long long)blockIdx.x + (long long)i * gridDim.x >= ntiles) break;
        }
        for (long long c = 0; c < nchunks; ++c, ++gc) {
          const int st = (int)(gc % kSt);
          const int set = (int)(gg % kSets);
          const long long use = gg / kSets;   // earlier groups on this accumulator set
          const bool first = c % kFlush == 0;
          const bool last = (c + 1) % kFlush == 0 || c + 1 == nchunks;
          // before a set is reused, its previous group must have been flushed
          if ((first && use > 0 &&
               !mbar_wait(smem_u32(&acc_empty[set]), (uint32_t)((use - 1) & 1), err)) ||
              !mbar_wait(smem_u32(&full[st]), (uint32_t)((gc / kSt) & 1), err)) {
            bad = 1;
            atomicOr(err, 1ull);
            goto mma_done;
          }
          fence_after();
          // descriptors of the stage's first A and B slices; a slice or K-step offset is
          // added to the start-address field (shared addresses < 256 KB: no carry out of it)
          const uint32_t a0 = sm0 + st * Cfg<S>::kStage, b0 = a0 + Cfg<S>::kAChunk;
          const uint32_t tacc = tmem + (uint32_t)set * 256u;   // this group's accumulator set
          const uint64_t da0 = smem_desc(a0, 128, kKcores * 128);
          const uint64_t db0 = smem_desc(b0, 128, kKcores * 128);
          const uint32_t acc0 = first ? 0u : 1u;
          // A digit i meets B digits 0 .. S-1-i in ONE MMA: the B digit slices lie one after
          // another in shared memory (the same 8-row-group stride), so together they are a
          // (S - i) N column operand, and its products land on the level accumulators
          // i .. S-1, which lie one after another in TMEM from column i N.
#pragma unroll
          for (int kk = 0; kk < kKr / 16; ++kk)
#pragma unroll
            for (int i = 0; i < S; ++i)
              mma_bf16(tacc + i * kN, da0 + (uint64_t)((i * kABytes + kk * 256) >> 4),
                       db0 + (uint64_t)((kk * 256) >> 4), idesc((S - i) * kN),
                       (i == 0 && kk == 0) ? acc0 : 1u);
          commit(smem_u32(&empty[st]));
          if (last) {
            commit(smem_u32(&acc_full[set]));
            ++gg;
          }
          mmas = (int)(gc + 1);
        }
      }
    mma_done:;
    }
  } else {  // epilogue warps: flush the levels every kFlush chunks, store each tile
    const int quarter = warp & 3, half = (warp - 2) / 4, ew = warp - 2;
    int gg = 0;   // flush groups of this CTA so far (tiles and chunks per step < 2^31)
    bool failed = false;
    // i: tiles of this CTA so far; t: the tile (tiles per step < 2^31)
    for (int i = 0, t = (int)blockIdx.x; !failed; ++i, t += (int)gridDim.x) {
      if constexpr (Q) {
        const int slot = i % kTq;
        if (!mbar_wait(smem_u32(&tq_full[slot]), (uint32_t)((i / kTq) & 1), err)) {
          if (lane == 0) {
            bad = 1;
            atomicOr(err, 1ull);
          }
          break;
        }
        t = tq[slot];
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&tq_empty[slot]));
        if (t < 0) break;
      } else {
        if (t >= ntiles) break;
      }
      long long bb, tm, tn;
      tile_coords(t, bb, tm, tn);
      // this thread's row of C (lane = row within the lane quarter) and, per lane j < 12,
      // its warp's column j: offsets from the digit kernel's tables (-1 past the edge)
      const long long crow =
          ((const long long*)(scratch + L.cr_off))[(bb * L.tiles_m + tm) * kMc + quarter * 32 + lane];
      if (lane < kNc / 2)
        cn_s[ew][lane] = ((const long long*)(scratch + L.cc_off))[tn * kNc + half * (kNc / 2) + lane];
      // this thread's row exponent and its warp's column exponents, per flush group
      const int* ea_g = (const int*)(scratch + L.ea_off) + (bb * L.tiles_m + tm) * L.groups * kMc +
                        quarter * 32 + lane;
      const int* eb_g = (const int*)(scratch + L.eb_off) + (bb * L.tiles_n + tn) * L.groups * kNc +
                        half * (kNc / 2);
      // blocks of 8 real columns of this warp that hold columns of C (a narrow step's last
      // column block has fewer than kNc; the others are neither read nor combined)
      const long long nv = s.N - tn * kNc;
      const int cols = (int)max(0LL, min((long long)(kCw / 2), nv - half * (kCw / 2)));
      const int c8n = (2 * cols + 7) / 8;
      float acc_h[kCw], acc_l[kCw];
#pragma unroll
      for (int j = 0; j < kCw; ++j) acc_h[j] = acc_l[j] = 0.f;
      for (int g = 0; g < ngroups; ++g, ++gg) {
        const int set = gg % kSets;
        const int eam = ea_g[g * kMc];
        if (lane < kNc / 2) eb_s[ew][lane] = eb_g[g * kNc + lane];
        __syncwarp();
        if (!mbar_wait(smem_u32(&acc_full[set]), (uint32_t)((gg / kSets) & 1), err)) {
          if (lane == 0) {
            bad = 1;
            atomicOr(err, 1ull);
          }
          failed = true;
          break;
        }
        fence_after();
        // level L holds an integer sum of digit products (below 2^24 in magnitude) at weight
        // 2^(-14-8L).  Per 8 columns: levels 0 and 1 are added exactly (TwoSum); levels 2 ..
        // S-1, at most 2^-16 of level 0's scale, are folded into the low part with FP32 FMAs,
        // whose rounding (below 2^-40 of level 0's scale) is under the digits' truncation.
        // The sum is scaled by the group's 2^(e(m) + e(n) - 14) (powers of two: exact) and
        // added to the float-float accumulators.
        const uint32_t ta0 =
            tmem + (uint32_t)set * 256u + ((uint32_t)(quarter * 32) << 16) + half * kCw;
#pragma unroll
        for (int c8 = 0; c8 < kCw / 8; ++c8) {
          if (c8 >= c8n) break;   // warp-uniform
          float hi[8], lo[8];
          tmem_ld8x2(ta0 + c8 * 8, ta0 + kN + c8 * 8, hi, lo);   // levels 0 and 1
#pragma unroll
          for (int i = 0; i < 8; ++i) two_sum(hi[i], lo[i] * 0.00390625f, hi[i], lo[i]);   // exact
#pragma unroll
          for (int lv = 2; lv < S; lv += 2) {
            float v[8], v2[8];
            const float w = __int_as_float((127 - 8 * lv) << 23);   // 2^(-8L) relative to level 0
            if (lv + 1 < S) {
              tmem_ld8x2(ta0 + lv * kN + c8 * 8, ta0 + (lv + 1) * kN + c8 * 8, v, v2);
              const float w2 = w * 0.00390625f;
#pragma unroll
              for (int i = 0; i < 8; ++i) lo[i] = fmaf(v2[i], w2, fmaf(v[i], w, lo[i]));
            } else {
              tmem_ld8(ta0 + lv * kN + c8 * 8, v);
#pragma unroll
              for (int i = 0; i < 8; ++i) lo[i] = fmaf(v[i], w, lo[i]);
            }
          }
#pragma unroll
          for (int i = 0; i < 8; i += 2) {
            float f1, f2;   // one exponent per complex column: (re, im) = columns i, i + 1
            pow2_pair(eam - 14 + eb_s[ew][(c8 * 8 + i) >> 1], f1, f2);
#pragma unroll
            for (int u = i; u < i + 2; ++u) {
              const float h = (hi[u] * f1) * f2, l = (lo[u] * f1) * f2;
              if (g == 0) {   // the first group starts the sums (a float pair, not renormalised)
                acc_h[c8 * 8 + u] = h;
                acc_l[c8 * 8 + u] = l;
              } else {
                ff_acc(acc_h[c8 * 8 + u], acc_l[c8 * 8 + u], h, l);
              }
            }
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&acc_empty[set]));
      }
      // ---- store the tile (the accumulators are released: the next tile's MMAs run):
      // scaled by the step's normalisation; this thread's columns hold the (re, im) pairs
      // of kCw / 2 complex columns of its row.  A tile whose wait gave up is written as NaN.
      Cx<ff>* C = arena + s.off_c;
#pragma unroll
      for (int j = 0; j < kCw / 2; ++j) {
        ff re = ff_norm(acc_h[2 * j], acc_l[2 * j]), im = ff_norm(acc_h[2 * j + 1], acc_l[2 * j + 1]);
        re.hi *= scale;
        re.lo *= scale;
        im.hi *= scale;
        im.lo *= scale;
        if (failed) re.hi = re.lo = im.hi = im.lo = __int_as_float(0x7fc00000);
        const long long cc = cn_s[ew][j];
        if (crow >= 0 && cc >= 0) {
          const Cx<ff> out{re, im};
          st(C + crow + cc, out);
          vmax = fmaxf(vmax, mag(out));
        }
      }
      __syncwarp();   // cn_s of this tile read before the next tile's offsets replace it
    }
  }
  __syncthreads();

  // ---- give-up path: before the tensor memory is freed, wait (with the same bound,
  // ignoring the error word) for this CTA's asynchronous work in flight: the bulk copies of
  // the last chunk issued on each stage, and every MMA issued (one more commit tracks all
  // of them).  If even these waits run out, the CTA exits regardless.
  if (bad) {
    if (warp == 0 && lane == 0)
      for (int c = issued > kSt ? issued - kSt : 0; c < issued; ++c)
        mbar_wait(smem_u32(&full[c % kSt]), (uint32_t)((c / kSt) & 1), nullptr);
    if (warp == 1 && lane == 0 && mmas > 0) {
      commit(smem_u32(&drain));
      mbar_wait(smem_u32(&drain), 0u, nullptr);
    }
    fence_before();
    __syncthreads();
    fence_after();
  }
  block_max_to_meta(vmax, meta + s.c);
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kCols)
                 : "memory");
}

}  // namespace pk
