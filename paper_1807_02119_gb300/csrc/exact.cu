// Exact evaluation: Z(q) modulo word-size primes, on the GPU.
//
// At integer q the Potts t(q) is a root of x^2 - (q - 2) x + 1, and with the standard
// weights every clause entry is an integer polynomial in t (off-diagonal 1, diagonal
// (-1)^mult t^-signsum, t^-1 = (q - 2) - t).  Z(q) is therefore an element a + b t of
// Z[t]/(t^2 - (q - 2) t + 1).  The same plan (network, order, slicing, step records) is
// contracted in F_p[t]/(t^2 - (q - 2) t + 1) for a prime p < 2^31: an element is a pair
// of residues (a, b), stored where a complex64 value would be (8 bytes), and
//     (a + b t)(c + d t) = (ac - bd) + (ad + bc + (q - 2) bd) t.
// Several primes determine Z(q), or quantities derived from it, by the Chinese remainder
// theorem.  No rescaling is needed: the arithmetic is exact.
//
// The kernels mirror the floating-point ones in their indexing only: the initial tensors
// follow their recipes (sum over the vertex spin of products of COPY legs and clause
// entries), every contraction step is C[n R + r] = sum_k A[row r, k] B[k, column n] through
// the step's stride runs, one thread per output, and the slice results are summed.
#include <cuda_runtime.h>

#include <algorithm>

#include "exact_ring.h"
#include "handles.h"
#include "pk_internal.h"

namespace pk {
namespace exact {

__device__ inline void runs(unsigned long long x, const Run* rr, int n, long long& oa, long long& ob) {
  oa = 0;
  ob = 0;
  for (int i = 0; i < n; ++i) {
    const unsigned long long sz = (unsigned long long)rr[i].size;
    const unsigned long long d = x % sz;
    x /= sz;
    oa += (long long)d * rr[i].sa;
    ob += (long long)d * rr[i].sb;
  }
}

// Initial tensor blockIdx.y of one slice: entry e = sum_s prod_j f_j(s, x_j), with f_j a
// COPY leg [s = x_j] or an absorbed clause matrix (diagonal (-1)^mult t^-signsum when
// s = x_j, off-diagonal 1), x_j the entry's digit at the slot's position or the slice's
// fixed value of a sliced index.
__global__ void __launch_bounds__(256) k_exact_build(const Recipe* rec, const Slot* slots, E* arena,
                                                     int q, Ring ring, long long slice, int n_sliced) {
  const Recipe R = rec[blockIdx.y];
  int sdig[64];
  {
    long long s = slice;
    for (int i = 0; i < n_sliced && i < 64; ++i) {
      sdig[i] = (int)(s % q);
      s /= q;
    }
  }
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < R.elems;
       e += (long long)gridDim.x * blockDim.x) {
    E v{0, 0};
    if (R.kind == 1) {
      v = E{1, 0};
    } else {
      for (int s = 0; s < q; ++s) {
        E pr{1, 0};
        bool zero = false;
        for (int j = 0; j < R.nslot; ++j) {
          const Slot sl = slots[R.slot0 + j];
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
              int32_t mult, signsum;
              slot_exact_unpack(sl.pad, mult, signsum);
              E dg = epow_t(-(long long)signsum, ring);
              if (mult & 1) dg = eneg(dg, ring);
              pr = emul(pr, dg, ring);
            }
          } else if (s != x) {
            zero = true;
            break;
          }
        }
        if (!zero) v = eadd(v, pr, ring);
      }
    }
    arena[R.offset + e] = v;
  }
}

// One contraction step, thread per output o = n R + r.
__global__ void __launch_bounds__(256) k_exact_step(const Step s, E* arena, Ring ring) {
  const E* A = arena + s.off_a;
  const E* B = arena + s.off_b;
  E* C = arena + s.off_c;
  const bool hasB = s.b >= 0;
  const unsigned long long total = (unsigned long long)s.R * (unsigned long long)s.N;
  for (unsigned long long o = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; o < total;
       o += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long n = o / (unsigned long long)s.R, r = o % (unsigned long long)s.R;
    long long oa, ob, nb, dummy;
    runs(r, s.row, s.nrow, oa, ob);
    runs(n, s.nr, s.nn, dummy, nb);
    E acc{0, 0};
    for (long long k = 0; k < s.K; ++k) {
      long long ka, kb;
      runs((unsigned long long)k, s.kr, s.nk, ka, kb);
      const E a = A[oa + ka];
      acc = eadd(acc, hasB ? emul(a, B[ob + nb + kb], ring) : a, ring);
    }
    C[o] = acc;
  }
}

// Slice result: the final (rank-0) tensor added into the running sum.
__global__ void k_exact_accum(const E* arena, long long off_final, E* sum, Ring ring) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *sum = eadd(*sum, arena[off_final], ring);
}

}  // namespace exact

// Z(q) of plan `p` modulo `prime` (before the host's loop factor), left in *d_sum as
// (a, b): every slice's initial tensors, steps and result, in the plan's own order.  The
// program must be uploaded (pk_upload) in `ws`; the arena is the complex64 one.
cudaError_t launch_exact(const Plan& p, uint32_t prime, void* ws, void* arena, void* d_sum,
                         cudaStream_t stream) {
  using namespace exact;
  char* base = (char*)ws;
  E* ar = (E*)arena;
  E* sum = (E*)d_sum;
  const Ring ring = make_ring(prime, p.q);
  cudaError_t e = cudaMemsetAsync(sum, 0, sizeof(E), stream);
  if (e != cudaSuccess) return e;
  if (p.n_init > 65535) return cudaErrorInvalidValue;
  int64_t maxel = 1;
  for (const auto& r : p.recipes) maxel = std::max<int64_t>(maxel, r.elems);
  const unsigned bx = (unsigned)std::min<int64_t>((maxel + 255) / 256, 1024);
  for (long long sl = 0; sl < p.n_slices; ++sl) {
    if (p.n_init > 0)
      k_exact_build<<<dim3(bx, (unsigned)p.n_init), 256, 0, stream>>>(
          (const Recipe*)(base + p.off_recipe), (const Slot*)(base + p.off_slots), ar, p.q, ring, sl,
          (int)p.sliced.size());
    for (const Step& st : p.steps) {
      const long long outs = st.R * st.N;
      const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>((outs + 255) / 256, 152 * 16));
      k_exact_step<<<grid, 256, 0, stream>>>(st, ar, ring);
    }
    k_exact_accum<<<1, 32, 0, stream>>>(ar, p.tensors[p.final_tensor].offset, sum, ring);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace pk
