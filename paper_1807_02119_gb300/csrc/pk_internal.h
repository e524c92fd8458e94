// Internal declarations shared by the host translation units of libpk.
#pragma once

#include <array>
#include <cstdint>
#include <string>
#include <vector>

#include "pk.h"

#ifdef __CUDACC__
#define PK_HD __host__ __device__
#else
#define PK_HD
#endif

namespace pk {

// ------------------------------------------------------------------ knots (Sec. II)
struct Knot {
  int32_t n_v = 0;         // Tait vertices (black regions)
  int32_t n_c = 0;         // crossings = Tait edges
  int32_t writhe = 0;      // sum of twist signs
  int32_t tau = 0;         // sum of Tait signs
  int32_t components = 1;  // link components of the diagram
  std::vector<std::array<int32_t, 3>> edges;  // (u, v, eps)
  std::vector<std::array<int32_t, 4>> pd;     // empty for graph input
  bool has_pd = false;
};

bool knot_from_pd(const int32_t* pd, int32_t n, int32_t outer_arc, int32_t outer_side, Knot& k,
                  std::string& err, const int32_t* signs = nullptr);
bool knot_from_graph(int32_t n_v, int32_t n_e, const int32_t* uve, int32_t writhe, Knot& k,
                     std::string& err);
// The signed Tait graph after repeated Reidemeister I (loops, spikes) and II (opposite-sign
// parallel pairs) simplification, with n_v, writhe and tau updated so that V is unchanged.
bool simplify_knot(const Knot& in, Knot& out);
bool grid_walk_pd(int32_t L, uint64_t seed, bool random_over_under, int32_t nmin, int32_t nmax,
                  std::vector<std::array<int32_t, 4>>& pd, int32_t& outer_arc,
                  int32_t& outer_side, std::string& err);

// ------------------------------------------------------------------ scaled scalars
struct Scaled {
  double re = 0, im = 0;
  int64_t e = 0;  // value = (re + i im) 2^e
  void norm();
};
Scaled s_mul(const Scaled& a, const Scaled& b);
Scaled s_pow(Scaled a, int64_t n);
Scaled s_from(double re, double im);

// ------------------------------------------------------------------ plans (Sec. III)
constexpr int kMaxRuns = 20;  // merged stride runs per index class (Step stays < 4 KB)

struct Run {
  int64_t size;
  int64_t sa, sb;  // element strides in operand A and operand B (0 when absent)
};

// One initial tensor: entry(i...) = sum_{s<q} prod_j f_j(s, x_j) where x_j is the value of
// slot j's index (a digit of the element, or a sliced index's fixed value) and
// f_j(s, x) = (s == x) ? diag_j : off_j for an absorbed clause matrix (off_j = 1 for the
// standard weights), [s == x] for a COPY leg.  kind CONST1 is the scalar 1.
struct Recipe {
  int32_t kind;            // 0 = vertex sum, 1 = const 1
  int32_t rank;            // free dims
  int32_t slot0, nslot;    // into Plan::slots
  int64_t elems;           // q^rank
  int64_t offset;          // element offset in the tensor arena
  int32_t meta;            // meta slot (tensor id)
  int32_t exp2;            // the entries stand for entry * 2^exp2: general clause weights
                           // are stored scaled by a power of two (max entry in [0.5, 1)),
                           // so that products of large or small weights neither overflow
                           // nor underflow before the steps' own rescaling; 0 otherwise
};

struct Slot {
  int32_t dimpos;          // position (stride q^dimpos) in the tensor, or -1 if sliced
  int32_t slice_ord;       // ordinal among sliced indices (valid when dimpos < 0)
  int32_t absorbed;        // 1: clause matrix, 0: COPY leg
  int32_t pad;             // absorbed, standard weights: slot_exact_pack(mult, signsum)
  double dre, dim;         // clause diagonal when absorbed
  double ore, oim;         // clause off-diagonal when absorbed
};

// Exact form of an absorbed clause diagonal under the standard weights: the product of
// `mult` Tait-edge diagonals -t^-eps with sum of signs `signsum` is (-1)^mult t^-signsum.
inline int32_t slot_exact_pack(int32_t mult, int32_t signsum) {
  return (int32_t)(((uint32_t)(signsum & 0xFFFF) << 16) | (uint32_t)(mult & 0xFFFF));
}
#if defined(__CUDACC__)
__host__ __device__
#endif
inline void slot_exact_unpack(int32_t pad, int32_t& mult, int32_t& signsum) {
  mult = pad & 0xFFFF;
  signsum = (int32_t)(int16_t)((uint32_t)pad >> 16);
}

enum KernelKind : int32_t { KROWS = 0, KSPLITK = 1, KGEMM = 2 };

// A stride run with its stride in C as well (GEMM view of a step).
struct Run4 {
  int64_t size;
  int64_t sa, sb, sc;
};

struct Step {
  int32_t a, b, c;         // tensor ids (a = larger operand; b = -1: constant 1)
  int32_t kernel;          // KernelKind
  int64_t off_a, off_b, off_c;  // element offsets in the tensor arena
  int64_t R, K, N;         // rows (batch x free-of-a), contracted, free-of-b
  int32_t nrow, nk, nn;    // runs per class
  Run row[kMaxRuns];       // inner -> outer; C stride of a row digit is implicit (contiguous)
  Run kr[kMaxRuns];
  Run nr[kMaxRuns];        // sa unused, sb = stride in B; C offset = n * R
  int32_t rank_c;
  int32_t chunks;          // split-K: K chunks
  // GEMM view: C[b, m, n] = sum_k A[b, m, k] B[b, k, n] with the rows split into batch
  // runs (present in both operands) and m runs (A only); every run carries its C stride.
  int64_t Bsz, M;          // R = Bsz * M
  int32_t ngb, ngm, ngn;
  int32_t a_kinner;        // A's unit-stride index is a contracted one
  int32_t b_kinner;        // B's unit-stride index is a contracted one
  int32_t tc;              // split precision: BF16 digits per operand on the tensor cores
                           // (4 or 5), 0 = the GEMM step runs on the CUDA cores
  Run4 gb[kMaxRuns];
  Run4 gm[kMaxRuns];
  Run4 gn[kMaxRuns];
};

// Per-tensor device bookkeeping: stored value x means x * 2^exp; maxbits is the bit
// pattern of max(|re|, |im|) over the stored tensor (IEEE order = integer order for
// non-negative values, so atomicMax on the bits is a max on the values).
struct Meta {
  unsigned long long maxbits;
  long long exp;
};
struct SliceResult {
  double re, im;
  long long exp;
  // In the total record (index n_slices) only, the evaluation's error word: bit 0 is set
  // when a bounded device wait gave up (the tensor-core GEMM's pipeline waits); bits 1 and
  // up hold status_nonfinite's code of the first tensor found non-finite by the finite
  // check.  Nonzero: the value is invalid.  Cleared by the first slice's bookkeeping reset
  // of every launch sequence.
  unsigned long long status;
};
// Error-word code of a non-finite entry in the result of `step` (-1: an initial tensor) of
// slice `slice`; decoded by nonfinite_slice / nonfinite_step.
PK_HD inline unsigned long long status_nonfinite(long long slice, int step) {
  return ((unsigned long long)(slice + 1) << 24 | (unsigned long long)(step + 2)) << 1;
}
inline long long nonfinite_slice(unsigned long long status) { return (long long)(status >> 25) - 1; }
inline int nonfinite_step(unsigned long long status) { return (int)((status >> 1) & 0xFFFFFF) - 2; }

// Split precision: a bulk (complex64) tensor read by a complex128 tail step is copied,
// widened, into the tail region; its copy gets its own bookkeeping slot.
struct ConvRec {
  int64_t src_off;   // complex64 elements into the arena
  int64_t dst_off;   // complex128 elements into the tail region
  int64_t elems;
  int32_t src_meta, dst_meta;
};
// A small step run inside a sequence kernel (one CTA runs consecutive small steps with a
// block barrier between them): the step's row, contraction and column runs only.
struct TinyStep {
  int32_t a, b, c;         // bookkeeping slots (b = -1: constant 1)
  int32_t nrow, nk, nn;
  int64_t off_a, off_b, off_c;
  int64_t R, K, N;
  Run row[kMaxRuns];
  Run kr[kMaxRuns];
  Run nr[kMaxRuns];
};
// Consecutive small steps [first, first + count) run as one launch.
struct Segment {
  int32_t first, count;
  int32_t tiny0;           // index of the first step's TinyStep record
};
constexpr int64_t kTinyK = 2048;          // contracted extent at most (offset table in shared memory)

struct TailStep {
  int32_t step;
  int32_t meta_a, meta_b;            // bookkeeping slots of the (possibly converted) operands
  int32_t pad;
  int64_t off_a, off_b, off_c;       // complex128 elements into the tail region
};


// GEMM steps of the split precision on the tensor cores: each operand element becomes S
// BF16 digits (exact 8-bit pieces; S = Step::tc, 4 or 5), stored per tile block and
// 16-complex-k chunk in the workspace after the arena, followed by the blocks' exponents,
// one per row (column) and flush group of tc_flush(S) chunks.
// A tile is kTcMc complex rows of A, each stored once as [Re A, Im A], by kTcNc complex
// columns of B, each stored as two real columns [Re B; -Im B] and [Im B; Re B] (the
// complex doubling sits on B, the operand the planner keeps smaller).
constexpr int kTcMc = 128, kTcNc = 24, kTcKc = 16;
PK_HD constexpr long long tc_a_chunk(int S) { return (long long)S * kTcMc * (2 * kTcKc) * 2; }
PK_HD constexpr long long tc_b_chunk(int S) { return (long long)S * (2 * kTcNc) * (2 * kTcKc) * 2; }
// Chunks per flush group: the S digit pairs of a level, 2 kTcKc real terms per chunk and
// digit products below 2^14 keep a level's FP32 sum exact (below 2^24) for this many chunks.
PK_HD constexpr int tc_flush(int S) { return ((1 << 10) - 1) / (S * 2 * kTcKc); }
// After the digits and exponents: the C offsets of every tile row (batch base included,
// Bsz x tiles_m x kTcMc) and tile column (tiles_n x kTcNc), -1 past the edge, written by
// the digit kernel for the GEMM's epilogue.
struct TcScratch {
  long long tiles_m, tiles_n, chunks, groups;
  long long a_off, b_off, ea_off, eb_off, cr_off, cc_off, bytes;
};
PK_HD inline TcScratch tc_scratch(long long Bsz, long long M, long long N, long long K, int S) {
  TcScratch x;
  x.tiles_m = (M + kTcMc - 1) / kTcMc;
  x.tiles_n = (N + kTcNc - 1) / kTcNc;
  x.chunks = (K + kTcKc - 1) / kTcKc;
  x.groups = (x.chunks + tc_flush(S) - 1) / tc_flush(S);
  x.a_off = 0;
  x.b_off = x.a_off + Bsz * x.tiles_m * x.chunks * tc_a_chunk(S);
  x.ea_off = x.b_off + Bsz * x.tiles_n * x.chunks * tc_b_chunk(S);
  x.eb_off = x.ea_off + ((Bsz * x.tiles_m * x.groups * kTcMc * 4 + 255) & ~255LL);
  x.cr_off = x.eb_off + ((Bsz * x.tiles_n * x.groups * kTcNc * 4 + 255) & ~255LL);
  x.cc_off = x.cr_off + ((Bsz * x.tiles_m * kTcMc * 8 + 255) & ~255LL);
  x.bytes = x.cc_off + ((x.tiles_n * kTcNc * 8 + 255) & ~255LL);
  return x;
}

// Reverse pass: one record per clause tensor (merged edge group) of a gradient plan.
// The adjoint dZ/dM of the group's matrix M (full shape q x q, or q for a loop vector)
// is read from the arena with the strides below and added into an accumulator.
struct GradLeaf {
  int32_t meta;            // bookkeeping slot of the adjoint; -1: the adjoint is the constant 1
  int32_t rank;            // 2: clause matrix over (u, v); 1: loop vector over u
  int32_t slice_ord[2];    // >= 0: full dim j is a sliced index with this ordinal
  int64_t offset;          // adjoint's element offset in the arena
  int64_t stride[2];       // adjoint's element stride of full dim j (0: broadcast)
};

// Per merged edge group of a general (weighted or gradient) plan: the clause tensor and
// the Tait edges whose entrywise product it is.
struct EdgeGroup {
  int32_t u, v;            // u < v, or u == v for loops
  int32_t leaf;            // initial tensor id
  int32_t slot;            // index of its absorbed slot in Plan::slots
  std::vector<int32_t> members;
};

// The program of a gradient plan: forward steps, then per checkpoint region the
// recomputed intermediates and the adjoint steps, all on one arena.
struct GradProgram {
  bool built = false;
  int32_t stride = 1;                // checkpoint stride in tree levels (<= 1: keep all)
  std::vector<Step> steps;           // launch order; meta slots in a, b, c
  std::vector<int8_t> phase;         // per step: 0 forward, 1 recompute, 2 adjoint
  std::vector<Recipe> recipes;       // initial tensors at their offsets in this arena
  std::vector<GradLeaf> leaves;      // one per EdgeGroup, same order
  std::vector<Segment> segments;     // runs of small steps launched as one sequence kernel
  std::vector<TinyStep> tiny;        // their records (in the program at off_tiny)
  int32_t n_meta = 0;
  int32_t n_checkpoints = 0;
  int64_t arena_elems = 0;
  int64_t partials = 0;
  int64_t root_offset = 0;
  int32_t root_meta = 0;
  double cmacs[3] = {0, 0, 0};       // per slice, by phase
  uint64_t off_recipe = 0, off_slots = 0, off_leaves = 0, off_tiny = 0, off_meta = 0,
           off_counter = 0, off_result = 0, off_scratch = 0, off_acc = 0, off_arena = 0;
  std::vector<uint8_t> program;      // recipes | slots | leaves | tiny steps, copied by pk_grad
  uint64_t ws_bytes(int32_t precision) const {
    return off_arena + (uint64_t)arena_elems * (precision == PK_C64 ? 8ull : 16ull);
  }
};

struct TensorInfo {
  std::vector<int32_t> dims;  // index ids, outermost first (row-major)
  int64_t elems = 1;
  int64_t offset = 0;         // element offset in arena
  int32_t born = -1, dies = -1;
};

struct Plan {
  int32_t q = 0;
  int32_t order_used = 0;
  Knot knot;
  // network
  int32_t n_idx = 0;
  std::vector<TensorInfo> tensors;  // initial tensors first, then one per step
  int32_t n_init = 0;
  std::vector<Recipe> recipes;
  std::vector<Slot> slots;
  std::vector<int32_t> slot_exp;     // per slot: power of two its clause values are scaled by
  std::vector<Step> steps;
  std::vector<int32_t> sliced;       // sliced index ids
  int64_t n_slices = 1;
  Scaled factor;                     // constant factors (loops), applied on the host
  int32_t loop_count = 0, loop_signsum = 0;  // the same factor exactly: prod of -t^-eps
  int32_t final_tensor = -1;
  // stats
  int32_t max_rank = 0;
  double log2_max_elems = 0;
  double cmacs = 0, bytes_c64 = 0;
  double est_cost = 0;   // the planner's estimated cost of the chosen sequence (all slices)
  int64_t arena_elems = 0;
  int64_t splitk_partials = 0;      // complex scratch entries for split-K steps
  // device program layout (byte offsets inside the workspace)
  uint64_t off_recipe = 0, off_slots = 0, off_meta = 0, off_result = 0, off_scratch = 0,
           off_counter = 0, off_arena = 0;
  uint64_t ws_bytes(int32_t precision) const;
  // byte offset of the split precision's digit scratch from the arena's start
  uint64_t tc_offset() const { return ((uint64_t)arena_elems * 16ull + 255) & ~uint64_t(255); }
  std::vector<uint8_t> program;      // recipe + slots blob copied by pk_upload
  // split precision: steps >= tail_first run in complex128 in a separate tail region;
  // bulk tensors they read are up-converted there first
  int32_t tail_first = 0;
  std::vector<ConvRec> conv;
  std::vector<Segment> segments;     // runs of small steps launched as one sequence kernel
  std::vector<TinyStep> tiny;        // their records (in the program at off_tiny)
  uint64_t off_tiny = 0;
  pk_tuning tuning{};                // launch shapes the plan was made with
  std::vector<TailStep> tail;        // one per step >= tail_first
  int64_t tail_elems = 0;            // complex128 elements of the tail region
  int64_t final_tail_off = 0;        // final tensor's offset in the tail region
  int32_t n_meta = 0;                // tensors + converted copies
  uint64_t off_tail = 0;             // byte offset of the tail region (split only)
  int64_t tc_bytes = 0;              // split precision: digit scratch of the largest
                                     // tensor-core step (after the arena)
  int32_t n_tc = 0;                  // tensor-core steps per slice
  uint64_t off_conv = 0;             // byte offset of the ConvRec records (in the program)
  // general networks (PK_FLAG_GRAD or custom weights): every edge group is a tensor
  bool general = false;
  bool std_weights = true;           // weights are (-t^-eps, 1) of t(q)
  std::vector<std::array<double, 4>> weights;  // per Tait edge: diag re, im, off re, im
  std::vector<EdgeGroup> groups;
  std::vector<std::vector<int32_t>> leaf_dims;  // initial tensors' dims before slicing
  GradProgram grad;
};

// Host-side check of every index map and of the memory layout of `p` for `precision`
// (verify.cpp); false with `err` naming the first violation.
bool verify_plan(const Plan& p, int32_t precision, std::string& err);

// The error of an evaluation's error word (SliceResult::status of the total record):
// PK_ENONFINITE for a finite-check code, PK_ETIMEOUT for an expired wait, with `err` set.
pk_status status_error(unsigned long long status, std::string& err);

// Host side of reading a result back: Z from the total record (normalised, times the
// plan's constant factor) and V = A(q) Z when V is not null.  PK_ETIMEOUT (with `err` set)
// when the record's status word is nonzero, PK_EINVAL when A(q)'s exponent condition fails.
pk_status decode_total(const Plan& P, const SliceResult& r, pk_scaled* Z, pk_scaled* V,
                       std::string& err);

// Step descriptor for C = sum over the indices of X and Y that are not in `out` of X Y
// (Y absent: the constant 1).  `a` is the operand with more indices (ties: X); the
// result's layout is written to `cdims`.
// tc_min_k, tc_min_n, tc_wide_n: split precision, row steps of GEMM shape (M >= 64) with
// N >= tc_min_n and either K >= tc_min_k or (K >= 4 and N >= tc_wide_n) also go to
// the tensor cores (Step::tc).
bool build_step(const std::vector<int32_t>& xd, const std::vector<int32_t>* yd,
                const std::vector<int32_t>& out, int32_t q, int32_t flags, Step& st,
                bool& swapped, std::vector<int32_t>& cdims, std::string& err, int64_t tc_min_k = 16,
                int64_t tc_min_n = 32, int64_t tc_wide_n = (int64_t)1 << 30, int64_t tc_min_work = 0);
bool make_plan(const Knot& k, int32_t q, const pk_plan_opts& opts, const pk_tuning& tune, Plan& p,
               std::string& err);
// Order search only (no slicing, no step records): out[0] largest tensor rank, out[1] log2
// of the summed R K N, out[2] initial tensors, out[3] indices, for the best candidate of
// `order` (by rank, then cost).  False for an unknown order or q.
bool order_stats(const Knot& k, int32_t q, int32_t order, int32_t restarts, double* out);
// Maximal runs (>= 2) of consecutive small row-kernel steps (at most tune.seq_outs outputs,
// K <= tune.seq_k <= kTinyK, at most tune.seq_work complex multiply-adds), with their
// compact records, for the sequence kernel k_seg.
void build_segments(const std::vector<Step>& steps, const pk_tuning& tune,
                    std::vector<Segment>& segments, std::vector<TinyStep>& tiny);
bool valid_tuning(const pk_tuning& t);
bool make_grad_program(Plan& p, int32_t stride, int32_t flags, const pk_tuning& tune, std::string& err);
// Writes the clause values of p.weights into p.slots and both program blobs.
void apply_weights(Plan& p);
// New per-edge weights (4 doubles per Tait edge; NULL: the standard weights of t(q)) for a
// general plan; false if a weight is not finite.
bool set_weights(Plan& p, const double* w);
// d log Z / dT_c for every Tait edge from the accumulated adjoints (acc: q*q complex per
// group, exp: power-of-two exponent per group) and Z; dlogV/dt at the standard weights.
// Returns false when Z is zero.
bool grad_finalize(const Plan& p, const double* acc, const int64_t* acc_exp, const Scaled& z,
                   double* dlogz, double* dlogv_dt);
void clause_diag(int32_t q, int32_t mult, int32_t signsum, double& re, double& im);
void t_of_q_value(int32_t q, double& re, double& im);  // t(q) of Eq. potts2jones
bool jones_defined(const Knot& k);  // A(q)'s exponent condition (knots: 4 | num, links: 2 | num)
Scaled jones_prefactor(const Knot& k, int32_t q);  // A(q) in its integer-exponent form

// Exact coefficients of V (jones_exact.cpp): the exponent window of a knot's V from its PD
// code; V(t(q)) mod p from Z(q) mod p; the coefficients mod p from values at several q;
// the signed integers from residues (the last prime checks).
int32_t jones_half(const Knot& k);  // 1: V has half-integer powers (the window is of V t^-1/2)
bool jones_window(const Knot& k, int32_t& lo, int32_t& hi);
void jones_value_mod(const Knot& k, int32_t q, uint32_t p, uint32_t za, uint32_t zb, uint32_t& va,
                     uint32_t& vb);
bool solve_coefficients_mod(const std::vector<int32_t>& qs, const std::vector<uint32_t>& vals, int32_t lo,
                            int32_t m, uint32_t p, std::vector<uint32_t>& c);
bool crt_signed(const std::vector<uint32_t>& primes, const std::vector<std::vector<uint32_t>>& res,
                std::vector<int64_t>& out);

}  // namespace pk
