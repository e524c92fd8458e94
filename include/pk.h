/*
 * pk.h -- C ABI of the GB300 library that evaluates the Jones polynomial V_K(t(q))
 * of a knot by exact contraction of the PACI tensor network (Meichanetzidis &
 * Kourtis, "Evaluating the Jones polynomial with tensor networks").
 *
 * Problem statement (Sec. III, first paragraph): given a knot diagram and an
 * integer q, compute the partition function Z(q) of the q-state Potts model with
 * anisotropic complex interactions on the knot's signed Tait graph, and from it
 * V_K(t(q)) = A(q) Z(q) (Eq. JonesPotts) with t(q) = (q + sqrt(q) sqrt(q-4) - 2)/2
 * (Eq. potts2jones).
 *
 * Conventions for every entry point:
 *  - Return value is a pk_status; nothing is thrown across the ABI.  On error the
 *    context's pk_last_error() holds a one-line message.
 *  - The caller owns every array it passes; inputs are copied, never retained.
 *  - Handles (pk_ctx, pk_knot, pk_plan) are opaque and freed by their *_destroy.
 *  - A context is used by one host thread at a time.
 *  - Device pointers are plain CUDA device addresses on the context's device.
 *  - Results Z and V are returned as pk_scaled because they leave the double
 *    range for large knots.
 */
#ifndef PK_H
#define PK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pk_ctx pk_ctx;
typedef struct pk_knot pk_knot;
typedef struct pk_plan pk_plan;

/* value = (re + i im) * 2^exp2; max(|re|,|im|) in [0.5, 1) unless the value is 0. */
typedef struct {
  double re, im;
  int64_t exp2;
} pk_scaled;

typedef enum {
  PK_OK = 0,
  PK_EINVAL = 1,     /* bad argument: q < 1, malformed PD code, bad sign, NULL pointer */
  PK_ENOTKNOT = 2,   /* kept for compatibility: no longer returned (links get V too)  */
  PK_ENOMEM = 3,     /* host allocation failed or workspace too small                  */
  PK_ETOOWIDE = 4,   /* plan exceeds the slicing limits                                 */
  PK_ECUDA = 5,      /* a CUDA runtime call failed                                      */
  PK_ETIMEOUT = 6,   /* a bounded device wait gave up (the tensor-core GEMM's pipeline
                        waits); the result is invalid.  Reported by pk_download, pk_eval and
                        pk_eval_noalloc from the evaluation's own error word, which every
                        launch sequence clears again: later evaluations are unaffected     */
  PK_ENODEVICE = 7,  /* operation needs a GPU context (device >= 0)                     */
  PK_EZERO = 8,      /* Z is zero, so log-derivatives are undefined                     */
  PK_ENONFINITE = 9  /* the finite check (PK_DEBUG_CHECK_FINITE) found NaN or Inf in a
                        tensor of the evaluation; pk_last_error names the slice and the
                        step (-1: an initial tensor) that wrote it                       */
} pk_status;

typedef enum {
  PK_C128 = 0,       /* complex128 storage, FP64 arithmetic                               */
  PK_C64 = 1,        /* complex64 storage, FP32 arithmetic; with pk_plan_opts.tail_steps
                        > 0 the final contractions run in complex128                      */
  PK_SPLIT = 2       /* split FP32: every real number is an unevaluated pair of floats
                        hi + lo (16 bytes per complex entry); products are split exactly
                        with an FMA (two-product) and sums carried in float pairs
                        (TwoSum), i.e. about 48 significant bits on the FP32 units       */
} pk_precision;

typedef enum {
  PK_ORDER_AUTO = 0,         /* cheapest (by complex multiply-adds) of the orders below     */
  PK_ORDER_GREEDY_EDGE = 1,  /* Sec. III "greedy": vertex tensors on Tait vertices, indices
                                on edges; contract the pair whose result has the smallest
                                degree (graph minors H, cost O(q^Delta_H))                  */
  PK_ORDER_GREEDY_SPIN = 2,  /* same greedy on the network whose COPY tensors are kept as
                                shared spin indices (clause matrices only)                  */
  PK_ORDER_ELIM_SPIN = 3,    /* spin network, order from min-degree spin elimination        */
  PK_ORDER_PARTITION = 4,    /* spin network, nested dissection: the tensors are bisected
                                recursively (level-structure split of a breadth-first order
                                from a pseudo-peripheral tensor, then single moves that
                                shrink the separator); each half's spins are eliminated
                                before the separator's; best of pk_plan_opts.restarts seeds.
                                Not among AUTO's candidates (min-fill is far cheaper on
                                grid-walk knots)                                             */
  PK_ORDER_FILL_SPIN = 5     /* spin network, min-fill elimination with randomised ties,
                                best of pk_plan_opts.restarts restarts                       */
} pk_order;

/* pk_plan_opts.flags: kernel-choice overrides for testing and tuning (default 0 lets
 * the planner choose per step by its shape). */
#define PK_FLAG_FORCE_GEMM 1 /* every two-operand step on the tiled GEMM kernel           */
#define PK_FLAG_FORCE_ROWS 2 /* every step on the row kernel                               */
#define PK_FLAG_NO_TC 8      /* PK_SPLIT: run GEMM-shaped steps on the CUDA cores (float-float
                                SIMT kernel) instead of the tensor cores                     */
#define PK_FLAG_TC_DIGITS4 16 /* PK_SPLIT tensor-core steps: four BF16 digits per operand
                                (10 digit-pair products, truncation near 2^-32 of a row's and
                                column's largest entries) instead of five (15 products, 2^-40) */
#define PK_FLAG_GRAD 4       /* also build the reverse (adjoint) program used by pk_grad.
                                The network then keeps every edge group as a tensor (a pair
                                of opposite-sign parallel edges is not dropped, loops become
                                vectors over their vertex's spin) and only spin-network
                                orders are used; Z is unchanged                              */

typedef struct {
  int32_t order;             /* pk_order                                                    */
  int32_t flags;             /* PK_FLAG_* bits, 0 by default                                */
  double max_log2_elems;     /* slice indices until no tensor exceeds 2^x elements (<= 31;
                                0 -> 31)                                                     */
  double max_log2_slices;    /* refuse (PK_ETOOWIDE) plans needing more slices (0 -> 40)    */
  int32_t tail_steps;        /* PK_C64: this many final contractions run in complex128
                                (<= 0: none)                                                 */
  int32_t restarts;          /* min-fill restarts for PK_ORDER_FILL_SPIN / AUTO (0 -> 8)    */
  int32_t checkpoint_stride; /* PK_FLAG_GRAD: the reverse pass keeps the forward
                                intermediates whose tree level (leaves 0, a step's result
                                1 + its operands' maximum) is a multiple of this and
                                recomputes the others from them (<= 1: keep all)             */
  const double* edge_weights;/* NULL for the Jones weights of Eq. clause, or 4 doubles per
                                Tait edge e (pk_knot_edges order): the clause matrix of e is
                                diag (w[4e] + i w[4e+1]) and off-diagonal (w[4e+2] + i
                                w[4e+3]): a general anisotropic complex Potts instance.
                                Read during pk_plan_create only.  V is then reported with
                                the A(q) of the standard weights (meaningless unless they
                                are those weights); such networks are general (see
                                PK_FLAG_GRAD) and use spin-network orders                   */
  int32_t refine;            /* subtree reconfiguration of the 16 cheapest candidate
                                sequences: pairwise bracketings of frontiers of up to
                                `refine` subtrees (4..10; larger values act as 10), and of
                                refine + 2 at the 12 widest nodes, chosen exactly by dynamic
                                programming under the ranking's cost model (0 -> none).
                                Planning effort only: Z is unchanged                          */
} pk_plan_opts;

typedef struct {
  double log2_max_elems;     /* largest tensor of one slice, log2 elements                  */
  double cmacs;              /* complex multiply-adds, all slices                           */
  double bytes_c64;          /* algorithmic bytes at 8 B/element: sum over steps of
                                |A| + |B| + |C|, all slices (x2 for complex128)             */
  int64_t n_slices;
  int32_t n_steps;           /* pairwise contraction steps per slice                        */
  int32_t max_rank;          /* Delta_H: largest tensor rank (indices) in one slice         */
  int32_t order_used;        /* pk_order actually used                                      */
  int32_t n_tensors;         /* initial tensors                                             */
  uint64_t workspace_c128;   /* device workspace bytes for PK_C128                          */
  uint64_t workspace_c64;    /* device workspace bytes for PK_C64                           */
  uint64_t workspace_split;  /* device workspace bytes for PK_SPLIT                         */
  int32_t n_segments;        /* runs of consecutive small steps launched as one sequence
                                kernel (one CTA, a block barrier between steps)              */
  int32_t n_segment_steps;   /* steps inside those runs                                     */
  double est_cost;           /* the planner's estimated cost of the chosen sequence, all
                                slices (the ranking's units: row-kernel multiply-adds)        */
} pk_plan_stats;

/* ---- tuning ------------------------------------------------------------------- */

/* Launch-shape parameters of the executor, chosen per GPU by measurement (the package's
 * autotune script sweeps them on the configured workloads and writes the table the
 * library is compiled with; pk_tuning_default returns that table).  A context starts with
 * the defaults; pk_ctx_set_tuning changes them for plans and batches created afterwards. */
typedef struct {
  int32_t batch_threads;     /* threads per CTA of the batch executor: 128, 256 or 512       */
  int32_t batch_ktab;        /* batch executor: contracted-index offsets of a step kept in
                                shared memory (steps with longer K recompute them): 256..2048 */
  int64_t seq_outs;          /* runs of small steps launched as one sequence kernel: outputs
                                per step at most (1..65536)                                   */
  int64_t seq_work;          /* ... complex multiply-adds per step at most (1..2^24)          */
  int64_t seq_k;             /* ... contracted extent per step at most (1..2048)              */
  int64_t tc_min_k;          /* PK_SPLIT: row steps of GEMM shape (M >= 64, N >= tc_min_n)
                                with this contracted extent or more run on the tensor cores
                                too (4..16; 16: only steps with K >= 16)                      */
  int64_t tc_db_groups;      /* PK_SPLIT: tensor-core steps with at least this many flush
                                groups of K (96 complex k each) run one CTA per SM with two
                                accumulator sets, so a group's flush overlaps the next group's
                                products; shorter steps run two CTAs per SM (0: never; 1..4096) */
  int64_t tc_min_n;          /* PK_SPLIT: ... and at least this many columns (8..32; a tile
                                has 24, so narrower steps leave part of it idle)              */
  int64_t cost_gemm_milli;   /* planner: cost of a complex multiply-add in a step that runs on
                                the tensor cores (M >= 64, N >= tc_min_n, K >= tc_min_k), in
                                thousandths of a row-kernel multiply-add (10..1000), when the
                                candidate orders are ranked                                    */
  int64_t cost_out_milli;    /* planner: cost of one output entry of a step (its store and
                                normalisation), in thousandths of a multiply-add (0..10^6)    */
  int64_t tc_wide_n;         /* PK_SPLIT: row steps of GEMM shape with K >= 4 (below tc_min_k)
                                also run on the tensor cores when they have at least this many
                                columns (16..2^30; 2^30: never)                               */
  int64_t cost_tcin_milli;   /* planner: cost of one operand entry (of A and of B) of a step
                                that runs on the tensor cores (its BF16 digits are written by a
                                conversion pass and read back by the GEMM), in thousandths of a
                                multiply-add (0..10^6)                                         */
  int64_t tc_min_work;       /* PK_SPLIT: row steps of GEMM shape (above) run on the tensor
                                cores only from this many complex multiply-adds per slice
                                (0..2^40; smaller ones stay on the row kernels)               */
} pk_tuning;

pk_status pk_tuning_default(pk_tuning* out);

/* ---- context ------------------------------------------------------------------ */

/* device >= 0: a GPU context on that device; stream (a cudaStream_t, may be NULL for
 * the legacy default stream) is where every launch goes.  device = -1: a host-only
 * context for knot input and planning (pk_eval returns PK_ENODEVICE). */
pk_status pk_ctx_create(int32_t device, void* stream, pk_ctx** out);
pk_status pk_ctx_set_stream(pk_ctx* ctx, void* stream);
/* Device-memory budget for the plans created afterwards (0: none, the default): a plan
 * whose workspace at any precision (pk_plan_workspace_bytes) would exceed `bytes` is sliced
 * further -- one index fewer on its largest tensor at a time, more slices of less memory
 * (Sec. III.B names memory as the bottleneck) -- until it fits; PK_ETOOWIDE from
 * pk_plan_create when the slice limit (pk_plan_opts.max_log2_slices) is reached first. */
pk_status pk_ctx_set_hbm_budget(pk_ctx* ctx, uint64_t bytes);
/* NULL restores the defaults.  PK_EINVAL for values outside the ranges of pk_tuning. */
pk_status pk_ctx_set_tuning(pk_ctx* ctx, const pk_tuning* t);
pk_status pk_ctx_get_tuning(const pk_ctx* ctx, pk_tuning* out);
const char* pk_last_error(const pk_ctx* ctx);
void pk_ctx_destroy(pk_ctx* ctx);

/* ---- knots (Sec. II) ------------------------------------------------------------ */

/* PD code: n crossings, pd[4*i .. 4*i+3] = (a, b, c, d); arcs labelled 0..2n-1 along
 * the orientation; a = incoming under-arc, then counter-clockwise; c = a+1 mod 2n.
 * outer_arc/outer_side (side 0 = left, 1 = right of that arc) name a region that the
 * Tait graph treats as the unbounded, white region (Sec. II); outer_arc = -1 picks
 * the colour class of the region right of arc 0 as black.  n = 0 is the unknot.
 * Errors: PK_EINVAL (labels, orientation or planarity wrong). */
pk_status pk_knot_from_pd(pk_ctx* ctx, const int32_t* pd, int32_t n, int32_t outer_arc,
                          int32_t outer_side, pk_knot** out);

/* A link diagram (one or more components; Sec. "Conclusions and outlook": Tait graphs,
 * and so the method, extend to links):
 * PD code as above but with any labels 0..2n-1 (each occurring twice; c is the arc
 * leaving through the under-strand, not necessarily a+1), and signs[i] = +1 or -1, the
 * twist sign of crossing i by the right-hand rule (+1: the over-strand leaves through
 * arm b, -1: through arm d), which fixes every component's orientation.  The diagram
 * must be connected (a split diagram has no Tait graph here).  V of a link lies in
 * Z[t^(1/2)]: it is evaluated with s = exp(Log t / 4), the principal fourth root of the
 * Potts t(q), in A(q) = (-1)^(w+n_v+1) s^(3w+tau+2n_v+2) (t+1)^-(n_v+1).
 * Errors: PK_EINVAL (labels, signs, orientation or planarity wrong). */
pk_status pk_link_from_pd(pk_ctx* ctx, const int32_t* pd, const int32_t* signs, int32_t n,
                          int32_t outer_arc, int32_t outer_side, pk_knot** out);

/* Signed Tait graph given directly: n_e edges uve[3*e..] = (u, v, eps), eps = +-1,
 * u, v in [0, n_v); writhe w.  Z is defined for any such graph (general PACI
 * instance, Sec. III); V uses tau = sum eps and needs 4 | 3w + tau + 2 n_v + 2. */
pk_status pk_knot_from_signed_graph(pk_ctx* ctx, int32_t n_v, int32_t n_e, const int32_t* uve,
                                    int32_t writhe, pk_knot** out);

/* Random grid-walk knot (Sec. III.A): permutations x, y of 0..L-1 from SplitMix64(seed)
 * by Fisher-Yates; redrawn from the same stream until the crossing count lies in
 * [ncross_min, ncross_max]; random_over_under != 0 draws one over/under bit per
 * crossing, else vertical strands pass over.  The unbounded region is white. */
pk_status pk_knot_from_grid_walk(pk_ctx* ctx, int32_t L, uint64_t seed, int32_t random_over_under,
                                 int32_t ncross_min, int32_t ncross_max, pk_knot** out);

pk_status pk_knot_info(const pk_knot* k, int32_t* n_v, int32_t* n_c, int32_t* writhe,
                       int32_t* tau, int32_t* components);
/* The simplified Tait graph of Sec. III.A as a new knot (signed graph, no PD code):
 * Reidemeister I removes loops (tau -= eps, w -= eps) and spikes, i.e. degree-1 vertices
 * (n_v -= 1, tau -= eps, w += eps); Reidemeister II removes parallel edge pairs of
 * opposite Tait signs; repeated until none applies.  V of the result equals V of k.
 * The caller owns *out (pk_knot_destroy). */
pk_status pk_knot_simplify(pk_ctx* ctx, const pk_knot* k, pk_knot** out);
/* Copies the signed Tait graph: uve[3*e..] = (u, v, eps) for each crossing (n_c edges). */
pk_status pk_knot_edges(const pk_knot* k, int32_t* uve);
/* Copies the PD code (4*n_c ints); PK_EINVAL for knots built from a signed graph. */
pk_status pk_knot_pd(const pk_knot* k, int32_t* pd);
void pk_knot_destroy(pk_knot* k);

/* ---- contraction plan (Sec. III: network G_T, contraction order, slicing) ------ */

/* q >= 1.  opts may be NULL (defaults).  PK_ETOOWIDE if slicing cannot meet the limits. */
pk_status pk_plan_create(pk_ctx* ctx, const pk_knot* k, int32_t q, const pk_plan_opts* opts,
                         pk_plan** out);
pk_status pk_plan_info(const pk_plan* p, pk_plan_stats* out);
/* The contraction-order search alone, without slicing or step records (for studies of
 * order quality, Sec. III and Fig. 3): runs `order` (not PK_ORDER_AUTO; `restarts` seeds
 * for PK_ORDER_FILL_SPIN and PK_ORDER_PARTITION, 0 -> 8) on the knot's network for q and
 * writes 4 doubles of the best candidate (fewest indices on its largest tensor, then the
 * least work): out[0] = that largest rank Delta_H (for PK_ORDER_GREEDY_EDGE the paper's
 * maximal degree over the graph minors; otherwise spin indices), out[1] = log2 of the
 * summed R K N of all pairwise steps, out[2] = initial tensors, out[3] = indices.
 * Errors: PK_EINVAL (order, q). */
pk_status pk_order_stats(const pk_knot* k, int32_t q, int32_t order, int32_t restarts, double* out);
/* Device workspace needed by pk_eval / pk_upload / pk_launch at this precision. */
pk_status pk_plan_workspace_bytes(const pk_plan* p, int32_t precision, uint64_t* bytes);
/* Plan introspection for host-side checks: writes n_steps records of 10 int64:
 * (a, b, c, R, K, N, rank_c, kernel, tc, Bsz) with a/b/c tensor ids, the GEMM extents
 * R (batch x free-of-A rows), K, N of one slice, the kernel kind (0 row, 1 split-K,
 * 2 GEMM), the digits per operand when the split precision runs the step on the tensor
 * cores (0 otherwise) and the batch extent (R = Bsz x M). */
pk_status pk_plan_steps(const pk_plan* p, int64_t* rec);
void pk_plan_destroy(pk_plan* p);

/* ---- evaluation --------------------------------------------------------------- */

/* Full evaluation on the context's stream; blocks until Z and V are on the host.
 * d_workspace: device buffer of at least pk_plan_workspace_bytes bytes, owned by the
 * caller; NULL lets the context allocate (and keep) one.  V: the Jones value for knots
 * and links (see pk_link_from_pd for the branch); PK_EINVAL with Z still valid if the
 * exponent 3w + tau + 2 n_v + 2 is not a multiple of 4 (knot) or 2 (link), which a
 * signed graph given by pk_knot_from_signed_graph can violate. */
pk_status pk_eval(pk_ctx* ctx, const pk_plan* p, int32_t precision, void* d_workspace,
                  uint64_t workspace_bytes, pk_scaled* Z, pk_scaled* V);

/* The three stages of pk_eval, asynchronous on the context's stream:
 * pk_upload copies the plan's initial-tensor recipe into the workspace (host->device);
 * pk_launch enqueues every kernel of every slice (the workspace must hold an uploaded
 * recipe of the same plan and precision); the first launch for a given workspace and
 * precision records the sequence into a CUDA graph (on a private stream of the
 * context), later launches replay it, so a plan should keep using the same buffers;
 * pk_download waits for the stream, copies the scaled result back and applies A(q). */
pk_status pk_upload(pk_ctx* ctx, const pk_plan* p, int32_t precision, void* d_workspace,
                    uint64_t workspace_bytes);
/* As pk_upload, but only the knot-derived part of the program: the initial-tensor recipes
 * and their slots (the program's first bytes).  The plan's other records (conversion and
 * sequence-kernel step records) stay as an earlier pk_upload of this plan and precision
 * left them in the same workspace, which the caller must have done (not checked).  For
 * repeated evaluations of the same plan.  *copied (may be NULL): the bytes copied. */
pk_status pk_upload_inputs(pk_ctx* ctx, const pk_plan* p, int32_t precision, void* d_workspace,
                           uint64_t workspace_bytes, uint64_t* copied);
pk_status pk_launch(pk_ctx* ctx, const pk_plan* p, int32_t precision, void* d_workspace,
                    uint64_t workspace_bytes);
pk_status pk_download(pk_ctx* ctx, const pk_plan* p, int32_t precision, const void* d_workspace,
                      pk_scaled* Z, pk_scaled* V);

/* Host-side last stage of pk_download, for checking it without a GPU: `record` is the
 * 32-byte total record an evaluation leaves in its workspace (double re, double im,
 * int64 exp2 of the contracted value, uint64 status word).  Writes Z (the value times the
 * plan's constant factor) and V = A(q) Z (if V is not NULL).  Errors: PK_ENONFINITE when
 * bits 1 and up of the status word hold a finite-check code (((slice + 1) << 24 | (step +
 * 2)) << 1), PK_ETIMEOUT when only bit 0 is set (a bounded device wait gave up); Z is then
 * meaningless; PK_EINVAL as pk_eval for V. */
pk_status pk_decode_result(const pk_plan* p, const void* record, pk_scaled* Z, pk_scaled* V);

/* The workspace of an evaluation is a small per-plan state (initial-tensor program,
 * per-tensor bookkeeping, slice results, split-K scratch: *state_bytes) followed by the
 * tensor arena (*arena_bytes); their sum is pk_plan_workspace_bytes.  They may also
 * live in two separate buffers: pk_upload and pk_download then take the state buffer,
 * and pk_launch_arena takes both (the profile entry point likewise).  Plans whose
 * launches are ordered on one stream may share one arena while each keeps its state
 * (and so its uploaded program) resident. */
pk_status pk_plan_state_bytes(const pk_plan* p, int32_t precision, uint64_t* state_bytes,
                              uint64_t* arena_bytes);
pk_status pk_launch_arena(pk_ctx* ctx, const pk_plan* p, int32_t precision, void* d_state,
                          uint64_t state_bytes, void* d_arena, uint64_t arena_bytes);

/* Internal plan records, for host-side verification of a plan without a GPU.
 * which = 0: the device program (recipe, slot and widening records, as uploaded);
 *         1: the step records; 2: per tensor (arena element offset, elements) int64
 *         pairs; 3: int64 scalars (q, n_init, n_steps, n_slices, n_sliced,
 *         final_tensor, off_recipe, off_slots, n_slots, sizeof step record,
 *         tail_first, n_tail, n_widen, off_widen, final tail offset, folded loops,
 *         their sum of Tait signs);
 *         4: three doubles (re, im, exp2) of the constant factor (loops of the graph)
 *         that multiplies the contracted value; 5: the complex128 tail-step records
 *         of PK_SPLIT.
 * With dst == NULL only *bytes is set.  The record layouts are those of
 * csrc/pk_internal.h (Recipe, Slot, Step, ConvRec, TailStep) and may change between
 * versions. */
pk_status pk_plan_debug_blob(const pk_plan* p, int32_t which, void* dst, uint64_t* bytes);

/* Runs the kernels of pk_launch once (same stream, same workspace, recipe already
 * uploaded; d_arena NULL = the arena inside the workspace, else as pk_launch_arena)
 * with a CUDA event pair around every launch, waits, and returns per kernel
 * class c (0 build, 1 rows: row, thread-per-output and sequence kernels, 2 split-K,
 * 3 results, 4 GEMM on CUDA cores, 5 GEMM on the tensor cores, 6 digit conversion for
 * the tensor-core GEMM): out[c] = milliseconds, out[7+c] = launches, out[14+c] =
 * algorithmic complex multiply-adds, out[21+c] = algorithmic bytes (|A| + |B| + |C| at
 * the precision's element size; for class 6 the operands it reads, |A| + |B|),
 * out[28+c] = milliseconds weighted per launch by the share of the GPU it fills
 * (min(1, CTAs / (multiprocessors x CTAs resident per multiprocessor)): the class's
 * share of a step in which many plans' launches run concurrently).  35 doubles. */
pk_status pk_profile(pk_ctx* ctx, const pk_plan* p, int32_t precision, void* d_workspace,
                     uint64_t workspace_bytes, void* d_arena, uint64_t arena_bytes, double* out);

/* ---- groups of plans run concurrently ------------------------------------------- */

/* n plans, each with its own full workspace (already uploaded with pk_upload), whose
 * launch sequences are recorded as independent branches of one CUDA graph, so the GPU
 * overlaps the plans' (often small, latency-bound) kernels.  pk_group_launch replays
 * it on the context's stream; results are read per plan with pk_download.  The
 * workspaces must stay allocated while the group exists. */
typedef struct pk_group pk_group;
pk_status pk_group_create(pk_ctx* ctx, const pk_plan* const* plans, int32_t n, int32_t precision,
                          void* const* d_workspaces, const uint64_t* workspace_bytes,
                          pk_group** out);
pk_status pk_group_launch(pk_ctx* ctx, pk_group* grp);
/* pk_upload (inputs_only = 0) or pk_upload_inputs (inputs_only != 0) of every plan of the
 * group into its workspace (asynchronous, the context's stream).  *copied (may be NULL):
 * the bytes copied over all plans.  This call and pk_group_download read the group's
 * plans: they must not be destroyed before the group. */
pk_status pk_group_upload(pk_ctx* ctx, pk_group* grp, int32_t inputs_only, uint64_t* copied);
/* The results of every plan of the group after a pk_group_launch: one device->host copy
 * per plan of its 32-byte result record into pinned memory, one wait for the stream, then
 * Z[i] and V[i] (V may be NULL) as pk_download gives them.  status (may be NULL): every
 * plan's pk_download status.  Returns PK_OK, or the first plan's failing status (with the
 * plan index in pk_last_error). */
pk_status pk_group_download(pk_ctx* ctx, pk_group* grp, pk_scaled* Z, pk_scaled* V,
                            int32_t* status);
void pk_group_destroy(pk_group* grp);
/* As pk_group_create, but inside the graph every kernel launch of every plan is
 * bracketed by two CUDA event-record nodes, so one pk_group_launch measures the duration
 * of each launch as it runs among the other plans' launches (the concurrent step, not a
 * serialised pass).  The extra nodes cost a little time per launch: use a separate
 * profiled group for measurement and a plain one for timing. */
pk_status pk_group_create_profiled(pk_ctx* ctx, const pk_plan* const* plans, int32_t n,
                                   int32_t precision, void* const* d_workspaces,
                                   const uint64_t* workspace_bytes, pk_group** out);
/* Waits for the context's stream, then reads the events of the last replay of a
 * profiled group: per kernel class as pk_profile (35 doubles), the milliseconds being the
 * sum over launches of each launch's in-replay duration.  PK_EINVAL for a plain group. */
pk_status pk_group_profile(pk_ctx* ctx, const pk_group* grp, double* out);
/* The last replay of a profiled group as a timeline: per kernel launch 6 doubles (plan
 * index in the group, kernel class as in pk_profile, start and end in milliseconds after
 * the first plan's first launch began -- negative when earlier --, complex multiply-adds,
 * algorithmic bytes), plans in group order, launches in launch order.  Writes at most
 * `capacity` launches and sets *count to the number of launches (PK_ENOMEM when larger
 * than capacity).  Waits for the context's stream first. */
pk_status pk_group_timeline(pk_ctx* ctx, const pk_group* grp, double* out, int64_t capacity,
                            int64_t* count);

/* ---- batched evaluation (many knots in one launch) ------------------------------- */

/* A batch of n planned knots (plans must outlive pk_batch_create only: their data is
 * copied) evaluated together at one precision by one persistent kernel: each CTA takes
 * the next knot from a work counter and performs its whole contraction (Sec. III),
 * so knots of uneven size balance across the GPU without any CTA waiting for another.
 * The counter reset and the launch are recorded once into a CUDA graph per workspace
 * and replayed by every pk_batch_launch. */
typedef struct pk_batch pk_batch;
pk_status pk_batch_create(pk_ctx* ctx, const pk_plan* const* plans, int32_t n, int32_t precision,
                          pk_batch** out);
/* Device workspace for the batch; *upload_bytes (may be NULL) is the part pk_batch_upload
 * copies host->device (knot headers, recipes and steps). */
pk_status pk_batch_workspace_bytes(const pk_batch* b, uint64_t* bytes, uint64_t* upload_bytes);
pk_status pk_batch_upload(pk_ctx* ctx, pk_batch* b, void* d_workspace, uint64_t workspace_bytes);
/* Copies only the knot-derived part of the image (knot headers, initial-tensor recipes and
 * their slots) host->device on the context's stream; the step records and index runs (the
 * plans' structure) stay as an earlier pk_batch_upload of this batch left them in the same
 * workspace, which the caller must have done (they are not checked).  For repeated
 * evaluations of the same planned knots.  *copied (may be NULL): the bytes copied.
 * Errors as pk_batch_upload. */
pk_status pk_batch_upload_inputs(pk_ctx* ctx, pk_batch* b, void* d_workspace,
                                 uint64_t workspace_bytes, uint64_t* copied);
pk_status pk_batch_launch(pk_ctx* ctx, pk_batch* b, void* d_workspace, uint64_t workspace_bytes);
/* Waits for the stream; Z[i], V[i] for knot or link i (V[i] = 0 and PK_EINVAL where the
 * A(q) exponent condition fails). */
pk_status pk_batch_download(pk_ctx* ctx, pk_batch* b, const void* d_workspace, pk_scaled* Z,
                            pk_scaled* V);
/* create + upload + launch + download + destroy. */
pk_status pk_eval_batch(pk_ctx* ctx, const pk_plan* const* plans, int32_t n, int32_t precision,
                        void* d_workspace, uint64_t workspace_bytes, pk_scaled* Z, pk_scaled* V);
void pk_batch_destroy(pk_batch* b);

/* Number of kernel launches pk_launch issues for this plan and precision. */
pk_status pk_plan_launches(const pk_plan* p, int32_t precision, int64_t* launches);

/* Allocation-free evaluation (the paper has no counterpart: this is a deployment aid).
 * Same result as pk_eval, for callers that cannot allocate device memory -- code embedded
 * in a host application whose allocator has reserved the GPU's memory, or a service that
 * forbids allocation once running.  The workspace is a file-scope static device array
 * of 64 MiB (67108864 bytes) that every GPU loading the library holds until exit; no
 * cudaMalloc, cudaFree or other allocating routine is called.  Plans whose
 * pk_plan_workspace_bytes exceeds 64 MiB are refused with PK_ENOMEM and a message in
 * pk_last_error.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it: make that first call
 * before any stream capture.  All calls on a device share the array, which keeps the
 * previous call's contents (each call re-uploads its program and clears its bookkeeping);
 * calls whose GPU work overlaps -- on different streams or contexts of the same device --
 * race on it.  Blocks until Z (and V, as in pk_eval) are on the host. */
pk_status pk_eval_noalloc(pk_ctx* ctx, const pk_plan* p, int32_t precision, pk_scaled* Z,
                          pk_scaled* V);

/* Host-side normalisation only: V = A(q) Z for the knot's (n_v, w, tau) (Eq. JonesPotts). */
pk_status pk_jones_from_z(const pk_knot* k, int32_t q, const pk_scaled* Z, pk_scaled* V);

/* ---- exact evaluation and the Jones polynomial (Sec. "Conclusions and outlook") ---- */

/* Z(q) exactly, modulo each of n_primes primes q < p < 2^31 (checked): at integer q the
 * Potts t is a root of t^2 - (q-2) t + 1, the standard clause entries are integer
 * polynomials in t, and the plan's contraction is run on the GPU in
 * F_p[t]/(t^2 - (q-2) t + 1).  zab[2i], zab[2i+1] = (a, b) with Z = a + b t mod primes[i]
 * (constant factors included).  d_workspace: at least pk_plan_workspace_bytes(PK_C64)
 * (NULL: the context's own); the program is uploaded into it.  Blocks until done.
 * Errors: PK_EINVAL (general weights, a complex128 tail, bad moduli), PK_ETOOWIDE (more
 * than 10^6 slices: each slice is a launch sequence), PK_ENOMEM. */
pk_status pk_eval_exact(pk_ctx* ctx, const pk_plan* p, const uint32_t* primes, int32_t n_primes,
                        void* d_workspace, uint64_t workspace_bytes, uint32_t* zab);

/* All coefficients of V(t) for a knot or link given by its PD code (pk_knot_from_pd or
 * pk_link_from_pd), by interpolation between exact values at integer q = 1, 2, ...: the
 * exponent window comes from the all-A and all-B smoothings (span <= crossings); each q
 * adds two linear equations (the t^0 and t^1 parts of V(t(q)) in
 * Z[t]/(t^2 - (q-2) t + 1)), solved modulo four primes near 2^31 (Z(q) mod p from
 * pk_eval_exact) and lifted to signed 64-bit integers by the Chinese remainder theorem
 * with the fourth prime as a check.  On return V = sum_j coef[j] t^(lowest + j + half/2),
 * j < count (count <= capacity, else PK_ENOMEM with count set); *half = 1 when V has
 * half-integer powers (links with an even number of components; the system is then
 * solved for V t^(-1/2)).  Plans for q up to about crossings/2 + 3 are built and
 * evaluated: feasible while those fit.  Errors: PK_EINVAL (no PD code, a singular or
 * inconsistent system, coefficients beyond 64 bits), PK_ETOOWIDE (a plan too wide). */
pk_status pk_jones_coefficients(pk_ctx* ctx, const pk_knot* k, int32_t capacity, int32_t* lowest,
                                int32_t* count, int64_t* coef, int32_t* half);

/* The two host stages of pk_jones_coefficients (no GPU needed).  pk_jones_plan: the
 * values of q (n_q of them, 1 .. n_q, into qs if not NULL) and the four moduli (into
 * primes if not NULL) the knot's exponent window needs.  pk_jones_solve: the coefficients
 * from zab[2 (iq n_primes + ip) + {0, 1}] = (a, b), Z(qs[iq]) = a + b t mod primes[ip]
 * (as pk_eval_exact gives them); the last modulus checks the reconstruction.  Errors:
 * PK_EINVAL (no PD code, bad moduli, a singular or inconsistent system, coefficients
 * beyond 64 bits), PK_ENOMEM (capacity; count set). */
pk_status pk_jones_plan(const pk_knot* k, int32_t* n_q, int32_t* qs, int32_t* n_primes, uint32_t* primes);
pk_status pk_jones_solve(const pk_knot* k, int32_t n_q, const int32_t* qs, int32_t n_primes,
                         const uint32_t* primes, const uint32_t* zab, int32_t capacity, int32_t* lowest,
                         int32_t* count, int64_t* coef, int32_t* half);

/* ---- reverse pass (adjoint contraction) ------------------------------------------
 *
 * Z = sum over spin states of prod_e T_e[s_u, s_v] (Sec. II) is linear in every entry
 * of every clause matrix T_e, so dZ/dT_e[a, b] is the same sum restricted to
 * s_u = a, s_v = b with T_e left out: (T_e[a,b] / Z) dZ/dT_e[a,b] is the (complex) joint
 * distribution of the two spins of edge e ("edge-resolved Potts correlations").  pk_grad
 * computes every dZ/dT_e in one reverse pass over the plan's contraction tree: for a step
 * C = sum A B the adjoints are dZ/dA = sum C' B and dZ/dB = sum A C' (C' = dZ/dC; no
 * complex conjugate: Z is holomorphic in every entry), each again a pairwise contraction
 * run by the same kernels, with the forward intermediates kept at every
 * pk_plan_opts.checkpoint_stride-th tree level and the others recomputed.  Parallel
 * edges share one tensor M = prod T_e (entrywise); dZ/dT_e = dZ/dM * prod_{e' != e} T_e'. */

/* Device workspace of pk_grad for a plan made with PK_FLAG_GRAD. */
pk_status pk_grad_workspace_bytes(const pk_plan* p, int32_t precision, uint64_t* bytes);

/* Z, V and the reverse pass.  d_workspace: NULL (the context's own buffer) or at least
 * pk_grad_workspace_bytes, 256-byte aligned.  dlogZ_dT (may be NULL): 2*n_e*q*q
 * doubles, entry ((e*q + a)*q + b) = re, im of (1/Z) dZ/dT_e[a, b] with a the spin of
 * edge e's first vertex and b of its second (pk_knot_edges order); for a loop only
 * a == b is defined, off-diagonal entries are 0.  dlogV_dt (may be NULL): 2 doubles,
 * (1/V) dV/dt at fixed q: the network's dimension q stays fixed while t moves through
 * the clause weights -t^-eps and through A = (-1)^(w+n_v+1) t^k (t+1)^-(n_v+1), giving
 * k/t - (n_v+1)/(t+1) + sum_e eps_e t^(-eps_e-1) sum_a (1/Z) dZ/dT_e[a,a].  It is not the
 * derivative of the Jones polynomial (which would move q as well); NaN when the plan's
 * weights are not the standard ones.  Errors: PK_EINVAL (plan without PK_FLAG_GRAD),
 * PK_EZERO (Z = 0), PK_ENOMEM, PK_ECUDA.  Blocks until the results are on the host. */
pk_status pk_grad(pk_ctx* ctx, const pk_plan* p, int32_t precision, void* d_workspace,
                  uint64_t workspace_bytes, pk_scaled* Z, pk_scaled* V, double* dlogZ_dT,
                  double* dlogV_dt);

/* Host-side last stage of pk_grad, for checking it without a GPU: acc holds, per edge
 * group g of the plan (pk_grad_stats out[7] groups), 2*q*q doubles of dZ/dM_g scaled by
 * 2^-acc_exp[g] (row-major over (spin of the group's lower vertex, spin of the higher);
 * a loop uses the first q entries), and Z.  Writes dlogZ_dT and dlogV_dt as pk_grad. */
pk_status pk_grad_from_accumulators(const pk_plan* p, const double* acc, const int64_t* acc_exp,
                                    const pk_scaled* Z, double* dlogZ_dT, double* dlogV_dt);

/* d log Z with respect to each Tait edge's two clause weights (the diagonal entry d_e and
 * the off-diagonal entry o_e of pk_plan_opts.edge_weights: T_e[a,a] = d_e, T_e[a,b] = o_e
 * for a != b), from pk_grad's dlogZ_dT (same layout): out[4e..4e+3] = re, im of
 * sum_a dlogZ_dT[e,a,a] and of sum_{a != b} dlogZ_dT[e,a,b] (holomorphic derivatives).
 * Host only. */
pk_status pk_grad_weights(const pk_plan* p, const double* dlogZ_dT, double* out);

/* Reverse-program statistics of a PK_FLAG_GRAD plan, 10 doubles: complex multiply-adds
 * per slice of the forward, recompute and adjoint steps; their step counts; arena
 * elements; forward intermediates kept as checkpoints; edge groups; slices. */
pk_status pk_grad_stats(const pk_plan* p, double* out);

/* New clause weights for a plan made with PK_FLAG_GRAD or edge_weights (same layout as
 * pk_plan_opts.edge_weights; NULL restores the standard weights of t(q)).  The order,
 * slicing and arena are unchanged; the next pk_upload / pk_eval / pk_grad uses them. */
pk_status pk_plan_set_weights(pk_plan* p, const double* edge_weights);

/* ---- debugging aids and slice-level resume ---------------------------------------- */

/* Debug flags of a context (0 by default).  While any is set, pk_launch and
 * pk_launch_arena (so pk_eval) enqueue the plan's kernels directly instead of replaying a
 * recorded graph; groups (pk_group_*), the batch executor, pk_grad, pk_eval_exact and
 * pk_eval_noalloc ignore them. */
#define PK_DEBUG_CHECK_FINITE 1 /* after the initial tensors and after every step (sequence
                                   runs split into single steps) scan the tensor just
                                   written for NaN / Inf; the first one found is reported by
                                   pk_download as PK_ENONFINITE                            */
#define PK_DEBUG_VERIFY 2       /* pk_plan_verify before every launch (PK_EINVAL on failure) */
#define PK_DEBUG_NVTX 4         /* an NVTX range around every kernel launch, named
                                   "step <i> <class>" (i = -1 for the initial tensors and the
                                   slice results; class as pk_profile's)                    */
pk_status pk_ctx_set_debug(pk_ctx* ctx, int32_t flags);

/* Host-side check of a plan's index maps and memory layout for `precision`, without a GPU.
 * Every gather and scatter of a step is an affine map given by stride runs, so it is
 * checked exhaustively: A's row and contracted runs (and B's batch, contracted and column
 * runs, and in the GEMM view C's runs) enumerate the operand's dense tensor exactly once
 * with extents R, K, N (Bsz, M); each step reads live tensors and writes its own; every
 * tensor lies inside the arena on a 512-byte boundary, and tensors live at the same step do
 * not overlap; sequence-kernel records equal their steps; the complex128 tail, the split
 * precision's digit scratch, the reverse program (PK_FLAG_GRAD) and the state records fit
 * the workspace of pk_plan_workspace_bytes.  PK_EINVAL with the first violation in msg
 * (NUL-terminated, at most msg_bytes; msg may be NULL). */
pk_status pk_plan_verify(const pk_plan* p, int32_t precision, char* msg, uint64_t msg_bytes);

/* Slices [first, first + count) of an evaluation (Sec. III: a sliced contraction is a sum
 * of independent sub-contractions with the sliced indices fixed; pk_plan_stats gives
 * n_slices): uploads the program, enqueues those slices directly (no graph; the context's
 * debug flags apply), waits, and writes each slice's contracted value -- without the
 * plan's constant factor -- to slices[0 .. count).  The values are plain data: a caller
 * can store them and resume a long evaluation from the first slice not yet done.
 * d_workspace as pk_eval.  Errors: PK_EINVAL (range), PK_ETIMEOUT / PK_ENONFINITE as
 * pk_download for the slices run. */
pk_status pk_eval_slices(pk_ctx* ctx, const pk_plan* p, int32_t precision, void* d_workspace,
                         uint64_t workspace_bytes, int64_t first, int64_t count,
                         pk_scaled* slices);
/* Z and V (NULL: not wanted) from all n = n_slices per-slice values of pk_eval_slices, in
 * slice order: summed at the largest exponent with compensated (Kahan) sums, times the
 * plan's constant factor, V = A(q) Z as pk_download.  Host only. */
pk_status pk_combine_slices(const pk_plan* p, const pk_scaled* slices, int64_t n, pk_scaled* Z,
                            pk_scaled* V);

#ifdef __cplusplus
}
#endif
#endif /* PK_H */
