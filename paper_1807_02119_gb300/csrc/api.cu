// C ABI (include/pk.h): handles, argument checks, workspace handling and the host-side
// normalisation V = A(q) Z (Eq. JonesPotts).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "pk_internal.h"

#include "exact_ring.h"
#include "handles.h"

namespace {

pk_status fail(pk_ctx* c, pk_status s, const std::string& m) {
  if (c) c->err = m;
  return s;
}
pk_status cuda_fail(pk_ctx* c, cudaError_t e, const char* where) {
  return fail(c, PK_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
int elem_bytes(int32_t precision) { return precision == PK_C128 ? 16 : 8; }
bool valid_precision(int32_t p) { return p == PK_C128 || p == PK_C64 || p == PK_SPLIT; }

pk_scaled to_abi(const pk::Scaled& s) {
  pk_scaled r;
  r.re = s.re;
  r.im = s.im;
  r.exp2 = s.e;
  return r;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (dev >= 0 && dev != prev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

pk_status check_ws_need(pk_ctx* ctx, uint64_t need, void*& ws, uint64_t& bytes) {
  if (ws == nullptr) {
    if (ctx->own_ws_bytes < need) {
      if (ctx->own_ws) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->own_ws);
        ctx->own_ws = nullptr;
        ctx->own_ws_bytes = 0;
      }
      cudaError_t e = cudaMalloc(&ctx->own_ws, need);
      if (e != cudaSuccess) return fail(ctx, PK_ENOMEM, "workspace cudaMalloc failed");
      ctx->own_ws_bytes = need;
    }
    ws = ctx->own_ws;
    bytes = ctx->own_ws_bytes;
  }
  if (bytes < need) return fail(ctx, PK_ENOMEM, "workspace smaller than the plan needs");
  if (((uintptr_t)ws & 255u) != 0) return fail(ctx, PK_EINVAL, "workspace must be 256-byte aligned");
  return PK_OK;
}

pk_status check_ws(pk_ctx* ctx, const pk_plan* p, int32_t precision, void*& ws, uint64_t& bytes) {
  return check_ws_need(ctx, p->p.ws_bytes(precision), ws, bytes);
}

// Enqueues the plan's kernels on the context's stream.  The launch sequence is recorded
// once into a CUDA graph on the context's private capture stream (for this state
// buffer, arena and precision) and replayed afterwards; very long sequences (many
// slices) are launched directly.
pk_status launch_recorded(pk_ctx* ctx, const pk_plan* p, int32_t precision, void* ws, void* arena) {
  const pk::Plan& P = p->p;
  if (ctx->debug) {  // debugging aids: verified, checked launches enqueued directly
    if (ctx->debug & PK_DEBUG_VERIFY) {
      std::string err;
      if (!pk::verify_plan(P, precision, err)) return fail(ctx, PK_EINVAL, "pk_plan_verify: " + err);
    }
    pk::LaunchOpts o;
    o.check_finite = (ctx->debug & PK_DEBUG_CHECK_FINITE) != 0;
    o.nvtx = (ctx->debug & PK_DEBUG_NVTX) != 0;
    cudaError_t e = pk::launch_plan_opts(P, precision, ws, arena, ctx->stream, o);
    return e == cudaSuccess ? PK_OK : cuda_fail(ctx, e, "launch");
  }
  const double nodes = (double)P.n_slices * (double)(P.steps.size() + 4);
  if (nodes > 20000.0) {
    cudaError_t e = pk::launch_plan(P, precision, ws, arena, ctx->stream);
    return e == cudaSuccess ? PK_OK : cuda_fail(ctx, e, "launch");
  }
  PlanGraph& g = const_cast<pk_plan*>(p)->graph;
  if (!(g.exec && g.ws == ws && g.arena == arena && g.precision == precision)) {
    if (g.exec) {
      cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
    }
    cudaError_t e = pk::prepare_kernels();
    if (e == cudaSuccess && !ctx->capture)
      e = cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "graph set-up");
    e = cudaStreamBeginCapture(ctx->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "begin capture");
    cudaError_t e1 = pk::launch_plan(P, precision, ws, arena, ctx->capture);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(ctx->capture, &graph);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail(ctx, e1 != cudaSuccess ? e1 : e2, "record launch sequence");
    }
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      g.exec = nullptr;
      return cuda_fail(ctx, e, "instantiate graph");
    }
    g.ws = ws;
    g.arena = arena;
    g.precision = precision;
  }
  cudaError_t e = cudaGraphLaunch(g.exec, ctx->stream);
  return e == cudaSuccess ? PK_OK : cuda_fail(ctx, e, "graph launch");
}

}  // namespace

namespace pk {

pk_status status_error(unsigned long long status, std::string& err) {
  if (status >> 1) {
    err = "the finite check found NaN or Inf in the result of step " +
          std::to_string(nonfinite_step(status)) + " of slice " +
          std::to_string(nonfinite_slice(status)) + " (step -1: an initial tensor)";
    return PK_ENONFINITE;
  }
  if (status != 0) {
    err = "a bounded wait of the tensor-core GEMM gave up: the result is invalid (status " +
          std::to_string(status) + ")";
    return PK_ETIMEOUT;
  }
  return PK_OK;
}

pk_status decode_total(const Plan& P, const SliceResult& r, pk_scaled* Z, pk_scaled* V,
                       std::string& err) {
  Scaled z;
  z.re = r.re;
  z.im = r.im;
  z.e = r.exp;
  z.norm();
  z = s_mul(z, P.factor);
  *Z = to_abi(z);
  const pk_status st = status_error(r.status, err);
  if (st != PK_OK) return st;
  if (V) {
    if (!jones_defined(P.knot)) {
      err = "3w + tau + 2 n_v + 2 not divisible by 4 (knot) or 2 (link)";
      return PK_EINVAL;
    }
    *V = to_abi(s_mul(jones_prefactor(P.knot, P.q), z));
  }
  return PK_OK;
}

}  // namespace pk

extern "C" {

pk_status pk_ctx_create(int32_t device, void* stream, pk_ctx** out) {
  if (!out) return PK_EINVAL;
  *out = nullptr;
  pk_ctx* c = new (std::nothrow) pk_ctx();
  if (!c) return PK_ENOMEM;
  c->device = device;
  c->stream = (cudaStream_t)stream;
  if (device >= 0) {
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device >= n) {
      delete c;
      return PK_ENODEVICE;
    }
    DeviceGuard g(device);
    if (cudaMallocHost((void**)&c->pinned_result, sizeof(pk::SliceResult)) != cudaSuccess) {
      delete c;
      return PK_ECUDA;
    }
  }
  *out = c;
  return PK_OK;
}

pk_status pk_tuning_default(pk_tuning* out) {
  if (!out) return PK_EINVAL;
  *out = kTunedDefault;
  return PK_OK;
}

pk_status pk_ctx_set_tuning(pk_ctx* ctx, const pk_tuning* t) {
  if (!ctx) return PK_EINVAL;
  if (!t) {
    ctx->tuning = kTunedDefault;
    return PK_OK;
  }
  if (!pk::valid_tuning(*t)) return fail(ctx, PK_EINVAL, "tuning value out of range");
  ctx->tuning = *t;
  return PK_OK;
}

pk_status pk_ctx_set_debug(pk_ctx* ctx, int32_t flags) {
  if (!ctx) return PK_EINVAL;
  if (flags & ~(PK_DEBUG_CHECK_FINITE | PK_DEBUG_VERIFY | PK_DEBUG_NVTX))
    return fail(ctx, PK_EINVAL, "unknown debug flag");
  ctx->debug = flags;
  return PK_OK;
}

pk_status pk_plan_verify(const pk_plan* p, int32_t precision, char* msg, uint64_t msg_bytes) {
  if (!p || !valid_precision(precision)) return PK_EINVAL;
  std::string err;
  const bool ok = pk::verify_plan(p->p, precision, err);
  if (msg && msg_bytes > 0) {
    const size_t n = std::min<size_t>(err.size(), (size_t)msg_bytes - 1);
    std::memcpy(msg, err.data(), n);
    msg[n] = 0;
  }
  return ok ? PK_OK : PK_EINVAL;
}

pk_status pk_ctx_set_hbm_budget(pk_ctx* ctx, uint64_t bytes) {
  if (!ctx) return PK_EINVAL;
  ctx->hbm_budget = bytes;
  return PK_OK;
}

pk_status pk_ctx_get_tuning(const pk_ctx* ctx, pk_tuning* out) {
  if (!ctx || !out) return PK_EINVAL;
  *out = ctx->tuning;
  return PK_OK;
}

pk_status pk_ctx_set_stream(pk_ctx* ctx, void* stream) {
  if (!ctx) return PK_EINVAL;
  ctx->stream = (cudaStream_t)stream;
  return PK_OK;
}

const char* pk_last_error(const pk_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void pk_ctx_destroy(pk_ctx* ctx) {
  if (!ctx) return;
  if (ctx->device >= 0) {
    DeviceGuard g(ctx->device);
    if (ctx->own_ws) {
      cudaStreamSynchronize(ctx->stream);
      cudaFree(ctx->own_ws);
    }
    if (ctx->pinned_result) cudaFreeHost(ctx->pinned_result);
    if (ctx->capture) cudaStreamDestroy(ctx->capture);
  }
  delete ctx;
}

pk_status pk_knot_from_pd(pk_ctx* ctx, const int32_t* pd, int32_t n, int32_t outer_arc,
                          int32_t outer_side, pk_knot** out) {
  if (!out) return fail(ctx, PK_EINVAL, "null output");
  *out = nullptr;
  pk_knot* k = new (std::nothrow) pk_knot();
  if (!k) return fail(ctx, PK_ENOMEM, "out of host memory");
  std::string err;
  if (!pk::knot_from_pd(pd, n, outer_arc, outer_side, k->k, err)) {
    delete k;
    return fail(ctx, PK_EINVAL, err);
  }
  *out = k;
  return PK_OK;
}

pk_status pk_link_from_pd(pk_ctx* ctx, const int32_t* pd, const int32_t* signs, int32_t n,
                          int32_t outer_arc, int32_t outer_side, pk_knot** out) {
  if (!out) return fail(ctx, PK_EINVAL, "null output");
  *out = nullptr;
  if (n > 0 && !signs) return fail(ctx, PK_EINVAL, "null twist signs");
  pk_knot* k = new (std::nothrow) pk_knot();
  if (!k) return fail(ctx, PK_ENOMEM, "out of host memory");
  std::string err;
  if (!pk::knot_from_pd(pd, n, outer_arc, outer_side, k->k, err, signs)) {
    delete k;
    return fail(ctx, PK_EINVAL, err);
  }
  *out = k;
  return PK_OK;
}

pk_status pk_knot_from_signed_graph(pk_ctx* ctx, int32_t n_v, int32_t n_e, const int32_t* uve,
                                    int32_t writhe, pk_knot** out) {
  if (!out) return fail(ctx, PK_EINVAL, "null output");
  *out = nullptr;
  pk_knot* k = new (std::nothrow) pk_knot();
  if (!k) return fail(ctx, PK_ENOMEM, "out of host memory");
  std::string err;
  if (!pk::knot_from_graph(n_v, n_e, uve, writhe, k->k, err)) {
    delete k;
    return fail(ctx, PK_EINVAL, err);
  }
  *out = k;
  return PK_OK;
}

pk_status pk_knot_from_grid_walk(pk_ctx* ctx, int32_t L, uint64_t seed, int32_t random_over_under,
                                 int32_t ncross_min, int32_t ncross_max, pk_knot** out) {
  if (!out) return fail(ctx, PK_EINVAL, "null output");
  *out = nullptr;
  std::vector<std::array<int32_t, 4>> pd;
  int32_t oa, os;
  std::string err;
  if (!pk::grid_walk_pd(L, seed, random_over_under != 0, ncross_min, ncross_max, pd, oa, os, err))
    return fail(ctx, PK_EINVAL, err);
  std::vector<int32_t> flat(4 * pd.size());
  for (size_t i = 0; i < pd.size(); ++i)
    for (int j = 0; j < 4; ++j) flat[4 * i + j] = pd[i][j];
  return pk_knot_from_pd(ctx, flat.data(), (int32_t)pd.size(), oa, os, out);
}

pk_status pk_knot_simplify(pk_ctx* ctx, const pk_knot* k, pk_knot** out) {
  if (!out || !k) return fail(ctx, PK_EINVAL, "null argument");
  *out = nullptr;
  pk_knot* r = new (std::nothrow) pk_knot();
  if (!r) return fail(ctx, PK_ENOMEM, "out of host memory");
  pk::simplify_knot(k->k, r->k);
  *out = r;
  return PK_OK;
}

pk_status pk_knot_info(const pk_knot* k, int32_t* n_v, int32_t* n_c, int32_t* writhe,
                       int32_t* tau, int32_t* components) {
  if (!k) return PK_EINVAL;
  if (n_v) *n_v = k->k.n_v;
  if (n_c) *n_c = k->k.n_c;
  if (writhe) *writhe = k->k.writhe;
  if (tau) *tau = k->k.tau;
  if (components) *components = k->k.components;
  return PK_OK;
}

pk_status pk_knot_edges(const pk_knot* k, int32_t* uve) {
  if (!k || (!uve && k->k.n_c > 0)) return PK_EINVAL;
  for (size_t e = 0; e < k->k.edges.size(); ++e)
    for (int j = 0; j < 3; ++j) uve[3 * e + j] = k->k.edges[e][j];
  return PK_OK;
}

pk_status pk_knot_pd(const pk_knot* k, int32_t* pd) {
  if (!k || !k->k.has_pd || (!pd && k->k.n_c > 0)) return PK_EINVAL;
  for (size_t i = 0; i < k->k.pd.size(); ++i)
    for (int j = 0; j < 4; ++j) pd[4 * i + j] = k->k.pd[i][j];
  return PK_OK;
}

void pk_knot_destroy(pk_knot* k) { delete k; }

pk_status pk_plan_create(pk_ctx* ctx, const pk_knot* k, int32_t q, const pk_plan_opts* opts,
                         pk_plan** out) {
  if (!out || !k) return fail(ctx, PK_EINVAL, "null argument");
  *out = nullptr;
  if (q < 1) return fail(ctx, PK_EINVAL, "q must be >= 1");
  pk_plan_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  pk_plan* p = new (std::nothrow) pk_plan();
  if (!p) return fail(ctx, PK_ENOMEM, "out of host memory");
  std::string err;
  const uint64_t budget = ctx ? ctx->hbm_budget : 0;
  for (;;) {
    if (!pk::make_plan(k->k, q, o, ctx ? ctx->tuning : kTunedDefault, p->p, err)) {
      delete p;
      if (err.find("slices") != std::string::npos || err.find("runs") != std::string::npos)
        return fail(ctx, PK_ETOOWIDE, err);
      return fail(ctx, PK_EINVAL, err);
    }
    const pk::Plan& P = p->p;
    const uint64_t need = std::max(P.ws_bytes(PK_C128), std::max(P.ws_bytes(PK_SPLIT), P.ws_bytes(PK_C64)));
    if (budget == 0 || need <= budget) break;
    // over the device-memory budget: one index fewer on the largest tensor (more slices)
    const double lq = std::log2((double)q);
    if (q < 2 || P.max_rank <= 1) {
      delete p;
      return fail(ctx, PK_ETOOWIDE, "no slicing fits the device-memory budget");
    }
    o.max_log2_elems = (P.max_rank - 1) * lq + 1e-9;
  }
  *out = p;
  return PK_OK;
}

pk_status pk_order_stats(const pk_knot* k, int32_t q, int32_t order, int32_t restarts, double* out) {
  if (!k || !out) return PK_EINVAL;
  return pk::order_stats(k->k, q, order, restarts, out) ? PK_OK : PK_EINVAL;
}

pk_status pk_plan_info(const pk_plan* p, pk_plan_stats* out) {
  if (!p || !out) return PK_EINVAL;
  const pk::Plan& P = p->p;
  out->log2_max_elems = P.log2_max_elems;
  out->cmacs = P.cmacs;
  out->bytes_c64 = P.bytes_c64;
  out->n_slices = P.n_slices;
  out->n_steps = (int32_t)P.steps.size();
  out->max_rank = P.max_rank;
  out->order_used = P.order_used;
  out->n_tensors = P.n_init;
  out->workspace_c128 = P.ws_bytes(PK_C128);
  out->workspace_c64 = P.ws_bytes(PK_C64);
  out->workspace_split = P.ws_bytes(PK_SPLIT);
  int32_t seg_steps = 0;
  for (const pk::Segment& g : P.segments) seg_steps += g.count;
  out->n_segments = (int32_t)P.segments.size();
  out->n_segment_steps = seg_steps;
  out->est_cost = P.est_cost;
  return PK_OK;
}

pk_status pk_plan_workspace_bytes(const pk_plan* p, int32_t precision, uint64_t* bytes) {
  if (!p || !bytes || !valid_precision(precision)) return PK_EINVAL;
  *bytes = p->p.ws_bytes(precision);
  return PK_OK;
}

pk_status pk_plan_steps(const pk_plan* p, int64_t* rec) {
  if (!p || (!rec && !p->p.steps.empty())) return PK_EINVAL;
  for (size_t i = 0; i < p->p.steps.size(); ++i) {
    const pk::Step& s = p->p.steps[i];
    int64_t* r = rec + 10 * i;
    r[0] = s.a;
    r[1] = s.b;
    r[2] = s.c;
    r[3] = s.R;
    r[4] = s.K;
    r[5] = s.N;
    r[6] = s.rank_c;
    r[7] = s.kernel;
    r[8] = s.tc;
    r[9] = s.Bsz;
  }
  return PK_OK;
}

pk_status pk_plan_debug_blob(const pk_plan* p, int32_t which, void* dst, uint64_t* bytes) {
  if (!p || !bytes) return PK_EINVAL;
  const pk::Plan& P = p->p;
  std::vector<uint8_t> buf;
  if (which == 0) {
    buf = P.program;
  } else if (which == 1) {
    buf.resize(sizeof(pk::Step) * P.steps.size());
    if (!P.steps.empty()) std::memcpy(buf.data(), P.steps.data(), buf.size());
  } else if (which == 2) {
    std::vector<int64_t> v;
    for (const auto& t : P.tensors) {
      v.push_back(t.offset);
      v.push_back(t.elems);
    }
    buf.resize(8 * v.size());
    if (!v.empty()) std::memcpy(buf.data(), v.data(), buf.size());
  } else if (which == 3) {
    int64_t v[17] = {P.q, P.n_init, (int64_t)P.steps.size(), P.n_slices, (int64_t)P.sliced.size(),
                     P.final_tensor, (int64_t)P.off_recipe, (int64_t)P.off_slots,
                     (int64_t)P.slots.size(), (int64_t)sizeof(pk::Step), P.tail_first,
                     (int64_t)P.tail.size(), (int64_t)P.conv.size(), (int64_t)P.off_conv,
                     P.final_tail_off, P.loop_count, P.loop_signsum};
    buf.resize(sizeof(v));
    std::memcpy(buf.data(), v, sizeof(v));
  } else if (which == 5) {
    buf.resize(sizeof(pk::TailStep) * P.tail.size());
    if (!P.tail.empty()) std::memcpy(buf.data(), P.tail.data(), buf.size());
  } else if (which == 4) {
    double v[3] = {P.factor.re, P.factor.im, (double)P.factor.e};
    buf.resize(sizeof(v));
    std::memcpy(buf.data(), v, sizeof(v));
  } else if (which >= 6 && which <= 9 && P.grad.built) {
    const pk::GradProgram& G = P.grad;
    if (which == 6) {
      buf.resize(sizeof(pk::Step) * G.steps.size());
      if (!G.steps.empty()) std::memcpy(buf.data(), G.steps.data(), buf.size());
    } else if (which == 7) {
      int64_t v[16] = {(int64_t)G.steps.size(), G.n_meta, G.arena_elems, G.root_offset,
                       G.root_meta, (int64_t)G.off_recipe, (int64_t)G.off_slots,
                       (int64_t)G.off_leaves, (int64_t)G.leaves.size(), P.n_slices,
                       (int64_t)sizeof(pk::GradLeaf), P.n_init, (int64_t)P.slots.size(), P.q,
                       (int64_t)P.sliced.size(), (int64_t)sizeof(pk::Slot)};
      buf.resize(sizeof(v));
      std::memcpy(buf.data(), v, sizeof(v));
    } else if (which == 8) {
      buf = G.program;
    } else {
      buf.resize(G.phase.size());
      if (!G.phase.empty()) std::memcpy(buf.data(), G.phase.data(), buf.size());
    }
  } else {
    return PK_EINVAL;
  }
  if (dst) {
    if (*bytes < buf.size()) return PK_ENOMEM;
    if (!buf.empty()) std::memcpy(dst, buf.data(), buf.size());
  }
  *bytes = buf.size();
  return PK_OK;
}

pk_status pk_plan_launches(const pk_plan* p, int32_t precision, int64_t* launches) {
  if (!p || !launches || !valid_precision(precision)) return PK_EINVAL;
  const pk::Plan& P = p->p;
  const int64_t widen = (precision == PK_C64 && !P.conv.empty()) ? 1 : 0;
  const int64_t digits = precision == PK_SPLIT ? (int64_t)P.n_tc : 0;  // one conversion launch per tensor-core step
  int64_t fused = 0;  // steps saved by sequence launches (runs of small steps)
  for (const pk::Segment& g : P.segments)
    if (precision != PK_C64 || g.first + g.count <= P.tail_first) fused += g.count - 1;
  *launches = P.n_slices * ((P.n_init > 0 ? 1 : 0) + (int64_t)P.steps.size() - fused + 1 + widen +
                            digits) + 1;
  return PK_OK;
}

void pk_plan_destroy(pk_plan* p) {
  if (!p) return;
  if (p->pinned_program) cudaFreeHost(p->pinned_program);
  if (p->pinned_grad) cudaFreeHost(p->pinned_grad);
  if (p->graph.exec) cudaGraphExecDestroy(p->graph.exec);
  if (p->grad_graph.exec) cudaGraphExecDestroy(p->grad_graph.exec);
  delete p;
}

pk_status pk_upload(pk_ctx* ctx, const pk_plan* p, int32_t precision, void* d_workspace,
                    uint64_t workspace_bytes) {
  if (!ctx || !p || !valid_precision(precision)) return fail(ctx, PK_EINVAL, "bad argument");
  if (ctx->device < 0) return fail(ctx, PK_ENODEVICE, "host-only context");
  DeviceGuard g(ctx->device);
  pk_status s = PK_OK;
  if (d_workspace == nullptr)
    s = check_ws(ctx, p, precision, d_workspace, workspace_bytes);
  else if (workspace_bytes < p->p.off_arena)
    s = fail(ctx, PK_ENOMEM, "buffer smaller than the plan state (pk_plan_state_bytes)");
  if (s != PK_OK) return s;
  const pk::Plan& P = p->p;
  if (P.program.empty()) return PK_OK;
  pk_plan* mp = const_cast<pk_plan*>(p);
  if (!mp->pinned_program) {
    if (cudaMallocHost((void**)&mp->pinned_program, P.program.size()) != cudaSuccess)
      return fail(ctx, PK_ENOMEM, "pinned host allocation failed");
    std::memcpy(mp->pinned_program, P.program.data(), P.program.size());
  }
  cudaError_t e = cudaMemcpyAsync(d_workspace, mp->pinned_program, P.program.size(),
                                  cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "upload");
  return PK_OK;
}

pk_status pk_upload_inputs(pk_ctx* ctx, const pk_plan* p, int32_t precision, void* d_workspace,
                           uint64_t workspace_bytes, uint64_t* copied) {
  if (!ctx || !p || !valid_precision(precision)) return fail(ctx, PK_EINVAL, "bad argument");
  if (ctx->device < 0) return fail(ctx, PK_ENODEVICE, "host-only context");
  DeviceGuard g(ctx->device);
  pk_status s = PK_OK;
  if (d_workspace == nullptr)
    s = check_ws(ctx, p, precision, d_workspace, workspace_bytes);
  else if (workspace_bytes < p->p.off_arena)
    s = fail(ctx, PK_ENOMEM, "buffer smaller than the plan state (pk_plan_state_bytes)");
  if (s != PK_OK) return s;
  const pk::Plan& P = p->p;
  // recipes and slots lie first in the program, the conversion and sequence records after
  const uint64_t n = std::min<uint64_t>(P.off_conv, P.program.size());
  if (copied) *copied = n;
  if (n == 0) return PK_OK;
  pk_plan* mp = const_cast<pk_plan*>(p);
  if (!mp->pinned_program) {
    if (cudaMallocHost((void**)&mp->pinned_program, P.program.size()) != cudaSuccess)
      return fail(ctx, PK_ENOMEM, "pinned host allocation failed");
    std::memcpy(mp->pinned_program, P.program.data(), P.program.size());
  }
  cudaError_t e = cudaMemcpyAsync(d_workspace, mp->pinned_program, n, cudaMemcpyHostToDevice,
                                  ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "upload");
  return PK_OK;
}

pk_status pk_launch(pk_ctx* ctx, const pk_plan* p, int32_t precision, void* d_workspace,
                    uint64_t workspace_bytes) {
  if (!ctx || !p || !valid_precision(precision)) return fail(ctx, PK_EINVAL, "bad argument");
  if (ctx->device < 0) return fail(ctx, PK_ENODEVICE, "host-only context");
  DeviceGuard g(ctx->device);
  pk_status s = check_ws(ctx, p, precision, d_workspace, workspace_bytes);
  if (s != PK_OK) return s;
  return launch_recorded(ctx, p, precision, d_workspace, (char*)d_workspace + p->p.off_arena);
  return PK_OK;
}

static pk_status check_split(pk_ctx* ctx, const pk_plan* p, int32_t precision, const void* state,
                             uint64_t state_bytes, const void* arena, uint64_t arena_bytes) {
  const uint64_t need_state = p->p.off_arena;
  const uint64_t need_arena = p->p.ws_bytes(precision) - p->p.off_arena;
  if (!state || !arena) return fail(ctx, PK_EINVAL, "null state or arena");
  if (state_bytes < need_state || arena_bytes < need_arena)
    return fail(ctx, PK_ENOMEM, "state or arena smaller than pk_plan_state_bytes");
  if ((((uintptr_t)state) & 255u) || (((uintptr_t)arena) & 255u))
    return fail(ctx, PK_EINVAL, "state and arena must be 256-byte aligned");
  return PK_OK;
}

pk_status pk_plan_state_bytes(const pk_plan* p, int32_t precision, uint64_t* state_bytes,
                              uint64_t* arena_bytes) {
  if (!p || !state_bytes || !arena_bytes || !valid_precision(precision)) return PK_EINVAL;
  *state_bytes = p->p.off_arena;
  *arena_bytes = p->p.ws_bytes(precision) - p->p.off_arena;
  return PK_OK;
}

pk_status pk_launch_arena(pk_ctx* ctx, const pk_plan* p, int32_t precision, void* d_state,
                          uint64_t state_bytes, void* d_arena, uint64_t arena_bytes) {
  if (!ctx || !p || !valid_precision(precision)) return fail(ctx, PK_EINVAL, "bad argument");
  if (ctx->device < 0) return fail(ctx, PK_ENODEVICE, "host-only context");
  DeviceGuard g(ctx->device);
  pk_status s = check_split(ctx, p, precision, d_state, state_bytes, d_arena, arena_bytes);
  if (s != PK_OK) return s;
  return launch_recorded(ctx, p, precision, d_state, d_arena);
}

pk_status pk_profile(pk_ctx* ctx, const pk_plan* p, int32_t precision, void* d_workspace,
                     uint64_t workspace_bytes, void* d_arena, uint64_t arena_bytes, double* out) {
  if (!ctx || !p || !out || !valid_precision(precision)) return fail(ctx, PK_EINVAL, "bad argument");
  if (ctx->device < 0) return fail(ctx, PK_ENODEVICE, "host-only context");
  DeviceGuard g(ctx->device);
  pk_status s;
  if (d_arena == nullptr) {
    s = check_ws(ctx, p, precision, d_workspace, workspace_bytes);
    d_arena = (char*)d_workspace + p->p.off_arena;
  } else {
    s = check_split(ctx, p, precision, d_workspace, workspace_bytes, d_arena, arena_bytes);
  }
  if (s != PK_OK) return s;
  cudaError_t e = pk::profile_plan(p->p, precision, d_workspace, d_arena, ctx->stream, out);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "profile");
  return PK_OK;
}

}  // extern "C"

struct pk_group {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int32_t n = 0;
  int32_t precision = 0;
  std::vector<const pk_plan*> plans;
  std::vector<void*> ws;
  std::vector<uint64_t> ws_bytes;
  pk::SliceResult* pinned = nullptr;   // every plan's total result record (pk_group_download)
  std::vector<pk::Prof*> profs;   // profiled groups: the per-launch events of every branch
};

namespace {

pk_status group_create(pk_ctx* ctx, const pk_plan* const* plans, int32_t n, int32_t precision,
                       void* const* d_workspaces, const uint64_t* workspace_bytes, bool profiled,
                       pk_group** out) {
  if (!ctx || !out || n < 0 || (n > 0 && (!plans || !d_workspaces || !workspace_bytes)) ||
      !valid_precision(precision))
    return fail(ctx, PK_EINVAL, "bad argument");
  if (ctx->device < 0) return fail(ctx, PK_ENODEVICE, "host-only context");
  *out = nullptr;
  DeviceGuard g(ctx->device);
  pk_group* grp = new (std::nothrow) pk_group();
  if (!grp) return fail(ctx, PK_ENOMEM, "out of host memory");
  grp->n = n;
  grp->precision = precision;
  grp->plans.assign(plans, plans + n);
  grp->ws.assign(d_workspaces, d_workspaces + n);
  grp->ws_bytes.assign(workspace_bytes, workspace_bytes + n);
  cudaError_t e = pk::prepare_kernels();
  if (e == cudaSuccess && !ctx->capture) e = cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaGraphCreate(&grp->graph, 0);
  for (int32_t i = 0; e == cudaSuccess && i < n; ++i) {
    void* ws = d_workspaces[i];
    uint64_t bytes = workspace_bytes[i];
    pk_status s = check_ws(ctx, plans[i], precision, ws, bytes);
    if (s != PK_OK || ws == nullptr) {
      pk_group_destroy(grp);
      return s != PK_OK ? s : fail(ctx, PK_EINVAL, "null workspace");
    }
    pk::Prof* prof = nullptr;
    if (profiled) {
      prof = pk::prof_new();
      grp->profs.push_back(prof);
    }
    e = cudaStreamBeginCapture(ctx->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) break;
    cudaError_t e1 = profiled ? pk::launch_plan_prof(plans[i]->p, precision, ws,
                                                     (char*)ws + plans[i]->p.off_arena, ctx->capture, prof)
                              : pk::launch_plan(plans[i]->p, precision, ws,
                                                (char*)ws + plans[i]->p.off_arena, ctx->capture);
    cudaGraph_t child = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(ctx->capture, &child);
    e = e1 != cudaSuccess ? e1 : e2;
    if (e == cudaSuccess) {
      cudaGraphNode_t node;
      e = cudaGraphAddChildGraphNode(&node, grp->graph, nullptr, 0, child);  // no dependencies
    }
    if (child) cudaGraphDestroy(child);
  }
  if (e == cudaSuccess && n > 0) e = cudaGraphInstantiate(&grp->exec, grp->graph, 0);
  if (e != cudaSuccess) {
    pk_group_destroy(grp);
    return cuda_fail(ctx, e, "group graph");
  }
  *out = grp;
  return PK_OK;
}

}  // namespace

extern "C" {

pk_status pk_group_create(pk_ctx* ctx, const pk_plan* const* plans, int32_t n, int32_t precision,
                          void* const* d_workspaces, const uint64_t* workspace_bytes,
                          pk_group** out) {
  return group_create(ctx, plans, n, precision, d_workspaces, workspace_bytes, false, out);
}

pk_status pk_group_create_profiled(pk_ctx* ctx, const pk_plan* const* plans, int32_t n,
                                   int32_t precision, void* const* d_workspaces,
                                   const uint64_t* workspace_bytes, pk_group** out) {
  return group_create(ctx, plans, n, precision, d_workspaces, workspace_bytes, true, out);
}

pk_status pk_group_profile(pk_ctx* ctx, const pk_group* grp, double* out) {
  if (!ctx || !grp || !out) return fail(ctx, PK_EINVAL, "bad argument");
  if (grp->profs.empty() && grp->n > 0) return fail(ctx, PK_EINVAL, "group was not created profiled");
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess) e = pk::prof_read(grp->profs.data(), (int)grp->profs.size(), out);
  return e == cudaSuccess ? PK_OK : cuda_fail(ctx, e, "group profile");
}

pk_status pk_group_timeline(pk_ctx* ctx, const pk_group* grp, double* out, int64_t capacity,
                            int64_t* count) {
  if (!ctx || !grp || !count || (capacity > 0 && !out)) return fail(ctx, PK_EINVAL, "bad argument");
  if (grp->profs.empty() && grp->n > 0) return fail(ctx, PK_EINVAL, "group was not created profiled");
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess)
    e = pk::prof_timeline(grp->profs.data(), (int)grp->profs.size(), out, capacity, count);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "group timeline");
  return *count > capacity ? fail(ctx, PK_ENOMEM, "timeline buffer too small") : PK_OK;
}

pk_status pk_group_launch(pk_ctx* ctx, pk_group* grp) {
  if (!ctx || !grp) return fail(ctx, PK_EINVAL, "bad argument");
  if (grp->n == 0) return PK_OK;
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaGraphLaunch(grp->exec, ctx->stream);
  return e == cudaSuccess ? PK_OK : cuda_fail(ctx, e, "group launch");
}

pk_status pk_group_upload(pk_ctx* ctx, pk_group* grp, int32_t inputs_only, uint64_t* copied) {
  if (!ctx || !grp) return fail(ctx, PK_EINVAL, "bad argument");
  uint64_t total = 0;
  for (int32_t i = 0; i < grp->n; ++i) {
    uint64_t n = grp->plans[i]->p.program.size();
    const pk_status s =
        inputs_only ? pk_upload_inputs(ctx, grp->plans[i], grp->precision, grp->ws[i], grp->ws_bytes[i], &n)
                    : pk_upload(ctx, grp->plans[i], grp->precision, grp->ws[i], grp->ws_bytes[i]);
    if (s != PK_OK) return s;
    total += n;
  }
  if (copied) *copied = total;
  return PK_OK;
}

pk_status pk_group_download(pk_ctx* ctx, pk_group* grp, pk_scaled* Z, pk_scaled* V,
                            int32_t* status) {
  if (!ctx || !grp || (grp->n > 0 && !Z)) return fail(ctx, PK_EINVAL, "bad argument");
  if (grp->n == 0) return PK_OK;
  DeviceGuard g(ctx->device);
  if (!grp->pinned &&
      cudaMallocHost((void**)&grp->pinned, sizeof(pk::SliceResult) * (size_t)grp->n) != cudaSuccess)
    return fail(ctx, PK_ENOMEM, "pinned host allocation failed");
  cudaError_t e = cudaSuccess;
  for (int32_t i = 0; e == cudaSuccess && i < grp->n; ++i) {
    const pk::Plan& P = grp->plans[i]->p;
    const char* src = (const char*)grp->ws[i] + P.off_result + sizeof(pk::SliceResult) * P.n_slices;
    e = cudaMemcpyAsync(grp->pinned + i, src, sizeof(pk::SliceResult), cudaMemcpyDeviceToHost,
                        ctx->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "group download");
  pk_status first = PK_OK;
  std::string err;
  for (int32_t i = 0; i < grp->n; ++i) {
    pk_scaled vv;
    const pk_status s = pk::decode_total(grp->plans[i]->p, grp->pinned[i], Z + i, V ? V + i : &vv, err);
    if (status) status[i] = s;
    if (s != PK_OK && first == PK_OK) {
      first = s;
      fail(ctx, s, "plan " + std::to_string(i) + ": " + err);
    }
  }
  return first;
}

void pk_group_destroy(pk_group* grp) {
  if (!grp) return;
  if (grp->pinned) cudaFreeHost(grp->pinned);
  if (grp->exec) cudaGraphExecDestroy(grp->exec);
  if (grp->graph) cudaGraphDestroy(grp->graph);
  for (pk::Prof* p : grp->profs) pk::prof_free(p);
  delete grp;
}

pk_status pk_jones_from_z(const pk_knot* k, int32_t q, const pk_scaled* Z, pk_scaled* V) {
  if (!k || !Z || !V || q < 1) return PK_EINVAL;
  if (!pk::jones_defined(k->k)) return PK_EINVAL;
  pk::Scaled z;
  z.re = Z->re;
  z.im = Z->im;
  z.e = Z->exp2;
  *V = to_abi(pk::s_mul(pk::jones_prefactor(k->k, q), z));
  return PK_OK;
}

pk_status pk_decode_result(const pk_plan* p, const void* record, pk_scaled* Z, pk_scaled* V) {
  if (!p || !record || !Z) return PK_EINVAL;
  pk::SliceResult r;
  std::memcpy(&r, record, sizeof(r));
  std::string err;
  return pk::decode_total(p->p, r, Z, V, err);
}

pk_status pk_download(pk_ctx* ctx, const pk_plan* p, int32_t precision, const void* d_workspace,
                      pk_scaled* Z, pk_scaled* V) {
  if (!ctx || !p || !Z || !valid_precision(precision)) return fail(ctx, PK_EINVAL, "bad argument");
  if (ctx->device < 0) return fail(ctx, PK_ENODEVICE, "host-only context");
  DeviceGuard g(ctx->device);
  const void* ws = d_workspace ? d_workspace : ctx->own_ws;
  if (!ws) return fail(ctx, PK_EINVAL, "no workspace");
  const pk::Plan& P = p->p;
  const char* src = (const char*)ws + P.off_result + sizeof(pk::SliceResult) * P.n_slices;
  cudaError_t e = cudaMemcpyAsync(ctx->pinned_result, src, sizeof(pk::SliceResult),
                                  cudaMemcpyDeviceToHost, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "download");
  e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronize");
  std::string err;
  const pk_status s = pk::decode_total(P, *ctx->pinned_result, Z, V, err);
  return s == PK_OK ? PK_OK : fail(ctx, s, err);
}

pk_status pk_eval(pk_ctx* ctx, const pk_plan* p, int32_t precision, void* d_workspace,
                  uint64_t workspace_bytes, pk_scaled* Z, pk_scaled* V) {
  pk_status s = pk_upload(ctx, p, precision, d_workspace, workspace_bytes);
  if (s != PK_OK) return s;
  s = pk_launch(ctx, p, precision, d_workspace, workspace_bytes);
  if (s != PK_OK) return s;
  return pk_download(ctx, p, precision, d_workspace, Z, V);
}

pk_status pk_eval_slices(pk_ctx* ctx, const pk_plan* p, int32_t precision, void* d_workspace,
                         uint64_t workspace_bytes, int64_t first, int64_t count,
                         pk_scaled* slices) {
  if (!ctx || !p || !slices || !valid_precision(precision)) return fail(ctx, PK_EINVAL, "bad argument");
  const pk::Plan& P = p->p;
  if (first < 0 || count < 1 || first > P.n_slices - count)
    return fail(ctx, PK_EINVAL, "slice range outside [0, n_slices)");
  pk_status s = pk_upload(ctx, p, precision, d_workspace, workspace_bytes);
  if (s != PK_OK) return s;
  DeviceGuard g(ctx->device);
  void* ws = d_workspace;
  if ((s = check_ws(ctx, p, precision, ws, workspace_bytes)) != PK_OK) return s;
  if (ctx->debug & PK_DEBUG_VERIFY) {
    std::string err;
    if (!pk::verify_plan(P, precision, err)) return fail(ctx, PK_EINVAL, "pk_plan_verify: " + err);
  }
  pk::LaunchOpts o;
  o.slice_first = first;
  o.slice_count = count;
  o.check_finite = (ctx->debug & PK_DEBUG_CHECK_FINITE) != 0;
  o.nvtx = (ctx->debug & PK_DEBUG_NVTX) != 0;
  cudaError_t e = pk::launch_plan_opts(P, precision, ws, (char*)ws + P.off_arena, ctx->stream, o);
  std::vector<pk::SliceResult> rec((size_t)count + 1);
  const char* res = (const char*)ws + P.off_result;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(rec.data(), res + sizeof(pk::SliceResult) * first,
                        sizeof(pk::SliceResult) * count, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&rec[count], res + sizeof(pk::SliceResult) * P.n_slices,
                        sizeof(pk::SliceResult), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "slices");
  std::string err;
  if ((s = pk::status_error(rec[count].status, err)) != PK_OK) return fail(ctx, s, err);
  for (int64_t i = 0; i < count; ++i) {
    pk::Scaled z;
    z.re = rec[i].re;
    z.im = rec[i].im;
    z.e = rec[i].exp;
    z.norm();
    slices[i] = to_abi(z);
  }
  return PK_OK;
}

pk_status pk_combine_slices(const pk_plan* p, const pk_scaled* slices, int64_t n, pk_scaled* Z,
                            pk_scaled* V) {
  if (!p || !slices || !Z || n != p->p.n_slices) return PK_EINVAL;
  int64_t emax = INT64_MIN;
  for (int64_t i = 0; i < n; ++i) {
    const double m = std::max(std::fabs(slices[i].re), std::fabs(slices[i].im));
    if (!std::isfinite(m)) return PK_EINVAL;
    if (m > 0) {
      int e;
      std::frexp(m, &e);
      emax = std::max<int64_t>(emax, slices[i].exp2 + e);
    }
  }
  pk::SliceResult tot{0, 0, 0, 0};
  if (emax != INT64_MIN) {
    double are = 0, aim = 0, cre = 0, cim = 0;  // Kahan-compensated, as the device sum
    for (int64_t i = 0; i < n; ++i) {
      const int64_t d = slices[i].exp2 - emax;
      const double f = d < -2000 ? 0.0 : std::ldexp(1.0, (int)d);
      const double yr = slices[i].re * f - cre, tr = are + yr;
      cre = (tr - are) - yr;
      are = tr;
      const double yi = slices[i].im * f - cim, ti = aim + yi;
      cim = (ti - aim) - yi;
      aim = ti;
    }
    tot.re = are;
    tot.im = aim;
    tot.exp = emax;
  }
  std::string err;
  return pk::decode_total(p->p, tot, Z, V, err);
}

pk_status pk_grad_workspace_bytes(const pk_plan* p, int32_t precision, uint64_t* bytes) {
  if (!p || !bytes || !valid_precision(precision) || !p->p.grad.built) return PK_EINVAL;
  *bytes = p->p.grad.ws_bytes(precision);
  return PK_OK;
}

pk_status pk_grad_stats(const pk_plan* p, double* out) {
  if (!p || !out || !p->p.grad.built) return PK_EINVAL;
  const pk::GradProgram& G = p->p.grad;
  double n[3] = {0, 0, 0};
  for (int8_t ph : G.phase) n[ph] += 1;
  const double v[10] = {G.cmacs[0], G.cmacs[1], G.cmacs[2], n[0], n[1], n[2],
                        (double)G.arena_elems, (double)G.n_checkpoints,
                        (double)G.leaves.size(), (double)p->p.n_slices};
  std::memcpy(out, v, sizeof(v));
  return PK_OK;
}

pk_status pk_grad_from_accumulators(const pk_plan* p, const double* acc, const int64_t* acc_exp,
                                    const pk_scaled* Z, double* dlogZ_dT, double* dlogV_dt) {
  if (!p || !Z || !p->p.grad.built || (!acc && !p->p.groups.empty()) ||
      (!acc_exp && !p->p.groups.empty()))
    return PK_EINVAL;
  pk::Scaled z;
  z.re = Z->re;
  z.im = Z->im;
  z.e = Z->exp2;
  return pk::grad_finalize(p->p, acc, acc_exp, z, dlogZ_dT, dlogV_dt) ? PK_OK : PK_EZERO;
}

pk_status pk_grad_weights(const pk_plan* p, const double* dlogZ_dT, double* out) {
  if (!p || !dlogZ_dT || !out) return PK_EINVAL;
  const int32_t q = p->p.q;
  const size_t n_e = p->p.knot.edges.size();
  for (size_t e = 0; e < n_e; ++e) {
    double dr = 0, di = 0, orr = 0, oi = 0;
    for (int32_t a = 0; a < q; ++a)
      for (int32_t b = 0; b < q; ++b) {
        const double* v = dlogZ_dT + 2 * ((e * q + a) * q + b);
        if (a == b) {
          dr += v[0];
          di += v[1];
        } else {
          orr += v[0];
          oi += v[1];
        }
      }
    out[4 * e] = dr;
    out[4 * e + 1] = di;
    out[4 * e + 2] = orr;
    out[4 * e + 3] = oi;
  }
  return PK_OK;
}

pk_status pk_plan_set_weights(pk_plan* p, const double* edge_weights) {
  if (!p || !p->p.general) return PK_EINVAL;
  if (!pk::set_weights(p->p, edge_weights)) return PK_EINVAL;
  if (p->pinned_program) {  // refilled from the new program by the next pk_upload
    cudaFreeHost(p->pinned_program);
    p->pinned_program = nullptr;
  }
  return PK_OK;
}

}  // extern "C"

namespace {

// The reverse-pass launch sequence recorded once per (workspace, precision) into a CUDA
// graph on the context's capture stream and replayed afterwards; very long sequences
// (many slices) are launched directly.
cudaError_t launch_grad_recorded(pk_ctx* ctx, const pk_plan* p, int32_t precision, void* ws) {
  const pk::Plan& P = p->p;
  const double nodes = (double)P.n_slices * (double)(P.grad.steps.size() + 4);
  if (nodes > 20000.0) return pk::launch_grad(P, precision, ws, ctx->stream);
  PlanGraph& g = const_cast<pk_plan*>(p)->grad_graph;
  if (!(g.exec && g.ws == ws && g.precision == precision)) {
    if (g.exec) {
      cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
    }
    cudaError_t e = pk::prepare_kernels();
    if (e == cudaSuccess && !ctx->capture)
      e = cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    e = cudaStreamBeginCapture(ctx->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t e1 = pk::launch_grad(P, precision, ws, ctx->capture);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(ctx->capture, &graph);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return e1 != cudaSuccess ? e1 : e2;
    }
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      g.exec = nullptr;
      return e;
    }
    g.ws = ws;
    g.precision = precision;
  }
  return cudaGraphLaunch(g.exec, ctx->stream);
}

}  // namespace

extern "C" {

pk_status pk_grad(pk_ctx* ctx, const pk_plan* p, int32_t precision, void* d_workspace,
                  uint64_t workspace_bytes, pk_scaled* Z, pk_scaled* V, double* dlogZ_dT,
                  double* dlogV_dt) {
  if (!ctx || !p || !valid_precision(precision)) return fail(ctx, PK_EINVAL, "bad argument");
  if (!p->p.grad.built) return fail(ctx, PK_EINVAL, "plan made without PK_FLAG_GRAD");
  if (ctx->device < 0) return fail(ctx, PK_ENODEVICE, "host-only context");
  DeviceGuard g(ctx->device);
  const pk::Plan& P = p->p;
  const pk::GradProgram& G = P.grad;
  pk_status s = check_ws_need(ctx, G.ws_bytes(precision), d_workspace, workspace_bytes);
  if (s != PK_OK) return s;
  const uint64_t nl = std::max<size_t>(1, G.leaves.size());
  const uint64_t acc_bytes = 16ull * (uint64_t)P.q * P.q * nl + 8ull * nl;
  const uint64_t prog = (G.program.size() + 255) & ~uint64_t(255);
  pk_plan* mp = const_cast<pk_plan*>(p);
  if (!mp->pinned_grad &&
      cudaMallocHost((void**)&mp->pinned_grad, prog + sizeof(pk::SliceResult) + acc_bytes) !=
          cudaSuccess) {
    mp->pinned_grad = nullptr;
    return fail(ctx, PK_ENOMEM, "pinned host allocation failed");
  }
  uint8_t* host = mp->pinned_grad;
  std::memcpy(host, G.program.data(), G.program.size());  // the current weights
  char* ws = (char*)d_workspace;
  cudaError_t e = cudaMemcpyAsync(ws, host, G.program.size(), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = launch_grad_recorded(ctx, p, precision, ws);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host + prog, ws + G.off_result + sizeof(pk::SliceResult) * P.n_slices,
                        sizeof(pk::SliceResult), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host + prog + sizeof(pk::SliceResult), ws + G.off_acc, acc_bytes,
                        cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "reverse pass");
  const pk::SliceResult* r = (const pk::SliceResult*)(host + prog);
  pk::Scaled z;
  z.re = r->re;
  z.im = r->im;
  z.e = r->exp;
  z.norm();
  z = pk::s_mul(z, P.factor);
  pk_scaled zs = to_abi(z);
  if (Z) *Z = zs;
  if (V) {
    pk_knot kk;
    kk.k = P.knot;
    pk_status sv = pk_jones_from_z(&kk, P.q, &zs, V);
    if (sv != PK_OK) return fail(ctx, sv, "3w + tau + 2 n_v + 2 not divisible by 4 (knot) or 2 (link)");
  }
  const double* acc = (const double*)(host + prog + sizeof(pk::SliceResult));
  const int64_t* acc_exp = (const int64_t*)(host + prog + sizeof(pk::SliceResult) +
                                            16ull * (uint64_t)P.q * P.q * nl);
  if (!pk::grad_finalize(P, acc, acc_exp, z, dlogZ_dT, dlogV_dt))
    return fail(ctx, PK_EZERO, "Z is zero: log-derivatives undefined");
  return PK_OK;
}


}  // extern "C"

// ------------------------------------------------------------------ exact evaluation
namespace {

constexpr int64_t kExactMaxSlices = 1000000;

bool is_prime32(uint32_t p) {
  if (p < 2) return false;
  for (uint32_t d = 2; (uint64_t)d * d <= p; ++d)
    if (p % d == 0) return false;
  return true;
}

// Z(q) mod each prime (loop factor included) for an uploaded plan.
pk_status exact_residues(pk_ctx* ctx, const pk_plan* p, const uint32_t* primes, int32_t n_primes,
                         void* ws, uint32_t* zab) {
  const pk::Plan& P = p->p;
  for (int32_t i = 0; i < n_primes; ++i) {
    void* sum = (char*)ws + P.off_result;
    cudaError_t e = pk::launch_exact(P, primes[i], ws, (char*)ws + P.off_arena, sum, ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ctx->pinned_result, sum, sizeof(pk::exact::E), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "exact evaluation");
    pk::exact::E z;
    std::memcpy(&z, ctx->pinned_result, sizeof(z));
    const pk::exact::Ring r = pk::exact::make_ring(primes[i], P.q);
    pk::exact::E f = pk::exact::epow_t(-(long long)P.loop_signsum, r);  // folded loops
    if (P.loop_count & 1) f = pk::exact::eneg(f, r);
    z = pk::exact::emul(z, f, r);
    zab[2 * i] = z.a;
    zab[2 * i + 1] = z.b;
  }
  return PK_OK;
}

}  // namespace

extern "C" {

pk_status pk_eval_exact(pk_ctx* ctx, const pk_plan* p, const uint32_t* primes, int32_t n_primes,
                        void* d_workspace, uint64_t workspace_bytes, uint32_t* zab) {
  if (!ctx || !p || !primes || n_primes < 1 || !zab) return fail(ctx, PK_EINVAL, "bad argument");
  if (ctx->device < 0) return fail(ctx, PK_ENODEVICE, "host-only context");
  const pk::Plan& P = p->p;
  if (P.general || !P.std_weights || !P.tail.empty())
    return fail(ctx, PK_EINVAL, "exact evaluation needs the standard weights and no complex128 tail");
  for (int32_t i = 0; i < n_primes; ++i)
    if (primes[i] <= (uint32_t)P.q || primes[i] >= (1u << 31) || !is_prime32(primes[i]))
      return fail(ctx, PK_EINVAL, "moduli must be primes between q and 2^31");
  if (P.n_slices > kExactMaxSlices)   // every slice is a launch sequence of its own
    return fail(ctx, PK_ETOOWIDE, "too many slices for the exact path");
  DeviceGuard g(ctx->device);
  void* ws = d_workspace;
  uint64_t bytes = workspace_bytes;
  pk_status s = check_ws(ctx, p, PK_C64, ws, bytes);
  if (s != PK_OK) return s;
  if ((s = pk_upload(ctx, p, PK_C64, ws, bytes)) != PK_OK) return s;
  return exact_residues(ctx, p, primes, n_primes, ws, zab);
}

pk_status pk_jones_plan(const pk_knot* k, int32_t* n_q, int32_t* qs_out, int32_t* n_primes,
                        uint32_t* primes_out) {
  if (!k || !n_q || !n_primes) return PK_EINVAL;
  int32_t lo = 0, hi = 0;
  if (!pk::jones_window(k->k, lo, hi)) return PK_EINVAL;
  const int32_t m = hi - lo + 1;
  // q = 1, 2, ... until two equations per q exceed the unknowns by four
  int32_t nq = 0;
  while (2 * nq < m + 4) ++nq;
  if (qs_out)
    for (int32_t i = 0; i < nq; ++i) qs_out[i] = i + 1;
  *n_q = nq;
  // moduli: the four largest primes below 2^31 (the last one checks the reconstruction)
  int32_t np = 0;
  for (uint32_t c = (1u << 31) - 1; np < 4; c -= 2)
    if (is_prime32(c)) {
      if (primes_out) primes_out[np] = c;
      ++np;
    }
  *n_primes = np;
  return PK_OK;
}

pk_status pk_jones_solve(const pk_knot* k, int32_t n_q, const int32_t* qs, int32_t n_primes,
                         const uint32_t* primes, const uint32_t* zab, int32_t capacity, int32_t* lowest,
                         int32_t* count, int64_t* coef, int32_t* half) {
  if (!k || n_q < 1 || !qs || n_primes < 2 || !primes || !zab || !lowest || !count || !half ||
      (capacity > 0 && !coef))
    return PK_EINVAL;
  *half = pk::jones_half(k->k);
  int32_t lo = 0, hi = 0;
  if (!pk::jones_window(k->k, lo, hi)) return PK_EINVAL;
  const int32_t m = hi - lo + 1;
  std::vector<int32_t> q(qs, qs + n_q);
  std::vector<uint32_t> pr(primes, primes + n_primes);
  for (int32_t i = 0; i < n_q; ++i)
    for (int32_t j = 0; j < n_primes; ++j)
      if (q[i] < 1 || pr[j] <= (uint32_t)q[i] || pr[j] >= (1u << 31) || !is_prime32(pr[j])) return PK_EINVAL;
  std::vector<std::vector<uint32_t>> res(n_primes);
  for (int32_t ip = 0; ip < n_primes; ++ip) {
    std::vector<uint32_t> vals(2 * (size_t)n_q);
    for (int32_t iq = 0; iq < n_q; ++iq) {
      const uint32_t* z = zab + 2 * ((size_t)iq * n_primes + ip);
      pk::jones_value_mod(k->k, q[iq], pr[ip], z[0] % pr[ip], z[1] % pr[ip], vals[2 * iq], vals[2 * iq + 1]);
    }
    if (!pk::solve_coefficients_mod(q, vals, lo, m, pr[ip], res[ip])) return PK_EINVAL;
  }
  std::vector<int64_t> c;
  if (!pk::crt_signed(pr, res, c)) return PK_EINVAL;
  int32_t first = 0, last = m - 1;
  while (first <= last && c[first] == 0) ++first;
  while (last >= first && c[last] == 0) --last;
  *lowest = first <= last ? lo + first : 0;
  *count = first <= last ? last - first + 1 : 0;
  if (*count > capacity) return PK_ENOMEM;
  for (int32_t j = 0; j < *count; ++j) coef[j] = c[first + j];
  return PK_OK;
}

pk_status pk_jones_coefficients(pk_ctx* ctx, const pk_knot* k, int32_t capacity, int32_t* lowest,
                                int32_t* count, int64_t* coef, int32_t* half) {
  if (!ctx || !k || !lowest || !count || !half || (capacity > 0 && !coef))
    return fail(ctx, PK_EINVAL, "bad argument");
  if (ctx->device < 0) return fail(ctx, PK_ENODEVICE, "host-only context");
  int32_t nq = 0, np = 0;
  if (pk_jones_plan(k, &nq, nullptr, &np, nullptr) != PK_OK)
    return fail(ctx, PK_EINVAL, "coefficients need a knot or link given by its PD code");
  std::vector<int32_t> qs(nq);
  std::vector<uint32_t> primes(np);
  pk_jones_plan(k, &nq, qs.data(), &np, primes.data());
  std::vector<uint32_t> zab(2 * (size_t)nq * np);
  DeviceGuard g(ctx->device);
  for (int32_t iq = 0; iq < nq; ++iq) {
    pk_plan* p = nullptr;
    pk_plan_opts o;
    std::memset(&o, 0, sizeof(o));
    pk_status s = pk_plan_create(ctx, k, qs[iq], &o, &p);
    if (s != PK_OK) return s;
    if (p->p.n_slices > kExactMaxSlices) {
      pk_plan_destroy(p);
      return fail(ctx, PK_ETOOWIDE, "too many slices for the exact path");
    }
    void* ws = nullptr;
    uint64_t bytes = 0;
    s = check_ws(ctx, p, PK_C64, ws, bytes);
    if (s == PK_OK) s = pk_upload(ctx, p, PK_C64, ws, bytes);
    if (s == PK_OK) s = exact_residues(ctx, p, primes.data(), np, ws, zab.data() + 2 * (size_t)iq * np);
    pk_plan_destroy(p);
    if (s != PK_OK) return s;
  }
  const pk_status s = pk_jones_solve(k, nq, qs.data(), np, primes.data(), zab.data(), capacity, lowest,
                                     count, coef, half);
  if (s == PK_ENOMEM) return fail(ctx, s, "coefficient buffer too small");
  if (s != PK_OK) return fail(ctx, s, "coefficient system singular or inconsistent, or beyond 64 bits");
  return PK_OK;
}

}  // extern "C"
