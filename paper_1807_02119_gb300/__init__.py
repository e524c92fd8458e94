"""Python binding of libpk (include/pk.h): argument marshalling only.

Every step of the evaluation runs in the library (host planning in C++, contraction
in CUDA kernels for sm_103a).  PyTorch supplies device memory (the workspace) and
the stream.  There is no CPU fallback: if libpk.so is missing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpk.so")

PK_C128, PK_C64, PK_SPLIT = 0, 1, 2
FLAG_FORCE_GEMM, FLAG_FORCE_ROWS, FLAG_GRAD, FLAG_NO_TC, FLAG_TC_DIGITS4 = 1, 2, 4, 8, 16
PRECISIONS = {"c128": PK_C128, "c64": PK_C64, "split": PK_SPLIT}
PRECISION_NAMES = {v: k for k, v in PRECISIONS.items()}
ORDERS = {"auto": 0, "greedy_edge": 1, "greedy_spin": 2, "elim_spin": 3, "partition": 4,
          "fill_spin": 5}
STATUS = {0: "PK_OK", 1: "PK_EINVAL", 2: "PK_ENOTKNOT", 3: "PK_ENOMEM", 4: "PK_ETOOWIDE",
          5: "PK_ECUDA", 6: "PK_ETIMEOUT", 7: "PK_ENODEVICE", 8: "PK_EZERO", 9: "PK_ENONFINITE"}
DEBUG_CHECK_FINITE, DEBUG_VERIFY, DEBUG_NVTX = 1, 2, 4

EXPORTED = [
    "pk_ctx_create", "pk_ctx_set_stream", "pk_last_error", "pk_ctx_destroy",
    "pk_knot_from_pd", "pk_link_from_pd", "pk_knot_from_signed_graph", "pk_knot_from_grid_walk", "pk_knot_info",
    "pk_knot_edges", "pk_knot_pd", "pk_knot_destroy", "pk_plan_create", "pk_plan_info",
    "pk_plan_workspace_bytes", "pk_plan_steps", "pk_plan_destroy", "pk_eval", "pk_upload",
    "pk_upload_inputs",
    "pk_launch", "pk_download", "pk_plan_launches", "pk_jones_from_z", "pk_plan_debug_blob",
    "pk_profile", "pk_eval_noalloc", "pk_plan_state_bytes", "pk_launch_arena",
    "pk_batch_create", "pk_batch_workspace_bytes", "pk_batch_upload", "pk_batch_upload_inputs",
    "pk_batch_launch",
    "pk_batch_download", "pk_eval_batch", "pk_batch_destroy", "pk_group_create",
    "pk_group_launch", "pk_group_upload", "pk_group_download", "pk_group_destroy",
    "pk_grad_workspace_bytes", "pk_grad",
    "pk_grad_from_accumulators", "pk_grad_stats", "pk_plan_set_weights", "pk_eval_exact",
    "pk_jones_coefficients", "pk_jones_plan", "pk_jones_solve", "pk_decode_result",
    "pk_group_create_profiled", "pk_group_profile", "pk_group_timeline",
    "pk_tuning_default", "pk_ctx_set_tuning", "pk_ctx_get_tuning", "pk_knot_simplify",
    "pk_order_stats", "pk_ctx_set_hbm_budget", "pk_grad_weights", "pk_ctx_set_debug",
    "pk_plan_verify", "pk_eval_slices", "pk_combine_slices",
]


class PkError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class pk_scaled(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double), ("exp2", C.c_int64)]


class pk_plan_opts(C.Structure):
    _fields_ = [("order", C.c_int32), ("flags", C.c_int32), ("max_log2_elems", C.c_double),
                ("max_log2_slices", C.c_double), ("tail_steps", C.c_int32),
                ("restarts", C.c_int32), ("checkpoint_stride", C.c_int32),
                ("edge_weights", C.POINTER(C.c_double)), ("refine", C.c_int32)]


class pk_tuning(C.Structure):
    _fields_ = [("batch_threads", C.c_int32), ("batch_ktab", C.c_int32), ("seq_outs", C.c_int64),
                ("seq_work", C.c_int64), ("seq_k", C.c_int64), ("tc_min_k", C.c_int64),
                ("tc_db_groups", C.c_int64), ("tc_min_n", C.c_int64),
                ("cost_gemm_milli", C.c_int64), ("cost_out_milli", C.c_int64),
                ("tc_wide_n", C.c_int64), ("cost_tcin_milli", C.c_int64),
                ("tc_min_work", C.c_int64)]


class pk_plan_stats(C.Structure):
    _fields_ = [("log2_max_elems", C.c_double), ("cmacs", C.c_double),
                ("bytes_c64", C.c_double), ("n_slices", C.c_int64), ("n_steps", C.c_int32),
                ("max_rank", C.c_int32), ("order_used", C.c_int32), ("n_tensors", C.c_int32),
                ("workspace_c128", C.c_uint64), ("workspace_c64", C.c_uint64),
                ("workspace_split", C.c_uint64), ("n_segments", C.c_int32),
                ("n_segment_steps", C.c_int32), ("est_cost", C.c_double)]


_lib = None


def default_tuning() -> dict:
    """pk_tuning_default: the table the library was compiled with (written by autotune.py)."""
    t = pk_tuning()
    _check(lib().pk_tuning_default(C.byref(t)))
    return {f: getattr(t, f) for f, _ in t._fields_}


def lib():
    """Load libpk.so (built by __graft_entry__.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run `python -c 'import __graft_entry__ as g; "
                          "g.build()'` (there is no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
    P = C.POINTER
    sig = {
        "pk_ctx_create": [i32, vp, P(vp)],
        "pk_ctx_set_stream": [vp, vp],
        "pk_ctx_destroy": [vp],
        "pk_knot_from_pd": [vp, P(i32), i32, i32, i32, P(vp)],
        "pk_link_from_pd": [vp, P(i32), P(i32), i32, i32, i32, P(vp)],
        "pk_eval_exact": [vp, vp, P(C.c_uint32), i32, vp, u64, P(C.c_uint32)],
        "pk_jones_coefficients": [vp, vp, i32, P(i32), P(i32), P(i64), P(i32)],
        "pk_jones_plan": [vp, P(i32), P(i32), P(i32), P(C.c_uint32)],
        "pk_jones_solve": [vp, i32, P(i32), i32, P(C.c_uint32), P(C.c_uint32), i32, P(i32), P(i32),
                           P(i64), P(i32)],
        "pk_knot_from_signed_graph": [vp, i32, i32, P(i32), i32, P(vp)],
        "pk_knot_from_grid_walk": [vp, i32, u64, i32, i32, i32, P(vp)],
        "pk_knot_info": [vp, P(i32), P(i32), P(i32), P(i32), P(i32)],
        "pk_knot_simplify": [vp, vp, P(vp)],
        "pk_order_stats": [vp, i32, i32, i32, P(C.c_double)],
        "pk_ctx_set_hbm_budget": [vp, u64],
        "pk_ctx_set_debug": [vp, i32],
        "pk_plan_verify": [vp, i32, C.c_char_p, u64],
        "pk_eval_slices": [vp, vp, i32, vp, u64, i64, i64, P(pk_scaled)],
        "pk_combine_slices": [vp, P(pk_scaled), i64, P(pk_scaled), P(pk_scaled)],
        "pk_grad_weights": [vp, P(C.c_double), P(C.c_double)],
        "pk_knot_edges": [vp, P(i32)],
        "pk_knot_pd": [vp, P(i32)],
        "pk_knot_destroy": [vp],
        "pk_plan_create": [vp, vp, i32, P(pk_plan_opts), P(vp)],
        "pk_plan_info": [vp, P(pk_plan_stats)],
        "pk_plan_workspace_bytes": [vp, i32, P(u64)],
        "pk_plan_steps": [vp, P(i64)],
        "pk_plan_destroy": [vp],
        "pk_eval": [vp, vp, i32, vp, u64, P(pk_scaled), P(pk_scaled)],
        "pk_upload": [vp, vp, i32, vp, u64],
        "pk_launch": [vp, vp, i32, vp, u64],
        "pk_download": [vp, vp, i32, vp, P(pk_scaled), P(pk_scaled)],
        "pk_decode_result": [vp, vp, P(pk_scaled), P(pk_scaled)],
        "pk_plan_launches": [vp, i32, P(i64)],
        "pk_jones_from_z": [vp, i32, P(pk_scaled), P(pk_scaled)],
        "pk_plan_debug_blob": [vp, i32, vp, P(u64)],
        "pk_profile": [vp, vp, i32, vp, u64, vp, u64, P(C.c_double)],
        "pk_eval_noalloc": [vp, vp, i32, P(pk_scaled), P(pk_scaled)],
        "pk_plan_state_bytes": [vp, i32, P(u64), P(u64)],
        "pk_launch_arena": [vp, vp, i32, vp, u64, vp, u64],
        "pk_batch_create": [vp, P(vp), i32, i32, P(vp)],
        "pk_batch_workspace_bytes": [vp, P(u64), P(u64)],
        "pk_batch_upload": [vp, vp, vp, u64],
        "pk_batch_upload_inputs": [vp, vp, vp, u64, P(u64)],
        "pk_batch_launch": [vp, vp, vp, u64],
        "pk_batch_download": [vp, vp, vp, P(pk_scaled), P(pk_scaled)],
        "pk_eval_batch": [vp, P(vp), i32, i32, vp, u64, P(pk_scaled), P(pk_scaled)],
        "pk_batch_destroy": [vp],
        "pk_group_create": [vp, P(vp), i32, i32, P(vp), P(u64), P(vp)],
        "pk_group_launch": [vp, vp],
        "pk_group_upload": [vp, vp, i32, P(u64)],
        "pk_upload_inputs": [vp, vp, i32, vp, u64, P(u64)],
        "pk_group_download": [vp, vp, P(pk_scaled), P(pk_scaled), P(i32)],
        "pk_group_create_profiled": [vp, P(vp), i32, i32, P(vp), P(u64), P(vp)],
        "pk_group_profile": [vp, vp, P(C.c_double)],
        "pk_group_timeline": [vp, vp, P(C.c_double), i64, P(i64)],
        "pk_tuning_default": [P(pk_tuning)],
        "pk_ctx_set_tuning": [vp, P(pk_tuning)],
        "pk_ctx_get_tuning": [vp, P(pk_tuning)],
        "pk_group_destroy": [vp],
        "pk_grad_workspace_bytes": [vp, i32, P(u64)],
        "pk_grad": [vp, vp, i32, vp, u64, P(pk_scaled), P(pk_scaled), P(C.c_double),
                    P(C.c_double)],
        "pk_grad_from_accumulators": [vp, P(C.c_double), P(i64), P(pk_scaled), P(C.c_double),
                                      P(C.c_double)],
        "pk_grad_stats": [vp, P(C.c_double)],
        "pk_plan_set_weights": [vp, P(C.c_double)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = None if name.endswith("destroy") else C.c_int
    L.pk_last_error.argtypes = [vp]
    L.pk_last_error.restype = C.c_char_p
    _lib = L
    return L


def _check(status, ctx=None):
    if status != 0:
        msg = lib().pk_last_error(ctx.h if ctx is not None else None)
        raise PkError(status, msg.decode() if msg else "")


@dataclass(frozen=True)
class Scaled:
    """value = (re + i im) * 2**exp2"""
    re: float
    im: float
    exp2: int

    @staticmethod
    def of(s: pk_scaled) -> "Scaled":
        return Scaled(s.re, s.im, s.exp2)

    @property
    def mantissa(self) -> complex:
        return complex(self.re, self.im)

    def to_complex(self) -> complex:
        import math
        try:
            return complex(math.ldexp(self.re, self.exp2), math.ldexp(self.im, self.exp2))
        except OverflowError:
            return complex(float("inf"), float("inf"))


class Context:
    """A library context.  device=-1 gives a host-only context (knots and plans)."""

    def __init__(self, device: int = -1, stream: int | None = None):
        h = C.c_void_p()
        st = lib().pk_ctx_create(device, C.c_void_p(stream or 0), C.byref(h))
        if st != 0:
            raise PkError(st, f"pk_ctx_create(device={device})")
        self.h = h
        self.device = device

    def set_stream(self, stream: int):
        _check(lib().pk_ctx_set_stream(self.h, C.c_void_p(stream)), self)

    def set_debug(self, flags: int = 0):
        """pk_ctx_set_debug: DEBUG_CHECK_FINITE | DEBUG_VERIFY | DEBUG_NVTX (0 turns them off)."""
        _check(lib().pk_ctx_set_debug(self.h, int(flags)), self)

    def set_hbm_budget(self, nbytes: int):
        """pk_ctx_set_hbm_budget: plans created afterwards slice until their workspace fits."""
        _check(lib().pk_ctx_set_hbm_budget(self.h, int(nbytes)), self)

    def tuning(self) -> dict:
        """The launch shapes plans and batches created now will use (pk_ctx_get_tuning)."""
        t = pk_tuning()
        _check(lib().pk_ctx_get_tuning(self.h, C.byref(t)), self)
        return {f: getattr(t, f) for f, _ in t._fields_}

    def set_tuning(self, **kw):
        """pk_ctx_set_tuning: change some launch shapes (others keep their current values);
        with no arguments, restore the compiled-in defaults."""
        if not kw:
            _check(lib().pk_ctx_set_tuning(self.h, None), self)
            return
        cur = self.tuning()
        cur.update(kw)
        _check(lib().pk_ctx_set_tuning(self.h, C.byref(pk_tuning(**cur))), self)

    def close(self):
        if self.h:
            lib().pk_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Knot:
    def __init__(self, h, ctx):
        self.h = h
        self.ctx = ctx

    @staticmethod
    def from_pd(ctx: Context, pd, outer=None) -> "Knot":
        flat = [int(v) for X in pd for v in X]
        arr = (C.c_int32 * max(1, len(flat)))(*flat)
        oa, os_ = (outer if outer is not None else (-1, 0))
        h = C.c_void_p()
        _check(lib().pk_knot_from_pd(ctx.h, arr, len(pd), oa, os_, C.byref(h)), ctx)
        return Knot(h, ctx)

    @staticmethod
    def from_link_pd(ctx: Context, pd, signs, outer=None) -> "Knot":
        """pk_link_from_pd: a link (or knot) diagram with the twist sign of every crossing
        (+1: over-strand leaves through arm b); V is then evaluated for links too."""
        flat = [int(v) for X in pd for v in X]
        arr = (C.c_int32 * max(1, len(flat)))(*flat)
        sg = (C.c_int32 * max(1, len(signs)))(*[int(x) for x in signs])
        oa, os_ = (outer if outer is not None else (-1, 0))
        h = C.c_void_p()
        _check(lib().pk_link_from_pd(ctx.h, arr, sg, len(pd), oa, os_, C.byref(h)), ctx)
        return Knot(h, ctx)

    @staticmethod
    def from_signed_graph(ctx: Context, n_v, edges, writhe) -> "Knot":
        flat = [int(v) for e in edges for v in e]
        arr = (C.c_int32 * max(1, len(flat)))(*flat)
        h = C.c_void_p()
        _check(lib().pk_knot_from_signed_graph(ctx.h, n_v, len(edges), arr, writhe, C.byref(h)), ctx)
        return Knot(h, ctx)

    @staticmethod
    def from_grid_walk(ctx: Context, L, seed, random_over_under=True, ncross_min=0,
                       ncross_max=1 << 30) -> "Knot":
        h = C.c_void_p()
        _check(lib().pk_knot_from_grid_walk(ctx.h, L, seed, int(random_over_under), ncross_min,
                                            ncross_max, C.byref(h)), ctx)
        return Knot(h, ctx)

    def simplified(self) -> "Knot":
        """pk_knot_simplify: the Reidemeister-simplified signed Tait graph (same V)."""
        h = C.c_void_p()
        _check(lib().pk_knot_simplify(self.ctx.h, self.h, C.byref(h)), self.ctx)
        return Knot(h, self.ctx)

    def order_stats(self, q: int, order: str, restarts: int = 0) -> dict:
        """pk_order_stats: the order search alone -- Delta_H (largest rank), log2 of the
        unsliced work, initial tensors and indices of the best candidate."""
        out = (C.c_double * 4)()
        _check(lib().pk_order_stats(self.h, q, ORDERS[order], restarts, out))
        return {"delta_h": int(out[0]), "log2_work": out[1], "tensors": int(out[2]),
                "indices": int(out[3])}

    def max_degree(self) -> int:
        """Delta_G: the largest vertex degree of the signed Tait graph (a loop counts twice)."""
        deg = [0] * self.info()["n_v"]
        for u, v, _ in self.edges():
            deg[u] += 1
            deg[v] += 1
        return max(deg) if deg else 0

    def info(self) -> dict:
        v = [C.c_int32() for _ in range(5)]
        _check(lib().pk_knot_info(self.h, *[C.byref(x) for x in v]))
        return dict(zip(("n_v", "n_c", "writhe", "tau", "components"), (x.value for x in v)))

    def edges(self):
        n = self.info()["n_c"]
        arr = (C.c_int32 * max(1, 3 * n))()
        _check(lib().pk_knot_edges(self.h, arr))
        return [(arr[3 * e], arr[3 * e + 1], arr[3 * e + 2]) for e in range(n)]

    def pd(self):
        n = self.info()["n_c"]
        arr = (C.c_int32 * max(1, 4 * n))()
        _check(lib().pk_knot_pd(self.h, arr))
        return [tuple(arr[4 * i:4 * i + 4]) for i in range(n)]

    def jones_from_z(self, q: int, z: Scaled) -> Scaled:
        zz = pk_scaled(z.re, z.im, z.exp2)
        vv = pk_scaled()
        _check(lib().pk_jones_from_z(self.h, q, C.byref(zz), C.byref(vv)))
        return Scaled.of(vv)

    def __del__(self):
        try:
            if self.h:
                lib().pk_knot_destroy(self.h)
                self.h = None
        except Exception:
            pass


def _weights_array(weights, n_e):
    """4 doubles per Tait edge (diag re, diag im, off re, off im) from an (n_e, 2) array
    of complex (diagonal, off-diagonal) clause weights."""
    flat = []
    for d, o in weights:
        d, o = complex(d), complex(o)
        flat += [d.real, d.imag, o.real, o.imag]
    if len(flat) != 4 * n_e:
        raise ValueError(f"expected {n_e} (diagonal, off-diagonal) weight pairs")
    return (C.c_double * max(1, len(flat)))(*flat)


class Plan:
    """A contraction plan.  grad=True also builds the reverse-pass program (pk_grad);
    weights: None (the Jones weights of Eq. clause) or one (diagonal, off-diagonal) complex
    pair per Tait edge; refine > 0: subtree reconfiguration of the cheapest candidate
    sequences with frontiers of up to `refine` subtrees (pk_plan_opts.refine)."""

    def __init__(self, ctx: Context, knot: Knot, q: int, order: str = "auto",
                 max_log2_elems: float = 0.0, max_log2_slices: float = 0.0, flags: int = 0,
                 tail_steps: int = 0, restarts: int = 0, grad: bool = False,
                 checkpoint_stride: int = 0, weights=None, refine: int = 0):
        w = None
        if weights is not None:
            w = _weights_array(weights, knot.info()["n_c"])
        o = pk_plan_opts(ORDERS[order], flags | (FLAG_GRAD if grad else 0), max_log2_elems,
                         max_log2_slices, tail_steps, restarts, checkpoint_stride,
                         C.cast(w, C.POINTER(C.c_double)) if w is not None else None, refine)
        h = C.c_void_p()
        _check(lib().pk_plan_create(ctx.h, knot.h, q, C.byref(o), C.byref(h)), ctx)
        self.h = h
        self.q = q
        self.knot = knot
        self.ctx = ctx
        self.n_e = knot.info()["n_c"]

    def set_weights(self, weights=None):
        """pk_plan_set_weights: new (diagonal, off-diagonal) pairs per Tait edge, or the
        standard weights of t(q) for None."""
        w = _weights_array(weights, self.n_e) if weights is not None else None
        _check(lib().pk_plan_set_weights(self.h, C.cast(w, C.POINTER(C.c_double))
                                         if w is not None else None), self.ctx)

    def grad_workspace_bytes(self, precision="c128") -> int:
        b = C.c_uint64()
        _check(lib().pk_grad_workspace_bytes(self.h, PRECISIONS[precision], C.byref(b)))
        return b.value

    def grad_stats(self) -> dict:
        out = (C.c_double * 10)()
        _check(lib().pk_grad_stats(self.h, out))
        keys = ("cmacs_forward", "cmacs_recompute", "cmacs_adjoint", "steps_forward",
                "steps_recompute", "steps_adjoint", "arena_elems", "checkpoints", "groups",
                "slices")
        return dict(zip(keys, list(out)))

    def stats(self) -> dict:
        s = pk_plan_stats()
        _check(lib().pk_plan_info(self.h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in s._fields_}

    def workspace_bytes(self, precision="c128") -> int:
        b = C.c_uint64()
        _check(lib().pk_plan_workspace_bytes(self.h, PRECISIONS[precision], C.byref(b)))
        return b.value

    def state_bytes(self, precision="c128"):
        """(state bytes, arena bytes) of the workspace split (pk_plan_state_bytes)."""
        s, a = C.c_uint64(), C.c_uint64()
        _check(lib().pk_plan_state_bytes(self.h, PRECISIONS[precision], C.byref(s), C.byref(a)))
        return s.value, a.value

    def launches(self, precision="c128") -> int:
        n = C.c_int64()
        _check(lib().pk_plan_launches(self.h, PRECISIONS[precision], C.byref(n)))
        return n.value

    def steps(self):
        n = self.stats()["n_steps"]
        arr = (C.c_int64 * max(1, 10 * n))()
        _check(lib().pk_plan_steps(self.h, arr))
        keys = ("a", "b", "c", "R", "K", "N", "rank_c", "kernel", "tc", "Bsz")
        return [dict(zip(keys, arr[10 * i:10 * i + 10])) for i in range(n)]

    def verify(self, precision="c128") -> str:
        """pk_plan_verify: '' when every index map and the memory layout check out, else the
        first violation."""
        buf = C.create_string_buffer(512)
        st = lib().pk_plan_verify(self.h, PRECISIONS[precision], buf, len(buf))
        if st not in (0, 1):
            _check(st)
        return "" if st == 0 else buf.value.decode()

    def combine_slices(self, slices):
        """pk_combine_slices: (Z, V) from all per-slice values (Scaled, in slice order)."""
        n = len(slices)
        arr = (pk_scaled * max(1, n))(*[pk_scaled(x.re, x.im, x.exp2) for x in slices])
        z, v = pk_scaled(), pk_scaled()
        st = lib().pk_combine_slices(self.h, arr, n, C.byref(z), C.byref(v))
        if st == 1 and n == self.stats()["n_slices"]:  # V undefined for this diagram
            _check(lib().pk_combine_slices(self.h, arr, n, C.byref(z), None))
            return Scaled.of(z), None
        _check(st)
        return Scaled.of(z), Scaled.of(v)

    def debug_blob(self, which: int) -> bytes:
        nb = C.c_uint64()
        _check(lib().pk_plan_debug_blob(self.h, which, None, C.byref(nb)))
        buf = (C.c_uint8 * max(1, nb.value))()
        _check(lib().pk_plan_debug_blob(self.h, which, buf, C.byref(nb)))
        return bytes(buf)[:nb.value]

    def __del__(self):
        try:
            if self.h:
                lib().pk_plan_destroy(self.h)
                self.h = None
        except Exception:
            pass


def _torch_stream(ctx: Context):
    import torch
    ctx.set_stream(torch.cuda.current_stream().cuda_stream)


def workspace(plan: Plan, precision="c128"):
    """A device workspace for `plan` from the PyTorch allocator."""
    import torch
    return torch.empty(plan.workspace_bytes(precision), dtype=torch.uint8,
                       device=f"cuda:{plan.ctx.device}")


def evaluate(plan: Plan, precision: str = "c128", ws=None):
    """Z(q) and V_K(t(q)) of the plan's knot on the GPU; returns (Z, V) as Scaled
    (V is None when the diagram is not a knot)."""
    ctx = plan.ctx
    if ctx.device < 0:
        raise PkError(7, "evaluate needs a GPU context")
    _torch_stream(ctx)
    if ws is None:
        ws = workspace(plan, precision)
    z, v = pk_scaled(), pk_scaled()
    st = lib().pk_eval(ctx.h, plan.h, PRECISIONS[precision], C.c_void_p(ws.data_ptr()),
                       ws.numel() * ws.element_size(), C.byref(z), C.byref(v))
    if st == 2:
        return Scaled.of(z), None
    _check(st, ctx)
    return Scaled.of(z), Scaled.of(v)


def evaluate_slices(plan: Plan, first: int, count: int, precision: str = "c128", ws=None):
    """pk_eval_slices: the contracted values of slices [first, first + count) as a list of
    Scaled (without the plan's constant factor; combine with Plan.combine_slices)."""
    ctx = plan.ctx
    if ctx.device < 0:
        raise PkError(7, "evaluate_slices needs a GPU context")
    _torch_stream(ctx)
    if ws is None:
        ws = workspace(plan, precision)
    out = (pk_scaled * count)()
    _check(lib().pk_eval_slices(ctx.h, plan.h, PRECISIONS[precision], C.c_void_p(ws.data_ptr()),
                                ws.numel() * ws.element_size(), int(first), int(count), out), ctx)
    return [Scaled.of(out[i]) for i in range(count)]


def plan_fingerprint(plan: Plan) -> str:
    """Digest of the plan's step records and scalars: equal for the same knot, q, options
    and library version, so a stored partial evaluation is only resumed on its own plan."""
    import hashlib
    h = hashlib.sha256()
    for which in (1, 3):
        h.update(plan.debug_blob(which))
    return h.hexdigest()


def evaluate_resumable(plan: Plan, path: str, precision: str = "c128", chunk: int = 64,
                       ws=None, run_slices=None, stop_after: int | None = None):
    """Z and V of a sliced evaluation that survives interruption: slices are run `chunk` at
    a time and, after each chunk, every value obtained so far is written to `path` (a JSON
    file replaced atomically, holding the plan's fingerprint and precision).  A later call
    with the same plan and path runs only the slices not yet stored.  `stop_after` ends the
    call (returning None) after that many chunks, for splitting a long evaluation across
    processes; `run_slices(first, count)` replaces the GPU call (evaluate_slices)."""
    import json
    n = plan.stats()["n_slices"]
    fp = plan_fingerprint(plan)
    done: dict[int, Scaled] = {}
    if os.path.exists(path):
        with open(path) as f:
            rec = json.load(f)
        if rec.get("fingerprint") != fp or rec.get("precision") != precision:
            raise ValueError(f"{path} belongs to another plan or precision")
        done = {int(k): Scaled(v[0], v[1], int(v[2])) for k, v in rec["slices"].items()}
    if run_slices is None:
        def run_slices(first, count):
            return evaluate_slices(plan, first, count, precision, ws)
    chunks = 0
    first = 0
    while first < n:
        if first in done:
            first += 1
            continue
        count = 1
        while count < chunk and first + count < n and first + count not in done:
            count += 1
        for i, v in enumerate(run_slices(first, count)):
            done[first + i] = v
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump({"fingerprint": fp, "precision": precision, "n_slices": n,
                       "slices": {str(k): [v.re, v.im, v.exp2] for k, v in sorted(done.items())}},
                      f)
        os.replace(tmp, path)
        first += count
        chunks += 1
        if stop_after is not None and chunks >= stop_after and len(done) < n:
            return None
    return plan.combine_slices([done[i] for i in range(n)])


def evaluate_exact(plan: Plan, primes, ws=None):
    """pk_eval_exact: Z(q) modulo each prime as (a, b) with Z = a + b t (t the Potts t(q)),
    computed on the GPU without rounding."""
    ctx = plan.ctx
    if ctx.device < 0:
        raise PkError(7, "evaluate_exact needs a GPU context")
    _torch_stream(ctx)
    n = len(primes)
    pr = (C.c_uint32 * n)(*[int(x) for x in primes])
    out = (C.c_uint32 * (2 * n))()
    if ws is None:
        ws = workspace(plan, "c64")
    _check(lib().pk_eval_exact(ctx.h, plan.h, pr, n, C.c_void_p(ws.data_ptr()),
                               ws.numel() * ws.element_size(), out), ctx)
    return [(out[2 * i], out[2 * i + 1]) for i in range(n)]


def jones_polynomial(ctx: Context, knot: Knot) -> dict:
    """pk_jones_coefficients: V(t) as {power of t: integer coefficient} (a link's half-integer
    powers as Fractions)."""
    if ctx.device < 0:
        raise PkError(7, "jones_polynomial needs a GPU context")
    _torch_stream(ctx)
    cap = 2 * knot.info()["n_c"] + 8
    coef = (C.c_int64 * cap)()
    lo, cnt, half = C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib().pk_jones_coefficients(ctx.h, knot.h, cap, C.byref(lo), C.byref(cnt), coef,
                                       C.byref(half)), ctx)
    return _poly(lo.value, cnt.value, coef, half.value)


def _poly(lo, cnt, coef, half):
    """{power of t: coefficient}; powers lowest + j + half/2 (Fractions when half)."""
    from fractions import Fraction
    out = {}
    for j in range(cnt):
        if coef[j]:
            out[lo + j + Fraction(1, 2) if half else lo + j] = coef[j]
    return out


def jones_plan(knot: Knot):
    """pk_jones_plan: (the q values, the moduli) the coefficient solve needs."""
    nq, npr = C.c_int32(), C.c_int32()
    _check(lib().pk_jones_plan(knot.h, C.byref(nq), None, C.byref(npr), None))
    qs = (C.c_int32 * nq.value)()
    pr = (C.c_uint32 * npr.value)()
    _check(lib().pk_jones_plan(knot.h, C.byref(nq), qs, C.byref(npr), pr))
    return list(qs), list(pr)


def jones_solve(knot: Knot, qs, primes, zab) -> dict:
    """pk_jones_solve (host only): V's coefficients from zab[iq][ip] = (a, b), Z(qs[iq]) =
    a + b t mod primes[ip]."""
    nq, npr = len(qs), len(primes)
    q_arr = (C.c_int32 * nq)(*qs)
    p_arr = (C.c_uint32 * npr)(*primes)
    flat = [int(v) for row in zab for pair in row for v in pair]
    z_arr = (C.c_uint32 * len(flat))(*flat)
    cap = 2 * knot.info()["n_c"] + 8
    coef = (C.c_int64 * cap)()
    lo, cnt, half = C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib().pk_jones_solve(knot.h, nq, q_arr, npr, p_arr, z_arr, cap, C.byref(lo), C.byref(cnt),
                                coef, C.byref(half)))
    return _poly(lo.value, cnt.value, coef, half.value)


def evaluate_noalloc(plan: Plan, precision: str = "c128"):
    """pk_eval_noalloc: like evaluate() but allocates nothing; the library's fixed 64 MiB
    per-device scratch array holds the workspace (see include/pk.h)."""
    ctx = plan.ctx
    if ctx.device < 0:
        raise PkError(7, "evaluate_noalloc needs a GPU context")
    z, v = pk_scaled(), pk_scaled()
    st = lib().pk_eval_noalloc(ctx.h, plan.h, PRECISIONS[precision], C.byref(z), C.byref(v))
    if st == 2:
        return Scaled.of(z), None
    _check(st, ctx)
    return Scaled.of(z), Scaled.of(v)


def upload(plan: Plan, precision: str, ws):
    _check(lib().pk_upload(plan.ctx.h, plan.h, PRECISIONS[precision], C.c_void_p(ws.data_ptr()),
                           ws.numel()), plan.ctx)


def upload_inputs(plan: Plan, precision: str, ws) -> int:
    """pk_upload_inputs: the knot-derived part of the program only (after one upload)."""
    n = C.c_uint64()
    _check(lib().pk_upload_inputs(plan.ctx.h, plan.h, PRECISIONS[precision],
                                  C.c_void_p(ws.data_ptr()), ws.numel(), C.byref(n)), plan.ctx)
    return n.value


def launch(plan: Plan, precision: str, ws):
    _check(lib().pk_launch(plan.ctx.h, plan.h, PRECISIONS[precision], C.c_void_p(ws.data_ptr()),
                           ws.numel()), plan.ctx)


def launch_arena(plan: Plan, precision: str, state, arena):
    """pk_launch_arena: the plan's state buffer and a (possibly shared) tensor arena."""
    _check(lib().pk_launch_arena(plan.ctx.h, plan.h, PRECISIONS[precision],
                                 C.c_void_p(state.data_ptr()), state.numel(),
                                 C.c_void_p(arena.data_ptr()), arena.numel()), plan.ctx)


def download(plan: Plan, precision: str, ws):
    z, v = pk_scaled(), pk_scaled()
    st = lib().pk_download(plan.ctx.h, plan.h, PRECISIONS[precision], C.c_void_p(ws.data_ptr()),
                           C.byref(z), C.byref(v))
    if st == 2:
        return Scaled.of(z), None
    _check(st, plan.ctx)
    return Scaled.of(z), Scaled.of(v)


def decode_result(plan: Plan, re: float, im: float, exp2: int, status: int = 0):
    """pk_decode_result (host only): (status code, Z, V) from a total record as the device
    leaves it (value (re + i im) 2^exp2 and the evaluation's error word)."""
    import struct
    rec = C.create_string_buffer(struct.pack("<ddqQ", re, im, exp2, status), 32)
    z, v = pk_scaled(), pk_scaled()
    st = lib().pk_decode_result(plan.h, rec, C.byref(z), C.byref(v))
    return st, Scaled.of(z), Scaled.of(v)


def profile(plan: Plan, precision: str, ws, arena=None):
    """Per kernel class (build, rows, splitk, results, gemm, gemm_tc): ms, launches, complex MACs,
    bytes of one pass of the plan's kernels, timed with CUDA events on the context's
    stream.  `arena` (optional) is a separate tensor arena as for launch_arena()."""
    out = (C.c_double * 35)()
    ap = C.c_void_p(arena.data_ptr()) if arena is not None else None
    an = arena.numel() if arena is not None else 0
    _check(lib().pk_profile(plan.ctx.h, plan.h, PRECISIONS[precision], C.c_void_p(ws.data_ptr()),
                            ws.numel(), ap, an, out), plan.ctx)
    return _classes(out)


CLASSES = ("build", "rows", "splitk", "results", "gemm", "gemm_tc", "digits")


def _classes(out):
    n = len(CLASSES)
    return {c: {"ms": out[i], "launches": out[n + i], "cmacs": out[2 * n + i],
                "bytes": out[3 * n + i], "fill_ms": out[4 * n + i]} for i, c in enumerate(CLASSES)}


class Batch:
    """pk_batch: many planned knots evaluated by one persistent launch (CUDA graph)."""

    def __init__(self, plans, precision="split"):
        self.plans = list(plans)
        self.ctx = self.plans[0].ctx
        self.precision = precision
        arr = (C.c_void_p * len(self.plans))(*[p.h.value for p in self.plans])
        h = C.c_void_p()
        _check(lib().pk_batch_create(self.ctx.h, arr, len(self.plans), PRECISIONS[precision],
                                     C.byref(h)), self.ctx)
        self.h = h

    def workspace_bytes(self):
        b, u = C.c_uint64(), C.c_uint64()
        _check(lib().pk_batch_workspace_bytes(self.h, C.byref(b), C.byref(u)))
        return b.value, u.value

    def upload(self, ws):
        _check(lib().pk_batch_upload(self.ctx.h, self.h, C.c_void_p(ws.data_ptr()), ws.numel()),
               self.ctx)

    def upload_inputs(self, ws) -> int:
        """pk_batch_upload_inputs: the knot-derived part only (after one upload); bytes copied."""
        n = C.c_uint64()
        _check(lib().pk_batch_upload_inputs(self.ctx.h, self.h, C.c_void_p(ws.data_ptr()),
                                            ws.numel(), C.byref(n)), self.ctx)
        return n.value

    def launch(self, ws):
        _check(lib().pk_batch_launch(self.ctx.h, self.h, C.c_void_p(ws.data_ptr()), ws.numel()),
               self.ctx)

    def download(self, ws):
        n = len(self.plans)
        z = (pk_scaled * n)()
        v = (pk_scaled * n)()
        st = lib().pk_batch_download(self.ctx.h, self.h, C.c_void_p(ws.data_ptr()), z, v)
        if st not in (0, 2):
            _check(st, self.ctx)
        return [Scaled.of(x) for x in z], [Scaled.of(x) for x in v]

    def __del__(self):
        try:
            if self.h:
                lib().pk_batch_destroy(self.h)
                self.h = None
        except Exception:
            pass


def evaluate_batch(plans, precision="split", ws=None):
    """Z and V of every plan's knot from one persistent launch; returns two lists."""
    import torch
    b = Batch(plans, precision)
    _torch_stream(b.ctx)
    if ws is None:
        ws = torch.empty(b.workspace_bytes()[0], dtype=torch.uint8, device=f"cuda:{b.ctx.device}")
    b.upload(ws)
    b.launch(ws)
    return b.download(ws)


class Group:
    """pk_group: plans (each with its own uploaded workspace) replayed concurrently as
    independent branches of one CUDA graph.  profiled=True brackets every launch with
    event-record nodes (pk_group_create_profiled); profile() then reads the last replay."""

    def __init__(self, plans, precision, workspaces, profiled=False):
        self.plans = list(plans)
        self.ctx = self.plans[0].ctx
        self.ws = list(workspaces)
        n = len(self.plans)
        parr = (C.c_void_p * n)(*[p.h.value for p in self.plans])
        warr = (C.c_void_p * n)(*[w.data_ptr() for w in self.ws])
        barr = (C.c_uint64 * n)(*[w.numel() for w in self.ws])
        h = C.c_void_p()
        fn = lib().pk_group_create_profiled if profiled else lib().pk_group_create
        _check(fn(self.ctx.h, parr, n, PRECISIONS[precision], warr, barr, C.byref(h)), self.ctx)
        self.h = h
        self.precision = PRECISIONS[precision]

    def launch(self):
        _check(lib().pk_group_launch(self.ctx.h, self.h), self.ctx)

    def upload(self, inputs_only=False) -> int:
        """pk_group_upload: every plan's program (or with inputs_only its knot-derived part,
        after one full upload) into its workspace; the bytes copied."""
        n = C.c_uint64()
        _check(lib().pk_group_upload(self.ctx.h, self.h, int(inputs_only), C.byref(n)), self.ctx)
        return n.value

    def download(self):
        """pk_group_download: [(Z, V)] of every plan, one wait for the stream."""
        n = len(self.plans)
        z, v, st = (pk_scaled * n)(), (pk_scaled * n)(), (C.c_int32 * n)()
        _check(lib().pk_group_download(self.ctx.h, self.h, z, v, st), self.ctx)
        return [(Scaled.of(a), Scaled.of(b)) for a, b in zip(z, v)]

    def profile(self):
        """Per kernel class: summed in-replay launch durations (ms), launches, complex
        multiply-adds, algorithmic bytes of the last replay."""
        out = (C.c_double * 35)()
        _check(lib().pk_group_profile(self.ctx.h, self.h, out), self.ctx)
        return _classes(out)

    def timeline(self):
        """The last replay of a profiled group, one tuple per launch: (plan index, class
        name, start ms, end ms, complex multiply-adds, algorithmic bytes)."""
        n = C.c_int64()
        cap = max(1, sum(p.launches(PRECISION_NAMES[self.precision]) for p in self.plans) * 2)
        buf = (C.c_double * (6 * cap))()
        _check(lib().pk_group_timeline(self.ctx.h, self.h, buf, cap, C.byref(n)), self.ctx)
        return [(int(buf[6 * i]), CLASSES[int(buf[6 * i + 1])], buf[6 * i + 2], buf[6 * i + 3],
                 buf[6 * i + 4], buf[6 * i + 5]) for i in range(n.value)]

    def __del__(self):
        try:
            if self.h:
                lib().pk_group_destroy(self.h)
                self.h = None
        except Exception:
            pass


# ----------------------------------------------------------------------------- reverse pass

def grad(plan: Plan, precision: str = "c128", ws=None):
    """pk_grad: Z, V, (1/Z) dZ/dT_e[a, b] for every Tait edge e (numpy complex128 array of
    shape (n_e, q, q)) and (1/V) dV/dt at fixed q.  The plan needs grad=True."""
    import numpy as np
    ctx = plan.ctx
    if ctx.device < 0:
        raise PkError(7, "grad needs a GPU context")
    _torch_stream(ctx)
    if ws is None:
        import torch
        ws = torch.empty(plan.grad_workspace_bytes(precision), dtype=torch.uint8,
                         device=f"cuda:{ctx.device}")
    q, n_e = plan.q, plan.n_e
    z, v = pk_scaled(), pk_scaled()
    dl = (C.c_double * max(1, 2 * n_e * q * q))()
    dv = (C.c_double * 2)()
    st = lib().pk_grad(ctx.h, plan.h, PRECISIONS[precision], C.c_void_p(ws.data_ptr()),
                       ws.numel() * ws.element_size(), C.byref(z), C.byref(v), dl, dv)
    knot_ok = st != 2
    if st == 2:  # not a knot: Z and the derivatives of log Z are still defined
        st = lib().pk_grad(ctx.h, plan.h, PRECISIONS[precision], C.c_void_p(ws.data_ptr()),
                           ws.numel() * ws.element_size(), C.byref(z), None, dl, None)
    _check(st, ctx)
    arr = np.frombuffer(dl, dtype=np.float64)[:2 * n_e * q * q].copy()
    dlogz = (arr[0::2] + 1j * arr[1::2]).reshape(n_e, q, q)
    return (Scaled.of(z), Scaled.of(v) if knot_ok else None, dlogz,
            complex(dv[0], dv[1]) if knot_ok else None)


def grad_from_accumulators(plan: Plan, acc, acc_exp, z: Scaled):
    """pk_grad_from_accumulators (host only): the last stage of pk_grad from per-group
    adjoint accumulators (acc: complex array (groups, q*q); acc_exp: int array)."""
    import numpy as np
    q, n_e = plan.q, plan.n_e
    a = np.ascontiguousarray(np.asarray(acc, dtype=np.complex128).reshape(-1)).view(np.float64)
    a = np.ascontiguousarray(a)
    ex = np.ascontiguousarray(np.asarray(acc_exp, dtype=np.int64))
    zz = pk_scaled(z.re, z.im, z.exp2)
    dl = (C.c_double * max(1, 2 * n_e * q * q))()
    dv = (C.c_double * 2)()
    _check(lib().pk_grad_from_accumulators(
        plan.h, a.ctypes.data_as(C.POINTER(C.c_double)) if a.size else None,
        ex.ctypes.data_as(C.POINTER(C.c_int64)) if ex.size else None, C.byref(zz), dl, dv))
    arr = np.frombuffer(dl, dtype=np.float64)[:2 * n_e * q * q].copy()
    return (arr[0::2] + 1j * arr[1::2]).reshape(n_e, q, q), complex(dv[0], dv[1])


def grad_weights(plan: Plan, dlogz):
    """pk_grad_weights (host only): (n_e, 2) complex array of d log Z / d(diagonal weight)
    and d log Z / d(off-diagonal weight) per Tait edge, from pk_grad's (n_e, q, q) array."""
    import numpy as np
    d = np.ascontiguousarray(np.asarray(dlogz, dtype=np.complex128)).view(np.float64)
    d = np.ascontiguousarray(d)
    out = (C.c_double * max(1, 4 * plan.n_e))()
    _check(lib().pk_grad_weights(plan.h, d.ctypes.data_as(C.POINTER(C.c_double)), out))
    arr = np.frombuffer(out, dtype=np.float64)[:4 * plan.n_e]
    return (arr[0::2] + 1j * arr[1::2]).reshape(plan.n_e, 2)


_LOGZ_FN = None


def _logz_function():
    global _LOGZ_FN
    if _LOGZ_FN is not None:
        return _LOGZ_FN
    import math

    import torch

    class LogZ(torch.autograd.Function):
        """log Z as a function of the clause weights, (n_e, 2) complex128 = (diagonal,
        off-diagonal) per Tait edge.  The forward runs pk_grad (contraction and reverse
        pass on the GPU); the backward returns the saved holomorphic derivatives in
        PyTorch's convention for complex inputs (grad_output times their conjugate)."""

        @staticmethod
        def forward(ctx, weights, plan, precision):
            plan.set_weights([(complex(d), complex(o)) for d, o in weights.detach().cpu().tolist()])
            z, _, dlogz, _ = grad(plan, precision)
            jac = torch.as_tensor(grad_weights(plan, dlogz), dtype=torch.complex128)
            ctx.save_for_backward(jac.to(weights.device))
            logz = complex(math.log(abs(z.mantissa)) + z.exp2 * math.log(2.0),
                           math.atan2(z.im, z.re))
            return torch.tensor(logz, dtype=torch.complex128, device=weights.device)

        @staticmethod
        def backward(ctx, g):
            (jac,) = ctx.saved_tensors
            return g * jac.conj(), None, None

    _LOGZ_FN = LogZ
    return LogZ


def log_z(plan: Plan, weights, precision: str = "c128"):
    """torch: log Z(weights) with autograd through the reverse pass (plan made with
    grad=True).  weights: complex128 tensor (n_e, 2) of (diagonal, off-diagonal) clause
    weights per Tait edge.  The imaginary part is the principal argument of Z."""
    return _logz_function().apply(weights, plan, precision)
