"""GPU checks of the debugging aids (finite check, plan verification, NVTX ranges) and of
evaluation by slices with resume, against the recorded-graph evaluation and the oracle.
"""
import math
import re

import pytest

import knotgen as kg
import oracle
import paper_1807_02119_gb300 as pk
from oracle.order import min_fill_order
from oracle.scaled import SC, rel_err

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "c64": 1e-4, "split": 1e-6}   # the tolerances of the other GPU parity tests
ALL_DEBUG = pk.DEBUG_CHECK_FINITE | pk.DEBUG_VERIFY | pk.DEBUG_NVTX


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = pk.Context(0)
    c.set_stream(torch.cuda.current_stream().cuda_stream)
    return c


def sc(s):
    return SC.of(s.mantissa, s.exp2)


def _knot(ctx, L, seed, lo=1, hi=10 ** 6):
    gk = kg.random_grid_knot(L, seed, True, lo, hi)
    return gk, pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer)


def _oracle_z(gk, q):
    g = oracle.tait_graph(gk.pd, outer=gk.outer)
    order, _ = min_fill_order(g.n_v, g.edges, q)
    return oracle.z_complex(g.n_v, g.edges, q, order=order, sum_inside=True)


def test_debug_launches_match_graph_and_oracle(ctx):
    """Every debug flag on (plan verified before the launch, NaN/Inf scan after the initial
    tensors and after every step with sequence runs split into single steps, an NVTX range
    per launch): the same Z as the recorded graph and the oracle, in all three precisions,
    including tensor-core steps with several flush groups (L=30 seed 35 at q=5) and a
    complex64 plan with a complex128 tail."""
    cases = [((20, 3), 3, "c128", {}), ((20, 3), 3, "c64", dict(tail_steps=2)),
             ((20, 3), 3, "split", {}), ((30, 35), 5, "split", {}), ((30, 35), 5, "c128", {})]
    zo_cache = {}
    for (L, seed), q, prec, kw in cases:
        gk, k = _knot(ctx, L, seed)
        if (L, seed, q) not in zo_cache:
            zo_cache[(L, seed, q)] = _oracle_z(gk, q)
        zo = zo_cache[(L, seed, q)]
        p = pk.Plan(ctx, k, q, **kw)
        assert p.verify(prec) == ""
        z0, _ = pk.evaluate(p, prec)
        ctx.set_debug(ALL_DEBUG)
        try:
            z1, _ = pk.evaluate(p, prec)
        finally:
            ctx.set_debug(0)
        # single steps instead of sequence runs may sum in another order
        assert rel_err(sc(z1), sc(z0)) <= (1e-13 if prec == "c128" else 1e-5 if prec == "c64" else 1e-9)
        assert rel_err(sc(z1), zo) <= TOL[prec], (L, seed, q, prec)


def test_finite_check_reports_a_planted_nan(ctx):
    """A NaN planted on the host into the uploaded program (one clause value of the
    initial tensors, written into the workspace after pk_upload) propagates to Z.  Without
    the check pk_download returns PK_OK with a NaN Z; with it pk_download reports
    PK_ENONFINITE for step -1 (the initial tensors) of slice 0, the first tensor written,
    and the next evaluation on the same context is clean."""
    import ctypes as C
    import struct
    import torch
    gk, k = _knot(ctx, 20, 3)
    p = pk.Plan(ctx, k, 3)
    sc_ = [int(v) for v in struct.unpack(f"<{len(p.debug_blob(3)) // 8}q", p.debug_blob(3))]
    off_slots, n_slots = sc_[7], sc_[8]
    prog = p.debug_blob(0)
    slot_sz = 48
    absorbed = [i for i in range(n_slots)
                if struct.unpack_from("<4i", prog, off_slots + i * slot_sz)[2] == 1]
    assert absorbed
    at = off_slots + absorbed[0] * slot_sz + 16          # the slot's diagonal (re)
    nan = torch.tensor(list(struct.pack("<d", float("nan"))), dtype=torch.uint8, device="cuda")
    L = pk.lib()
    for flags in (0, pk.DEBUG_CHECK_FINITE):
        ws = pk.workspace(p, "c128")
        nb = ws.numel()
        ctx.set_debug(flags)
        try:
            assert L.pk_upload(ctx.h, p.h, 0, C.c_void_p(ws.data_ptr()), nb) == 0
            ws[at:at + 8].copy_(nan)                     # same stream: after the upload
            assert L.pk_launch(ctx.h, p.h, 0, C.c_void_p(ws.data_ptr()), nb) == 0
            z, v = pk.pk_scaled(), pk.pk_scaled()
            st = L.pk_download(ctx.h, p.h, 0, C.c_void_p(ws.data_ptr()), C.byref(z), C.byref(v))
        finally:
            ctx.set_debug(0)
        if flags == 0:
            assert st == 0 and math.isnan(z.re)
        else:
            assert st == 9
            msg = L.pk_last_error(ctx.h).decode()
            assert "step -1 of slice 0" in msg, msg
    z2, _ = pk.evaluate(p, "c128")
    assert rel_err(sc(z2), _oracle_z(gk, 3)) <= TOL["c128"]


def test_large_and_small_weights_on_the_gpu(ctx):
    """Clause matrices scaled by exact powers of two 2^s_e, |s_e| up to 1000 (raw entry
    products would leave the FP64 range, and the float range of the split precision by
    far): Z equals the oracle's Z of the unscaled knot times 2^(sum s_e), in complex128 and
    in split precision with tensor-core steps (L=30 seed 35, q=5)."""
    from oracle.potts import clause_diag
    for (L, seed), q in (((20, 3), 3), ((30, 35), 5)):
        gk, k = _knot(ctx, L, seed)
        rng = kg.SplitMix64(7 * L + q)
        w, tot = [], 0
        for (_, _, eps) in k.edges():
            s_e = int(rng.below(2001)) - 1000
            w.append((clause_diag(q, eps) * 2.0 ** s_e, 2.0 ** s_e + 0j))
            tot += s_e
        zo = _oracle_z(gk, q) * SC.of(1.0 + 0j, tot)
        p = pk.Plan(ctx, k, q, weights=w)
        for prec in ("c128", "split"):
            z, _ = pk.evaluate(p, prec)
            assert rel_err(sc(z), zo) <= TOL[prec], (L, seed, q, prec)


def test_slices_sum_to_the_evaluation_and_resume(ctx, tmp_path):
    """A 61-crossing knot at q=3 sliced into 81 sub-contractions (Sec. III slicing): the
    per-slice values of pk_eval_slices, taken in three uneven ranges, combine to pk_eval's
    Z and the oracle's; evaluate_resumable interrupted after two chunks and resumed by a
    new plan object gives the same Z bit for bit."""
    gk, k = _knot(ctx, 24, 11)
    zo = _oracle_z(gk, 3)
    mr = pk.Plan(ctx, k, 3).stats()["max_rank"]
    lim = (mr - 2) * math.log2(3)
    for prec in ("c128", "split"):
        p = pk.Plan(ctx, k, 3, max_log2_elems=lim)
        n = p.stats()["n_slices"]
        assert n >= 27
        z_all, v_all = pk.evaluate(p, prec)
        vals = []
        for first, count in ((0, 5), (5, n - 12), (n - 7, 7)):
            vals += pk.evaluate_slices(p, first, count, prec)
        z, v = p.combine_slices(vals)
        assert rel_err(sc(z), sc(z_all)) <= (1e-12 if prec == "c128" else 1e-9)
        assert rel_err(sc(v), sc(v_all)) <= (1e-12 if prec == "c128" else 1e-9)
        assert rel_err(sc(z), zo) <= TOL[prec]
        # the finite check on a range leaves its values unchanged
        ctx.set_debug(pk.DEBUG_CHECK_FINITE)
        try:
            again = pk.evaluate_slices(p, 5, 9, prec)
        finally:
            ctx.set_debug(0)
        assert all(rel_err(sc(a), sc(b)) <= 1e-12 for a, b in zip(again, vals[5:14]))
        path = str(tmp_path / f"{prec}.json")
        assert pk.evaluate_resumable(p, path, prec, chunk=10, stop_after=2) is None
        p2 = pk.Plan(ctx, k, 3, max_log2_elems=lim)
        z3, v3 = pk.evaluate_resumable(p2, path, prec, chunk=10)
        assert (z3, v3) == (z, v)
        with pytest.raises(pk.PkError):
            pk.evaluate_slices(p, n - 1, 2, prec)
