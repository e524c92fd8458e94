"""pk_eval_noalloc, the evaluation entry point for callers that cannot allocate device
memory (for example code inside a host application whose own allocator has reserved the
GPU's memory).  It must give the same Z and V as pk_eval, on consecutive calls that reuse
its fixed scratch array, and refuse plans that do not fit that array.

This file is named so that pytest collects it last; it also passes on its own in a fresh
process (the first call on the device sets the scratch address up).
"""
import ctypes as C

import pytest

import knotgen as kg
import paper_1807_02119_gb300 as pk
from oracle.scaled import SC, rel_err

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "c64": 1e-4}   # the tolerances of the other GPU parity tests
NOALLOC_LIMIT = 64 << 20


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = pk.Context(0)
    c.set_stream(torch.cuda.current_stream().cuda_stream)
    return c


def call_noalloc(plan, prec):
    """Through the C ABI directly: status, Z, V."""
    z, v = pk.pk_scaled(), pk.pk_scaled()
    st = pk.lib().pk_eval_noalloc(plan.ctx.h, plan.h, pk.PRECISIONS[prec], C.byref(z), C.byref(v))
    return st, pk.Scaled.of(z), pk.Scaled.of(v)


def sc(s):
    return SC.of(s.mantissa, s.exp2)


def _plans(ctx):
    out = []
    (tiny,) = kg.knot_suite("tiny")
    cases = [(tiny.pd, tiny.outer, 2), (kg.braid_closure_pd([1, 1, 1], 2), None, 3)]
    for s in range(4):
        gk = kg.random_grid_knot(16, 2100 + s, True, 20, 45)
        cases += [(gk.pd, gk.outer, 3), (gk.pd, gk.outer, 5)]
    gk = kg.random_grid_knot(18, 2200, True, 40, 70)
    cases.append((gk.pd, gk.outer, 3))
    for pd, outer, q in cases:
        k = pk.Knot.from_pd(ctx, pd, outer=outer)
        p = pk.Plan(ctx, k, q)
        if p.workspace_bytes("c128") <= NOALLOC_LIMIT:
            out.append(p)
    # a full-size knot of the L=40 workload whose workspace is several MiB
    for seed in range(1, 40):
        big = kg.random_grid_knot(40, seed, True, 100, 400)
        p = pk.Plan(ctx, pk.Knot.from_pd(ctx, big.pd, outer=big.outer), 3)
        if 4 << 20 < p.workspace_bytes("c128") <= NOALLOC_LIMIT:
            out.append(p)
            break
    # one sliced plan (several slices share the scratch within one call)
    k = pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer)
    full = pk.Plan(ctx, k, 2).stats()["log2_max_elems"]
    out.append(pk.Plan(ctx, k, 2, max_log2_elems=full - 2))
    return out


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_noalloc_matches_pk_eval_twice(ctx, prec):
    plans = _plans(ctx)
    assert len(plans) >= 8
    refs = [pk.evaluate(p, prec) for p in plans]
    for rnd in range(2):                       # two calls in a row for every plan
        for p, (zr, vr) in zip(plans, refs):
            st, z, v = call_noalloc(p, prec)
            assert st == 0, pk.lib().pk_last_error(ctx.h)
            assert rel_err(sc(z), sc(zr)) <= TOL[prec], (rnd, p.q)
            assert rel_err(sc(v), sc(vr)) <= TOL[prec], (rnd, p.q)


def test_noalloc_refuses_oversized_plan(ctx):
    gk = kg.random_grid_knot(40, 4, True, 100, 400)   # 40 GB workspace at q=5 in complex128
    p = pk.Plan(ctx, pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer), 5)
    assert p.workspace_bytes("c128") > NOALLOC_LIMIT
    st, _, _ = call_noalloc(p, "c128")
    assert st == 3
    assert b"static scratch" in pk.lib().pk_last_error(ctx.h)
