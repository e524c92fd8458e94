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
import oracle
import paper_1807_02119_gb300 as pk
from oracle.scaled import SC, rel_err

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "c64": 1e-4, "split": 1e-6}   # the tolerances of the other GPU parity tests
NOALLOC_LIMIT = 64 << 20
# L=30 grid-walk knots whose q=5 plans put GEMM-shaped steps on the tensor cores (split
# precision: digit scratch after the arena) and still fit the 64 MiB scratch array: seed
# 35 (119 crossings, two such steps, K up to 625 complex: several flush groups) and
# seed 8 (113 crossings, K up to 125)
TC_KNOTS = ((30, 35, 60, 160), (30, 8, 60, 160))


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


def _tc_plans(ctx):
    out = []
    for L, seed, lo, hi in TC_KNOTS:
        gk = kg.random_grid_knot(L, seed, True, lo, hi)
        p = pk.Plan(ctx, pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer), 5)
        out.append((gk, p))
    return out


def _plans(ctx, prec="c128"):
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
        if p.workspace_bytes(prec) <= NOALLOC_LIMIT:
            out.append(p)
    # a full-size knot of the L=40 workload whose workspace is several MiB
    for seed in range(1, 40):
        big = kg.random_grid_knot(40, seed, True, 100, 400)
        p = pk.Plan(ctx, pk.Knot.from_pd(ctx, big.pd, outer=big.outer), 3)
        if 4 << 20 < p.workspace_bytes(prec) <= NOALLOC_LIMIT:
            out.append(p)
            break
    # one sliced plan (several slices share the scratch within one call)
    k = pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer)
    full = pk.Plan(ctx, k, 2).stats()["log2_max_elems"]
    out.append(pk.Plan(ctx, k, 2, max_log2_elems=full - 2))
    if prec == "split":
        out += [p for _, p in _tc_plans(ctx) if p.workspace_bytes(prec) <= NOALLOC_LIMIT]
    return out


@pytest.mark.parametrize("prec", ["c128", "c64", "split"])
def test_noalloc_matches_pk_eval_twice(ctx, prec):
    plans = _plans(ctx, prec)
    assert len(plans) >= 8
    if prec == "split":   # the tensor-core GEMM and its digit scratch run inside the array
        assert sum(any(st["kernel"] == 2 for st in p.steps()) for p in plans) >= 2
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


def test_noalloc_split_tensor_core_plans_match_oracle(ctx):
    """The split precision's tensor-core steps through the static scratch array against
    the CPU oracle (Sec. II spin sum, Eq. JonesPotts), on two calls in a row."""
    for gk, p in _tc_plans(ctx):
        assert p.workspace_bytes("split") <= NOALLOC_LIMIT
        assert any(st["kernel"] == 2 and st["K"] > 96 for st in p.steps())
        g = oracle.tait_graph(gk.pd, outer=gk.outer)
        from oracle.order import min_fill_order
        order, _ = min_fill_order(g.n_v, g.edges, 5)
        zo = oracle.z_complex(g.n_v, g.edges, 5, order=order, sum_inside=True)
        vo = oracle.jones_from_z(zo, g, 5)
        for rnd in range(2):
            st, z, v = call_noalloc(p, "split")
            assert st == 0, pk.lib().pk_last_error(ctx.h)
            assert rel_err(sc(z), zo) <= TOL["split"], (gk.seed, rnd)
            assert rel_err(sc(v), vo) <= TOL["split"], (gk.seed, rnd)
