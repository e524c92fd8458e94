"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances: complex128 relative error <= 1e-10 on Z and V; complex64 (FP32 arithmetic)
relative error <= C64_TOL, and V within 1e-10 (c128) of exactly 1, +-1, 1 at the easy
points q = 1, 2, 4.
"""
import math

import pytest

import knotgen as kg
import oracle
import paper_1807_02119_gb300 as pk
from oracle.potts import exact_to_complex
from oracle.scaled import SC, rel_err

pytestmark = pytest.mark.gpu

C128_TOL = 1e-10
C64_TOL = 1e-4


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pk.lib()
    return pk.Context(0)


def sc(s):
    return SC.of(s.mantissa, s.exp2)


def run(ctx, pd, q, prec, outer=None, **kw):
    k = pk.Knot.from_pd(ctx, pd, outer=outer)
    p = pk.Plan(ctx, k, q, **kw)
    z, v = pk.evaluate(p, prec)
    return sc(z), (sc(v) if v is not None else None), p


def oracle_zv(pd, q, outer=None):
    g = oracle.tait_graph(pd, outer=outer, black=None if outer else 0)
    z = oracle.z_complex(g.n_v, g.edges, q)
    return z, oracle.jones_from_z(z, g, q)


TREFOIL = kg.braid_closure_pd([1, 1, 1], 2)
FIG8 = kg.braid_closure_pd([1, -2, 1, -2], 3)


def test_tiny_config_q2(ctx):
    (gk,) = kg.knot_suite("tiny")
    z, v, _ = run(ctx, gk.pd, 2, "c128", outer=gk.outer)
    zo, vo = oracle_zv(gk.pd, 2, outer=gk.outer)
    assert rel_err(z, zo) <= C128_TOL
    assert rel_err(v, vo) <= C128_TOL
    vc = v.to_complex()
    assert abs(vc.imag) < 1e-10 and abs(abs(vc.real) - 1) < 1e-10


@pytest.mark.parametrize("prec,tol", [("c128", C128_TOL), ("c64", C64_TOL)])
def test_closed_forms(ctx, prec, tol):
    cases = [(TREFOIL, {1: 1, 3: 1, 4: -1}), (FIG8, {-2: 1, -1: -1, 0: 1, 1: -1, 2: 1}),
             ([], {0: 1}), (kg.kink([], 0, 2), {0: 1})]
    for pd, poly in cases:
        for q in range(1, 7):
            _, v, _ = run(ctx, pd, q, prec)
            want = exact_to_complex(kg_eval(poly, q), 1, q)
            assert rel_err(v, want) <= tol, (pd, q, prec)


def kg_eval(poly, q):
    from oracle.ring import Zt
    return Zt(q).eval_laurent(poly)


@pytest.mark.parametrize("order", ["greedy_edge", "greedy_spin", "elim_spin", "fill_spin", "partition"])
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_random_knots_vs_oracle(ctx, order, prec):
    worst = 0.0
    for s in range(10):
        gk = kg.random_grid_knot(16, 500 + s, True, 20, 45)
        for q in (2, 3, 5):
            z, v, _ = run(ctx, gk.pd, q, prec, outer=gk.outer, order=order)
            zo, vo = oracle_zv(gk.pd, q, outer=gk.outer)
            ez, ev = rel_err(z, zo), rel_err(v, vo)
            worst = max(worst, ez, ev)
            assert ez <= (C128_TOL if prec == "c128" else C64_TOL), (s, q, ez)
    print(f"[{order} {prec}] worst relative error {worst:.3e}")


def test_slicing_gpu(ctx):
    for s in range(4):
        gk = kg.random_grid_knot(18, 700 + s, True, 40, 70)
        k = pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer)
        for q in (2, 3):
            full = pk.Plan(ctx, k, q).stats()["log2_max_elems"]
            lim = full - 1.5 * math.log2(q)      # forces at least one sliced index
            z, v, p = run(ctx, gk.pd, q, "c128", outer=gk.outer, max_log2_elems=lim)
            assert p.stats()["n_slices"] > 1
            zo, _ = oracle_zv(gk.pd, q, outer=gk.outer)
            assert rel_err(z, zo) <= C128_TOL


def test_splitk_steps(ctx):
    """Plans whose final contractions have few outputs and long K go to the split-K kernel."""
    found = 0
    for s in range(40):
        gk = kg.random_grid_knot(20, 900 + s, True, 50, 90)
        k = pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer)
        p = pk.Plan(ctx, k, 3, order="greedy_edge")
        if any(st["kernel"] == 1 for st in p.steps()):
            for prec, tol in (("c128", C128_TOL), ("c64", C64_TOL)):
                z, _ = pk.evaluate(p, prec)
                zo, _ = oracle_zv(gk.pd, 3, outer=gk.outer)
                assert rel_err(sc(z), zo) <= tol
            found += 1
            if found >= 2:
                break
    assert found >= 1


def test_easy_points_full_size(ctx):
    """Full-size L=40 knots of the 64-knot workload: V = 1 at q = 1 and q = 4, V = +-1 at
    q = 2 (properties that hold at any size), in complex128."""
    ks = kg.knot_suite("scale")
    for gk in ks[:6]:
        for q, want in ((1, [1]), (4, [1]), (2, [1, -1])):
            _, v, _ = run(ctx, gk.pd, q, "c128", outer=gk.outer)
            vc = v.to_complex()
            assert min(abs(vc - w) for w in want) < 1e-10, (gk.seed, q, vc)


def test_full_size_orders_agree_and_oracle_sample(ctx):
    """Two contraction orders give the same Z at full size; a sample of q=3 knots of the
    64-knot workload is checked against the oracle."""
    ks = kg.knot_suite("scale")
    for gk in ks[:4]:
        z1, v1, _ = run(ctx, gk.pd, 3, "c128", outer=gk.outer, order="elim_spin")
        z2, v2, _ = run(ctx, gk.pd, 3, "c128", outer=gk.outer, order="greedy_spin")
        assert rel_err(z1, z2) <= C128_TOL
        zo, vo = oracle_zv(gk.pd, 3, outer=gk.outer)
        assert rel_err(z1, zo) <= C128_TOL and rel_err(v1, vo) <= C128_TOL


def test_reidemeister_copy_same_v(ctx):
    rng = kg.SplitMix64(31)
    for s in range(4):
        gk = kg.random_grid_knot(16, 800 + s, True, 20, 40)
        moved = kg.randomize(gk.pd, rng, 8)
        for q in (3, 5):
            _, v1, _ = run(ctx, gk.pd, q, "c128")
            _, v2, _ = run(ctx, moved, q, "c128")
            assert rel_err(v2, v1) <= C128_TOL


def test_repeat_calls_same_workspace(ctx):
    import torch
    gk = kg.random_grid_knot(16, 42, True, 30, 40)
    k = pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer)
    p = pk.Plan(ctx, k, 3)
    ws = pk.workspace(p, "c128")
    z1, _ = pk.evaluate(p, "c128", ws)
    z2, _ = pk.evaluate(p, "c128", ws)
    assert (z1.re, z1.im, z1.exp2) == (z2.re, z2.im, z2.exp2)   # deterministic
    torch.cuda.synchronize()


@pytest.mark.parametrize("prec,tol", [("c128", C128_TOL), ("c64", C64_TOL)])
def test_forced_gemm_kernel(ctx, prec, tol):
    """Every two-operand step on the tiled GEMM kernel: ragged 64 x 64 edge tiles, tiny
    extents, batch indices and both unit-stride layouts of each operand."""
    worst = 0.0
    for s in range(8):
        gk = kg.random_grid_knot(16, 1200 + s, True, 20, 45)
        for order in ("greedy_edge", "greedy_spin", "elim_spin"):
            for q in (2, 3, 5):
                z, v, p = run(ctx, gk.pd, q, prec, outer=gk.outer, order=order,
                              flags=pk.FLAG_FORCE_GEMM)
                assert any(st["kernel"] == 2 for st in p.steps())
                zo, vo = oracle_zv(gk.pd, q, outer=gk.outer)
                e = rel_err(z, zo)
                worst = max(worst, e)
                assert e <= tol, (s, order, q, e)
    print(f"[forced GEMM {prec}] worst relative error {worst:.3e}")


def test_forced_rows_kernel(ctx):
    for s in range(4):
        gk = kg.random_grid_knot(16, 1300 + s, True, 20, 45)
        for q in (3, 5):
            z, _, _ = run(ctx, gk.pd, q, "c128", outer=gk.outer, order="greedy_edge",
                          flags=pk.FLAG_FORCE_ROWS)
            zo, _ = oracle_zv(gk.pd, q, outer=gk.outer)
            assert rel_err(z, zo) <= C128_TOL


SPLIT_TOL = 1e-6   # split FP32 (float-float arithmetic, complex128 tail) target


@pytest.mark.parametrize("order", ["greedy_edge", "greedy_spin", "elim_spin", "fill_spin", "partition"])
def test_split_precision_vs_oracle(ctx, order):
    worst = 0.0
    for s in range(10):
        gk = kg.random_grid_knot(16, 500 + s, True, 20, 45)
        for q in (2, 3, 5):
            z, v, _ = run(ctx, gk.pd, q, "split", outer=gk.outer, order=order)
            zo, vo = oracle_zv(gk.pd, q, outer=gk.outer)
            ez, ev = rel_err(z, zo), rel_err(v, vo)
            worst = max(worst, ez, ev)
            assert ez <= SPLIT_TOL and ev <= SPLIT_TOL, (s, q, ez, ev)
    print(f"[{order} split] worst relative error {worst:.3e}")


def test_split_forced_gemm(ctx):
    """Float-float GEMM kernel on every two-operand step."""
    worst = 0.0
    for s in range(6):
        gk = kg.random_grid_knot(16, 1200 + s, True, 20, 45)
        for q in (3, 5):
            zo, _ = oracle_zv(gk.pd, q, outer=gk.outer)
            for order in ("greedy_edge", "elim_spin"):
                z, _, p = run(ctx, gk.pd, q, "split", outer=gk.outer, order=order,
                              flags=pk.FLAG_FORCE_GEMM)
                e = rel_err(z, zo)
                worst = max(worst, e)
                assert e <= SPLIT_TOL, (s, q, order, e)
    print(f"[split forced GEMM] worst relative error {worst:.3e}")


def test_c64_with_fp64_tail(ctx):
    """complex64 bulk with the last 1, 4 or all contractions widened to complex128."""
    worst = {}
    for s in range(6):
        gk = kg.random_grid_knot(16, 1200 + s, True, 20, 45)
        for q in (3, 5):
            zo, _ = oracle_zv(gk.pd, q, outer=gk.outer)
            for tail in (1, 4, 1000):
                z, _, p = run(ctx, gk.pd, q, "c64", outer=gk.outer, order="greedy_edge",
                              tail_steps=tail)
                e = rel_err(z, zo)
                worst[tail] = max(worst.get(tail, 0.0), e)
                assert e <= C64_TOL, (s, q, tail, e)
    print("[c64 + FP64 tail] worst relative error by tail length", worst)


def test_split_closed_forms_and_slices(ctx):
    for pd, poly in ((TREFOIL, {1: 1, 3: 1, 4: -1}), (FIG8, {-2: 1, -1: -1, 0: 1, 1: -1, 2: 1}),
                     ([], {0: 1})):
        for q in range(1, 7):
            _, v, _ = run(ctx, pd, q, "split")
            assert rel_err(v, exact_to_complex(kg_eval(poly, q), 1, q)) <= SPLIT_TOL
    gk = kg.random_grid_knot(18, 700, True, 40, 70)
    k = pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer)
    full = pk.Plan(ctx, k, 3).stats()["log2_max_elems"]
    z, _, p = run(ctx, gk.pd, 3, "split", outer=gk.outer, max_log2_elems=full - 3)
    assert p.stats()["n_slices"] > 1
    assert rel_err(z, oracle_zv(gk.pd, 3, outer=gk.outer)[0]) <= SPLIT_TOL
