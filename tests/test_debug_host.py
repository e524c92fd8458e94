"""Host-side checks of the debugging aids and of slice-level resume (no GPU).

* pk_plan_verify accepts the plans the planner makes, over every order, kernel choice,
  slicing, complex128 tail, tensor-core digit scratch and reverse program;
* pk_combine_slices sums per-slice values exactly as a rational sum would (within one
  rounding) and applies the plan's constant factor and A(q) as pk_download does;
* evaluate_resumable stores its progress, resumes from the first missing slice and
  refuses a file made for another plan.
"""
import json
import math
import os
import struct
from fractions import Fraction

import pytest

import knotgen as kg
import paper_1807_02119_gb300 as pk
from oracle.scaled import SC, rel_err


@pytest.fixture(scope="module")
def ctx():
    return pk.Context(-1)


def _knots(ctx):
    out = [pk.Knot.from_pd(ctx, kg.braid_closure_pd([1, 1, 1], 2)),
           pk.Knot.from_pd(ctx, kg.braid_closure_pd(kg.torus_braid(3, 5), 3)),
           pk.Knot.from_pd(ctx, kg.kink(kg.braid_closure_pd([1, -2, 1, -2], 3), 0, 1))]
    for L, seed in ((14, 3), (18, 5), (24, 11), (30, 35)):
        gk = kg.random_grid_knot(L, seed, True, 1)
        out.append(pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer))
    return out


PRECS = ("c128", "c64", "split")


def test_verify_accepts_planner_output(ctx):
    n = 0
    for k in _knots(ctx):
        for q in (2, 3, 5):
            for order in ("auto", "greedy_edge", "greedy_spin", "elim_spin", "partition", "fill_spin"):
                p = pk.Plan(ctx, k, q, order=order, restarts=2)
                for prec in PRECS:
                    assert p.verify(prec) == "", (q, order, prec, p.verify(prec))
                n += 1
            for kw in (dict(flags=pk.FLAG_FORCE_GEMM), dict(flags=pk.FLAG_FORCE_ROWS),
                       dict(flags=pk.FLAG_TC_DIGITS4), dict(flags=pk.FLAG_NO_TC),
                       dict(max_log2_elems=6.0), dict(tail_steps=3),
                       dict(grad=True, checkpoint_stride=2), dict(grad=True, max_log2_elems=6.0)):
                try:
                    p = pk.Plan(ctx, k, q, **kw)
                except pk.PkError as e:     # slicing limit: more slices than allowed
                    assert e.status == 4
                    continue
                for prec in PRECS:
                    assert p.verify(prec) == "", (q, kw, prec, p.verify(prec))
                n += 1
    assert n >= 7 * 3 * 12


def test_verify_covers_tensor_core_and_sliced_plans(ctx):
    """Plans of L=30 grid walks at q=5: GEMM steps with several flush groups on the tensor
    cores (digit scratch), and the same knots sliced two indices below their widest
    tensor."""
    for seed in (35, 8):
        gk = kg.random_grid_knot(30, seed, True, 1)
        k = pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer)
        p = pk.Plan(ctx, k, 5, restarts=8)
        assert any(s["K"] > 96 for s in p.steps() if s["kernel"] == 2)
        assert p.verify("split") == ""
        ps = pk.Plan(ctx, k, 5, max_log2_elems=(p.stats()["max_rank"] - 2) * math.log2(5))
        assert ps.stats()["n_slices"] > 1 and ps.verify("split") == "" and ps.verify("c64") == ""


def test_debug_flags(ctx):
    ctx.set_debug(pk.DEBUG_CHECK_FINITE | pk.DEBUG_VERIFY | pk.DEBUG_NVTX)
    ctx.set_debug(0)
    with pytest.raises(pk.PkError):
        ctx.set_debug(8)


def _sliced_plan(ctx, q=3):
    """A 30-crossing grid walk sliced two indices below its widest tensor (27 slices)."""
    gk = kg.random_grid_knot(20, 3, True, 1)
    k = pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer)
    p = pk.Plan(ctx, k, q, max_log2_elems=2 * math.log2(q))
    assert p.stats()["n_slices"] >= 8
    return k, p


def _synthetic_slices(n, seed=1):
    """Dyadic values with exponents spread over 80 binades and mixed signs."""
    rng = kg.SplitMix64(seed)
    out = []
    for i in range(n):
        re = ((rng.next() >> 11) / 2.0 ** 53) * (1 if rng.next() & 1 else -1)
        im = ((rng.next() >> 11) / 2.0 ** 53) * (1 if rng.next() & 1 else -1)
        m = max(abs(re), abs(im))
        e = math.frexp(m)[1]
        out.append(pk.Scaled(math.ldexp(re, -e), math.ldexp(im, -e), int(rng.next() % 80) - 40 + e))
    return out


def test_combine_slices_matches_rational_sum(ctx):
    k, p = _sliced_plan(ctx)
    n = p.stats()["n_slices"]
    vals = _synthetic_slices(n)
    z, v = p.combine_slices(vals)
    sre = sum(Fraction(x.re) * Fraction(2) ** x.exp2 for x in vals)
    sim = sum(Fraction(x.im) * Fraction(2) ** x.exp2 for x in vals)
    fre, fim, fexp = struct.unpack("<3d", p.debug_blob(4))
    want = SC.of(complex(float(sre), float(sim)), 0) * SC.of(complex(fre, fim), int(fexp))
    assert rel_err(SC.of(z.mantissa, z.exp2), want) < 1e-14
    assert v == k.jones_from_z(3, z)
    # the per-slice order does not matter beyond rounding; a wrong count is refused
    z2, _ = p.combine_slices(vals[::-1])
    assert rel_err(SC.of(z2.mantissa, z2.exp2), SC.of(z.mantissa, z.exp2)) < 1e-14
    with pytest.raises(pk.PkError):
        p.combine_slices(vals[:-1])
    zero, _ = p.combine_slices([pk.Scaled(0.0, 0.0, 0)] * n)
    assert zero.re == 0 and zero.im == 0


def test_resumable_evaluation_host(ctx, tmp_path):
    """The resume logic with the GPU call replaced: an interrupted run leaves the values of
    its finished chunks in the file, the next run evaluates only the rest, and the result
    equals pk_combine_slices over all values."""
    k, p = _sliced_plan(ctx)
    n = p.stats()["n_slices"]
    vals = _synthetic_slices(n, seed=7)
    calls = []

    def run(first, count):
        calls.append((first, count))
        return vals[first:first + count]

    path = str(tmp_path / "z.json")
    assert pk.evaluate_resumable(p, path, "c128", chunk=3, run_slices=run, stop_after=2) is None
    assert calls == [(0, 3), (3, 3)]
    rec = json.load(open(path))
    assert sorted(int(x) for x in rec["slices"]) == list(range(6))
    # a second process (a new plan object of the same knot and options) continues
    p2 = pk.Plan(ctx, k, 3, max_log2_elems=2 * math.log2(3))
    calls.clear()
    z, v = pk.evaluate_resumable(p2, path, "c128", chunk=3, run_slices=run)
    assert calls[0] == (6, 3) and sum(c for _, c in calls) == n - 6
    assert (z, v) == p.combine_slices(vals)
    # nothing left to run: the stored values alone give the result
    calls.clear()
    assert pk.evaluate_resumable(p2, path, "c128", run_slices=run) == (z, v) and calls == []
    # a file of another plan or precision is refused
    p3 = pk.Plan(ctx, k, 2, max_log2_elems=3.0)
    with pytest.raises(ValueError):
        pk.evaluate_resumable(p3, path, "c128", run_slices=run)
    with pytest.raises(ValueError):
        pk.evaluate_resumable(p2, path, "split", run_slices=run)
    os.remove(path)


def _scaled_jones_weights(edges, q, seed):
    """The Jones clause weights of each edge times an exact power of two 2^s_e with
    |s_e| up to 1000 (entries near the ends of the FP64 range); returns (weights, sum s_e)."""
    from oracle.potts import clause_diag
    rng = kg.SplitMix64(seed)
    w, tot = [], 0
    for (_, _, eps) in edges:
        s = int(rng.below(2001)) - 1000
        w.append((clause_diag(q, eps) * 2.0 ** s, 2.0 ** s + 0j))
        tot += s
    return w, tot


def test_large_and_small_weights_stay_in_range(ctx):
    """Scaling every clause matrix T_e by an exact power of two 2^s_e multiplies Z by
    2^(sum s_e) (Z is multilinear in the clause matrices).  With s_e up to +-1000 any
    product of two raw entries would overflow or underflow FP64; the library stores each
    clause scaled into [0.5, 1) with its power of two carried as the initial tensor's
    exponent, so the CPU replay of the plan's own records matches the oracle's Z of the
    unscaled knot times 2^(sum s_e)."""
    from plan_replay import replay
    import oracle
    for L, seed in ((14, 3), (18, 5)):
        gk = kg.random_grid_knot(L, seed, True, 1)
        k = pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer)
        g = oracle.tait_graph(gk.pd, outer=gk.outer)
        for q in (2, 3, 5):
            w, tot = _scaled_jones_weights(k.edges(), q, 100 * L + q)
            zo = oracle.z_complex(g.n_v, g.edges, q) * SC.of(1.0 + 0j, tot)
            for kw in ({}, dict(max_log2_elems=2 * math.log2(q))):
                p = pk.Plan(ctx, k, q, weights=w, **kw)
                assert p.verify("c128") == ""
                z, e = replay(p)
                assert rel_err(SC.of(z, e), zo) <= 1e-10, (L, q, kw)
            # new weights through pk_plan_set_weights keep the scaling
            p.set_weights([(d * 2.0 ** 7, o * 2.0 ** 7) for d, o in w])
            z, e = replay(p)
            assert rel_err(SC.of(z, e), zo * SC.of(1.0 + 0j, 7 * len(w))) <= 1e-10
