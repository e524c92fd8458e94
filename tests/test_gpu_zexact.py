"""Exact evaluation on the GPU: Z(q) modulo primes (pk_eval_exact) against the oracle's
exact Z in Z[t], and the full Jones polynomial (pk_jones_coefficients) against the
Kauffman bracket (small knots) and against the oracle's exact V(t(q)) at q = 5, 6, 7
(knots beyond the bracket's 2^n states).  Named to be collected after the core GPU parity
files (and before the allocation-free entry point's file, which is collected last)."""
import time

import pytest

import knotgen as kg
import oracle
import paper_1807_02119_gb300 as pk
from oracle.kauffman import jones_poly
from oracle.ring import Zt

pytestmark = pytest.mark.gpu

PRIMES = [2147483647, 2147483629, 2147483587]


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = pk.Context(0)
    c.set_stream(torch.cuda.current_stream().cuda_stream)
    return c


def _knots():
    out = [(kg.braid_closure_pd([1, 1, 1], 2), None), (kg.braid_closure_pd([1, -2, 1, -2], 3), None)]
    for s in range(3):
        gk = kg.random_grid_knot(14, 700 + s, True, 20, 40)
        out.append((gk.pd, gk.outer))
    return out


def test_exact_residues_match_oracle(ctx):
    for pd, outer in _knots():
        k = pk.Knot.from_pd(ctx, pd, outer=outer)
        g = oracle.tait_graph(pd, outer=outer)
        for q in (2, 3, 5, 6):
            a, b = oracle.z_exact(g.n_v, g.edges, q)
            want = [(a % p, b % p) for p in PRIMES]
            for kw in ({}, {"order": "greedy_edge"}, {"order": "fill_spin"}):
                assert pk.evaluate_exact(pk.Plan(ctx, k, q, **kw), PRIMES) == want, (q, kw)


def _sliced_plan(ctx, k, q):
    """A plan sliced into a few (3..243) slices: the widest tensor's limit is lowered in
    steps of 0.5 from the unsliced width until slicing starts."""
    lim = pk.Plan(ctx, k, q).stats()["log2_max_elems"]
    while lim > 1.0:
        lim -= 0.5
        p = pk.Plan(ctx, k, q, max_log2_elems=lim)
        if p.stats()["n_slices"] > 1:
            assert p.stats()["n_slices"] <= 243
            return p
    raise AssertionError("no sliced plan")


def test_exact_residues_sliced(ctx):
    gk = kg.random_grid_knot(14, 711, True, 25, 40)
    k = pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer)
    g = oracle.tait_graph(gk.pd, outer=gk.outer)
    for q in (3, 5):
        p = _sliced_plan(ctx, k, q)
        a, b = oracle.z_exact(g.n_v, g.edges, q)
        assert pk.evaluate_exact(p, PRIMES) == [(a % m, b % m) for m in PRIMES]


def test_polynomial_matches_bracket(ctx):
    cases = [kg.braid_closure_pd(w, n) for w, n in
             (([1, 1, 1], 2), ([1, -2, 1, -2], 3), ([1] * 7, 2), ([1, 2] * 4, 3), ([1, 2, 3] * 5, 4))]
    for s in range(4):
        cases.append(kg.random_grid_knot(10, 100 + s, True, 8, 16).pd)
    for pd in cases:
        k = pk.Knot.from_pd(ctx, pd)
        assert pk.jones_polynomial(ctx, k) == jones_poly(pd)


def test_polynomial_beyond_the_bracket(ctx):
    """25-40 crossings: the polynomial evaluated exactly in Z[t] at t(q) equals the oracle's
    exact V(t(q)) (a different route: the Potts sum in Z[t] with its own order); V(1) = 1
    and the span is at most the crossing number."""
    for s in range(3):
        gk = kg.random_grid_knot(16, 800 + s, True, 25, 40)
        k = pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer)
        t0 = time.perf_counter()
        poly = pk.jones_polynomial(ctx, k)
        dt = time.perf_counter() - t0
        n = len(gk.pd)
        assert sum(poly.values()) == 1
        assert max(poly) - min(poly) <= n
        for q in (5, 6, 7):
            num, den = oracle.jones_exact(gk.pd, q, outer=gk.outer)
            R = Zt(q)
            v = R.eval_laurent(poly)
            assert (v[0] * den, v[1] * den) == tuple(num), (n, q)
        print(f"[jones polynomial] {n} crossings: span {max(poly) - min(poly)}, {dt:.2f} s")
