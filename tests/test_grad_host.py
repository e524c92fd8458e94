"""Reverse-pass programs of PK_FLAG_GRAD plans, checked on the CPU (no GPU).

tests/plan_replay.replay_grad runs the library's own records (recipes at their arena
offsets, forward / recompute / adjoint steps, leaf accumulation records) with numpy; the
library's host stage (pk_grad_from_accumulators) turns the accumulators into
(1/Z) dZ/dT_e, which must match the oracle's reverse pass on the same signed graph.
"""
import numpy as np
import pytest

import knotgen as kg
import oracle.grad as og
import paper_1807_02119_gb300 as pk
from oracle.scaled import SC
from plan_replay import replay_grad


@pytest.fixture(scope="module")
def ctx():
    return pk.Context(-1)


def _host_grad(plan):
    (zm, ze), acc, ae = replay_grad(plan)
    z = SC.of(zm, ze)
    d, dv = pk.grad_from_accumulators(plan, acc, ae, pk.Scaled(z.m.real, z.m.imag, z.e))
    return z, d, dv


def _sliced_plan(ctx, k, q, **kw):
    """A plan sliced into a few (3..243) slices: the widest tensor's limit is lowered
    step by step from the unsliced width until slicing starts."""
    full = pk.Plan(ctx, k, q, **kw).stats()["log2_max_elems"]
    lim = full
    while lim > 1.0:
        lim -= 0.5
        p = pk.Plan(ctx, k, q, max_log2_elems=lim, **kw)
        if p.stats()["n_slices"] > 1:
            assert p.stats()["n_slices"] <= 243
            return p
    raise AssertionError("no sliced plan")


def _knots():
    out = [kg.braid_closure_pd([1, 1, 1], 2), kg.braid_closure_pd([1, -2, 1, -2], 3),
           kg.kink(kg.braid_closure_pd([1, 1, 1], 2), 0, 1),
           kg.kink(kg.kink([], 0, 0), 1, 2)]
    rng = kg.SplitMix64(31)
    base = kg.random_grid_knot(12, 41, True, 10, 20).pd
    out.append(kg.randomize(base, rng, 4))            # R-I loops and R-II parallel pairs
    for s in range(4):
        out.append(kg.random_grid_knot(14, 60 + s, True, 15, 35).pd)
    return out


def _check(plan, knot, q, weights=None, tol=1e-10):
    info, edges = knot.info(), knot.edges()
    z, d, dv = _host_grad(plan)
    zo, do = og.dlogz(info["n_v"], edges, q, weights)
    assert abs(z.m * 2.0 ** (z.e - zo.e) - zo.m) <= tol * abs(zo.m)
    scale = max(1.0, float(np.max(np.abs(do)))) if do.size else 1.0
    assert d.shape == do.shape
    assert np.max(np.abs(d - do), initial=0.0) <= tol * scale
    if weights is None and info["components"] == 1:
        dvo = og.dlogv_dt(info["n_v"], edges, q, info["writhe"], info["tau"])
        assert abs(dv - dvo) <= tol * max(1.0, abs(dvo))
    return d


@pytest.mark.parametrize("q", [2, 3, 5])
def test_grad_replay_matches_oracle(ctx, q):
    for pd in _knots():
        k = pk.Knot.from_pd(ctx, pd)
        for stride in (0, 2, 3):
            p = pk.Plan(ctx, k, q, grad=True, checkpoint_stride=stride)
            _check(p, k, q)


def test_grad_orders_and_kernels(ctx):
    for pd in _knots()[4:8]:
        k = pk.Knot.from_pd(ctx, pd)
        for order in ("greedy_spin", "elim_spin", "fill_spin"):
            for flags in (0, pk.FLAG_FORCE_GEMM, pk.FLAG_FORCE_ROWS):
                p = pk.Plan(ctx, k, 3, order=order, flags=flags, grad=True, checkpoint_stride=2)
                _check(p, k, 3)


def test_grad_sliced(ctx):
    """Slicing: every slice's clause-tensor adjoints land on the sub-block of their full
    matrix that the slice fixes."""
    for s in range(2):
        gk = kg.random_grid_knot(14, 120 + s, True, 15, 35)
        k = pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer)
        for q in (2, 3):
            p = _sliced_plan(ctx, k, q, grad=True, checkpoint_stride=s % 3)
            _check(p, k, q)


def test_grad_general_weights_and_set_weights(ctx):
    rng = np.random.default_rng(5)
    for pd in _knots()[2:6]:
        k = pk.Knot.from_pd(ctx, pd)
        n_e = k.info()["n_c"]
        w = [(complex(*rng.standard_normal(2)), complex(*rng.standard_normal(2)))
             for _ in range(n_e)]
        p = pk.Plan(ctx, k, 3, weights=w, grad=True, checkpoint_stride=2)
        _check(p, k, 3, weights=w)
        w2 = [(d * 0.5 + 1j, o - 0.25) for d, o in w]
        p.set_weights(w2)
        _check(p, k, 3, weights=w2)
        p.set_weights(None)
        _check(p, k, 3)


def test_grad_program_stats(ctx):
    gk = kg.random_grid_knot(20, 9, True, 40, 60)
    k = pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer)
    keep = pk.Plan(ctx, k, 3, grad=True, checkpoint_stride=1).grad_stats()
    assert keep["steps_recompute"] == 0 and keep["cmacs_recompute"] == 0
    assert keep["cmacs_adjoint"] <= 2 * keep["cmacs_forward"] + 1e-9
    prev = keep["arena_elems"]
    for stride in (2, 4, 8):
        st = pk.Plan(ctx, k, 3, grad=True, checkpoint_stride=stride).grad_stats()
        assert st["steps_recompute"] > 0
        assert st["cmacs_recompute"] <= st["cmacs_forward"]
        assert st["checkpoints"] < keep["checkpoints"]
        assert st["arena_elems"] <= keep["arena_elems"]
        prev = st["arena_elems"]
    assert prev <= keep["arena_elems"]


def test_grad_errors_and_unknot(ctx):
    k = pk.Knot.from_pd(ctx, kg.braid_closure_pd([1, 1, 1], 2))
    with pytest.raises(pk.PkError):
        pk.Plan(ctx, k, 3).grad_stats()                      # no reverse program
    with pytest.raises(pk.PkError):
        pk.Plan(ctx, k, 3, order="greedy_edge", grad=True)   # edge network has no groups
    with pytest.raises(pk.PkError):
        pk.Plan(ctx, k, 3).set_weights(None)                 # standard network
    u = pk.Knot.from_pd(ctx, [])
    p = pk.Plan(ctx, u, 3, grad=True)
    z, d, dv = _host_grad(p)
    assert d.shape == (0, 3, 3)
    t = og.t_of_q(3)
    assert abs(dv - (1 / t - 2 / (t + 1))) < 1e-14         # V = 1: only A(t) and Z = q
    assert abs(z.m * 2.0 ** z.e - 3) < 1e-14


def test_grad_weights_sums_the_diagonal_and_off_diagonal():
    """pk_grad_weights: per Tait edge the sums of dlogZ/dT over the diagonal and over the
    off-diagonal entries, the derivatives with respect to the two clause weights."""
    import numpy as np
    ctx = pk.Context(-1)
    k = pk.Knot.from_pd(ctx, kg.braid_closure_pd([1, 1, 1], 2))
    p = pk.Plan(ctx, k, 3, grad=True)
    rng = np.random.default_rng(3)
    d = rng.normal(size=(p.n_e, 3, 3)) + 1j * rng.normal(size=(p.n_e, 3, 3))
    got = pk.grad_weights(p, d)
    eye = np.eye(3, dtype=bool)
    want = np.stack([d[:, eye].sum(axis=1), d[:, ~eye].sum(axis=1)], axis=1)
    assert np.allclose(got, want, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("q", [3, 5])
def test_grad_reconfigured_plan_matches_oracle(ctx, q):
    """A gradient plan whose contraction tree was rebracketed (pk_plan_opts.refine): the
    reverse program follows the new tree and the adjoints still match the oracle's."""
    for pd in _knots()[4:]:
        k = pk.Knot.from_pd(ctx, pd)
        for stride in (0, 2):
            p = pk.Plan(ctx, k, q, grad=True, checkpoint_stride=stride, refine=8)
            _check(p, k, q)
