"""Host-side checks of libpk (no GPU): exports, knot input, grid walks, plans.

Plans are replayed on the CPU from the library's own records (tests/plan_replay.py)
and compared with the oracle, so the planner's index bookkeeping, layouts, stride
runs, slicing and exponent tracking are checked before any kernel runs.
"""
import math
import re

import pytest

import knotgen as kg
import oracle
import paper_1807_02119_gb300 as pk
from oracle.scaled import SC, rel_err
from plan_replay import replay

HEADER = __file__.rsplit("/tests/", 1)[0] + "/include/pk.h"


@pytest.fixture(scope="module")
def ctx():
    return pk.Context(-1)


def test_library_exports_every_declared_symbol():
    names = set(re.findall(r"\b(pk_[a-z0-9_]+)\s*\(", open(HEADER).read()))
    assert len(names) >= 20
    L = pk.lib()
    for n in sorted(names):
        assert hasattr(L, n), n
    assert names <= set(pk.EXPORTED) | {"pk_last_error"}


def _pds():
    out = [kg.braid_closure_pd([1, 1, 1], 2), kg.braid_closure_pd([1, -2, 1, -2], 3), [],
           kg.kink([], 0, 1), kg.braid_closure_pd(kg.torus_braid(3, 5), 3)]
    for s in range(25):
        out.append(kg.random_grid_knot(14, s, bool(s % 2), 1).pd)
    rng = kg.SplitMix64(9)
    out.append(kg.randomize(out[5], rng, 5))
    return out


def test_knot_from_pd_matches_oracle(ctx):
    for pd in _pds():
        k = pk.Knot.from_pd(ctx, pd)
        g = oracle.tait_graph(pd, black=0)
        info = k.info()
        assert (info["n_v"], info["n_c"], info["writhe"], info["tau"], info["components"]) == \
            (g.n_v, g.n_crossings, g.writhe, g.tau, g.components)
        edges = k.edges()
        for q in (2, 3, 5):
            assert oracle.z_exact(info["n_v"], edges, q) == oracle.z_exact(g.n_v, g.edges, q)


def test_outer_region(ctx):
    for s in range(8):
        gk = kg.random_grid_knot(12, 40 + s, True, 2)
        k = pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer)
        g = oracle.tait_graph(gk.pd, outer=gk.outer)
        assert k.info()["n_v"] == g.n_v and k.info()["tau"] == g.tau


def test_grid_walk_matches_generator(ctx):
    for (L, seed, rou, lo, hi) in ((12, 0, True, 16, 16), (14, 3, False, 1, 99), (20, 11, True, 30, 60)):
        k = pk.Knot.from_grid_walk(ctx, L, seed, rou, lo, hi)
        g = kg.random_grid_knot(L, seed, rou, lo, hi)
        assert k.pd() == [tuple(x) for x in g.pd]
        assert k.info()["n_v"] == oracle.tait_graph(g.pd, outer=g.outer).n_v


def test_invalid_inputs(ctx):
    with pytest.raises(pk.PkError) as e:
        pk.Knot.from_pd(ctx, [(0, 1, 2, 3)])
    assert e.value.status == 1
    with pytest.raises(pk.PkError):
        pk.Knot.from_pd(ctx, [(0, 2, 1, 3), (2, 0, 3, 1)])  # under-strand not a -> a+1
    k = pk.Knot.from_pd(ctx, kg.braid_closure_pd([1, 1, 1], 2))
    with pytest.raises(pk.PkError) as e:
        pk.Plan(ctx, k, 0)
    assert e.value.status == 1
    with pytest.raises(pk.PkError):
        pk.Knot.from_signed_graph(ctx, 2, [(0, 2, 1)], 0)
    with pytest.raises(pk.PkError):
        pk.Knot.from_signed_graph(ctx, 2, [(0, 1, 0)], 0)


def test_link_pd_is_rejected(ctx):
    """Arc labels run consecutively along one component, so a two-component PD code
    (Hopf link) cannot satisfy the convention and is refused."""
    with pytest.raises(pk.PkError) as e:
        pk.Knot.from_pd(ctx, [(0, 3, 1, 2), (2, 1, 3, 0)])
    assert e.value.status == 1


def _z_oracle(pd, q):
    g = oracle.tait_graph(pd, black=0)
    return oracle.z_complex(g.n_v, g.edges, q)


@pytest.mark.parametrize("order", ["greedy_edge", "greedy_spin", "elim_spin", "fill_spin", "partition",
                                   "auto"])
def test_plan_replay_matches_oracle(ctx, order):
    for pd in _pds()[:18]:
        k = pk.Knot.from_pd(ctx, pd)
        for q in (1, 2, 3, 5):
            p = pk.Plan(ctx, k, q, order=order)
            z, e = replay(p)
            got = SC.of(z, e)
            want = _z_oracle(pd, q)
            assert rel_err(got, want) < 1e-10 or (abs(want.m) == 0 and abs(z) < 1e-12), (pd, q, order)


@pytest.mark.parametrize("order", ["greedy_edge", "greedy_spin", "fill_spin", "auto"])
def test_reconfigured_plan_replay_matches_oracle(ctx, order):
    """Subtree reconfiguration (pk_plan_opts.refine) rebrackets the pairwise products only:
    the replayed plan still gives the oracle's Z, its records pass the plan verifier, and
    at q = 5 it finds cheaper sequences than the unrefined plan on most knots."""
    cheaper = 0
    for i, pd in enumerate(_pds()[5:20]):
        k = pk.Knot.from_pd(ctx, pd)
        for q in (2, 3, 5):
            p = pk.Plan(ctx, k, q, order=order, refine=8)
            assert p.verify("split") == "" and p.verify("c128") == ""
            z, e = replay(p)
            assert rel_err(SC.of(z, e), _z_oracle(pd, q)) < 1e-10, (i, q, order)
            if q == 5:
                cheaper += p.stats()["cmacs"] < pk.Plan(ctx, k, q, order=order).stats()["cmacs"]
    assert cheaper >= 1


def test_reconfiguration_never_raises_the_estimated_cost(ctx):
    """The planner keeps a rebracketed sequence only when its estimated cost (after
    slicing) is lower, so refine > 0 can only lower pk_plan_stats.est_cost."""
    for s in range(6):
        k = pk.Knot.from_pd(ctx, kg.random_grid_knot(24, 300 + s, True, 40, 120).pd)
        for q in (3, 5):
            base = pk.Plan(ctx, k, q, restarts=16).stats()["est_cost"]
            ref = pk.Plan(ctx, k, q, restarts=16, refine=8).stats()["est_cost"]
            assert 0 < ref <= base * (1 + 1e-12), (s, q, base, ref)


def test_reconfigured_plan_with_slicing(ctx):
    """Reconfiguration keeps every new intermediate within the slicing bound."""
    for s in range(4):
        pd = kg.random_grid_knot(16, 100 + s, True, 20, 60).pd
        k = pk.Knot.from_pd(ctx, pd)
        for q, lim in ((2, 4.0), (3, 4.8), (5, 7.0)):
            p = pk.Plan(ctx, k, q, max_log2_elems=lim, refine=10)
            st = p.stats()
            assert st["log2_max_elems"] <= lim + 1e-9
            z, e = replay(p)
            assert rel_err(SC.of(z, e), _z_oracle(pd, q)) < 1e-10, (s, q)


def test_plan_replay_with_slicing(ctx):
    for s in range(6):
        pd = kg.random_grid_knot(16, 100 + s, True, 20, 60).pd
        k = pk.Knot.from_pd(ctx, pd)
        for order, q, lim in (("greedy_edge", 2, 4.0), ("greedy_spin", 3, 4.8), ("elim_spin", 2, 3.0)):
            p = pk.Plan(ctx, k, q, order=order, max_log2_elems=lim)
            st = p.stats()
            assert st["log2_max_elems"] <= lim + 1e-9
            assert st["n_slices"] >= 1
            z, e = replay(p)
            assert rel_err(SC.of(z, e), _z_oracle(pd, q)) < 1e-10, (s, order)


def test_plan_stats_and_steps(ctx):
    pd = kg.random_grid_knot(20, 5, True, 40, 80).pd
    k = pk.Knot.from_pd(ctx, pd)
    p = pk.Plan(ctx, k, 3, order="greedy_spin")
    st = p.stats()
    steps = p.steps()
    assert st["n_steps"] == len(steps)
    assert abs(st["cmacs"] - sum(s["R"] * s["K"] * s["N"] for s in steps)) < 1e-6 * st["cmacs"]
    assert st["workspace_c128"] > st["workspace_c64"]
    fused = st["n_segment_steps"] - st["n_segments"]      # runs of small steps: one launch
    assert st["n_segments"] > 0
    assert p.launches() == 1 + st["n_slices"] * (2 + st["n_steps"] - fused)


def test_jones_normalisation_host(ctx):
    """pk_jones_from_z applies A(q) (Eq. JonesPotts): with the oracle's Z it must
    reproduce the oracle's V."""
    for pd in _pds()[:10]:
        k = pk.Knot.from_pd(ctx, pd)
        g = oracle.tait_graph(pd, black=0)
        for q in (1, 2, 3, 5, 6):
            z = oracle.z_complex(g.n_v, g.edges, q)
            v = k.jones_from_z(q, pk.Scaled(z.m.real, z.m.imag, z.e))
            want = oracle.jones(pd, q, black=0)
            assert rel_err(SC.of(v.mantissa, v.exp2), want) < 1e-12


def test_plan_replay_forced_kernels(ctx):
    """Forcing every step onto the GEMM (or row) kernel keeps the plan valid: the GEMM
    view's batch/m/n/k stride runs address the same outputs as the row view."""
    for s in range(6):
        pd = kg.random_grid_knot(15, 60 + s, True, 15, 40).pd
        k = pk.Knot.from_pd(ctx, pd)
        for flags in (pk.FLAG_FORCE_GEMM, pk.FLAG_FORCE_ROWS):
            for order in ("greedy_edge", "greedy_spin", "elim_spin"):
                p = pk.Plan(ctx, k, 3, order=order, flags=flags)
                kinds = {st["kernel"] for st in p.steps()}
                if flags == pk.FLAG_FORCE_ROWS:
                    assert kinds <= {0}
                z, e = replay(p)
                assert rel_err(SC.of(z, e), _z_oracle(pd, 3)) < 1e-10


def test_plan_replay_split_tail_layout(ctx):
    """The complex128 tail of PK_SPLIT (widened inputs, tail-region offsets, separate
    bookkeeping slots) addresses the same contraction as the plain plan."""
    for s in range(5):
        pd = kg.random_grid_knot(15, 80 + s, True, 15, 40).pd
        k = pk.Knot.from_pd(ctx, pd)
        for tail in (0, 1, 7, -1, 1000):
            for order in ("greedy_spin", "elim_spin"):
                p = pk.Plan(ctx, k, 3, order=order, tail_steps=tail)
                z, e = replay(p, split=True)
                assert rel_err(SC.of(z, e), _z_oracle(pd, 3)) < 1e-10, (s, tail, order)
                st = p.stats()
                assert st["workspace_split"] > 0
    # sliced plan with a tail
    pd = kg.random_grid_knot(16, 101, True, 20, 60).pd
    k = pk.Knot.from_pd(ctx, pd)
    p = pk.Plan(ctx, k, 2, order="greedy_edge", max_log2_elems=4.0, tail_steps=3)
    assert p.stats()["n_slices"] > 1
    z, e = replay(p, split=True)
    assert rel_err(SC.of(z, e), _z_oracle(pd, 2)) < 1e-10


def test_decode_result_status_word(ctx):
    """The host side of reading a result: the total record's status word (set on the GPU
    when a bounded wait of the tensor-core GEMM gives up) becomes PK_ETIMEOUT; a zero word
    gives Z = value x the plan's loop factor and V = A(q) Z (Eq. JonesPotts), as
    pk_jones_from_z computes it."""
    k = pk.Knot.from_pd(ctx, kg.kink(kg.braid_closure_pd([1, 1, 1], 2), 0, 1))  # a loop factor
    for q in (2, 3, 5):
        p = pk.Plan(ctx, k, q)
        fre, fim, fexp = __import__("struct").unpack("<3d", p.debug_blob(4))
        st, z, v = pk.decode_result(p, 0.75, -0.25, 40, 0)
        assert st == 0
        want = SC.of(complex(0.75, -0.25), 40) * SC.of(complex(fre, fim), int(fexp))
        assert rel_err(SC.of(z.mantissa, z.exp2), want) < 1e-15
        assert v == k.jones_from_z(q, z)
        st, z2, _ = pk.decode_result(p, 0.75, -0.25, 40, 1)
        assert st == 6              # PK_ETIMEOUT (bit 0): the value is not to be used
        for sl, step in ((0, -1), (0, 0), (3, 17), (1 << 30, 5000)):
            code = ((sl + 1) << 24 | (step + 2)) << 1      # the finite check's code
            for word in (code, code | 1):
                st, z2, _ = pk.decode_result(p, 0.75, -0.25, 40, word)
                assert st == 9      # PK_ENONFINITE takes precedence over an expired wait
    # the record layout the device writes: 32 bytes, status in the last 8
    assert pk.STATUS[6] == "PK_ETIMEOUT" and pk.STATUS[9] == "PK_ENONFINITE"


def test_tuning_table_and_ranges(ctx):
    """pk_tuning: the compiled-in table is the context's start value; set/get round-trip,
    values outside the documented ranges are refused, NULL restores the table."""
    d = pk.default_tuning()
    assert ctx.tuning() == d
    assert d["batch_threads"] in (128, 256, 512) and 256 <= d["batch_ktab"] <= 2048
    c = pk.Context(-1)
    c.set_tuning(seq_outs=8192, seq_work=1 << 16, batch_threads=512, batch_ktab=512)
    assert c.tuning() == dict(d, seq_outs=8192, seq_work=1 << 16, batch_threads=512, batch_ktab=512)
    for bad in ({"batch_threads": 100}, {"batch_ktab": 4096}, {"seq_k": 4096}, {"seq_outs": 0},
                {"tc_min_k": 3}, {"tc_min_k": 17}, {"tc_db_groups": -1}, {"tc_db_groups": 5000},
                {"tc_min_n": 7}, {"tc_min_n": 33}, {"cost_gemm_milli": 5},
                {"cost_gemm_milli": 1001}, {"cost_out_milli": -1}, {"cost_out_milli": 1000001}, {"tc_wide_n": 15},
                {"tc_wide_n": (1 << 30) + 1}, {"cost_tcin_milli": -1}, {"cost_tcin_milli": 1000001},
                {"tc_min_work": -1}, {"tc_min_work": (1 << 40) + 1}):
        with pytest.raises(pk.PkError):
            c.set_tuning(**bad)
    c.set_tuning()
    assert c.tuning() == d


@pytest.mark.parametrize("outs,work", [(1, 1), (8192, 1 << 16)])
def test_plan_replay_under_other_sequence_thresholds(outs, work):
    """Plans made with other sequence-run thresholds (no runs at all; long runs) replay
    to the oracle's Z: the thresholds only group launches."""
    c = pk.Context(-1)
    c.set_tuning(seq_outs=outs, seq_work=work)
    for s in range(3):
        gk = kg.random_grid_knot(16, 300 + s, True, 20, 40)
        k = pk.Knot.from_pd(c, gk.pd, outer=gk.outer)
        p = pk.Plan(c, k, 3)
        st = p.stats()
        if outs == 1:
            assert st["n_segments"] == 0
        g = oracle.tait_graph(gk.pd, outer=gk.outer)
        zo = oracle.z_complex(g.n_v, g.edges, 3)
        z, e = replay(p)
        assert rel_err(SC.of(z, e), zo) < 1e-10


def test_hbm_budget_slices_until_the_workspace_fits():
    """A device-memory budget on the context: plans slice further until every precision's
    workspace fits, still replay to the oracle's Z; a budget below any slicing is refused
    with PK_ETOOWIDE."""
    c = pk.Context(-1)
    gk = kg.random_grid_knot(30, 35, True, 60, 160)        # 119 crossings, arena 263 KB
    k = pk.Knot.from_pd(c, gk.pd, outer=gk.outer)
    g = oracle.tait_graph(gk.pd, outer=gk.outer)
    free = pk.Plan(c, k, 3)
    state, arena = free.state_bytes("c128")     # the state part does not shrink with slicing
    budget = state + (3 * arena) // 5
    c.set_hbm_budget(budget)
    p = pk.Plan(c, k, 3)
    assert max(p.workspace_bytes(x) for x in ("c128", "c64", "split")) <= budget
    assert p.stats()["n_slices"] > free.stats()["n_slices"]
    z, e = replay(p)
    assert rel_err(SC.of(z, e), oracle.z_complex(g.n_v, g.edges, 3)) < 1e-10
    c.set_hbm_budget(1024)
    with pytest.raises(pk.PkError) as ex:
        pk.Plan(c, k, 3)
    assert ex.value.status == 4


@pytest.mark.parametrize("work", [1 << 12, 1 << 20])
def test_plan_replay_with_tensor_core_work_floor(work):
    """tc_min_work keeps small GEMM-shaped row steps off the tensor cores (and their C in
    the row kernels' layout); the plans still replay to the oracle's Z."""
    c = pk.Context(-1)
    c.set_tuning(tc_min_work=work)
    for s in range(3):
        pd = kg.random_grid_knot(20, 400 + s, True, 40, 80).pd
        for q in (3, 5):
            p = pk.Plan(c, pk.Knot.from_pd(c, pd), q, refine=6)
            z, e = replay(p)
            assert rel_err(SC.of(z, e), _z_oracle(pd, q)) < 1e-10, (s, q)
            small = [st for st in p.steps() if st["tc"] and st["kernel"] == 0 and
                     st["R"] * st["K"] * st["N"] < work]
            assert not small


def test_device_calls_refuse_a_host_only_context(ctx):
    """Upload, launch and download entry points need a GPU context: on a host-only context
    they return PK_ENODEVICE (7) before touching any pointer."""
    import ctypes as C
    k = pk.Knot.from_pd(ctx, kg.braid_closure_pd([1, 1, 1], 2))
    p = pk.Plan(ctx, k, 3)
    L = pk.lib()
    n = C.c_uint64()
    buf = C.c_void_p(1 << 20)   # never dereferenced: the context check comes first
    assert L.pk_upload(ctx.h, p.h, 0, buf, 1 << 30) == 7
    assert L.pk_upload_inputs(ctx.h, p.h, 0, buf, 1 << 30, C.byref(n)) == 7
    assert L.pk_launch(ctx.h, p.h, 0, buf, 1 << 30) == 7
    z, v = pk.pk_scaled(), pk.pk_scaled()
    assert L.pk_download(ctx.h, p.h, 0, buf, C.byref(z), C.byref(v)) == 7
