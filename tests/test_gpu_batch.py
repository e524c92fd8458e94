"""Batched evaluation (one persistent launch for many knots) against single evaluations
and the CPU oracle."""
import pytest

import knotgen as kg
import oracle
import paper_1807_02119_gb300 as pk
from oracle.scaled import SC, rel_err

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "split": 1e-6, "c64": 1e-4}


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


def _plans(ctx, knots, q):
    return [pk.Plan(ctx, pk.Knot.from_pd(ctx, k.pd, outer=k.outer), q) for k in knots]


@pytest.mark.parametrize("prec", ["c128", "split", "c64"])
def test_batch_matches_single(ctx, prec):
    knots = kg.knot_suite("batch")[:96]          # 18..122 crossings, uneven
    plans = _plans(ctx, knots, 3)
    Z, V = pk.evaluate_batch(plans, prec)
    worst = 0.0
    for p, z, v in zip(plans, Z, V):
        zs, vs = pk.evaluate(p, prec)
        e = max(rel_err(sc(z), sc(zs)), rel_err(sc(v), sc(vs)))
        worst = max(worst, e)
        assert e <= TOL[prec], e
    print(f"[batch {prec}] worst relative difference to single evaluation {worst:.3e}")


def test_batch_vs_oracle(ctx):
    knots = kg.knot_suite("batch")[:24]
    plans = _plans(ctx, knots, 3)
    for prec in ("c128", "split"):
        Z, V = pk.evaluate_batch(plans, prec)
        for k, z, v in zip(knots, Z, V):
            g = oracle.tait_graph(k.pd, outer=k.outer)
            zo = oracle.z_complex(g.n_v, g.edges, 3)
            vo = oracle.jones_from_z(zo, g, 3)
            assert rel_err(sc(z), zo) <= TOL[prec]
            assert rel_err(sc(v), vo) <= TOL[prec]


def _oracle_zv(job):
    """Z and V of one knot by the CPU oracle (spawned worker: imports its own modules)."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle
    from oracle.order import min_fill_order
    pd, outer, q = job
    g = oracle.tait_graph(pd, outer=outer)
    order, _ = min_fill_order(g.n_v, g.edges, q, restarts=4)
    z = oracle.z_complex(g.n_v, g.edges, q, order=order, sum_inside=True)
    return z, oracle.jones_from_z(z, g, q)


def test_batch_vs_oracle_512(ctx):
    """The batch workload's first 512 knots (18..122 crossings, q = 3) in ONE persistent
    launch, split and complex128, against the CPU oracle knot by knot."""
    import multiprocessing as mp
    import os
    knots = kg.knot_suite("batch")[:512]
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        ref = pool.map(_oracle_zv, [(k.pd, k.outer, 3) for k in knots], chunksize=8)
    plans = _plans(ctx, knots, 3)
    for prec in ("split", "c128"):
        Z, V = pk.evaluate_batch(plans, prec)
        worst = 0.0
        for i, (z, v, (zo, vo)) in enumerate(zip(Z, V, ref)):
            e = max(rel_err(sc(z), zo), rel_err(sc(v), vo))
            assert e <= TOL[prec], (i, prec, e)
            worst = max(worst, e)
        print(f"[batch {prec}] 512 knots in one launch, worst relative error vs the oracle {worst:.2e}")


def test_batch_mixed_q_slices_and_trivial(ctx):
    """Different q in one batch, sliced plans, the unknot and a kink; relaunch gives
    bit-identical results (the recorded graph is replayed)."""
    import torch
    knots = kg.knot_suite("batch")[100:112]
    plans = []
    for i, k in enumerate(knots):
        kn = pk.Knot.from_pd(ctx, k.pd, outer=k.outer)
        q = (2, 3, 5)[i % 3]
        full = pk.Plan(ctx, kn, q).stats()["log2_max_elems"]
        plans.append(pk.Plan(ctx, kn, q, max_log2_elems=max(1.0, full - 2.5) if i % 2 else 0.0))
    plans.append(pk.Plan(ctx, pk.Knot.from_pd(ctx, []), 3))
    plans.append(pk.Plan(ctx, pk.Knot.from_pd(ctx, kg.kink([], 0, 1)), 5))
    assert any(p.stats()["n_slices"] > 1 for p in plans)
    b = pk.Batch(plans, "split")
    ws = torch.empty(b.workspace_bytes()[0], dtype=torch.uint8, device="cuda")
    b.upload(ws)
    b.launch(ws)
    Z1, V1 = b.download(ws)
    b.launch(ws)
    Z2, V2 = b.download(ws)
    assert [(z.re, z.im, z.exp2) for z in Z1] == [(z.re, z.im, z.exp2) for z in Z2]
    for p, z, v in zip(plans, Z1, V1):
        zs, vs = pk.evaluate(p, "c128")
        assert rel_err(sc(z), sc(zs)) <= TOL["split"]
        assert rel_err(sc(v), sc(vs)) <= TOL["split"]
    assert abs(V1[-2].to_complex() - 1) < 1e-12 and abs(V1[-1].to_complex() - 1) < 1e-12


@pytest.mark.parametrize("prec", ["split", "c128"])
def test_group_concurrent_replay(ctx, prec):
    """Plans recorded as independent graph branches (run concurrently) give the same
    results as evaluating them one by one, on two replays."""
    import torch
    knots = kg.knot_suite("scale")[:6]
    plans = []
    for k in knots:
        kn = pk.Knot.from_pd(ctx, k.pd, outer=k.outer)
        plans += [pk.Plan(ctx, kn, q) for q in (2, 3)]
    ws = [torch.empty(p.workspace_bytes(prec) + 256, dtype=torch.uint8, device="cuda")
          for p in plans]
    for p, w in zip(plans, ws):
        pk.upload(p, prec, w)
    g = pk.Group(plans, prec, ws)
    for rnd in range(2):
        if rnd:   # the group's own upload and one-wait download
            for w in ws:
                w.zero_()
            g.upload()
        g.launch()
        got = [pk.download(p, prec, w) for p, w in zip(plans, ws)]
        together = g.download()
        for p, (z, v), (z2, v2) in zip(plans, got, together):
            assert (z.mantissa, z.exp2, v.mantissa, v.exp2) == (z2.mantissa, z2.exp2, v2.mantissa, v2.exp2)
            zs, vs = pk.evaluate(p, prec)
            assert rel_err(sc(z), sc(zs)) <= TOL[prec] and rel_err(sc(v), sc(vs)) <= TOL[prec]


def test_batch_launch_shapes_agree(ctx):
    """Every batch launch shape the autotuner may choose (threads per CTA, offsets kept in
    shared memory) gives the default shape's results."""
    knots = kg.knot_suite("batch")[:64]
    ref = None
    c = pk.Context(0)
    import torch
    c.set_stream(torch.cuda.current_stream().cuda_stream)
    for th in (128, 256, 512):
        for kt in (256, 2048):
            c.set_tuning(batch_threads=th, batch_ktab=kt)
            plans = _plans(c, knots, 3)
            Z, V = pk.evaluate_batch(plans, "split")
            if ref is None:
                ref = Z
            for z, zr in zip(Z, ref):
                assert rel_err(sc(z), sc(zr)) <= TOL["split"], (th, kt)


def test_batch_upload_inputs_restores_the_knot_part(ctx):
    """pk_batch_upload_inputs copies only the knot-derived part of the image (the first
    `copied` bytes of the workspace: knot headers, recipes, slots); with that part wiped on
    the device, it alone must bring back the same Z and V, bit for bit."""
    import torch
    knots = kg.knot_suite("batch")[:64]
    plans = _plans(ctx, knots, 3)
    b = pk.Batch(plans, "split")
    nbytes, upbytes = b.workspace_bytes()
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    b.upload(ws)
    b.launch(ws)
    z0, v0 = b.download(ws)
    n = b.upload_inputs(ws)
    assert 0 < n < upbytes
    for rnd in range(2):
        ws[:n].zero_()
        assert b.upload_inputs(ws) == n
        b.launch(ws)
        z1, v1 = b.download(ws)
        for a, c in zip(z0 + v0, z1 + v1):
            assert a.mantissa == c.mantissa and a.exp2 == c.exp2, rnd


def test_plan_and_group_upload_inputs(ctx):
    """pk_upload_inputs / pk_group_upload(inputs_only) copy only the knot-derived part of a
    program (its first `copied` bytes); with that part wiped on the device, it alone brings
    back the same Z and V, bit for bit, for a single plan and for a group."""
    import torch
    knots = kg.knot_suite("scale")[:4]
    plans = []
    for k in knots:
        kn = pk.Knot.from_pd(ctx, k.pd, outer=k.outer)
        plans += [pk.Plan(ctx, kn, q) for q in (3, 5)]
    prec = "split"
    ws = [torch.empty(p.workspace_bytes(prec) + 256, dtype=torch.uint8, device="cuda")
          for p in plans]
    ref = []
    for p, w in zip(plans, ws):
        pk.upload(p, prec, w)
        pk.launch(p, prec, w)
        ref.append(pk.download(p, prec, w))
    n0 = pk.upload_inputs(plans[0], prec, ws[0])
    assert 0 < n0 <= len(plans[0].debug_blob(0))
    ws[0][:n0].zero_()
    assert pk.upload_inputs(plans[0], prec, ws[0]) == n0
    pk.launch(plans[0], prec, ws[0])
    z, v = pk.download(plans[0], prec, ws[0])
    assert (z.mantissa, z.exp2, v.mantissa, v.exp2) == (ref[0][0].mantissa, ref[0][0].exp2,
                                                        ref[0][1].mantissa, ref[0][1].exp2)
    g = pk.Group(plans, prec, ws)
    total = g.upload(inputs_only=True)
    assert 0 < total < sum(len(p.debug_blob(0)) for p in plans) + 1
    for p, w in zip(plans, ws):
        w[:pk.upload_inputs(p, prec, w)].zero_()
    torch.cuda.synchronize()
    assert g.upload(inputs_only=True) == total
    g.launch()
    for (z, v), (zr, vr) in zip(g.download(), ref):
        assert (z.mantissa, z.exp2, v.mantissa, v.exp2) == (zr.mantissa, zr.exp2, vr.mantissa, vr.exp2)
