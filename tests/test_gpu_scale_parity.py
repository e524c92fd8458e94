"""The bench's scale workload at full size against the CPU oracle, evaluation by
evaluation.

64 random grid-walk knots (L = 40, seeds 1..64, 100..400 crossings, random over/under) at
q = 2, 3, 5: 192 evaluations, run in the launch configuration bench.py times -- plans with
256 min-fill restarts and subtree reconfiguration built on all host cores, one resident
workspace per plan, every plan's launch sequence an independent branch of one CUDA graph --
and compared with the
oracle's Z(q) (Sec. II spin sum) and V = A(q) Z (Eq. JonesPotts) stored in
tests/golden/scale_oracle.txt (written by tests/golden/make_scale_oracle.py from `oracle`
only).  The q = 5 plans carry the tensor-core GEMM steps at their real shapes (several
flush groups of K, stacked digit MMAs, up to 25 batch indices); the 6 q = 5 pairs the
oracle cannot reach within 5^12 entries per factor are compared between the precisions.
"split4" is the split precision with four BF16 digits per operand on the tensor cores
(PK_FLAG_TC_DIGITS4) instead of five: its truncation (about 2^-32 of a row's and a column's
largest entries per product) misses the 1e-6 target on this workload (1.25e-6 at seed 58,
q = 5, on earlier plans; 7.0e-6 on the reconfigured ones, measured on GB300), which is why
five digits are the default.  One digit fewer per operand raises the truncation bound by
2^8, so split4 is held to 2^8 times the split tolerance.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import pytest

import knotgen as kg
import paper_1807_02119_gb300 as pk
from oracle.scaled import SC, rel_err

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "scale_oracle.txt")
RESTARTS = 256   # min-fill restarts per plan, as bench.py builds the workload's plans
REFINE = 8       # subtree reconfiguration (frontiers of up to 8 subtrees), as bench.py
TOL = {"split": 1e-6, "split4": 256e-6, "split_db": 1e-6, "split_narrow": 1e-6, "c128": 1e-10}
QS = (2, 3, 5)


def load_golden():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#"):
            continue
        f = line.split()
        seed, q, w = int(f[0]), int(f[1]), int(f[2])
        if f[3] == "-":
            out[(seed, q)] = None
            continue
        z = SC.of(complex(float.fromhex(f[3]), float.fromhex(f[4])), int(f[5]))
        v = SC.of(complex(float.fromhex(f[6]), float.fromhex(f[7])), int(f[8]))
        out[(seed, q)] = (z, v)
    return out


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = pk.Context(0)
    c.set_stream(torch.cuda.current_stream().cuda_stream)
    return c


def _plans(ctx, flags=0, qs=QS, **tuning):
    """The workload's plans; `tuning` fields are set on a context of their own."""
    if tuning:
        import torch
        ctx = pk.Context(0)
        ctx.set_stream(torch.cuda.current_stream().cuda_stream)
        ctx.set_tuning(**tuning)
    knots = [kg.random_grid_knot(40, s, True, 100, 400) for s in range(1, 65)]
    kn = [pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer) for gk in knots]
    jobs = [(gk.seed, k, q) for gk, k in zip(knots, kn) for q in qs]
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        plans = list(ex.map(lambda j: pk.Plan(ctx, j[1], j[2], restarts=RESTARTS, flags=flags,
                                                     refine=REFINE), jobs))
    return [(seed, q) for seed, _, q in jobs], plans


@pytest.fixture(scope="module")
def workload(ctx):
    return _plans(ctx)


def sc(s):
    return SC.of(s.mantissa, s.exp2)


def run_group(plans, prec):
    import torch
    ws = [torch.empty(p.workspace_bytes(prec) + 256, dtype=torch.uint8, device="cuda")
          for p in plans]
    for p, w in zip(plans, ws):
        pk.upload(p, prec, w)
    g = pk.Group(plans, prec, ws)
    g.launch()
    res = [pk.download(p, prec, w) for p, w in zip(plans, ws)]
    del g, ws
    torch.cuda.empty_cache()
    return res


def test_golden_covers_the_tensor_core_shapes(workload):
    keys, plans = workload
    gold = load_golden()
    assert set(gold) == set(keys)
    assert sum(v is not None for v in gold.values()) >= 180
    multi = [k for k, p in zip(keys, plans) if gold[k] is not None and
             any(st["kernel"] == 2 and st["K"] > 96 for st in p.steps())]
    # q = 5 plans whose tensor-core steps have K > 96 complex (several flush groups),
    # including K = 3125 steps
    assert len(multi) >= 40, len(multi)
    assert any(st["K"] == 3125 and st["kernel"] == 2
               for k, p in zip(keys, plans) if gold[k] is not None for st in p.steps())


@pytest.mark.parametrize("prec", ["split", "split4", "split_db", "split_narrow", "c128"])
def test_scale_workload_vs_oracle(ctx, workload, prec):
    """split_db: every tensor-core step on the double-buffered GEMM (one CTA per SM, two
    accumulator sets); split_narrow: row steps of GEMM shape down to K = 4 and N = 8 on the
    tensor cores too (tiles with most of their 24 columns idle)."""
    if prec == "split4":
        keys, plans = _plans(ctx, pk.FLAG_TC_DIGITS4)
    elif prec == "split_db":
        keys, plans = _plans(ctx, tc_db_groups=1)
    elif prec == "split_narrow":
        keys, plans = _plans(ctx, tc_min_k=4, tc_min_n=8)
        import ctypes as C
        from plan_replay import Step
        narrow = 0
        for p in plans:
            b = p.debug_blob(1)
            narrow += sum(st.tc > 0 and st.N < 32 for st in
                          (Step * (len(b) // C.sizeof(Step))).from_buffer_copy(b))
        assert narrow >= 500, narrow      # tensor-core steps with N < 32 (mostly 25 = 5^2)
    else:
        keys, plans = workload
    gold = load_golden()
    res = run_group(plans, "split" if prec.startswith("split") else prec)
    worst, worst_tc, n_tc, n_cmp = 0.0, 0.0, 0, 0
    for key, p, (z, v) in zip(keys, plans, res):
        ref = gold[key]
        if ref is None:
            if key[1] == 2:    # V(i) = +-1 for every knot
                c = v.to_complex()
                assert abs(abs(c.real) - 1) < 1e-9 and abs(c.imag) < 1e-9, key
            continue
        e = max(rel_err(sc(z), ref[0]), rel_err(sc(v), ref[1]))
        assert e <= TOL[prec], (key, e)
        worst = max(worst, e)
        n_cmp += 1
        if any(st["kernel"] == 2 and st["K"] > 96 for st in p.steps()):
            n_tc += 1
            worst_tc = max(worst_tc, e)
    print(f"[scale {prec}] {n_cmp} evaluations vs the oracle, worst {worst:.2e}; "
          f"{n_tc} with multi-group GEMM steps, worst {worst_tc:.2e}")


def test_scale_workload_beyond_the_oracle(workload):
    """The pairs too wide for the oracle: split (tensor cores) against complex128 (FP64
    on the CUDA cores) at the split tolerance."""
    keys, plans = workload
    gold = load_golden()
    wide = [(k, p) for k, p in zip(keys, plans) if gold[k] is None]
    assert wide
    ps = [p for _, p in wide]
    rs, rc = run_group(ps, "split"), run_group(ps, "c128")
    for (k, _), (zs, vs), (zc, vc) in zip(wide, rs, rc):
        e = max(rel_err(sc(zs), sc(zc)), rel_err(sc(vs), sc(vc)))
        assert e <= TOL["split"], (k, e)


def test_double_buffered_gemm_is_bit_identical(ctx):
    """The two GEMM variants form the same products and flush the groups in the same order:
    the q = 5 evaluations agree bit for bit (every tensor-core step double-buffered against
    none)."""
    keys, p1 = _plans(ctx, qs=(5,), tc_db_groups=0)
    _, p2 = _plans(ctx, qs=(5,), tc_db_groups=1)
    assert sum(any(st["kernel"] == 2 and st["K"] > 96 for st in p.steps()) for p in p1) >= 40
    r1, r2 = run_group(p1, "split"), run_group(p2, "split")
    for k, (z1, v1), (z2, v2) in zip(keys, r1, r2):
        assert (z1, v1) == (z2, v2), k
