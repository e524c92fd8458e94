"""The tensor-core GEMM path of the split precision (k_gemm_tc: tcgen05 BF16 digit
products, exact FP32 accumulation per level) against complex128 and against the same
precision on the CUDA cores (PK_FLAG_NO_TC), and the whole split pipeline against the
CPU oracle."""
import pytest

import knotgen as kg
import oracle
import paper_1807_02119_gb300 as pk
from oracle.scaled import SC, rel_err

pytestmark = pytest.mark.gpu

SPLIT_TOL = 1e-6


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


def test_tc_forced_gemm_small(ctx):
    """Every two-operand step forced onto the GEMM kernel: ragged tiles (M, N not
    multiples of 64, K not a multiple of 32), several batch indices, q = 2, 3, 5."""
    worst = 0.0
    for s in range(6):
        gk = kg.random_grid_knot(15, 60 + s, True, 15, 40)
        k = pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer)
        g = oracle.tait_graph(gk.pd, outer=gk.outer)
        for q in (2, 3, 5):
            p = pk.Plan(ctx, k, q, flags=pk.FLAG_FORCE_GEMM)
            assert any(st["kernel"] == 2 for st in p.steps())
            z, v = pk.evaluate(p, "split")
            zo = oracle.z_complex(g.n_v, g.edges, q)
            e = rel_err(sc(z), zo)
            worst = max(worst, e)
            assert e <= SPLIT_TOL, (s, q, e)
    print(f"[tc forced] worst relative error vs the oracle {worst:.2e}")


def test_tc_matches_cuda_core_gemm_full_size(ctx):
    """Knots of the L=40 workload at q = 3 and 5, where the widest steps are large
    GEMMs: tensor-core split, CUDA-core split and complex128 agree."""
    worst = 0.0
    for gk in [kg.random_grid_knot(40, s, True, 100, 400) for s in (1, 2, 3, 5)]:
        k = pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer)
        for q in (3, 5):
            p = pk.Plan(ctx, k, q)
            if not any(st["kernel"] == 2 for st in p.steps()):
                continue
            z_tc, v_tc = pk.evaluate(p, "split")
            z_sm, v_sm = pk.evaluate(pk.Plan(ctx, k, q, flags=pk.FLAG_NO_TC), "split")
            z_64, v_64 = pk.evaluate(p, "c128")
            e = max(rel_err(sc(z_tc), sc(z_64)), rel_err(sc(v_tc), sc(v_64)))
            worst = max(worst, e)
            assert e <= SPLIT_TOL, (gk.seed, q, e)
            assert rel_err(sc(z_sm), sc(z_64)) <= SPLIT_TOL
    print(f"[tc full size] worst relative error vs complex128 {worst:.2e}")
