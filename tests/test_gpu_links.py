"""Links on the GPU: Z and V of multi-component diagrams (pk_link_from_pd) in complex128
and split precision against the oracle (Potts value, principal fourth root of t) and, for
small ones, the Kauffman bracket."""
import pytest

import knotgen as kg
import oracle
import paper_1807_02119_gb300 as pk
from oracle.kauffman import jones_poly
from oracle.ring import laurent_eval_complex
from test_links import LINKS

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "split": 1e-6}


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = pk.Context(0)
    c.set_stream(torch.cuda.current_stream().cuda_stream)
    return c


def _random_links(count, seed):
    """Seeded random braid words on 3-5 strands (every generator used) whose closures
    have at least two components, 20-40 crossings."""
    rng = kg.SplitMix64(seed)
    out = []
    while len(out) < count:
        ns = 3 + rng.below(3)
        n = 20 + rng.below(21)
        word = [(1 + rng.below(ns - 1)) * (1 if rng.bit() else -1) for _ in range(n)]
        try:
            pd, signs, comps = kg.braid_closure_link(word, ns)
        except ValueError:
            continue
        if comps >= 2:
            out.append((pd, signs, comps))
    return out


@pytest.mark.parametrize("prec", ["c128", "split"])
def test_links_small_match_bracket(ctx, prec):
    for word, ns in LINKS:
        pd, signs, comps = kg.braid_closure_link(word, ns)
        k = pk.Knot.from_link_pd(ctx, pd, signs)
        v = jones_poly(pd, signs)
        for q in (2, 3, 4, 5, 6):
            _, vg = pk.evaluate(pk.Plan(ctx, k, q), prec)
            vb = laurent_eval_complex(v, oracle.t_of_q(q))
            assert abs(vg.to_complex() - vb) <= TOL[prec] * max(1.0, abs(vb)), (word, q)


@pytest.mark.parametrize("prec", ["c128", "split"])
def test_random_links_match_oracle(ctx, prec):
    for pd, signs, comps in _random_links(6, 2024):
        k = pk.Knot.from_link_pd(ctx, pd, signs)
        assert k.info()["components"] == comps
        g = oracle.tait_graph(pd, signs=signs)
        for q in (3, 5):
            zg, vg = pk.evaluate(pk.Plan(ctx, k, q), prec)
            vo = oracle.jones_from_z(oracle.z_complex(g.n_v, g.edges, q), g, q)
            vgs = oracle.scaled.SC.of(vg.mantissa, vg.exp2)
            assert oracle.scaled.rel_err(vgs, vo) <= TOL[prec], (comps, q)
