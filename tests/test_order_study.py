"""The paper's statistics of grid-walk knots and contraction orders (Sec. III.A-B,
Figs. 2-3), reproduced on the host with the library's generator, Reidemeister
simplification and order search, at smaller sizes than the paper's (L <= 50, 20 knots
per L instead of L <= 100 and 200 knots):

* Fig. 2: <n_v> and <n_c> of the simplified Tait graphs grow as L^2 (the paper fits
  log-log slopes 2.013 and 2.074), <n_c>/<n_v> rises towards ~2 (above 13/7 for random
  planar graphs), and the mean maximal degree <Delta_G> grows only slowly (logarithmic);
* Fig. 3: the mean largest rank <Delta_H> met while contracting grows linearly in L for
  the paper's greedy and for the partition order.
The simplification itself is pinned against the oracle: V is unchanged."""
import math
import types

import pytest

import knotgen as kg
import oracle
import paper_1807_02119_gb300 as pk
from paper_1807_02119_gb300 import order_study as st
from oracle.scaled import rel_err


@pytest.fixture(scope="module")
def ctx():
    return pk.Context(-1)


@pytest.fixture(scope="module")
def study(ctx):
    rows = []
    for L in range(10, 51, 4):
        rows += st.sample(pk, ctx, L, 20)
    return st.summarise(rows, fit_last=7)


def test_simplification_keeps_v(ctx):
    """Reidemeister I (loops, spikes) and II (opposite-sign parallel pairs) on the signed
    Tait graph with the (n_v, w, tau) updates of pk_knot_simplify: V from the oracle's
    spin sum and A(q) is unchanged, for kinked closed braids and grid-walk knots."""
    rng = kg.SplitMix64(5)
    cases = [kg.kink(kg.braid_closure_pd([1, 1, 1], 2), 0, i) for i in range(4)]
    cases.append(kg.randomize(kg.braid_closure_pd([1, -2, 1, -2], 3), rng, 6))
    cases += [kg.random_grid_knot(10, s, bool(s % 2), 1).pd for s in range(20)]
    shrunk = 0
    for pd in cases:
        k = pk.Knot.from_pd(ctx, pd)
        s = k.simplified()
        g = oracle.tait_graph(pd)
        i = s.info()
        gs = types.SimpleNamespace(n_v=i["n_v"], writhe=i["writhe"], tau=i["tau"])
        shrunk += i["n_c"] < g.n_crossings
        for q in (2, 3, 5, 6):
            v0 = oracle.jones_from_z(oracle.z_complex(g.n_v, g.edges, q), g, q)
            v1 = oracle.jones_from_z(oracle.z_complex(i["n_v"], s.edges(), q), gs, q)
            assert rel_err(v1, v0) < 1e-10, (pd, q)
        edges = s.edges()
        assert all(u != v for u, v, _ in edges)                        # no loops
        deg = [0] * i["n_v"]
        for u, v, _ in edges:
            deg[u] += 1
            deg[v] += 1
        assert i["n_v"] == 1 or min(deg) >= 2                          # no spikes
        pairs = {}
        for u, v, e in edges:
            pairs.setdefault((min(u, v), max(u, v)), set()).add(e)
        assert all(len(x) == 1 for x in pairs.values())                # no opposite pairs
    assert shrunk >= 10


def test_fig2_quadratic_growth_and_ratio(study):
    assert 1.8 <= study["slope_n_v"] <= 2.3, study["slope_n_v"]
    assert 1.8 <= study["slope_n_c"] <= 2.3, study["slope_n_c"]
    per = study["per_L"]
    assert per[-1]["ratio"] > per[1]["ratio"]                 # rising towards ~2
    assert 13 / 7 - 0.05 <= per[-1]["ratio"] <= 2.05


def test_fig2_maximal_degree_grows_slowly(study):
    per = [e for e in study["per_L"] if e["L"] > 22]
    d0, d1 = per[0]["delta_g"], per[-1]["delta_g"]
    assert d1 < 1.4 * d0                                       # far below linear in L
    assert max(e["delta_g"] for e in per) < 10


def test_fig3_linear_delta_h(study):
    for o in ("greedy_edge", "partition"):
        f = study["delta_h_fit_" + o]
        assert f["slope"] > 0 and f["r2"] > 0.97, (o, f)
    per = study["per_L"]
    # the partition order (spin network, recursive bisection with Fiduccia-Mattheyses
    # refinement) is never worse than the paper's greedy on average here
    assert all(e["partition"] <= e["greedy_edge"] + 1e-9 for e in per)
