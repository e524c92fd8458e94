"""The Jones polynomial's coefficients by interpolation between exact values at integer q
(the conclusions' extension), host stages on the CPU: pk_jones_plan / pk_jones_solve fed
with the oracle's exact Z(q) in Z[t] reduced modulo the library's primes must give the
Kauffman bracket's polynomial, for knots and links; bad data must be refused, not
rounded."""
import pytest

import knotgen as kg
import oracle
import paper_1807_02119_gb300 as pk
from oracle.kauffman import jones_poly


@pytest.fixture(scope="module")
def ctx():
    return pk.Context(-1)


def _residues(pd, outer, qs, primes):
    g = oracle.tait_graph(pd, outer=outer)
    rows = []
    for q in qs:
        a, b = oracle.z_exact(g.n_v, g.edges, q)      # Z(q) = a + b t exactly
        rows.append([(a % p, b % p) for p in primes])
    return rows


def _cases():
    out = [(kg.braid_closure_pd(w, n), None) for w, n in
           (([1, 1, 1], 2), ([-1, -1, -1], 2), ([1, -2, 1, -2], 3), ([1] * 5, 2), ([1] * 7, 2),
            ([1, 2] * 4, 3), ([1, 2, 3] * 5, 4))]
    out.append((kg.kink(kg.braid_closure_pd([1, 1, 1], 2), 0, 1), None))
    for s in range(6):
        gk = kg.random_grid_knot(10, 100 + s, True, 8, 16)
        out.append((gk.pd, gk.outer))
    return out


@pytest.mark.parametrize("i", range(14))
def test_solve_matches_bracket(ctx, i):
    pd, outer = _cases()[i]
    k = pk.Knot.from_pd(ctx, pd, outer=outer)
    qs, primes = pk.jones_plan(k)
    assert qs == list(range(1, len(qs) + 1)) and len(primes) == 4
    assert 2 * len(qs) <= k.info()["n_c"] + 1 + 5      # span <= crossings
    got = pk.jones_solve(k, qs, primes, _residues(pd, outer, qs, primes))
    assert got == jones_poly(pd)


def test_unknot_and_kinks(ctx):
    for pd in ([], kg.kink([], 0, 0), kg.kink(kg.kink([], 0, 0), 1, 2)):
        k = pk.Knot.from_pd(ctx, pd)
        qs, primes = pk.jones_plan(k)
        assert pk.jones_solve(k, qs, primes, _residues(pd, None, qs, primes)) == {0: 1}


def test_inconsistent_data_is_refused(ctx):
    pd = kg.braid_closure_pd([1] * 5, 2)
    k = pk.Knot.from_pd(ctx, pd)
    qs, primes = pk.jones_plan(k)
    rows = _residues(pd, None, qs, primes)
    rows[-1][0] = ((rows[-1][0][0] + 1) % primes[0], rows[-1][0][1])   # one wrong residue
    with pytest.raises(pk.PkError):
        pk.jones_solve(k, qs, primes, rows)
    rows = _residues(pd, None, qs, primes)
    rows[0][3] = ((rows[0][3][0] + 7) % primes[3], rows[0][3][1])      # the check prime disagrees
    with pytest.raises(pk.PkError):
        pk.jones_solve(k, qs, primes, rows)


@pytest.mark.parametrize("word,ns", [([1, -1], 2), ([1, 1], 2), ([-1, -1], 2), ([1, 1, 1, 1], 2),
                                     ([1] * 6, 2), ([1, 2] * 3, 3), ([1, -2, 1, 2, 2, -1, 2], 3),
                                     ([1, 2, 3, 1, 2, 3, -2, 1], 4)])
def test_solve_links_match_bracket(ctx, word, ns):
    """Links: half-integer powers (an even number of components) through W = V t^(-1/2)."""
    pd, signs, comps = kg.braid_closure_link(word, ns)
    k = pk.Knot.from_link_pd(ctx, pd, signs)
    g = oracle.tait_graph(pd, signs=signs)
    qs, primes = pk.jones_plan(k)
    rows = []
    for q in qs:
        a, b = oracle.z_exact(g.n_v, g.edges, q)
        rows.append([(a % p, b % p) for p in primes])
    assert pk.jones_solve(k, qs, primes, rows) == jones_poly(pd, signs)


def test_graphs_are_refused(ctx):
    with pytest.raises(pk.PkError):
        pk.jones_plan(pk.Knot.from_signed_graph(ctx, 2, [(0, 1, 1), (0, 1, 1), (0, 1, 1)], 3))


def _sliced(ctx, k, q):
    lim = pk.Plan(ctx, k, q).stats()["log2_max_elems"]
    while lim > 1.0:
        lim -= 0.5
        p = pk.Plan(ctx, k, q, max_log2_elems=lim)
        if p.stats()["n_slices"] > 1:
            return p if p.stats()["n_slices"] <= 243 else None
    return None


def test_exact_records_replay_matches_oracle(ctx):
    """The records the exact kernels read (recipes with the packed clause data, steps,
    slices, the folded loops' factor), replayed modulo p, give the oracle's exact Z(q) for
    every q the interpolation uses (1 .. n_q, including q = 1 and 4), every order, and
    sliced plans."""
    from plan_replay import replay_exact
    p = 2147483629
    cases = [(kg.braid_closure_pd([1, 1, 1], 2), None),
             (kg.kink(kg.braid_closure_pd([1, -2, 1, -2], 3), 0, 1), None)]
    for s in range(2):
        gk = kg.random_grid_knot(10, 300 + s, True, 10, 18)
        cases.append((gk.pd, gk.outer))
    for pd, outer in cases:
        k = pk.Knot.from_pd(ctx, pd, outer=outer)
        g = oracle.tait_graph(pd, outer=outer)
        qs, _ = pk.jones_plan(k)
        for q in qs:
            a, b = oracle.z_exact(g.n_v, g.edges, q)
            want = (a % p, b % p)
            plans = [pk.Plan(ctx, k, q, order=o) for o in ("auto", "greedy_edge", "elim_spin")]
            if q in (3, 5):
                sp = _sliced(ctx, k, q)
                if sp is not None:
                    plans.append(sp)
            for pl in plans:
                assert replay_exact(pl, p) == want, (len(pd), q)
