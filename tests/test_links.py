"""Links (several components), on the CPU: the oracle against pins that do not go
through the Potts model, and the library's host path (PD parsing with crossing signs,
plan replay, the A(q) prefactor with the principal fourth root of t) against the oracle.

The paper's conclusions note that Tait graphs, and so the method, extend to links.  V of
a link lies in Z[t^(1/2)]; both sides evaluate its half-integer powers with the principal
branch s = exp(Log t / 4) of the Potts t(q).

Pins:
* the skein relation t^-1 V(L+) - t V(L-) = (t^(1/2) - t^(-1/2)) V(L0) on closures of
  sigma_1^n (textbook; V(unknot) = 1, V(2-component unlink) = -t^(1/2) - t^(-1/2)),
  which fixes V of every T(2, n) independently of the bracket and of the Potts model;
* V(1) = (-2)^(c-1) for a c-component link;
* V(mirror)(t) = V(1/t) (as Laurent polynomials in t^(1/2));
* the bracket state sum against the oracle's Potts value at q = 2, 3, 5, 6, and the
  library's host V against both.
"""
from fractions import Fraction

import pytest

import knotgen as kg
import oracle
import paper_1807_02119_gb300 as pk
from oracle.kauffman import jones_poly
from oracle.ring import laurent_eval_complex
from oracle.scaled import SC
from plan_replay import replay

HALF = Fraction(1, 2)

LINKS = [
    ([1, -1], 2),                  # 2-component unlink (Reidemeister II diagram)
    ([1, 1], 2),                   # positive Hopf link
    ([-1, -1], 2),                 # negative Hopf link
    ([1, 1, 1, 1], 2),             # T(2, 4)
    ([1, 1, 1, 1, 1, 1], 2),       # T(2, 6)
    ([1, 2] * 3, 3),               # T(3, 3), three components
    ([1, -2, 1, 2, 2, -1, 2], 3),  # mixed signs, two components
    ([1, 2, 3, 1, 2, 3, -2, 1], 4),
    ([1, 1, 1], 2),                # the trefoil, through the link path
]


def _norm(poly):
    return {k: v for k, v in poly.items() if v}


def _mul(p, r):
    out = {}
    for i, x in p.items():
        for j, y in r.items():
            out[i + j] = out.get(i + j, 0) + x * y
    return _norm(out)


def _add(p, r):
    out = dict(p)
    for k, v in r.items():
        out[k] = out.get(k, 0) + v
    return _norm(out)


def _key(e):
    e = Fraction(e)
    return int(e) if e.denominator == 1 else e


def _skein_torus_2(n_max):
    """V of the closure of sigma_1^n from V_n = t^2 V_{n-2} + t (t^(1/2) - t^(-1/2)) V_{n-1}."""
    vs = [{HALF: -1, -HALF: -1}, {0: 1}]
    step = {Fraction(3, 2): 1, HALF: -1}            # t (t^(1/2) - t^(-1/2))
    for _ in range(2, n_max + 1):
        vs.append(_add(_mul({2: 1}, vs[-2]), _mul(step, vs[-1])))
    return [{_key(k): v for k, v in p.items()} for p in vs]


def test_bracket_matches_skein_on_torus_links():
    ref = _skein_torus_2(10)
    for n in range(1, 11):
        pd, signs, comps = kg.braid_closure_link([1] * n, 2)
        assert comps == (2 if n % 2 == 0 else 1)
        assert jones_poly(pd, signs) == ref[n], n
    assert ref[2] == {HALF: -1, Fraction(5, 2): -1}      # the Hopf link


@pytest.mark.parametrize("word,ns", LINKS)
def test_value_at_one_and_mirror(word, ns):
    pd, signs, comps = kg.braid_closure_link(word, ns)
    v = jones_poly(pd, signs)
    assert sum(v.values()) == (-2) ** (comps - 1)
    mpd, msigns, _ = kg.braid_closure_link([-g for g in word], ns)
    assert jones_poly(mpd, msigns) == {_key(-k): c for k, c in v.items()}


@pytest.mark.parametrize("word,ns", LINKS)
def test_potts_oracle_matches_bracket(word, ns):
    pd, signs, comps = kg.braid_closure_link(word, ns)
    g = oracle.tait_graph(pd, signs=signs)
    assert g.components == comps
    assert (3 * g.writhe + g.tau + 2 * g.n_v + 2) % (4 if comps == 1 else 2) == 0
    v = jones_poly(pd, signs)
    for q in (2, 3, 5, 6):
        vb = laurent_eval_complex(v, oracle.t_of_q(q))
        vo = oracle.jones_from_z(oracle.z_complex(g.n_v, g.edges, q), g, q)
        vo = vo.m * 2.0 ** vo.e
        assert abs(vo - vb) <= 1e-9 * max(1.0, abs(vb)), (word, q, vo, vb)


@pytest.fixture(scope="module")
def ctx():
    return pk.Context(-1)


@pytest.mark.parametrize("word,ns", LINKS)
def test_library_host_path(ctx, word, ns):
    """pk_link_from_pd (components, writhe, tau), the plan's Z replayed on the CPU and
    pk_jones_from_z against the oracle and the bracket."""
    pd, signs, comps = kg.braid_closure_link(word, ns)
    k = pk.Knot.from_link_pd(ctx, pd, signs)
    g = oracle.tait_graph(pd, signs=signs)
    info = k.info()
    assert (info["components"], info["writhe"], info["tau"], info["n_v"]) == \
        (comps, g.writhe, g.tau, g.n_v)
    v = jones_poly(pd, signs)
    for q in (1, 2, 3, 4, 5, 6):
        zm, ze = replay(pk.Plan(ctx, k, q))
        z = SC.of(zm, ze)
        zo = oracle.z_complex(g.n_v, g.edges, q)
        vl = k.jones_from_z(q, pk.Scaled(z.m.real, z.m.imag, z.e)).to_complex()
        vb = laurent_eval_complex(v, oracle.t_of_q(q))
        scale = max(1.0, abs(vb))
        assert abs(vl - vb) <= 1e-9 * scale, (word, q, vl, vb)
        zz = zo.m * 2.0 ** zo.e
        assert abs(z.m * 2.0 ** z.e - zz) <= 1e-9 * max(1.0, abs(zz))


def test_knot_through_link_entry_matches(ctx):
    """A knot given with its crossing signs parses to the same Tait data."""
    for word, ns in (([1, 1, 1], 2), ([1, -2, 1, -2], 3), ([1, 1, 1, 1, 1], 2)):
        pd = kg.braid_closure_pd(word, ns)
        pd2, signs, comps = kg.braid_closure_link(word, ns)
        assert comps == 1
        a = pk.Knot.from_pd(ctx, pd).info()
        b = pk.Knot.from_link_pd(ctx, pd2, signs).info()
        assert a == b


def test_link_input_errors(ctx):
    pd, signs, _ = kg.braid_closure_link([1, 1], 2)
    with pytest.raises(pk.PkError):
        pk.Knot.from_link_pd(ctx, pd, [1, 0])          # a sign must be +-1
    with pytest.raises(pk.PkError):
        pk.Knot.from_link_pd(ctx, pd, [1, -1])         # inconsistent orientation
    with pytest.raises(ValueError):
        kg.braid_closure_link([1, 1], 3)               # split diagram (sigma_2 unused)


@pytest.mark.parametrize("word,ns", [([1, 1], 2), ([1, 1, 1, 1], 2), ([1, 2] * 3, 3), ([1, -2, 1, 2, 2, -1, 2], 3)])
def test_link_reverse_pass_host(ctx, word, ns):
    """(1/V) dV/dt at fixed q for links: the library's host stage (its A(q) exponent is a
    multiple of 1/2 here) on the replayed reverse program against the oracle."""
    import numpy as np

    import oracle.grad as og
    from plan_replay import replay_grad
    pd, signs, _ = kg.braid_closure_link(word, ns)
    k = pk.Knot.from_link_pd(ctx, pd, signs)
    info = k.info()
    g = oracle.tait_graph(pd, signs=signs)
    for q in (3, 5):
        p = pk.Plan(ctx, k, q, grad=True, checkpoint_stride=2)
        (zm, ze), acc, ae = replay_grad(p)
        z = SC.of(zm, ze)
        d, dv = pk.grad_from_accumulators(p, acc, ae, pk.Scaled(z.m.real, z.m.imag, z.e))
        dvo = og.dlogv_dt(g.n_v, g.edges, q, g.writhe, g.tau)
        assert (info["writhe"], info["tau"], info["n_v"]) == (g.writhe, g.tau, g.n_v)
        assert abs(dv - dvo) <= 1e-9 * max(1.0, abs(dvo)), (word, q, dv, dvo)
        assert np.all(np.isfinite(d))
