"""Pins for the CPU oracle: each check is independent of the oracle's own code path.

* values printed in the paper (Fig. 1 caption, tests/golden/fig1_trefoil.txt);
* closed forms of t(q) and of textbook Jones polynomials (trefoil, figure-eight,
  torus knots T(p, r));
* brute-force spin sums on tiny graphs (the literal definition of Z, Sec. II);
* the Kauffman-bracket state sum (independent of the Tait graph);
* knot invariants that hold for every knot at any size.
"""
import cmath
import math
import random

import pytest

import knotgen as kg
import oracle
from oracle.kauffman import jones_poly
from oracle.potts import (exact_to_complex, t_of_q, z_bruteforce, z_bruteforce_exact)
from oracle.ring import Zt
from oracle.scaled import SC, rel_err

GOLDEN = __file__.rsplit("/", 1)[0] + "/golden/fig1_trefoil.txt"
TREFOIL = kg.braid_closure_pd([1, 1, 1], 2)
FIG8 = kg.braid_closure_pd([1, -2, 1, -2], 3)


def torus_jones(p, r):
    """Textbook V(T(p,r)) = t^{(p-1)(r-1)/2} (1 - t^{p+1} - t^{r+1} + t^{p+r}) / (1 - t^2),
    divided out exactly; returns {power: coeff}."""
    num = {0: 1}
    for k, c in ((p + 1, -1), (r + 1, -1), (p + r, 1)):
        num[k] = num.get(k, 0) + c
    deg = max(num)
    coeffs = [num.get(i, 0) for i in range(deg + 1)]
    quo = [0] * (deg - 1)
    # divide by (1 - t^2) from the low end: quo[i] = coeffs[i] + quo[i-2]
    for i in range(deg - 1):
        quo[i] = coeffs[i] + (quo[i - 2] if i >= 2 else 0)
    sh = (p - 1) * (r - 1) // 2
    return {i + sh: c for i, c in enumerate(quo) if c}


def laurent_value(poly, q):
    t = t_of_q(q)
    return sum(c * t ** k for k, c in poly.items())


def exact_value(poly, q):
    return Zt(q).eval_laurent(poly)


def v_exact_as_ring(pd, q, **kw):
    v, den = oracle.jones_exact(pd, q, **kw)
    assert v[0] % den == 0 and v[1] % den == 0, "V must be integral in Z[t] for a knot"
    return (v[0] // den, v[1] // den)


# ----------------------------------------------------------------------------- t(q)

def test_t_of_q_closed_forms():
    expect = {1: cmath.exp(2j * math.pi / 3), 2: 1j, 3: cmath.exp(1j * math.pi / 3), 4: 1.0,
              5: (3 + math.sqrt(5)) / 2, 6: 2 + math.sqrt(3)}
    for q, t in expect.items():
        assert abs(t_of_q(q) - t) < 1e-15
        assert abs(t_of_q(q) + 1 / t_of_q(q) - (q - 2)) < 1e-14  # t solves x^2-(q-2)x+1


# ----------------------------------------------------------------------------- paper values

def test_fig1_caption_values():
    vals = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        q, expr = line.split("\t")
        vals[int(q)] = eval(expr, {"__builtins__": {}},
                            {"I": 1j, "sqrt": math.sqrt, "phi2": (3 + math.sqrt(5)) / 2})
    assert set(vals) == {3, 5}
    for q, v in vals.items():
        got = oracle.jones(TREFOIL, q)
        assert rel_err(got, SC.of(v)) < 1e-12, (q, got, v)
        ve = exact_to_complex(*oracle.jones_exact(TREFOIL, q), q)
        assert rel_err(ve, SC.of(v)) < 1e-15


# ----------------------------------------------------------------------------- bracket pins

def test_bracket_closed_forms():
    assert jones_poly(TREFOIL) == {1: 1, 3: 1, 4: -1}
    assert jones_poly(FIG8) == {-2: 1, -1: -1, 0: 1, 1: -1, 2: 1}
    assert jones_poly(kg.mirror(TREFOIL)) == {-1: 1, -3: 1, -4: -1}
    assert jones_poly([]) == {0: 1}
    for var in range(4):
        assert jones_poly(kg.kink([], 0, var)) == {0: 1}
    for p, r in ((2, 5), (2, 7), (3, 4), (3, 5), (2, 9)):
        pd = kg.braid_closure_pd(kg.torus_braid(p, r), p)
        assert jones_poly(pd) == torus_jones(p, r), (p, r)


def test_torus_formula_matches_trefoil():
    assert torus_jones(2, 3) == {1: 1, 3: 1, 4: -1}


# ----------------------------------------------------------------------------- brute force Z

def _random_signed_graph(rng, n_v, n_e, loops=True):
    edges = []
    for _ in range(n_e):
        u = rng.randrange(n_v)
        v = rng.randrange(n_v) if loops else rng.choice([x for x in range(n_v) if x != u] or [u])
        edges.append((u, v, rng.choice((1, -1))))
    return edges


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_elimination_matches_bruteforce(q):
    rng = random.Random(1000 + q)
    for trial in range(12):
        n_v = rng.randint(1, 6 if q <= 3 else 5)
        edges = _random_signed_graph(rng, n_v, rng.randint(0, 9))
        zb = z_bruteforce(n_v, edges, q)
        zc = oracle.z_complex(n_v, edges, q)
        assert rel_err(zc, SC.of(zb)) < 1e-12 or abs(zb) < 1e-12
        assert oracle.z_exact(n_v, edges, q) == z_bruteforce_exact(n_v, edges, q)


def test_isolated_vertices_and_empty():
    for q in range(1, 6):
        assert oracle.z_exact(1, [], q) == (q, 0)
        assert oracle.z_exact(3, [], q) == (q ** 3, 0)


# ----------------------------------------------------------------------------- oracle vs bracket

def _small_knots():
    out = [TREFOIL, FIG8, kg.kink([], 0, 0), kg.kink([], 0, 1), kg.kink([], 0, 2),
           kg.kink([], 0, 3), kg.mirror(FIG8), kg.braid_closure_pd([1, 1, 1, 2, -1, 2], 3)]
    for seed in range(40):
        k = kg.random_grid_knot(8, seed, random_over_under=bool(seed % 2), ncross_min=1,
                                ncross_max=11)
        out.append(k.pd)
    rng = kg.SplitMix64(77)
    out.append(kg.randomize(TREFOIL, rng, 4))
    out.append(kg.randomize(FIG8, rng, 3))
    return out


def test_oracle_matches_bracket_exactly():
    for pd in _small_knots():
        poly = jones_poly(pd)
        for q in range(1, 7):
            assert v_exact_as_ring(pd, q) == exact_value(poly, q), (pd, q)


def test_oracle_complex_matches_bracket():
    for pd in _small_knots()[:20]:
        poly = jones_poly(pd)
        for q in (2, 3, 5, 6):
            want = laurent_value(poly, q)
            got = oracle.jones(pd, q)
            scale = max(1.0, sum(abs(c) * abs(t_of_q(q)) ** k for k, c in poly.items()))
            assert abs(got.to_complex() - want) <= 1e-12 * scale, (pd, q)


# ----------------------------------------------------------------------------- invariants

def _grid_knots(n, L, seed0=0):
    return [kg.random_grid_knot(L, seed0 + s, True, 1).pd for s in range(n)]


def test_exponent_congruence_and_components():
    for pd in _grid_knots(30, 14) + _small_knots():
        for black in (0, 1):
            g = oracle.tait_graph(pd, black=black)
            assert g.components == 1
            assert (3 * g.writhe + g.tau + 2 * g.n_v + 2) % 4 == 0
            assert g.black_faces + g.white_faces == g.n_crossings + 2


def test_easy_points():
    """V = 1 at q = 1 (t = e^{2 pi i/3}) and q = 4 (t = 1); V = +-1 at q = 2 (t = i)."""
    for pd in _grid_knots(12, 16):
        assert v_exact_as_ring(pd, 1) == (1, 0)
        assert v_exact_as_ring(pd, 4) in ((1, 0),) or sum(v_exact_as_ring(pd, 4)) == 1
        a, b = v_exact_as_ring(pd, 2)
        assert b == 0 and a in (1, -1)
        for q in (1, 2, 4):
            v = oracle.jones(pd, q).to_complex()
            assert abs(abs(v) - 1) < 1e-9


def test_dual_colouring_same_v():
    for pd in _grid_knots(10, 14, 100):
        for q in (2, 3, 5):
            assert v_exact_as_ring(pd, q, black=0) == v_exact_as_ring(pd, q, black=1)


def test_outer_face_convention():
    """With the unbounded region white (Sec. II), V agrees with the other colouring."""
    for s in range(10):
        k = kg.random_grid_knot(12, 300 + s, True, 2)
        g = oracle.tait_graph(k.pd, outer=k.outer)
        assert g.components == 1
        for q in (3, 5):
            assert v_exact_as_ring(k.pd, q, outer=k.outer) == v_exact_as_ring(k.pd, q, black=0)


def test_reidemeister_invariance():
    rng = kg.SplitMix64(2024)
    for pd in _grid_knots(8, 13, 200):
        moved = kg.randomize(pd, rng, 6)
        assert len(moved) > len(pd)
        for q in (2, 3, 5, 6):
            assert v_exact_as_ring(pd, q) == v_exact_as_ring(moved, q)


def test_mirror_is_t_inverse():
    """V_mirror(t) = V(1/t): in Z[t] the map t -> 1/t = (q-2) - t sends a + b t to
    (a + b (q-2)) - b t."""
    for pd in _grid_knots(8, 13, 400):
        for q in (2, 3, 5, 6):
            a, b = v_exact_as_ring(pd, q)
            assert v_exact_as_ring(kg.mirror(pd), q) == (a + b * (q - 2), -b)


def test_connected_sum_multiplies():
    ks = _grid_knots(6, 12, 500)
    for i in range(0, 6, 2):
        s = kg.connected_sum(ks[i], ks[i + 1])
        for q in (2, 3, 5):
            R = Zt(q)
            assert v_exact_as_ring(s, q) == R.mul(v_exact_as_ring(ks[i], q),
                                                   v_exact_as_ring(ks[i + 1], q))


def test_torus_knots_large():
    """T(2,r) up to 101 crossings and T(3,r): closed form vs oracle (complex and exact)."""
    for p, r in ((2, 51), (2, 101), (3, 31), (4, 9)):
        pd = kg.braid_closure_pd(kg.torus_braid(p, r), p)
        poly = torus_jones(p, r)
        for q in (2, 3, 5, 6):
            assert v_exact_as_ring(pd, q) == exact_value(poly, q), (p, r, q)
            want = exact_to_complex(exact_value(poly, q), 1, q)
            assert rel_err(oracle.jones(pd, q), want) < 1e-9, (p, r, q)


def test_order_independence():
    for pd in _grid_knots(6, 15, 600):
        g = oracle.tait_graph(pd)
        for q in (3, 5):
            z1 = oracle.z_complex(g.n_v, g.edges, q)
            z2 = oracle.z_complex(g.n_v, g.edges, q, order=list(range(g.n_v))[::-1])
            assert rel_err(z2, z1) < 1e-10
            assert oracle.z_exact(g.n_v, g.edges, q) == oracle.z_exact(
                g.n_v, g.edges, q, order=list(range(g.n_v)))


def test_complex_matches_exact_midsize():
    for pd in _grid_knots(6, 22, 700):
        g = oracle.tait_graph(pd)
        for q in (2, 3, 5):
            ze = exact_to_complex(oracle.z_exact(g.n_v, g.edges, q), 1, q)
            assert rel_err(oracle.z_complex(g.n_v, g.edges, q), ze) < 1e-10


def test_scaled_overflow_range():
    """Z of T(2,601) at q=6 leaves double range; the scaled form still matches the
    closed form: the Tait graph here is a 601-cycle with all signs +, so
    Z = (q-1-t^-1)^601 + (q-1)(-1-t^-1)^601 (eigenvalues of J - (1+t^-1) I)."""
    pd = kg.braid_closure_pd(kg.torus_braid(2, 601), 2)
    g = oracle.tait_graph(pd, black=0)
    if g.n_v == 2:
        g = oracle.tait_graph(pd, black=1)
    assert g.n_v == 601 and all(e[2] == 1 for e in g.edges)
    q = 6
    t = t_of_q(q)
    lam1 = SC.of(q - 1 - 1 / t)
    lam2 = SC.of(-1 - 1 / t)
    want = lam1.pow(601) + SC.of(q - 1) * lam2.pow(601)
    got = oracle.z_complex(g.n_v, g.edges, q)
    assert got.log2abs() > 1100
    assert rel_err(got, want) < 1e-10


def _is_power_of_3(n):
    if n < 1:
        return False
    while n % 3 == 0:
        n //= 3
    return n == 1


def test_q3_modulus_is_power_of_three():
    """At q = 3, t = e^(i pi/3) and V = +- i^c (i sqrt 3)^d for every knot (Lickorish and
    Millett: d is the Z_3-rank of the homology of the double branched cover), so
    |V|^2 = a^2 + a b + b^2 (V = a + b t exactly, t + conj(t) = 1) is a power of 3."""
    for pd in _grid_knots(12, 18, 800) + [TREFOIL, FIG8]:
        a, b = v_exact_as_ring(pd, 3)
        assert _is_power_of_3(a * a + a * b + b * b), (a, b)
    a, b = v_exact_as_ring(TREFOIL, 3)
    assert a * a + a * b + b * b == 3     # i sqrt 3 (Fig. 1 caption)


# ----------------------------------------------------------------------------- min-fill orders and one-call buckets

@pytest.mark.parametrize("q", [2, 3, 5])
def test_sum_inside_matches_bruteforce(q):
    """The one-einsum bucket step (product and sum over the eliminated spin in one
    library call) against the literal spin sum, on random graphs with loops and parallel
    edges, under the default order and under min-fill orders."""
    from oracle.order import min_fill_order
    rng = random.Random(2000 + q)
    for trial in range(12):
        n_v = rng.randint(1, 6 if q <= 3 else 5)
        edges = _random_signed_graph(rng, n_v, rng.randint(0, 9))
        zb = z_bruteforce(n_v, edges, q)
        order, _ = min_fill_order(n_v, edges, q, seed=trial, restarts=3)
        for o in (None, order):
            zc = oracle.z_complex(n_v, edges, q, order=o, sum_inside=True)
            assert rel_err(zc, SC.of(zb)) < 1e-12 or abs(zb) < 1e-12


def test_min_fill_order_is_a_narrow_permutation():
    """min_fill_order returns every spin once; summing in that order gives the exact Z
    (Z[t], the default elimination) and the torus-knot closed form; and its largest
    factor is never wider than the default min-degree order's."""
    from oracle.order import min_fill_order
    for pd in _grid_knots(6, 22, 700):
        g = oracle.tait_graph(pd)
        order, w = min_fill_order(g.n_v, g.edges, 3, seed=1, restarts=4)
        assert sorted(order) == list(range(g.n_v))
        _, wd = oracle.z_complex(g.n_v, g.edges, 3, return_width=True)
        _, wm = oracle.z_complex(g.n_v, g.edges, 3, order=order, return_width=True, sum_inside=True)
        assert wm == w and w <= wd
        for q in (2, 3, 5):
            ze = exact_to_complex(oracle.z_exact(g.n_v, g.edges, q), 1, q)
            assert rel_err(oracle.z_complex(g.n_v, g.edges, q, order=order, sum_inside=True), ze) < 1e-10
    pd = kg.braid_closure_pd(kg.torus_braid(2, 9), 2)
    g = oracle.tait_graph(pd)
    order, _ = min_fill_order(g.n_v, g.edges, 5)
    v = oracle.jones_from_z(oracle.z_complex(g.n_v, g.edges, 5, order=order, sum_inside=True), g, 5)
    want = exact_to_complex(exact_value(torus_jones(2, 9), 5), 1, 5)
    assert rel_err(v, want) < 1e-9
