"""Pins for the oracle's reverse pass (oracle/grad.py), each independent of its code path:

* the literal definition dZ/dT_e[a, b] = sum over spin states with s_u = a, s_v = b of
  the product of every other edge's entry, summed by brute force on tiny graphs (with
  loops, parallel edges and general complex weights);
* central finite differences of the forward sweep along random directions of the edge
  weights, and of V(t) along t;
* identities that hold for every graph: Z is linear in each T_e (so
  sum_ab T_e[a,b] dlogZ/dT_e[a,b] = 1), the colour-permutation symmetry of the weights
  (equal diagonal entries, equal off-diagonal entries, and every single-spin marginal
  equal to 1/q).
"""
import cmath
import itertools
import math
import random

import numpy as np
import pytest

import knotgen as kg
import oracle
from oracle.grad import (dlogv_dt, dlogz, jones_weights, prefactor_at, standard_weights,
                         z_and_adjoints, z_weighted)
from oracle.potts import t_of_q


def _entry(w, a, b):
    d, o = w
    return complex(d) if a == b else complex(o)


def _brute_dz(n_v, edges, q, weights, e, a, b):
    """sum over states with s_u = a, s_v = b of prod_{e' != e} T_e'[s_u', s_v']."""
    u, v, _ = edges[e]
    tot = 0j
    for sig in itertools.product(range(q), repeat=n_v):
        if sig[u] != a or sig[v] != b:
            continue
        p = 1 + 0j
        for k, ((x, y, _), w) in enumerate(zip(edges, weights)):
            if k != e:
                p *= _entry(w, sig[x], sig[y])
        tot += p
    return tot


def _random_graph(rng, n_v, n_e):
    edges = []
    for _ in range(n_e):
        u, v = rng.randrange(n_v), rng.randrange(n_v)
        edges.append((u, v, rng.choice((1, -1))))
    # a parallel pair and a loop for sure
    edges.append(edges[0][:2] + (-edges[0][2],))
    edges.append((0, 0, 1))
    return edges


@pytest.mark.parametrize("q", [2, 3, 4])
def test_adjoints_match_bruteforce_definition(q):
    rng = random.Random(500 + q)
    for trial in range(6):
        n_v = rng.randint(2, 5 if q <= 3 else 4)
        edges = _random_graph(rng, n_v, rng.randint(1, 6))
        if trial % 2:
            weights = [(complex(rng.uniform(-2, 2), rng.uniform(-2, 2)),
                        complex(rng.uniform(-2, 2), rng.uniform(-2, 2))) for _ in edges]
        else:
            weights = standard_weights(edges, q)
        z, adj = z_and_adjoints(n_v, edges, q, weights)
        for e, ((u, v, _), (arr, ex)) in enumerate(zip(edges, adj)):
            for a in range(q):
                for b in range(q):
                    if u == v and a != b:
                        continue
                    want = _brute_dz(n_v, edges, q, weights, e, a, b)
                    got = (arr[a] if u == v else arr[a, b]) * 2.0 ** ex
                    assert abs(got - want) <= 1e-12 * max(1.0, abs(want)), (trial, e, a, b)


def _dlog(zp, zm):
    """log(zp / zm) on the principal branch of the ratio (near 1), so the branch cut of
    log never falls between the two points."""
    return cmath.log(zp.m / zm.m) + (zp.e - zm.e) * math.log(2.0)


@pytest.mark.parametrize("q", [2, 3, 5])
def test_adjoints_match_finite_differences(q):
    """Directional derivative along a random complex direction of all (d, o) weights
    against central differences of log Z with h = 1e-6."""
    rng = np.random.default_rng(q)
    h = 1e-6
    for seed in range(3):
        gk = kg.random_grid_knot(12, 900 + seed, True, 12, 30)
        g = oracle.tait_graph(gk.pd, outer=gk.outer)
        w0 = standard_weights(g.edges, q)
        dirs = rng.standard_normal((len(g.edges), 2)) + 1j * rng.standard_normal((len(g.edges), 2))
        _, d = dlogz(g.n_v, g.edges, q, w0)
        eye = np.eye(q, dtype=bool)
        lin = 0j
        for k, (u, v, _) in enumerate(g.edges):
            lin += dirs[k, 0] * d[k][eye].sum()
            if u != v:
                lin += dirs[k, 1] * d[k][~eye].sum()
        wp = [(a + h * dd[0], b + h * dd[1]) for (a, b), dd in zip(w0, dirs)]
        wm = [(a - h * dd[0], b - h * dd[1]) for (a, b), dd in zip(w0, dirs)]
        fd = _dlog(z_weighted(g.n_v, g.edges, q, wp), z_weighted(g.n_v, g.edges, q, wm)) / (2 * h)
        assert abs(fd - lin) <= 1e-6 * max(1.0, abs(lin)), (seed, fd, lin)


def test_adjoint_identities():
    for seed in range(8):
        gk = kg.random_grid_knot(14, 700 + seed, True, 15, 40)
        g = oracle.tait_graph(gk.pd, outer=gk.outer)
        for q in (2, 3, 5, 6):
            w = standard_weights(g.edges, q)
            _, d = dlogz(g.n_v, g.edges, q, w)
            for k, ((u, v, _), (dg, off)) in enumerate(zip(g.edges, w)):
                T = np.full((q, q), off, dtype=np.complex128)
                T[np.diag_indices(q)] = dg
                if u == v:
                    assert abs(np.sum(np.diag(d[k]) * dg) - 1) < 1e-9
                    continue
                P = T * d[k]          # joint distribution of (s_u, s_v)
                assert abs(P.sum() - 1) < 1e-9
                assert np.allclose(P.sum(axis=1), 1.0 / q, atol=1e-9)
                assert np.allclose(P.sum(axis=0), 1.0 / q, atol=1e-9)
                assert np.allclose(np.diag(d[k]), d[k][0, 0], atol=1e-9 * abs(d[k]).max())
                offd = d[k][~np.eye(q, dtype=bool)]
                assert np.allclose(offd, offd[0], atol=1e-9 * abs(d[k]).max())


@pytest.mark.parametrize("q", [2, 3, 5])
def test_dlogv_dt_matches_finite_differences(q):
    h = 1e-6
    for seed in range(3):
        gk = kg.random_grid_knot(12, 800 + seed, True, 10, 25)
        g = oracle.tait_graph(gk.pd, outer=gk.outer)
        t = t_of_q(q)

        def vat(tt):
            z = z_weighted(g.n_v, g.edges, q, jones_weights(g.edges, q, tt))
            return prefactor_at(tt, g.n_v, g.writhe, g.tau) * z

        # at t(q) itself the forward is the oracle's V
        v = prefactor_at(t, g.n_v, g.writhe, g.tau) * z_weighted(
            g.n_v, g.edges, q, jones_weights(g.edges, q, t))
        vo = oracle.jones(gk.pd, q, outer=gk.outer)
        assert abs(v.m * 2.0 ** (v.e - vo.e) - vo.m) < 1e-10
        fd = _dlog(vat(t + h), vat(t - h)) / (2 * h)
        an = dlogv_dt(g.n_v, g.edges, q, g.writhe, g.tau)
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (seed, fd, an)
