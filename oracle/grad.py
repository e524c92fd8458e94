"""Derivatives of Z over the edge weights: a complex128 reverse pass (test infrastructure).

Z = sum_sigma prod_e T_e[sigma_u, sigma_v] (Sec. II) is linear in every entry of every
clause matrix, and dZ/dT_e[a, b] is the same spin sum with the factor T_e left out and
sigma_u = a, sigma_v = b held fixed.  Here every edge is its own factor (parallel edges
are not merged, a loop is a vector over its vertex's spin holding T_e[s, s]) and the
weights may be general: T_e = o_e everywhere off the diagonal and d_e on it; the Jones
weights of Eq. clause are d_e = -t^-eps_e, o_e = 1.

Forward: the spin elimination of `elim.py` (min-degree order, numpy broadcasting, a
power-of-two exponent per factor), with every elimination recorded.  Backward: for an
elimination g = sum_v prod_i F_i, the adjoint of each factor is
    dZ/dF_i = sum over the spins of the elimination that F_i does not hold of
              (dZ/dg, constant along v) * prod_{j != i} F_j,
and the adjoint of each scalar left at the end is the product of the others.  Every
factor enters exactly one elimination, so no adjoint needs accumulating.
"""
from __future__ import annotations

import cmath
import math

import numpy as np

from .elim import _expand
from .potts import clause_diag, t_of_q
from .scaled import SC


def standard_weights(edges, q):
    """(d, o) per edge for the Jones weights: d = -t^-eps, o = 1."""
    return [(clause_diag(q, eps), 1.0 + 0j) for (_, _, eps) in edges]


def _normalise(arr, e):
    m = float(np.max(np.abs(arr))) if arr.size else 0.0
    if m == 0.0 or not math.isfinite(m):
        return arr, e
    _, k = math.frexp(m)
    return arr * (2.0 ** -k), e + k


def _factors(n_v, edges, q, weights):
    facs = []
    for (u, v, _), (d, o) in zip(edges, weights):
        if u == v:
            facs.append(((u,), np.full(q, complex(d), dtype=np.complex128), 0))
        else:
            f = np.full((q, q), complex(o), dtype=np.complex128)
            f[np.diag_indices(q)] = complex(d)
            facs.append(((u, v), f, 0))
    for v in range(n_v):
        facs.append(((v,), np.ones(q, dtype=np.complex128), 0))
    return facs


def z_and_adjoints(n_v, edges, q, weights=None):
    """Z as SC and, per edge, dZ/dT_e as (array, exp): a (q, q) array over (s_u, s_v),
    or a (q,) array of the diagonal entries for a loop."""
    if weights is None:
        weights = standard_weights(edges, q)
    facs = _factors(n_v, edges, q, weights)
    scopes = [s for s, _, _ in facs]
    vals = [(a, e) for _, a, e in facs]
    alive = {i: set(s) for i, s in enumerate(scopes)}
    var_facs = {v: set() for v in range(n_v)}
    for i, s in alive.items():
        for v in s:
            var_facs[v].add(i)
    tape = []
    remaining = set(range(n_v))
    while remaining:
        best = None
        for u in sorted(remaining):
            nb = set()
            for i in var_facs[u]:
                nb |= alive[i]
            nb.discard(u)
            key = (len(nb), u)
            if best is None or key < best[0]:
                best = (key, u)
        v = best[1]
        idx = sorted(var_facs[v])
        U = sorted(set().union(*[alive[i] for i in idx]))
        prod, e = None, 0
        for i in idx:
            x = _expand(vals[i][0], list(scopes[i]), U)
            prod = x if prod is None else prod * x
            e += vals[i][1]
        prod = np.broadcast_to(prod, [q] * len(U))
        new = np.asarray(prod.sum(axis=U.index(v)))
        new, e = _normalise(new, e)
        nid = len(scopes)
        scopes.append(tuple(u for u in U if u != v))
        vals.append((new, e))
        for i in idx:
            for u in alive[i]:
                var_facs[u].discard(i)
            del alive[i]
        alive[nid] = set(scopes[nid])
        for u in scopes[nid]:
            var_facs[u].add(nid)
        remaining.discard(v)
        tape.append((v, idx, U, nid))
    # scalars left at the end: Z is their product
    rest = sorted(alive)
    z = SC.of(1.0)
    for i in rest:
        z = z * SC.of(complex(np.asarray(vals[i][0]).reshape(())), vals[i][1])
    adj = {}
    for i in rest:
        a = SC.of(1.0)
        for j in rest:
            if j != i:
                a = a * SC.of(complex(np.asarray(vals[j][0]).reshape(())), vals[j][1])
        adj[i] = (np.asarray(a.m), a.e)
    for (v, idx, U, nid) in reversed(tape):
        gbar, ge = adj.pop(nid)
        g = np.expand_dims(gbar, U.index(v))
        for i in idx:
            term, e = g, ge
            for j in idx:
                if j != i:
                    term = term * _expand(vals[j][0], list(scopes[j]), U)
                    e += vals[j][1]
            term = np.broadcast_to(term, [q] * len(U))
            keep = [U.index(x) for x in scopes[i]]
            drop = tuple(ax for ax in range(len(U)) if ax not in keep)
            r = term.sum(axis=drop) if drop else np.array(term)
            # the kept axes are in U order; put them in the factor's scope order
            kept_sorted = sorted(keep)
            r = np.transpose(r, [kept_sorted.index(k) for k in keep])
            adj[i] = _normalise(np.asarray(r), e)
    return z, [adj[e] for e in range(len(edges))]


def dlogz(n_v, edges, q, weights=None):
    """(1/Z) dZ/dT_e[a, b] for every edge, complex128 array (n_e, q, q); loops fill the
    diagonal only.  Returns (Z, array)."""
    z, ad = z_and_adjoints(n_v, edges, q, weights)
    out = np.zeros((len(edges), q, q), dtype=np.complex128)
    for k, ((u, v, _), (arr, e)) in enumerate(zip(edges, ad)):
        scale = math.ldexp(1.0, max(-2000, min(2000, e - z.e))) / z.m
        if u == v:
            out[k][np.diag_indices(q)] = arr * scale
        else:
            out[k] = arr * scale
    return z, out


def z_weighted(n_v, edges, q, weights):
    """Z for general per-edge (d, o) weights (the forward sweep of z_and_adjoints)."""
    return z_and_adjoints(n_v, edges, q, weights)[0]


def jones_weights(edges, q, t):
    """Clause weights of Eq. clause at a given t (the network's dimension q unchanged)."""
    return [(-(t ** (-eps)), 1.0 + 0j) for (_, _, eps) in edges]


def prefactor_at(t, n_v, writhe, tau) -> SC:
    """A of Eq. JonesPotts at a given t, through the principal fourth root s of t."""
    s = cmath.exp(cmath.log(t) / 4)
    return (SC.of(-(s ** 2) - s ** -2).pow(-n_v - 1) * SC.of(-(s ** 3)).pow(writhe) *
            SC.of(s).pow(tau))


def dlogv_dt(n_v, edges, q, writhe, tau):
    """(1/V) dV/dt at fixed q: the derivative of log A(t) (from its form in s = t^(1/4):
    d log(-s^2 - s^-2)/dt = (t - 1) / (2 t (t + 1)), d log s / dt = 1 / (4 t)) plus the
    chain rule through every clause diagonal d_e = -t^-eps_e (dd_e/dt = eps_e t^(-eps_e-1))."""
    t = t_of_q(q)
    _, d = dlogz(n_v, edges, q)
    r = (-(n_v + 1) * (t - 1) / (2 * t * (t + 1)) + 3 * writhe / (4 * t) + tau / (4 * t))
    for k, (_, _, eps) in enumerate(edges):
        r += eps * t ** (-eps - 1) * np.trace(d[k])
    return complex(r)
