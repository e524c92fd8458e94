"""Z(q) = sum_sigma prod_edges T[sigma_u, sigma_v] by summing out one spin at a time.

This is the plain definition of Sec. II with the sum distributed over the product:
collect every factor that depends on spin v, multiply them (numpy broadcasting),
sum over sigma_v, and put the resulting factor back.  The order is min-degree
(eliminate the spin whose new factor has the fewest spins; ties -> smallest id).
Factors are edges' q x q clause matrices, loops' diagonals and, for every vertex,
a constant all-ones vector (so an isolated vertex contributes q).

Two arithmetics:
* `z_complex`: complex128 with a separate power-of-two exponent per factor
  (renormalised after every elimination), returned as a scaled complex `SC`.
* `z_exact`:   exact in Z[t] with Python integers (object arrays holding the two
  coordinates a, b of a + b t), using t^2 = (q-2) t - 1.
"""
from __future__ import annotations

import math

import numpy as np

from .potts import clause_diag
from .scaled import SC


def _index_scopes(n_v, scopes):
    """Live factor scopes and, per spin, the factors that contain it."""
    alive = {i: set(s) for i, s in enumerate(scopes)}
    var_facs = {v: set() for v in range(n_v)}
    for i, s in alive.items():
        for v in s:
            var_facs[v].add(i)
    return alive, var_facs


def _expand(arr, vars_, U):
    """View of `arr` (axes in vars_ order) broadcastable against axes U."""
    present = [u for u in U if u in vars_]
    a = np.transpose(arr, [vars_.index(u) for u in present])
    return a.reshape([a.shape[present.index(u)] if u in vars_ else 1 for u in U])


def _eliminate(n_v, factors, multiply, sum_axis, normalise, max_width=None, order=None,
               bucket=None):
    """Generic bucket elimination; `factors` is a list of (vars tuple, payload).  With
    `bucket` (a callable taking the bucket's [(payload, vars)] and the kept spins) the
    product of the bucket's factors and the sum over the eliminated spin are one call."""
    scopes = [tuple(v) for v, _ in factors]
    payloads = [p for _, p in factors]
    alive, var_facs = _index_scopes(n_v, scopes)
    remaining = set(range(n_v))
    width = 0
    forced = list(order) if order is not None else None
    while remaining:
        if forced:
            v = forced.pop(0)
        else:
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
        U = sorted(set().union(*[alive[i] for i in idx])) if idx else [v]
        width = max(width, len(U))
        if max_width is not None and len(U) > max_width:
            raise MemoryError(f"elimination width {len(U)} exceeds {max_width}")
        newscope = tuple(u for u in U if u != v)
        if bucket is not None and idx:
            newp = bucket([(payloads[i], list(scopes[i])) for i in idx], list(newscope))
        else:
            prod = None
            for i in idx:
                term = (payloads[i], list(scopes[i]), U)
                prod = multiply(prod, term)
            newp = sum_axis(prod, U.index(v))
        newp = normalise(newp)
        for i in idx:
            for u in alive[i]:
                var_facs[u].discard(i)
            del alive[i]
        nid = len(scopes)
        scopes.append(newscope)
        payloads.append(newp)
        alive[nid] = set(newscope)
        for u in newscope:
            var_facs[u].add(nid)
        remaining.discard(v)
    # all remaining factors are scalars
    result = None
    for i in alive:
        result = multiply(result, (payloads[i], [], []))
    return result, width


def z_complex(n_v, edges, q, max_width=None, order=None, return_width=False, sum_inside=False):
    """Z(q) in complex128 with per-factor power-of-two exponents -> SC.

    sum_inside=True forms each bucket's new factor sum_{sigma_v} prod_i f_i with one
    numpy einsum call (a library contraction routine) instead of materialising the
    product over all the bucket's spins first: the same sum, with arrays q times smaller,
    so that knots of a few hundred crossings (with an order from `order.min_fill_order`)
    stay within the host's memory."""
    diag = {+1: clause_diag(q, +1), -1: clause_diag(q, -1)}
    factors = []
    for (u, v, eps) in edges:
        if u == v:
            f = np.full(q, diag[eps], dtype=np.complex128)
            factors.append(((u,), (f, 0)))
        else:
            f = np.ones((q, q), dtype=np.complex128)
            f[np.diag_indices(q)] = diag[eps]
            factors.append(((u, v), (f, 0)))
    for v in range(n_v):
        factors.append(((v,), (np.ones(q, dtype=np.complex128), 0)))

    def multiply(acc, term):
        (arr, e), vars_, U = term
        x = _expand(arr, vars_, U) if vars_ else arr
        if acc is None:
            return (x, e)
        return (acc[0] * x, acc[1] + e)

    def sum_axis(p, ax):
        arr, e = p
        return (np.asarray(arr.sum(axis=ax)), e)

    def normalise(p):
        arr, e = p
        m = float(np.max(np.abs(arr))) if arr.size else 0.0
        if m == 0.0 or not math.isfinite(m):
            return (arr, e)
        _, k = math.frexp(m)
        return (arr * (2.0 ** -k), e + k)

    def bucket(terms, keep):
        label = {}   # einsum labels are small integers: number the bucket's spins
        for _, vars_ in terms:
            for u in vars_:
                label.setdefault(u, len(label))
        ops = []
        for (arr, _), vars_ in terms:
            ops += [arr, [label[u] for u in vars_]]
        e = sum(ex for (_, ex), _ in terms)
        out = np.einsum(*ops, [label[u] for u in keep], optimize="greedy")
        return (np.asarray(out, dtype=np.complex128), e)

    res, width = _eliminate(n_v, factors, multiply, sum_axis, normalise, max_width, order,
                            bucket if sum_inside else None)
    arr, e = res
    z = SC.of(complex(np.asarray(arr).reshape(())), e)
    return (z, width) if return_width else z


def z_exact(n_v, edges, q, max_width=None, order=None):
    """Z(q) exactly as (a, b) with Z = a + b t(q), a and b Python integers."""
    c = q - 2
    dg = {+1: (-(q - 2), 1), -1: (0, -1)}   # -t^-1 = t - (q-2);  -t
    factors = []

    def obj(shape, val):
        a = np.empty(shape, dtype=object)
        a.fill(val)
        return a

    for (u, v, eps) in edges:
        if u == v:
            factors.append(((u,), (obj(q, dg[eps][0]), obj(q, dg[eps][1]))))
        else:
            A = obj((q, q), 1)
            B = obj((q, q), 0)
            for s in range(q):
                A[s, s] = dg[eps][0]
                B[s, s] = dg[eps][1]
            factors.append(((u, v), (A, B)))
    for v in range(n_v):
        factors.append(((v,), (obj(q, 1), obj(q, 0))))

    def multiply(acc, term):
        (A, B), vars_, U = term
        if vars_:
            A, B = _expand(A, vars_, U), _expand(B, vars_, U)
        if acc is None:
            return (A, B)
        C, D = acc
        return (C * A - D * B, C * B + D * A + c * (D * B))

    def sum_axis(p, ax):
        A, B = p
        return (np.asarray(A.sum(axis=ax), dtype=object), np.asarray(B.sum(axis=ax), dtype=object))

    res, _ = _eliminate(n_v, factors, multiply, sum_axis, lambda p: p, max_width, order)
    A, B = res
    return (int(np.asarray(A).reshape(())), int(np.asarray(B).reshape(())))
