"""Spin elimination orders for the oracle's `elim` (test infrastructure).

The value of Z does not depend on the order in which spins are summed out (the sum
over all spin states is distributed over the product, Sec. II); only the size of the
intermediate factors does.  The plain min-degree order of `elim` makes factors far wider
than needed on knots of a few hundred crossings, so the oracle can also take an order
from the textbook min-fill heuristic: repeatedly sum out the spin whose neighbours in
the interaction graph (spins sharing a factor with it) miss the fewest edges among
themselves, ties broken by a seeded random draw, and keep the best of several draws by
(largest factor, total entries).  Nothing here is shared with the library's planner.
"""
from __future__ import annotations

import random


def _fill(adj, v):
    """Pairs of v's neighbours that are not yet adjacent."""
    nb = list(adj[v])
    f = 0
    for i in range(len(nb)):
        ai = adj[nb[i]]
        for j in range(i + 1, len(nb)):
            if nb[j] not in ai:
                f += 1
    return f


def _one_order(n_v, pairs, rng, q):
    adj = {v: set() for v in range(n_v)}
    for u, v in pairs:
        adj[u].add(v)
        adj[v].add(u)
    fill = {v: _fill(adj, v) for v in range(n_v)}
    order, width, cost = [], 0, 0
    while adj:
        best = min(fill.values())
        cands = [v for v, f in fill.items() if f == best]
        v = cands[rng.randrange(len(cands))] if len(cands) > 1 else cands[0]
        nb = adj.pop(v)
        del fill[v]
        width = max(width, len(nb) + 1)
        cost += q ** (len(nb) + 1)
        touched = set(nb)
        for u in nb:
            adj[u].discard(v)
            new = nb - adj[u] - {u}
            adj[u] |= new
            touched |= adj[u]
        for u in touched:
            if u in adj:
                fill[u] = _fill(adj, u)
        order.append(v)
    return order, width, cost


def min_fill_order(n_v, edges, q=2, seed=0, restarts=8):
    """An elimination order of the spins 0..n_v-1 for the signed graph `edges` ((u, v,
    eps) triples; loops ignored): best of `restarts` seeded min-fill draws by (largest
    number of spins in one factor, sum of q^spins over the eliminations).  Returns
    (order, width)."""
    pairs = {(min(u, v), max(u, v)) for (u, v, _) in edges if u != v}
    rng = random.Random(seed)
    best = None
    for _ in range(max(1, restarts)):
        order, width, cost = _one_order(n_v, sorted(pairs), rng, q)
        if best is None or (width, cost) < (best[1], best[2]):
            best = (order, width, cost)
    return best[0], best[1]
