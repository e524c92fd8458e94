"""Jones polynomial from the Kauffman bracket state sum of a PD code.

Independent of the Tait graph and of the Potts model: it pins them.  (The paper
uses the Jones polynomial as a knot invariant in Sec. I; the bracket is the
textbook state-sum definition of it.)

* A smoothing state S picks, at every crossing (a, b, c, d), either the
  A-smoothing or the B-smoothing.  The A-regions of a crossing are the two
  corners swept when the over-strand (b-d) is turned counter-clockwise: the
  corners (b, c) and (d, a); the A-smoothing opens them into one region, so it
  joins arc ends a-b and c-d.  The B-smoothing joins a-d and b-c.
* <K> = sum_S A^{#A(S) - #B(S)} d^{|S| - 1},  d = -A^2 - A^-2, |S| = loops of S.
* V(t) = (-A^3)^{-w} <K> with t = A^-4 (w = writhe, right-hand rule).
Returned as {power of t: integer coefficient}; for a link the powers are multiples of
1/2 (Fraction keys).  The bracket needs no orientation; the writhe does: a knot's PD
labels give it, a link passes the twist signs of its crossings.
"""
from __future__ import annotations

from collections import Counter, defaultdict
from fractions import Fraction


def _writhe(pd):
    two_n = 2 * len(pd)
    w = 0
    for (a, b, c, d) in pd:
        via_b = (b == a) if two_n == 2 else (b == (d + 1) % two_n)
        w += 1 if via_b else -1
    return w


def _poly_mul(p, r):
    out = defaultdict(int)
    for i, x in p.items():
        for j, y in r.items():
            out[i + j] += x * y
    return {k: v for k, v in out.items() if v}


def bracket(pd):
    """<K> as {power of A: coefficient}."""
    n = len(pd)
    if n == 0:
        return {0: 1}
    if n > 22:
        raise ValueError("state sum limited to 22 crossings")
    two_n = 2 * n
    hist = Counter()
    for mask in range(1 << n):
        parent = list(range(two_n))

        def find(u):
            while parent[u] != u:
                parent[u] = parent[parent[u]]
                u = parent[u]
            return u

        loops = two_n
        for k, (a, b, c, d) in enumerate(pd):
            pairs = ((a, b), (c, d)) if (mask >> k) & 1 else ((a, d), (b, c))
            for x, y in pairs:
                rx, ry = find(x), find(y)
                if rx != ry:
                    parent[rx] = ry
                    loops -= 1
        na = bin(mask).count("1")
        hist[(na - (n - na), loops)] += 1
    d = {2: -1, -2: -1}
    dpow = {0: {0: 1}}
    out = defaultdict(int)
    for (ab, loops), cnt in hist.items():
        k = loops - 1
        while k not in dpow:
            m = max(dpow)
            dpow[m + 1] = _poly_mul(dpow[m], d)
        for e, cf in dpow[k].items():
            out[ab + e] += cnt * cf
    return {k: v for k, v in out.items() if v}


def jones_poly(pd, signs=None):
    """V(t) as {power of t: coefficient} from the bracket (integer powers for a knot,
    multiples of 1/2 as Fractions for a link given with its crossing signs)."""
    w = _writhe(pd) if signs is None else sum(signs)
    br = bracket(pd)
    sign = -1 if w % 2 else 1
    out = {}
    for e, c in br.items():
        ea = e - 3 * w             # (-A^3)^-w = (-1)^w A^-3w
        if signs is None and ea % 4:
            raise ValueError("not a knot: A-exponent not divisible by 4")
        if ea % 2:
            raise ValueError("A-exponent of a link bracket must be even")
        p = Fraction(-ea, 4)
        key = int(p) if p.denominator == 1 else p
        out[key] = out.get(key, 0) + sign * c
    return {k: v for k, v in out.items() if v}
