"""Seeded synthetic knot diagrams shared by the oracle, the tests and the benchmark.

This module only *produces inputs*: knot diagrams as planar-diagram (PD) codes.  It
holds none of the method's arithmetic (no Tait graph, no Potts weights, no
contraction); both the CPU oracle and the GPU library consume its PD codes
independently.

PD convention (used everywhere in this repository): arcs are labelled
0 .. 2n-1 consecutively along the knot's orientation, so the arc after arc k is
(k+1) mod 2n.  A crossing is a 4-tuple (a, b, c, d): a is the incoming
under-arc, then b, c, d follow counter-clockwise around the crossing; c is the
outgoing under-arc (c = a+1 mod 2n) and the over-strand runs between b and d.
A link (several components) cannot be labelled along one strand; `braid_closure_link`
labels it component by component and returns the twist sign of every crossing
(+1: the over-strand leaves through b), which fixes the orientation instead.

Random knots follow the random grid walk of Sec. III.A: two random permutations
x, y of 0..L-1 give the closed walk (x_i, y_i) -> (x_i, y_{i+1}) -> (x_{i+1}, y_{i+1});
vertical segments pass over horizontal ones unless the caller asks for a random
over/under choice per crossing.  Randomness comes from SplitMix64 (Steele,
Lea & Flood, OOPSLA 2014), so the C++ generator in the library reproduces the
same diagrams bit for bit.
"""
from __future__ import annotations

from dataclasses import dataclass, field

MASK64 = (1 << 64) - 1

__all__ = [
    "SplitMix64", "GridKnot", "grid_walk_pd", "random_grid_knot", "braid_closure_pd",
    "braid_closure_link",
    "over_out_is_b", "kink", "poke", "mirror", "connected_sum", "randomize",
    "rotate_labels", "torus_braid", "knot_suite",
]


class SplitMix64:
    """SplitMix64 generator (published constants; 64-bit state)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def below(self, n: int) -> int:
        """Integer in [0, n) by the multiply-high map of one 64-bit draw."""
        return (self.next() * n) >> 64

    def bit(self) -> int:
        return self.next() >> 63

    def permutation(self, n: int) -> list[int]:
        """Fisher-Yates shuffle of 0..n-1, swapping from the top down."""
        a = list(range(n))
        for i in range(n - 1, 0, -1):
            j = self.below(i + 1)
            a[i], a[j] = a[j], a[i]
        return a


# --------------------------------------------------------------------------- grid walk

def _grid_crossings(xs, ys):
    """Crossings (i, j) of vertical segment V_i with horizontal segment H_j, in
    lexicographic (i, j) order."""
    import numpy as np
    x = np.asarray(xs)
    y = np.asarray(ys)
    xn, yn = np.roll(x, -1), np.roll(y, -1)
    ylo, yhi = np.minimum(y, yn), np.maximum(y, yn)        # V_i spans y_i .. y_{i+1}
    xlo, xhi = np.minimum(x, xn), np.maximum(x, xn)        # H_j spans x_j .. x_{j+1} at y_{j+1}
    hit = ((xlo[None, :] < x[:, None]) & (x[:, None] < xhi[None, :]) &
           (ylo[:, None] < yn[None, :]) & (yn[None, :] < yhi[:, None]))
    ii, jj = np.nonzero(hit)                                 # row-major: sorted by (i, j)
    return [(int(i), int(j)) for i, j in zip(ii, jj)]


def grid_walk_pd(xs, ys, over_bits=None):
    """PD code of the grid walk given by permutations xs, ys (Sec. III.A).

    over_bits[c] = 1 keeps the vertical strand over at crossing c (crossings in
    lexicographic (i, j) order), 0 puts the horizontal strand over; None means
    vertical always over, as in the paper.  Returns (pd, outer) where outer is
    (arc, side) naming a side (0 = left, 1 = right) of an arc that borders the
    unbounded region, or None for a crossingless walk.
    """
    L = len(xs)
    cr = _grid_crossings(xs, ys)
    n = len(cr)
    if n == 0:
        return [], None
    # events along the curve: segment order V_0, H_0, V_1, H_1, ...
    ev = []  # (segment, distance, crossing, is_vertical)
    for c, (i, j) in enumerate(cr):
        ev.append((2 * i, abs(ys[(j + 1) % L] - ys[i]), c, True))
        ev.append((2 * j + 1, abs(xs[i] - xs[j]), c, False))
    ev.sort()
    vpos = [0] * n
    hpos = [0] * n
    for m, (_, _, c, isv) in enumerate(ev):
        if isv:
            vpos[c] = m
        else:
            hpos[c] = m
    two_n = 2 * n
    pd = []
    for c, (i, j) in enumerate(cr):
        dv = (0, 1 if ys[(i + 1) % L] > ys[i] else -1)
        dh = (1 if xs[(j + 1) % L] > xs[j] else -1, 0)
        v_in, v_out = (vpos[c] - 1) % two_n, vpos[c]
        h_in, h_out = (hpos[c] - 1) % two_n, hpos[c]
        vert_over = True if over_bits is None else bool(over_bits[c])
        if vert_over:
            du, do = dh, dv
            a, cc, o_in, o_out = h_in, h_out, v_in, v_out
        else:
            du, do = dv, dh
            a, cc, o_in, o_out = v_in, v_out, h_in, h_out
        # arm counter-clockwise after the incoming-under arm points along R(-du)
        east_of_a = (du[1], -du[0])
        if do == east_of_a:
            pd.append((a, o_out, cc, o_in))
        else:
            pd.append((a, o_in, cc, o_out))
    # unbounded region: west of the vertical segment at x = 0
    i0 = xs.index(0)
    ymid_seg = 2 * i0
    half = abs(ys[(i0 + 1) % L] - ys[i0]) / 2.0
    key = (ymid_seg, half)
    m_last = -1
    for m, e in enumerate(ev):
        if (e[0], e[1]) <= key:
            m_last = m
    arc = m_last % two_n
    north = ys[(i0 + 1) % L] > ys[i0]
    side = 0 if north else 1
    return pd, (arc, side)


@dataclass
class GridKnot:
    L: int
    seed: int
    xs: list
    ys: list
    over_bits: list | None
    pd: list
    outer: tuple | None
    draws: int = 1
    extra: dict = field(default_factory=dict)

    @property
    def n_crossings(self):
        return len(self.pd)


def random_grid_knot(L: int, seed: int, random_over_under: bool = False,
                     ncross_min: int = 0, ncross_max: int = 1 << 30,
                     max_draws: int = 200000) -> GridKnot:
    """Random grid-walk knot; redraws from the same seeded stream until the raw
    crossing count lies in [ncross_min, ncross_max].  Each draw takes the x
    permutation, then the y permutation, then (only for an accepted draw with
    random_over_under) one bit per crossing."""
    rng = SplitMix64(seed)
    for d in range(1, max_draws + 1):
        xs = rng.permutation(L)
        ys = rng.permutation(L)
        n = len(_grid_crossings(xs, ys))
        if ncross_min <= n <= ncross_max:
            bits = [rng.bit() for _ in range(n)] if random_over_under else None
            pd, outer = grid_walk_pd(xs, ys, bits)
            return GridKnot(L, seed, xs, ys, bits, pd, outer, d)
    raise RuntimeError(f"no grid walk with {ncross_min}..{ncross_max} crossings "
                       f"after {max_draws} draws (L={L}, seed={seed})")


# --------------------------------------------------------------------------- braids

def braid_closure_pd(word, n_strands: int):
    """PD code of the closure of a braid word (+i = sigma_i: strand i passes over
    strand i+1, strands running upward; -i = its inverse).  Raises ValueError if
    the closure has more than one component."""
    parent = {}

    def find(u):
        while parent[u] != u:
            parent[u] = parent[parent[u]]
            u = parent[u]
        return u

    ids = [0]

    def new():
        k = ids[0]
        ids[0] += 1
        parent[k] = k
        return k

    cur = [new() for _ in range(n_strands)]
    start = list(cur)
    raw = []
    for g in word:
        i = abs(g) - 1
        if not (0 <= i < n_strands - 1):
            raise ValueError("generator out of range")
        in_l, in_r = cur[i], cur[i + 1]
        o1, o2 = new(), new()  # o1: left strand, now at i+1; o2: right strand, now at i
        if g > 0:
            raw.append((in_r, o1, o2, in_l))
        else:
            raw.append((in_l, in_r, o1, o2))
        cur[i], cur[i + 1] = o2, o1
    for p in range(n_strands):
        ra, rb = find(cur[p]), find(start[p])
        if ra != rb:
            parent[ra] = rb
    if not raw:
        if n_strands != 1:
            raise ValueError("crossingless closure of several strands is a link")
        return []
    raw = [tuple(find(u) for u in x) for x in raw]
    nxt = {}
    for (a, b, c, d) in raw:
        nxt[a] = c
        # over strand: in -> out, orientation from the braid (upward)
    # over strand direction: for sigma_i (+) over goes in_l -> o1 = d -> b;
    # for sigma_i^-1 over goes in_r -> o2 = b -> d.
    for g, (a, b, c, d) in zip(word, raw):
        if g > 0:
            nxt[d] = b
        else:
            nxt[b] = d
    arcs = set(nxt.keys())
    first = raw[0][0]
    label = {}
    u = first
    k = 0
    while u not in label:
        label[u] = k
        k += 1
        u = nxt[u]
    if len(label) != len(arcs):
        raise ValueError("braid closure is a link, not a knot")
    return [tuple(label[u] for u in x) for x in raw]


def braid_closure_link(word, n_strands: int):
    """Closure of a braid word as a possibly multi-component diagram: (pd, signs,
    components).  Arcs are labelled component by component along the orientation
    (strands running upward); signs[i] = +1 when crossing i is sigma_j (over-strand
    leaving through arm b), -1 for sigma_j^-1.  Every generator sigma_1 ..
    sigma_{n_strands-1} must occur, so that the diagram is connected."""
    if not word:
        raise ValueError("a link diagram needs crossings")
    if sorted({abs(g) for g in word}) != list(range(1, n_strands)):
        raise ValueError("every generator must occur (a split diagram has no Tait graph)")
    parent = {}

    def find(u):
        while parent[u] != u:
            parent[u] = parent[parent[u]]
            u = parent[u]
        return u

    ids = [0]

    def new():
        k = ids[0]
        ids[0] += 1
        parent[k] = k
        return k

    cur = [new() for _ in range(n_strands)]
    start = list(cur)
    raw = []
    for g in word:
        i = abs(g) - 1
        in_l, in_r = cur[i], cur[i + 1]
        o1, o2 = new(), new()   # o1: left strand, now at i+1; o2: right strand, now at i
        raw.append((in_r, o1, o2, in_l) if g > 0 else (in_l, in_r, o1, o2))
        cur[i], cur[i + 1] = o2, o1
    for p in range(n_strands):
        ra, rb = find(cur[p]), find(start[p])
        if ra != rb:
            parent[ra] = rb
    raw = [tuple(find(u) for u in x) for x in raw]
    signs = [1 if g > 0 else -1 for g in word]
    nxt = {}
    for (a, b, c, d), sg in zip(raw, signs):
        nxt[a] = c
        if sg > 0:
            nxt[d] = b
        else:
            nxt[b] = d
    label = {}
    comps = 0
    for x in raw:             # a component may pass only over: start from every arc
        for a in x:
            if a in label:
                continue
            comps += 1
            u = a
            while u not in label:
                label[u] = len(label)
                u = nxt[u]
    if len(label) != len(nxt):
        raise ValueError("inconsistent braid closure")
    return [tuple(label[u] for u in x) for x in raw], signs, comps


def torus_braid(p: int, r: int):
    """Braid word (sigma_1 ... sigma_{p-1})^r whose closure is the torus knot T(p, r)."""
    return list(range(1, p)) * r


# --------------------------------------------------------------------------- PD moves

def over_out_is_b(pd) -> list[bool]:
    """For each crossing, True if the over-strand leaves through arm b."""
    two_n = 2 * len(pd)
    res = []
    for (a, b, c, d) in pd:
        if two_n == 2:
            res.append(b == a)
        else:
            res.append(b == (d + 1) % two_n)
    return res


def _incoming(pd, ob, k, pos):
    if pos == 0:
        return True
    if pos == 2:
        return False
    if pos == 1:
        return not ob[k]
    return ob[k]


def kink(pd, x: int, variant: int):
    """Reidemeister I: add a curl on arc x (variant 0..3 picks over/under of the
    first pass and the side of the loop; variants 0 and 3 add a positive crossing)."""
    n = len(pd)
    two_n2 = 2 * n + 2
    if n == 0:
        x = 0
    ob = over_out_is_b(pd)
    out = []
    for k, X in enumerate(pd):
        Y = []
        for pos, y in enumerate(X):
            if y == x:
                Y.append((x + 2) % two_n2 if _incoming(pd, ob, k, pos) else x)
            elif y > x:
                Y.append(y + 2)
            else:
                Y.append(y)
        out.append(tuple(Y))
    x1, x2 = (x + 1) % two_n2, (x + 2) % two_n2
    new = [(x, x2, x1, x1), (x1, x, x2, x1), (x, x1, x1, x2), (x1, x1, x2, x)][variant]
    out.append(new)
    return out


def poke(pd, k: int, b_over: bool):
    """Reidemeister II: push a finger of arm b of crossing k across arm a through
    their shared corner, over (b_over) or under arc a.  Returns None when the
    corner is not usable (an arm's arc meets crossing k twice)."""
    a, b = pd[k][0], pd[k][1]
    if a == b or list(pd[k]).count(a) != 1 or list(pd[k]).count(b) != 1:
        return None
    ob = over_out_is_b(pd)
    b_out = ob[k]
    a1, a2, a3 = 3 * a, 3 * a + 1, 3 * a + 2
    b1, b2, b3 = 3 * b, 3 * b + 1, 3 * b + 2
    out = []
    for kk, X in enumerate(pd):
        Y = []
        for pos, y in enumerate(X):
            if kk == k and pos == 0:
                Y.append(a3)
            elif kk == k and pos == 1:
                Y.append(b1 if b_out else b3)
            elif y == a:
                Y.append(a1)
            elif y == b:
                Y.append(b3 if b_out else b1)
            else:
                Y.append(3 * y)
        out.append(tuple(Y))
    if b_out:
        if b_over:
            out += [(a2, b1, a3, b2), (a1, b3, a2, b2)]
        else:
            out += [(b1, a3, b2, a2), (b2, a1, b3, a2)]
    else:
        if b_over:
            out += [(a1, b1, a2, b2), (a2, b3, a3, b2)]
        else:
            out += [(b1, a2, b2, a1), (b2, a2, b3, a3)]
    keys = sorted({y for X in out for y in X})
    relab = {kk: i for i, kk in enumerate(keys)}
    return [tuple(relab[y] for y in X) for X in out]


def mirror(pd):
    """Mirror image: every crossing switches over and under."""
    ob = over_out_is_b(pd)
    res = []
    for (a, b, c, d), is_b in zip(pd, ob):
        res.append((d, a, b, c) if is_b else (b, c, d, a))
    return res


def rotate_labels(pd, s: int):
    """Shift every arc label by s (moves the base point along the knot)."""
    two_n = 2 * len(pd)
    if two_n == 0:
        return []
    return [tuple((y + s) % two_n for y in X) for X in pd]


def connected_sum(pd1, pd2):
    """Connected sum, cutting both knots on their last arc."""
    if not pd1:
        return list(pd2)
    if not pd2:
        return list(pd1)
    n1, n2 = 2 * len(pd1), 2 * len(pd2)
    ob1, ob2 = over_out_is_b(pd1), over_out_is_b(pd2)
    last1, last2 = n1 - 1, n1 + n2 - 1
    out = []
    for k, X in enumerate(pd1):
        out.append(tuple(last2 if (y == n1 - 1 and _incoming(pd1, ob1, k, p)) else y
                         for p, y in enumerate(X)))
    for k, X in enumerate(pd2):
        out.append(tuple(last1 if (y == n2 - 1 and _incoming(pd2, ob2, k, p)) else y + n1
                         for p, y in enumerate(X)))
    return out


def randomize(pd, rng: SplitMix64, n_moves: int, kinds=("R1", "R2")):
    """Apply n_moves random Reidemeister I / II moves, then a random base-point
    shift and crossing-order shuffle.  The knot type (and so V) is unchanged."""
    cur = list(pd)
    done = 0
    tries = 0
    while done < n_moves and tries < 100 * (n_moves + 1):
        tries += 1
        kind = kinds[rng.below(len(kinds))]
        if kind == "R1" or not cur:
            x = rng.below(max(1, 2 * len(cur)))
            cur = kink(cur, x, rng.below(4))
            done += 1
        else:
            k = rng.below(len(cur))
            res = poke(cur, k, bool(rng.bit()))
            if res is not None:
                cur = res
                done += 1
    if cur:
        cur = rotate_labels(cur, rng.below(2 * len(cur)))
        order = rng.permutation(len(cur))
        cur = [cur[i] for i in order]
    return cur


# --------------------------------------------------------------------------- workloads

def knot_suite(name: str):
    """Named seeded workloads.

    tiny    : L=12, seed 0, redrawn until exactly 16 crossings, random over/under.
    scale   : L=40, seeds 1..64, each redrawn until 100..400 crossings, random over/under.
    batch   : 4096 knots; knot s targets a crossing count t drawn uniformly in 20..120
              from SplitMix64(0xB47C4), uses the grid side L = round(sqrt(t / 0.1))
              (inverting the mean crossing count ~0.1 L^2, as Sec. III.B inverts its
              fit of <n_c>(L)) and is redrawn from seed s until it has t-2..t+2
              crossings, random over/under.
    grad    : one knot with 300 crossings; L=53 (the grid side whose typical
              crossing count is about 300), seed 7, random over/under.
    large   : 8 knots with 600..1000 crossings at L=86, seeds 1..8, random over/under.
    large_moved : a copy of each `large` knot after 16 random Reidemeister I/II moves,
              a base-point shift and a crossing shuffle (SplitMix64(0x1A7E + i) for knot
              i); PD codes only (no embedding), returned as GridKnot with outer None.
    """
    if name == "tiny":
        return [random_grid_knot(12, 0, True, 16, 16)]
    if name == "scale":
        return [random_grid_knot(40, s, True, 100, 400) for s in range(1, 65)]
    if name == "batch":
        tr = SplitMix64(0xB47C4)
        out = []
        for s in range(4096):
            target = 20 + tr.below(101)
            L = max(6, int(round((target / 0.1) ** 0.5)))
            out.append(random_grid_knot(L, s, True, target - 2, target + 2))
        return out
    if name == "grad":
        return [random_grid_knot(53, 7, True, 300, 300)]
    if name == "large":
        return [random_grid_knot(86, s, True, 600, 1000) for s in range(1, 9)]
    if name == "large_moved":
        out = []
        for i, k in enumerate(knot_suite("large")):
            pd = randomize(k.pd, SplitMix64(0x1A7E + i), 16)
            out.append(GridKnot(k.L, k.seed, k.xs, k.ys, k.over_bits, pd, None, k.draws,
                                {"moves": 16}))
        return out
    raise KeyError(name)
