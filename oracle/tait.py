"""Knot diagram -> signed Tait graph (Sec. II).

Steps, in the order the paper gives them:

1. Orientation and twist signs.  Each crossing gets epsilon_c = +1 when the
   strands cross "clockwise", i.e. by the right-hand rule
   sign((over direction) x (under direction))_z = +1; the writhe is w = sum epsilon_c.
2. Bicolouring.  Regions of the diagram are coloured black/white so that regions
   on the two sides of an arc differ; the unbounded region is white.
3. Tait graph G.  Vertices are the black regions; each crossing is an edge between
   the black regions that meet at it (loops and parallel edges allowed).
4. Tait sign.  Leaving the crossing along the over-strand, if the region on the
   left is black the crossing gets varepsilon_c = +1, otherwise -1;
   tau = sum varepsilon_c.

Faces are found from the PD code alone: with arms a (south, incoming under),
b (east), c (north), d (west) in counter-clockwise order, the corner between two
consecutive arms glues the side of one arc to the side of the next.  A PD code
carries no unbounded region, so the caller either names a side of an arc that
borders it (`outer = (arc, side)`, side 0 = left, 1 = right, as the grid-walk
generator reports) or the colour class is chosen by `black` (0: the class of the
region right of arc 0 is black, 1: the other).  Both classes give the same V.

Orientation.  A knot's PD code labels its arcs 0..2n-1 along the orientation, so the
under-strand runs a -> a+1 and the over-strand's direction follows from its labels.  A
link (several components) cannot be labelled that way; it is given with `signs`, the
twist sign of every crossing (+1: the over-strand leaves through arm b, -1: through arm
d, which is the right-hand rule of step 1), and any labels occurring twice each.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass
class TaitGraph:
    n_v: int
    edges: list          # [(u, v, eps)] with eps = Tait sign +-1
    writhe: int
    tau: int
    n_crossings: int
    components: int
    twist: list          # per-crossing twist sign
    black_faces: int
    white_faces: int


def _over_leaves_via_b(pd):
    two_n = 2 * len(pd)
    out = []
    for (a, b, c, d) in pd:
        if two_n == 2:
            # one crossing: the under-strand uses arc a then arc c; the over-strand
            # enters on arc c and leaves on arc a
            out.append(b == a)
        else:
            out.append(b == (d + 1) % two_n)
    return out


def tait_graph(pd, outer=None, black=None, signs=None) -> TaitGraph:
    n = len(pd)
    if n == 0:
        # a crossingless circle: one black region inside, white outside
        return TaitGraph(1, [], 0, 0, 0, 1, [], 1, 1)
    two_n = 2 * n
    labels = sorted(y for X in pd for y in X)
    if labels != sorted(list(range(two_n)) * 2):
        raise ValueError("each arc label 0..2n-1 must occur exactly twice")
    if signs is None:
        for (a, b, c, d) in pd:
            if c != (a + 1) % two_n:
                raise ValueError("under-strand must run a -> a+1")
        via_b = _over_leaves_via_b(pd)
    else:
        if len(signs) != n or any(x not in (1, -1) for x in signs):
            raise ValueError("one twist sign +-1 per crossing")
        via_b = [x > 0 for x in signs]

    # components: follow arc -> next arc through each crossing
    nxt = {}
    for (a, b, c, d), vb in zip(pd, via_b):
        nxt[a] = c
        if vb:
            nxt[d] = b
        else:
            nxt[b] = d
    if len(nxt) != two_n or sorted(nxt.values()) != list(range(two_n)):
        raise ValueError("inconsistent over-strand orientation")
    seen = set()
    comps = 0
    for s in range(two_n):
        if s in seen:
            continue
        comps += 1
        u = s
        while u not in seen:
            seen.add(u)
            u = nxt[u]

    # faces: union-find over arc sides; node 2*arc = left side, 2*arc+1 = right side
    parent = list(range(2 * two_n))

    def find(u):
        while parent[u] != u:
            parent[u] = parent[parent[u]]
            u = parent[u]
        return u

    def union(u, v):
        ru, rv = find(u), find(v)
        if ru != rv:
            parent[ru] = rv

    for (a, b, c, d), vb in zip(pd, via_b):
        arms = [a, b, c, d]
        outgoing = [False, vb, True, not vb]
        for i in range(4):
            x, y = arms[i], arms[(i + 1) % 4]
            ox, oy = outgoing[i], outgoing[(i + 1) % 4]
            # corner between arm i and the next arm counter-clockwise:
            # it is left of arm i if arm i leaves, right of it if it enters;
            # it is right of arm i+1 if that arm leaves, left of it if it enters
            sx = 2 * x + (0 if ox else 1)
            sy = 2 * y + (1 if oy else 0)
            union(sx, sy)
    roots = sorted({find(u) for u in range(2 * two_n)})
    if len(roots) != n + 2:
        raise ValueError(f"diagram is not planar: {len(roots)} faces for {n} crossings")
    fid = {r: i for i, r in enumerate(roots)}
    face_of = [fid[find(u)] for u in range(2 * two_n)]

    # 2-colouring: the two sides of every arc differ
    nf = len(roots)
    adj = [[] for _ in range(nf)]
    for arc in range(two_n):
        l, r = face_of[2 * arc], face_of[2 * arc + 1]
        adj[l].append(r)
        adj[r].append(l)
    colour = [-1] * nf
    colour[0] = 0
    stack = [0]
    while stack:
        f = stack.pop()
        for g in adj[f]:
            if colour[g] < 0:
                colour[g] = 1 - colour[f]
                stack.append(g)
            elif colour[g] == colour[f]:
                raise ValueError("regions cannot be 2-coloured")
    if outer is not None:
        arc, side = outer
        white = colour[face_of[2 * arc + side]]
        black_c = 1 - white
    else:
        ref = colour[face_of[2 * 0 + 1]]
        black_c = ref if (black in (None, 0)) else 1 - ref
    black_faces = sorted(f for f in range(nf) if colour[f] == black_c)
    vid = {f: i for i, f in enumerate(black_faces)}

    edges = []
    twist = []
    for (a, b, c, d), vb in zip(pd, via_b):
        eps_twist = 1 if vb else -1
        twist.append(eps_twist)
        # the four corners alternate colour; corners (a,b) and (c,d) are opposite,
        # as are (b,c) and (d,a)
        f_ab = face_of[2 * a + 1]          # right of the incoming under-arc a
        f_bc = face_of[2 * c + 1]          # right of the outgoing under-arc c
        f_cd = face_of[2 * c + 0]
        f_da = face_of[2 * a + 0]
        if colour[f_ab] == black_c:
            u, v = f_ab, f_cd
        else:
            u, v = f_bc, f_da
        assert colour[u] == black_c and colour[v] == black_c
        over_out = b if vb else d
        left_of_over_exit = face_of[2 * over_out + 0]
        eps = 1 if colour[left_of_over_exit] == black_c else -1
        edges.append((vid[u], vid[v], eps))
    w = sum(twist)
    tau = sum(e[2] for e in edges)
    return TaitGraph(len(black_faces), edges, w, tau, n, comps, twist,
                     len(black_faces), nf - len(black_faces))
