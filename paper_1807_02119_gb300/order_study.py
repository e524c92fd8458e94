"""Statistics of the grid-walk knots and of contraction orders (Sec. III.A-B, Figs. 2-3).

For grid sides L the script samples knots with the paper's generator (random grid walks,
vertical strands always over: pk_knot_from_grid_walk), simplifies each signed Tait graph
by Reidemeister I and II moves (pk_knot_simplify) and reports, per L:

* Fig. 2: the means of n_v and n_c of the simplified graphs, their ratio, and the mean
  maximal degree Delta_G, with log-log fits of n_v and n_c against L over the largest L;
* Fig. 3: the mean largest rank Delta_H met while contracting the graph with the paper's
  greedy (edge network, PK_ORDER_GREEDY_EDGE) and with the partition order (recursive
  bisection with Fiduccia-Mattheyses refinement, PK_ORDER_PARTITION), the per-instance
  share where the partition order is better, linear fits of Delta_H against L, and the
  same comparison binned by n_c.  Min-fill (PK_ORDER_FILL_SPIN) is listed for reference.

Delta_H counts the indices of the largest intermediate tensor, so a contraction costs
O(q^Delta_H) for every order.  Only the host planner is used (no GPU).

Usage: python -m paper_1807_02119_gb300.order_study [--L 6:100:4] [--n 50] [--json out.json]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ORDERS = ("greedy_edge", "partition", "fill_spin")


def fit(xs, ys):
    """Least-squares line y = a x + b: (a, b, r^2)."""
    n = len(xs)
    mx, my = sum(xs) / n, sum(ys) / n
    sxx = sum((x - mx) ** 2 for x in xs)
    sxy = sum((x - mx) * (y - my) for x, y in zip(xs, ys))
    a = sxy / sxx
    b = my - a * mx
    ss = sum((y - my) ** 2 for y in ys)
    res = sum((y - a * x - b) ** 2 for x, y in zip(xs, ys))
    return a, b, (1 - res / ss) if ss > 0 else 1.0


def sample(pk, ctx, L, n, seed0=0, restarts=4, orders=ORDERS):
    """Per knot: n_c before and after simplification, n_v, Delta_G, Delta_H per order."""
    rows = []
    for s in range(n):
        k = pk.Knot.from_grid_walk(ctx, L, seed0 + s, False)
        g = k.simplified()
        info = g.info()
        r = {"L": L, "seed": seed0 + s, "n_c_raw": k.info()["n_c"], "n_c": info["n_c"],
             "n_v": info["n_v"], "delta_g": g.max_degree()}
        for o in orders:
            r[o] = g.order_stats(2, o, restarts)["delta_h"] if info["n_c"] > 0 else 0
        rows.append(r)
    return rows


def summarise(rows, fit_last=10):
    Ls = sorted({r["L"] for r in rows})
    per_L = []
    for L in Ls:
        rs = [r for r in rows if r["L"] == L]
        m = lambda key: sum(r[key] for r in rs) / len(rs)
        sem = lambda key: (math.sqrt(sum((r[key] - m(key)) ** 2 for r in rs) / max(1, len(rs) - 1))
                           / math.sqrt(len(rs)))
        e = {"L": L, "n": len(rs), "n_v": m("n_v"), "n_c": m("n_c"), "delta_g": m("delta_g"),
             "delta_g_sem": sem("delta_g")}
        e["ratio"] = e["n_c"] / e["n_v"] if e["n_v"] else float("nan")
        for o in ORDERS:
            if o in rs[0]:
                e[o] = m(o)
                e[o + "_sem"] = sem(o)
        if "partition" in rs[0]:
            e["partition_better"] = sum(r["partition"] < r["greedy_edge"] for r in rs) / len(rs)
            e["partition_worse"] = sum(r["partition"] > r["greedy_edge"] for r in rs) / len(rs)
        per_L.append(e)
    tail = [e for e in per_L if e["n_v"] > 0][-fit_last:]
    lx = [math.log(e["L"]) for e in tail]
    out = {"per_L": per_L,
           "fit_last": len(tail),
           "slope_n_v": fit(lx, [math.log(e["n_v"]) for e in tail])[0],
           "slope_n_c": fit(lx, [math.log(e["n_c"]) for e in tail])[0]}
    for o in ORDERS:
        if o in per_L[0]:
            a, b, r2 = fit([e["L"] for e in tail], [e[o] for e in tail])
            out["delta_h_fit_" + o] = {"slope": a, "intercept": b, "r2": r2}
    big = [e for e in per_L if e["L"] > 22]   # Fig. 2 (inset) fits Delta_G for L > 22
    if len(big) >= 2:
        a, b, r2 = fit([math.log(e["L"]) for e in big], [e["delta_g"] for e in big])
        out["delta_g_fit_log"] = {"slope": a, "intercept": b, "r2": r2, "from_L": big[0]["L"]}
    # the comparison by crossing number (bins of the simplified n_c)
    bins = {}
    for r in rows:
        if r["n_c"] == 0 or "partition" not in r:
            continue
        b = int(r["n_c"] // 200) * 200
        d = bins.setdefault(b, [0, 0.0, 0.0])
        d[0] += 1
        d[1] += r["greedy_edge"]
        d[2] += r["partition"]
    out["by_n_c"] = [{"n_c_from": b, "n": d[0], "greedy_edge": d[1] / d[0], "partition": d[2] / d[0]}
                     for b, d in sorted(bins.items())]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", default="6:100:4", help="first:last:step grid sides")
    ap.add_argument("--n", type=int, default=50, help="knots per grid side")
    ap.add_argument("--restarts", type=int, default=4)
    ap.add_argument("--json", default=None)
    args = ap.parse_args()
    sys.path.insert(0, os.path.dirname(HERE))
    import paper_1807_02119_gb300 as pk
    a, b, c = (int(x) for x in args.L.split(":"))
    ctx = pk.Context(-1)
    rows = []
    for L in range(a, b + 1, c):
        rows += sample(pk, ctx, L, args.n, restarts=args.restarts)
    s = summarise(rows)
    print(f"{'L':>4} {'<n_v>':>8} {'<n_c>':>8} {'ratio':>6} {'<D_G>':>6} "
          f"{'greedy':>7} {'partition':>9} {'min-fill':>8} {'part<greedy':>11} {'part>greedy':>11}")
    for e in s["per_L"]:
        print(f"{e['L']:4d} {e['n_v']:8.1f} {e['n_c']:8.1f} {e['ratio']:6.3f} {e['delta_g']:6.2f} "
              f"{e['greedy_edge']:7.2f} {e['partition']:9.2f} {e['fill_spin']:8.2f} "
              f"{e['partition_better']:11.2f} {e['partition_worse']:11.2f}")
    print(f"log-log slopes over the last {s['fit_last']} L: n_v {s['slope_n_v']:.3f}, n_c {s['slope_n_c']:.3f}")
    for o in ORDERS:
        f = s["delta_h_fit_" + o]
        print(f"Delta_H {o}: {f['slope']:.3f} L + {f['intercept']:.2f} (r^2 {f['r2']:.3f})")
    f = s.get("delta_g_fit_log")
    if f:
        print(f"Delta_G (L > 22): {f['slope']:.3f} ln L + {f['intercept']:.2f} (r^2 {f['r2']:.3f})")
    for d in s["by_n_c"]:
        print(f"n_c in [{d['n_c_from']}, {d['n_c_from'] + 200}): {d['n']:4d} knots, Delta_H greedy "
              f"{d['greedy_edge']:.2f}, partition {d['partition']:.2f}")
    if args.json:
        with open(args.json, "w") as fh:
            json.dump({"rows": rows, "summary": s}, fh)


if __name__ == "__main__":
    main()
