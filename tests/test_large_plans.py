"""Planning the 600-1000-crossing workload (no GPU): which (knot, q) evaluations fit a
contraction budget.  The knots are 8 grid walks at L=86 plus a copy of each after
Reidemeister moves; the work of a plan is its complex multiply-adds over all slices."""
import pytest

import knotgen as kg
import paper_1807_02119_gb300 as pk

BUDGET = 1e14   # complex multiply-adds per evaluation (about 200 s in split on one GB300)


@pytest.fixture(scope="module")
def plans():
    ctx = pk.Context(-1)
    out = {}
    for name in ("large", "large_moved"):
        for i, gk in enumerate(kg.knot_suite(name)):
            k = pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer)
            for q in (2, 3, 4, 6):
                try:
                    p = pk.Plan(ctx, k, q, restarts=64 if q > 2 else 8)
                    out[(name, i, q)] = p.stats()
                except pk.PkError as e:
                    assert e.status == 4          # PK_ETOOWIDE
                    out[(name, i, q)] = None
    return out


def test_large_feasibility_report(plans):
    rows = []
    for (name, i, q), st in sorted(plans.items()):
        rows.append((name, i, q, None if st is None else st["cmacs"]))
    # q = 2: every knot and copy fits easily, unsliced below 2^31 entries
    assert all(c is not None and c < 1e11 for n, i, q, c in rows if q == 2)
    # q = 4 and q = 6 are beyond the budget on every knot
    assert all(c is None or c > BUDGET for n, i, q, c in rows if q in (4, 6))
    # q = 3: some knots fit, some do not (the work spans several orders of magnitude)
    q3 = [c for n, i, q, c in rows if q == 3]
    assert min(q3) < BUDGET < max(q3)
    for r in rows:
        print(*r)
