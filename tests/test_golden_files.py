"""The stored oracle values under tests/golden/ are the oracle's: a few entries of
scale_oracle.txt are recomputed here with the same oracle calls its generator makes
(min-fill order, one-call bucket step) and must agree bit for bit."""
import os
import sys

import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, GOLDEN)


def _rows():
    out = {}
    for line in open(os.path.join(GOLDEN, "scale_oracle.txt")):
        if not line.startswith("#"):
            f = line.split()
            out[(int(f[0]), int(f[1]))] = f
    return out


def test_scale_oracle_file_complete():
    rows = _rows()
    assert set(rows) == {(s, q) for s in range(1, 65) for q in (2, 3, 5)}
    import make_scale_oracle as m
    for (s, q), f in rows.items():
        assert (f[3] == "-") == (not m.fits(q, int(f[2]))), (s, q)


@pytest.mark.parametrize("key", [(3, 2), (17, 3), (64, 5), (60, 5)])
def test_scale_oracle_entries_recomputed(key):
    import make_scale_oracle as m
    seed, q, w, z, v = m.one(key)
    f = _rows()[key]
    assert int(f[2]) == w
    assert f[3:6] == [z.m.real.hex(), z.m.imag.hex(), str(z.e)]
    assert f[6:9] == [v.m.real.hex(), v.m.imag.hex(), str(v.e)]
