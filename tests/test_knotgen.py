"""The shared seeded input generator: PD codes are well formed and reproducible."""
import knotgen as kg


def _valid(pd):
    two_n = 2 * len(pd)
    labels = sorted(y for X in pd for y in X)
    assert labels == sorted(list(range(two_n)) * 2)
    for (a, b, c, d) in pd:
        assert c == (a + 1) % two_n


def test_splitmix64_reference_values():
    # first outputs of SplitMix64 seeded with 0 (published test vector of the generator)
    r = kg.SplitMix64(0)
    assert [r.next() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                            0x06C45D188009454F]


def test_grid_knots_valid_and_seeded():
    for s in range(20):
        k1 = kg.random_grid_knot(14, s, bool(s % 2), 1)
        k2 = kg.random_grid_knot(14, s, bool(s % 2), 1)
        assert k1.pd == k2.pd and k1.outer == k2.outer
        _valid(k1.pd)


def test_tiny_suite_has_16_crossings():
    (k,) = kg.knot_suite("tiny")
    assert k.n_crossings == 16 and k.L == 12 and k.seed == 0


def test_moves_keep_pd_valid():
    rng = kg.SplitMix64(5)
    pd = kg.random_grid_knot(12, 3, True, 4).pd
    for _ in range(10):
        pd = kg.randomize(pd, rng, 3)
        _valid(pd)
    _valid(kg.mirror(pd))
    _valid(kg.connected_sum(pd, kg.braid_closure_pd([1, 1, 1], 2)))
