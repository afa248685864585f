"""The band-width autotuner's table lookup (host logic, no GPU): the entry of the nearest tuned order
at or below n, else the smallest; no entry -> 0 (the library default)."""
from paper_2502_02460_gb300 import tune


def test_pick_band_nearest_order_below():
    table = {"entries": {"f64/plain": {"1024": {"b": 16}, "4096": {"b": 32}, "8192": {"b": 64}},
                         "c128/mixed": {"2048": {"b": 32}}}}
    assert tune.pick_band(1024, False, False, table) == 16
    assert tune.pick_band(3000, False, False, table) == 16
    assert tune.pick_band(4096, False, False, table) == 32
    assert tune.pick_band(100000, False, False, table) == 64
    assert tune.pick_band(500, False, False, table) == 16  # below every tuned order: the smallest
    assert tune.pick_band(9000, True, True, table) == 32
    assert tune.pick_band(9000, True, False, table) == 0  # not tuned: the library's default
    assert tune.pick_band(9000, False, True, {}) == 0


def test_candidates_fit_the_bulge_kernel():
    # three b x b complex blocks (+1 padding column) must fit a CTA's 227 KB of shared memory
    for b in tune.CANDIDATES:
        assert 3 * b * (b + 1) * 16 <= 227 * 1024
    assert 3 * 128 * 129 * 8 > 227 * 1024  # why 128 is not a candidate


def test_committed_table_is_well_formed():
    """The table shipped with the package: every form, entries from the candidates, the fastest time's b."""
    table = tune.load(tune.TABLE)
    assert set(table["entries"]) == {"f64/plain", "f64/mixed", "c128/plain", "c128/mixed"}
    for form, orders in table["entries"].items():
        for order, ent in orders.items():
            assert ent["b"] in tune.CANDIDATES
            times = {int(b): t for b, t in ent["ms"].items()}
            assert min(times, key=times.get) == ent["b"], (form, order)
            cx, mixed = form.startswith("c128"), form.endswith("mixed")
            assert tune.pick_band(int(order), cx, mixed, table) == ent["b"]
