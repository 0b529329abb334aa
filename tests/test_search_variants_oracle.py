"""Pins of the per-DM-row search variant of the oracle: rows with identical
value sets reduce it to the whole-buffer search; a per-row offset or positive
scale leaves a row's candidates unchanged (the whole-buffer search does not
have this invariance)."""
import numpy as np

import oracle


def _keys(c):
    return [(int(r["dm_idx"]), int(r["t"]), int(r["width_idx"])) for r in c]


def test_rows_with_equal_statistics_reduce_to_the_global_search():
    r = np.random.default_rng(1)
    base = r.standard_normal(3000) * 4.0
    base[1234:1238] += 20.0
    rows = np.stack([np.roll(base, 17 * j) for j in range(6)])      # same multiset per row
    c_row, mus, sgs = oracle.search_per_row(rows, [1, 2, 4, 8], 5.0)
    mu, sg = oracle.stats(rows)
    c_glob = oracle.search(rows, [1, 2, 4, 8], mu, sg, 5.0)
    assert np.allclose(mus, mu, rtol=0, atol=1e-12) and np.allclose(sgs, sg, rtol=1e-12)
    assert _keys(c_row) == _keys(c_glob) and len(c_row) > 0


def test_row_offset_and_scale_invariance():
    r = np.random.default_rng(2)
    rows = r.standard_normal((5, 2000))
    rows[2, 700:703] += 8.0
    rows[4, 100:116] += 2.5
    c0, mu0, sg0 = oracle.search_per_row(rows, [1, 2, 4, 16], 4.0)
    moved = rows.copy()
    moved[2] = moved[2] * 3.0 + 50.0         # exact in double? (scale by 3 and shift)
    moved[4] = moved[4] + 1000.0
    c1, mu1, sg1 = oracle.search_per_row(moved, [1, 2, 4, 16], 4.0)
    assert _keys(c0) == _keys(c1)
    assert np.isclose(mu1[2], mu0[2] * 3 + 50) and np.isclose(sg1[2], sg0[2] * 3)
    # the whole-buffer search is not invariant: the shifted row dominates
    mu, sg = oracle.stats(moved)
    assert _keys(oracle.search(moved, [1, 2, 4, 16], mu, sg, 4.0)) != _keys(c0)
