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


def test_stream_carry_tests_every_window_once():
    # with the threshold at -inf every window of the concatenated stream is a
    # candidate, found exactly once: N - w + 1 per row and width
    r = np.random.default_rng(3)
    x = r.standard_normal((3, 4 * 64))
    chunks = [x[:, c * 64:(c + 1) * 64] for c in range(4)]
    widths = [1, 2, 5, 16]
    res = oracle.search_stream(chunks, widths, -1e9, carry=True)
    n = {}
    for c, cc in enumerate(res):
        for row in cc:
            start = c * 64 + int(row["t"])
            key = (int(row["dm_idx"]), start, int(row["width_idx"]))
            n[key] = n.get(key, 0) + 1
    assert all(v == 1 for v in n.values())
    for p, w in enumerate(widths):
        for j in range(3):
            assert sum(1 for (jj, s, pp) in n if jj == j and pp == p) == 4 * 64 - w + 1
    # without the carry: the per-chunk search
    res0 = oracle.search_stream(chunks, widths, -1e9, carry=False)
    assert all(len(a) == 3 * sum(64 - w + 1 for w in widths) for a in res0)


def test_stream_carry_finds_a_pulse_on_the_boundary():
    r = np.random.default_rng(4)
    x = r.standard_normal((2, 256))
    x[1, 124:132] += 3.0                       # 8 samples straddling the boundary at 128
    chunks = [x[:, :128], x[:, 128:]]
    with_c = oracle.search_stream(chunks, [1, 2, 4, 8], 6.0, carry=True)[1]
    without = oracle.search_stream(chunks, [1, 2, 4, 8], 6.0, carry=False)[1]
    hit = [(int(c["dm_idx"]), int(c["t"]), int(c["width_idx"])) for c in with_c]
    assert (1, -4, 3) in hit and all(int(c["t"]) >= 0 for c in without)
