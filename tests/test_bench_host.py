"""Host-side accounting of bench.py (no GPU): the shared-memory words one
kernel 5 launch moves, which its roofline line divides by the kernel time,
against a plain loop over DM blocks and subbands."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402


def _words_loop(d, foff, db, tile, cs=4):
    ndm, nch = d.shape
    total = 0
    for b in range(-(-ndm // db)):
        trials = [min(b * db + j, ndm - 1) for j in range(db)]
        for s in range(nch // cs):
            spans = {}
            for j in trials:
                sub = [int(v) for v in d[j, s * cs:(s + 1) * cs]]
                ref = sub[0] if foff < 0 else sub[-1]
                key = tuple(v - ref for v in sub)
                lo, hi = spans.get(key, (ref, ref))
                spans[key] = (min(lo, ref), max(hi, ref))
            total += sum(hi - lo + tile for lo, hi in spans.values()) * (cs + 1) + db * tile
    return total


@pytest.mark.parametrize("foff", [-0.39, 0.39])
@pytest.mark.parametrize("db,tile", [(8, 64), (12, 32)])
def test_share_words_matches_loop(foff, db, tile):
    # 16 channels, 37 trials (ragged last block), both band orientations
    fch1 = 150.0 if foff < 0 else 150.0 - 15 * abs(foff)
    dms = [0.7 * i for i in range(37)]
    d, _ = oracle.delays(16, fch1, foff, 327.68e-6, dms)
    d = np.asarray(d)
    assert bench.share_words(d, foff, db, tile) == _words_loop(d, foff, db, tile)


def test_share_words_single_pattern():
    # all trials with the same delays (DM 0): one pattern of span 0 per subband
    d = np.zeros((5, 8), np.int32)
    assert bench.share_words(d, -1.0, 4, 32) == 2 * 2 * ((32 * 5) + 4 * 32)


@pytest.mark.parametrize("seed", range(6))
def test_pipeline_schedule_covers_every_tile(seed):
    # dd_process_host's chunks: the tile ranges partition all tiles, the copied
    # columns only grow and end at the pitch, and every tile launched after
    # chunk c reads only columns that chunk c's copies have completed
    from paper_1107_2516_gb300 import build as ddbuild
    from paper_1107_2516_gb300 import dd as ddc
    ddbuild.build()
    rng = np.random.default_rng(seed)
    for _ in range(200):
        tile = int(rng.choice([256, 384, 512, 640]))
        nout = int(rng.integers(1, 40 * tile))
        reach = int(rng.integers(tile, tile + 30000))
        pitch = nout + reach - tile + int(rng.integers(0, 64))
        col, til = ddc.dd_host_chunk_schedule(nout, pitch, tile, reach)
        ntile = -(-nout // tile)
        assert 1 <= len(col) <= 8 and len(col) == min(8, ntile)
        assert til[-1] == ntile and np.all(np.diff(np.concatenate([[0], til])) > 0)
        assert col[-1] == pitch and np.all(np.diff(col) >= 0)
        for c in range(len(col)):
            assert min(pitch, int(til[c]) * tile + reach) <= col[c]


def test_traffic_reported_only_for_unchanged_sources(monkeypatch):
    # a recorded ncu traffic figure is reported while the kernel's sources
    # still hash to the digest taken with it, and dropped once they change
    dig = bench.kernel_source_digest(5)
    assert len(dig) == 64 and dig != bench.kernel_source_digest(3)
    monkeypatch.setattr(bench, "PROFILED_TRAFFIC", {(11, 16): (21.41e9, dig), (9, 16): (25.6e9, "0" * 64)})
    assert bench.profiled_traffic(5, (11, 16, 16, 6)) == 21.41e9
    assert bench.profiled_traffic(5, (9, 16, 16, 4)) is None
    assert bench.profiled_traffic(5, (10, 16, 8, 4)) is None
    assert bench.profiled_traffic(5, None) is None
