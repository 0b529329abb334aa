"""Kernel 5's tables as the library builds them (dd_share_tables, host only, no
GPU): the two stages of the kernel executed in numpy from those tables give
the oracle's brute-force sums, and every index stays inside the buffer it
addresses.

Stage 1: for subband s of DM block b and the time tile at t0, P[e] (e < E)
sums the subband's 4 staged input rows at the staged element b_c + e of the
pattern e belongs to; the rows hold input columns t0 + base[b][c] onwards,
rlen[b][c] of them or as many as the input has (the rest of a staged row is
never written: NaN here).  Stage 2: trial j adds P[q_j + i] to its output sample t0 + i."""
import numpy as np
import pytest

import oracle
import synth
import paper_1107_2516_gb300 as dd
from paper_1107_2516_gb300 import build as ddbuild
from paper_1107_2516_gb300 import dd as ddc

CS = 4
NPMAX, MAXW = 16, 8          # pattern slots per record; warps the stage-1 split records
SHAPES = {9: (512, 32), 10: (256, 32), 11: (512, 48), 12: (512, 64)}     # config: (tile, trials per block)
# warps the stage-1 rows are split over (config 12: its 8 stage-1 warps), and
# warp 0's share in percent of another warp's (it also issues the copies)
SPLIT = {9: 4, 10: 4, 11: 6, 12: 8}
W0 = {9: 70, 10: 70, 11: 70, 12: 50}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ddbuild.build()
    dd.load()


def emulate(x, nsamp, d, foff, dtype, config):
    """The kernel's sums from the library's tables (None if the shape cannot run)."""
    t = ddc.dd_share_tables(d, foff, dtype, config)
    if t is None:
        return None
    rec, base, rlen, rs = t["rec"], t["base"], t["rlen"], t["rs"]
    al_el = 16 if dtype == dd.DD_U8 else 8 if dtype == dd.DD_F16 else 4
    assert np.all(rlen <= rs) and np.all(rlen % al_el == 0) and np.all(rlen > 0)
    tile, db = SHAPES[config]
    ndm, nch = d.shape
    nblk, nsub, _ = rec.shape
    al = 16 if dtype == dd.DD_U8 else 4
    nsamp_al = (nsamp + al - 1) // al * al
    nout = nsamp - int(d.max())
    ntile = -(-nout // tile)
    out = np.full((nblk * db, ntile * tile), np.nan)
    for b in range(nblk):
        for j in range(ntile):
            t0 = j * tile
            acc = np.zeros((db, tile))
            for s in range(nsub):
                stage = np.full(CS * rs, np.nan)
                for c in range(CS):
                    # the kernel copies the channel's own row length (its trials' reach), not rs
                    g = t0 + int(base[b, s * CS + c])
                    n = max(0, min(int(rlen[b, s * CS + c]), nsamp_al - g))
                    stage[c * rs:c * rs + n] = x[s * CS + c, g:g + n]
                r = rec[b, s]
                E = int(r[db])
                pats = r[db + 4:db + 4 + NPMAX * 8].reshape(-1, 8)
                ends = pats[:, 0]
                e = np.arange(E)
                p = np.searchsorted(ends[ends > 0], e, side="right")
                assert E == int(ends[p.max()]) and np.all(np.diff(ends[:p.max() + 1]) > 0)
                P = np.zeros(E)
                for c in range(CS):
                    idx = pats[p, 1 + c] + e
                    # channel c's term comes from channel c's staged row
                    assert idx.min() >= c * rs and idx.max() < (c + 1) * rs
                    P += stage[idx]
                q = r[:db].astype(np.int64)
                assert q.min() >= 0 and q.max() + tile <= E
                acc += P[q[:, None] + np.arange(tile)[None, :]]
            out[b * db:(b + 1) * db, t0:t0 + tile] = acc
    return out[:ndm, :nout]


CASES = [
    # nchans, fch1, foff, tsamp, DMs, nsamp, dtype (ragged last block and tile in each)
    (128, 150.0, -0.0234375, 163.84e-6, [0.1 * i for i in range(60)], 2700, "f32"),       # 11-15 patterns
    (96, 150.0 - 95 * 0.0234375, 0.0234375, 163.84e-6, [0.1 * i for i in range(50)], 2300, "u8"),  # ascending
    (256, 150.0, -0.046875, 163.84e-6, [0.05 * i for i in range(100)], 3000, "f32"),      # 13 / 17 patterns
    (128, 150.0, -0.0234375, 163.84e-6, [0.05 * i for i in range(100)], 2900, "f32"),     # every shape (64 + 36 trials)
]


@pytest.mark.parametrize("config", [9, 10, 11, 12])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_kernel5_tables_reproduce_brute_force(case, config):
    nch, fch1, foff, ts, dms, nsamp, dt = CASES[case]
    d, m = oracle.delays(nch, fch1, foff, ts, dms)
    d = np.asarray(d)
    al = 16 if dt == "u8" else 4
    pitch = (nsamp + al - 1) // al * al + al
    x = synth.noise_f32(nch, nsamp, 11 + case, pitch=pitch)
    if dt == "u8":
        x = synth.quantize_u8(x)
    got = emulate(x.astype(np.float64), nsamp, d, foff, dd.DD_U8 if dt == "u8" else dd.DD_F32, config)
    if got is None:
        # more than 16 delay patterns in some (block, subband): the shape refuses the plan
        pytest.skip("shape unavailable for this plan")
    ref = oracle.dedisperse(x, d, nsamp - m)
    assert not np.isnan(got).any()
    if dt == "u8":
        assert np.array_equal(got.astype(np.int64), ref)
    else:
        assert np.max(np.abs(got - ref)) <= 1e-9 * nch


def test_kernel5_tables_refuse_many_patterns():
    # the small workload's 128 channels and 0.1 DM steps give 29 patterns per
    # (32-trial block, subband): more than the 16 the records hold
    wl = synth.workload("small_f32")
    d, _ = oracle.delays(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list)
    assert ddc.dd_share_tables(np.asarray(d), wl.foff, dd.DD_F32, 9) is None


def test_kernel5_tables_bad_config():
    d = np.zeros((4, 8), np.int32)
    with pytest.raises(dd.DDError):
        ddc.dd_share_tables(d, -1.0, dd.DD_F32, 5)


def _split(R, nw, w0):
    """Row boundaries b_0 .. b_nw: warp 0 weighs w0 (percent), the others 100,
    boundaries rounded half up in integers."""
    tot = w0 + 100 * (nw - 1)
    return [0] + [(R * (w0 + 100 * (w - 1)) + tot // 2) // tot for w in range(1, nw + 1)]


def _stage1_rows(rec_row, db, nw, w0):
    """Kernel 5's stage-1 work split, restated: the patterns' sums (index space
    e < E) cut into rows of 32 inside each pattern; warp w of nw takes rows
    [b_w, b_w+1) (_split: warp 0 a w0-percent share) and lane l element
    row_start + l of each.  The
    record's per-pattern start / rows-before fields and per-warp first row and
    pattern must be exactly these.  Returns how often each e is summed."""
    E = int(rec_row[db])
    pat = rec_row[db + 4:db + 4 + NPMAX * 8].reshape(NPMAX, 8).astype(np.int64)
    ends = pat[:, 0]
    npat = int(np.nonzero(ends == E)[0][0]) + 1
    starts = np.concatenate([[0], ends[:npat - 1]])
    rows = (ends[:npat] - starts + 31) // 32
    incl = np.cumsum(rows)
    excl = incl - rows
    assert np.array_equal(pat[:npat, 1 + CS], starts) and np.array_equal(pat[:npat, 2 + CS], excl)
    R = int(incl[-1])
    wt = rec_row[db + 4 + NPMAX * 8:].astype(np.int64)
    cover = np.zeros(E, np.int64)
    bnd = _split(R, nw, w0)
    assert bnd[-1] == R and all(bnd[i] <= bnd[i + 1] for i in range(nw))
    for w in range(nw):
        r0, r1 = bnd[w], bnd[w + 1]
        assert wt[w] == r0 and wt[w + 1] == r1
        if r0 < r1:
            assert wt[MAXW + 1 + w] == int(np.searchsorted(incl, r0, side="right"))
        for r in range(r0, r1):
            p = int(np.searchsorted(incl, r, side="right"))
            e = starts[p] + 32 * (r - excl[p]) + np.arange(32)
            e = e[e < ends[p]]
            assert e.size and e.min() >= starts[p]
            cover[e] += 1
    return cover


@pytest.mark.parametrize("config", [9, 10, 11, 12])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_stage1_rows_cover_every_sum_once(case, config):
    nch, fch1, foff, ts, dms, nsamp, dt = CASES[case]
    d, _ = oracle.delays(nch, fch1, foff, ts, dms)
    t = ddc.dd_share_tables(np.asarray(d), foff, dd.DD_U8 if dt == "u8" else dd.DD_F32, config)
    if t is None:
        pytest.skip("shape unavailable for this plan")
    _, db = SHAPES[config]
    nw = SPLIT[config]
    rec = t["rec"]
    for b in range(rec.shape[0]):
        for s in range(rec.shape[1]):
            assert np.all(_stage1_rows(rec[b, s], db, nw, W0[config]) == 1), (b, s)


def test_stage1_rows_cover_every_sum_once_lofar():
    # the benchmark plan's tables (every block, every 16th subband), configs 9, 11 and 12
    wl = synth.workload("lofar_f32")
    d, _ = oracle.delays(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list)
    for config in (9, 11, 12):
        nw = SPLIT[config]
        t = ddc.dd_share_tables(np.asarray(d), wl.foff, dd.DD_F32, config)
        assert t is not None
        _, db = SHAPES[config]
        rec = t["rec"]
        for b in range(rec.shape[0]):
            for s in range(0, rec.shape[1], 16):
                assert np.all(_stage1_rows(rec[b, s], db, nw, W0[config]) == 1), (config, b, s)



def test_tile_rotation_is_a_permutation():
    # whole-plan kernel 5 launches rotate each DM block's time tiles back by
    # its middle-channel row start in whole tiles (k_b); restated here on the
    # benchmark plan's tables: every (block, tile) pair is taken exactly once,
    # and the rotations spread the blocks over the delay span they stage
    wl = synth.workload("lofar_f32")
    d, m = oracle.delays(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list)
    nout = wl.nsamp - int(m)
    for config in (11, 12):
        t = ddc.dd_share_tables(np.asarray(d), wl.foff, dd.DD_F32, config)
        tile, _ = SHAPES[config]
        base = t["base"]
        nblk, nch = base.shape
        ntile = -(-nout // tile)
        k = (base[:, nch // 2].astype(np.int64) // tile) % ntile
        s = np.arange(ntile)
        taken = (s[None, :] + ntile - k[:, None]) % ntile          # tile of slot s, per block
        assert all(np.array_equal(np.sort(row), s) for row in taken)
        # the rotations follow the middle channel's delay: monotone over the blocks,
        # from 0 at DM 0 to about half the maxshift (in tiles) at the top
        assert k[0] == 0 and np.all(np.diff(k) >= 0)
        assert 0.3 * m / tile < k[-1] < 0.7 * m / tile
