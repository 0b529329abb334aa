"""Pins of the oracle's one-point and one-row helpers (point_f32, row_f32,
subband_point_f32), which check outputs too large for the whole-buffer oracle.

Each helper is compared element by element with the whole-buffer function it
samples (dedisperse, subband_dedisperse: pinned in test_oracle_pins.py and
test_subband_oracle.py) and with a numpy gather-and-sum written here, on small
plans that include a padded pitch, an ascending band and a ragged channel
count.  A helper that drops a channel, reads the wrong row or pitch, or
offsets t fails here."""
import numpy as np
import pytest

import oracle
import synth

TSAMP = 327.68e-6


def _plan(nch, fch1, foff, ndm, step):
    dms = np.arange(ndm, dtype=np.float64) * step
    d, m = oracle.delays(nch, fch1, foff, TSAMP, dms)
    return dms, d, m


def _gather_sum(x, drow, t):
    c = np.arange(x.shape[0])
    return float(np.sum(x[c, t + drow].astype(np.float64)))


CASES = [
    # (nchans, fch1, foff, nsamp, pitch, ndm, dm step)
    (64, 150.0, -0.1953125, 1500, 1500, 9, 0.35),      # descending band, pitch = nsamp
    (37, 150.0, -0.39, 1300, 1312, 7, 0.5),            # ragged channel count, padded pitch
    (48, 120.0, 0.25, 1400, 1408, 6, 0.4),             # ascending band (reference = last channel)
]


@pytest.mark.parametrize("nch,fch1,foff,nsamp,pitch,ndm,step", CASES)
def test_point_and_row_equal_whole_buffer(nch, fch1, foff, nsamp, pitch, ndm, step):
    dms, d, m = _plan(nch, fch1, foff, ndm, step)
    assert m > 0
    x = synth.noise_f32(nch, nsamp, seed=nch, pitch=pitch)
    x[:, nsamp:] = 1e6                          # padding must never be read
    nout = nsamp - m
    full = oracle.dedisperse(x[:, :nsamp].copy(), d, nout)
    for i in range(ndm):
        row = oracle.row_f32(x, d[i], nout)
        assert row.shape == (nout,)
        assert np.array_equal(row, full[i]), i
        for t in (0, 1, nout // 2, nout - 2, nout - 1):
            p = oracle.point_f32(x, d[i], t)
            assert p == full[i, t], (i, t)
            assert abs(p - _gather_sum(x, d[i], t)) <= 1e-12 * nch


def test_point_impulse_response():
    # a single 1 at (c, s) is seen by point(t) exactly when t + d[c] == s
    nch, nsamp = 5, 40
    drow = np.array([0, 3, 7, 7, 11], np.int64)
    for c in range(nch):
        for s in range(nsamp):
            x = np.zeros((nch, nsamp), np.float32)
            x[c, s] = 1.0
            for t in range(nsamp - int(drow.max())):
                want = 1.0 if t + drow[c] == s else 0.0
                assert oracle.point_f32(x, drow, t) == want, (c, s, t)


@pytest.mark.parametrize("nch,fch1,foff,nsub,G", [(64, 150.0, -0.1953125, 8, 3),
                                                  (48, 120.0, 0.25, 6, 4),
                                                  (32, 150.0, -0.39, 32, 2)])
def test_subband_point_equals_whole_buffer(nch, fch1, foff, nsub, G):
    ndm, nsamp, pitch = 11, 1600, 1616
    dms = np.arange(ndm, dtype=np.float64) * 0.3
    nom, d1, d2, m = oracle.subband_tables(nch, fch1, foff, TSAMP, dms, G, nsub)
    x = synth.noise_f32(nch, nsamp, seed=5 + nsub, pitch=pitch)
    x[:, nsamp:] = 1e6
    nout = nsamp - m
    full = oracle.subband_dedisperse(x[:, :nsamp].copy(), d1, d2, G, nout)
    cs = nch // nsub
    chan = np.arange(nch)
    for j in range(ndm):
        eff = d2[j][chan // cs] + d1[j // G]           # effective per-channel delay
        for t in (0, 7, nout // 3, nout - 1):
            p = oracle.subband_point_f32(x, d1, d2, G, j, t)
            assert p == full[j, t], (j, t)
            assert abs(p - _gather_sum(x, eff, t)) <= 1e-12 * nch
