"""Pins of the CPU oracle to things other than itself.

Each test ties one oracle function to a closed form (exact rational evaluation
of Eq. 1), a library routine (numpy sums, convolution, mean/std, float16
conversion), an invariant (constant input, impulse response, DM = 0), brute
force on tiny inputs, or the paper's own worked numbers (Table 2's fake pulsar,
Section 4).  A plausible mistake anywhere in the oracle -- a dropped term, a
wrong sign, a transposed index -- fails at least one of them.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth


def _exact_delay(fch1, foff, nchans, tsamp_s, dm, c):
    """Eq. 1 / tsamp in exact rational arithmetic on the given doubles."""
    f = Fraction(fch1) + c * Fraction(foff)
    f_top = Fraction(fch1) if foff < 0 else Fraction(fch1) + (nchans - 1) * Fraction(foff)
    k = Fraction(415, 100) * 10 ** 6 * (1 / (f * f) - 1 / (f_top * f_top))
    return k * Fraction(dm) / (Fraction(tsamp_s) * 1000)


def _round_half_away(x: Fraction) -> int:
    fl = math.floor(x)
    return fl + 1 if x - fl >= Fraction(1, 2) else fl


# ---------------------------------------------------------------- delays (Eq. 1)

@pytest.mark.parametrize("name", ["small_f32", "lofar_f32"])
def test_delays_match_exact_rational_eq1(name):
    wl = synth.workload(name)
    dms = wl.dm_list
    d, m = oracle.delays(wl.nchans, wl.fch1, wl.foff, wl.tsamp, dms)
    rows = range(wl.ndm) if wl.ndm <= 64 else range(0, wl.ndm, 97)
    chans = range(wl.nchans) if wl.nchans <= 128 else range(0, wl.nchans, 7)
    near_ties = 0
    for i in rows:
        for c in chans:
            x = _exact_delay(wl.fch1, wl.foff, wl.nchans, wl.tsamp, float(dms[i]), c)
            frac = x - math.floor(x)
            if abs(frac - Fraction(1, 2)) < Fraction(1, 10 ** 9):
                near_ties += 1
                continue
            assert d[i, c] == _round_half_away(x), (i, c, float(x))
    assert near_ties == 0


def test_delay_hand_worked_values(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "delay_hand_worked.json")))
    for case in g["cases"]:
        dl = case["dm_list"]
        dms = dl["start"] + np.arange(dl["n"], dtype=np.float64) * dl["step"]
        d, m = oracle.delays(case["nchans"], case["fch1_mhz"], case["foff_mhz"], case["tsamp_s"], dms)
        assert m == case["maxshift"]
        c = case["channel"]
        for pt in case["points"]:
            x = oracle.delay_exact(case["fch1_mhz"], case["foff_mhz"], case["nchans"],
                                   case["tsamp_s"], pt["dm"], c)
            assert abs(x - pt["x_samples"]) < 1e-9 * pt["x_samples"]
            d1, _ = oracle.delays(case["nchans"], case["fch1_mhz"], case["foff_mhz"],
                                  case["tsamp_s"], [pt["dm"]])
            assert d1[0, c] == pt["delay"]
        eq2 = oracle.maxshift_eq2(case["nchans"], case["fch1_mhz"], case["foff_mhz"],
                                  case["tsamp_s"], float(dms[-1]))
        assert abs(eq2 - m) / m < 0.01


def test_delay_invariants():
    # descending and ascending bands
    for foff in (-0.1953125, 0.1953125):
        fch1 = 150.0 if foff < 0 else 125.1953125
        dms = np.arange(40, dtype=np.float64) * 0.25
        d, m = oracle.delays(128, fch1, foff, 327.68e-6, dms)
        assert np.all(d[0] == 0)                          # DM = 0: no delay
        top = 0 if foff < 0 else 127
        assert np.all(d[:, top] == 0)                     # reference channel never shifts
        assert np.all(np.diff(d, axis=0) >= 0)            # monotone in DM
        if foff < 0:
            assert np.all(np.diff(d, axis=1) >= 0)        # lower frequency -> later
        else:
            assert np.all(np.diff(d, axis=1) <= 0)
        assert m == d.max()
        for i in (1, 17, 39):
            for c in (0, 5, 64, 127):
                x = oracle.delay_exact(fch1, foff, 128, 327.68e-6, float(dms[i]), c)
                assert abs(d[i, c] - x) <= 0.5
    # delays scale linearly with DM (Eq. 1 is linear in DM): x(2*dm) = 2*x(dm)
    x1 = oracle.delay_exact(150.0, -0.01171875, 1024, 163.84e-6, 12.5, 700)
    x2 = oracle.delay_exact(150.0, -0.01171875, 1024, 163.84e-6, 25.0, 700)
    assert abs(x2 - 2 * x1) < 1e-9 * x2
    # and inversely with the sampling time
    x3 = oracle.delay_exact(150.0, -0.01171875, 1024, 2 * 163.84e-6, 12.5, 700)
    assert abs(2 * x3 - x1) < 1e-9 * x1


def test_delays_reject_bad_arguments():
    with pytest.raises(ValueError):
        oracle.delays(0, 150.0, -0.1, 1e-4, [0.0])
    with pytest.raises(ValueError):
        oracle.delays(2000, 150.0, -0.1, 1e-4, [0.0])        # band crosses 0 MHz
    with pytest.raises(ValueError):
        oracle.delays(16, 150.0, -0.1, 1e-4, [-1.0])


# ------------------------------------------------------------- binary16 decoding

def test_half_decoder_all_bit_patterns():
    bits = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16)
    ref = bits.view(np.float16).astype(np.float64)
    got = np.array([oracle.half_to_double(int(b)) for b in bits])
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan], ref[~nan])


# ------------------------------------------------- brute-force sum (Section 3.1)

def _tiny_loop(data, d, nout):
    nch = data.shape[0]
    out = [[0.0] * nout for _ in range(d.shape[0])]
    for i in range(d.shape[0]):
        for t in range(nout):
            for c in range(nch):
                out[i][t] += float(data[c][t + d[i][c]])
    return np.array(out)


def test_dedisperse_brute_force_tiny():
    rng = np.random.default_rng(7)
    for nch, nsamp in ((1, 5), (3, 16), (4, 16)):
        data = rng.standard_normal((nch, nsamp)).astype(np.float32)
        d = rng.integers(0, 5, size=(3, nch)).astype(np.int64)
        nout = nsamp - int(d.max())
        got = oracle.dedisperse(data, d, nout)
        np.testing.assert_allclose(got, _tiny_loop(data, d, nout), rtol=0, atol=1e-12)


def test_dedisperse_impulse_response():
    # A single 1 at (c, s): out[i][t] == 1 exactly when t + d[i][c] == s.
    d = np.array([[0, 2, 5], [0, 1, 3], [0, 0, 0]], dtype=np.int64)
    nch, nsamp = 3, 12
    nout = nsamp - int(d.max())
    for c in range(nch):
        for s in range(nsamp):
            data = np.zeros((nch, nsamp), np.float32)
            data[c, s] = 1.0
            out = oracle.dedisperse(data, d, nout)
            want = np.zeros_like(out)
            for i in range(d.shape[0]):
                t = s - d[i, c]
                if 0 <= t < nout:
                    want[i, t] = 1.0
            assert np.array_equal(out, want), (c, s)


def test_dm_zero_row_is_channel_sum_and_constant_input():
    wl = synth.workload("small_f32")
    data = synth.noise_f32(wl.nchans, wl.nsamp, seed=11)
    d, m = oracle.delays(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list)
    nout = wl.nsamp - m
    out = oracle.dedisperse(data, d, nout)
    ref = np.sum(data[:, :nout].astype(np.float64), axis=0)
    np.testing.assert_allclose(out[0], ref, rtol=0, atol=1e-11)
    # constant input v gives C*v everywhere (Section 4: all elements the same value)
    const = np.full_like(data, 0.75)
    outc = oracle.dedisperse(const, d, nout)
    assert np.all(outc == wl.nchans * 0.75)


def test_integer_and_half_paths_agree_with_float_path():
    wl = synth.workload("small_f32")
    x = synth.noise_f32(wl.nchans, 2048, seed=3)
    dms = wl.dm_list[:16]
    d, m = oracle.delays(wl.nchans, wl.fch1, wl.foff, wl.tsamp, dms)
    nout = 2048 - m
    q = synth.quantize_u8(x)
    oi = oracle.dedisperse(q, d, nout)
    of = oracle.dedisperse(q.astype(np.float32), d, nout)
    assert oi.dtype == np.int64
    assert np.array_equal(oi.astype(np.float64), of)
    h = synth.to_f16_bits(x)
    oh = oracle.dedisperse(h, d, nout)
    oh_ref = oracle.dedisperse(h.view(np.float16).astype(np.float32), d, nout)
    assert np.array_equal(oh, oh_ref)


# --------------------------------------------- statistics and threshold search

def test_stats_match_numpy():
    rng = np.random.default_rng(5)
    x = rng.standard_normal((37, 1001)) * 3.0 + 10.0
    mu, sg = oracle.stats(x)
    assert abs(mu - np.mean(x)) < 1e-12 * abs(np.mean(x))
    assert abs(sg - np.std(x)) < 1e-12 * np.std(x)
    xi = rng.integers(0, 200000, size=(13, 999)).astype(np.int64)
    mu, sg = oracle.stats(xi)
    assert abs(mu - np.mean(xi.astype(np.float64))) < 1e-9
    assert abs(sg - np.std(xi.astype(np.float64))) < 1e-9 * np.std(xi.astype(np.float64))


def _search_by_convolution(out, widths, mu, sigma, k):
    res = set()
    for i in range(out.shape[0]):
        for wi, w in enumerate(widths):
            b = np.convolve(out[i].astype(np.float64), np.ones(w), mode="valid")
            thr = w * mu + k * sigma * math.sqrt(w)
            for t in np.nonzero(b > thr)[0]:
                res.add((i, int(t), wi))
    return res


def test_search_matches_convolution():
    rng = np.random.default_rng(9)
    out = rng.standard_normal((5, 3000))
    out[1, 100:104] += 6.0
    out[3, 2990:3000] += 4.0                 # near the end: windows must not cross it
    out[4, 0] += 9.0
    widths = [1, 2, 4, 8, 3]
    mu, sg = oracle.stats(out)
    k = 4.0
    got = oracle.search(out, widths, mu, sg, k)
    ref = _search_by_convolution(out, widths, mu, sg, k)
    assert {(int(r["dm_idx"]), int(r["t"]), int(r["width_idx"])) for r in got} == ref
    keys = [(int(r["dm_idx"]), int(r["t"]), int(r["width_idx"])) for r in got]
    assert keys == sorted(keys)
    for r in got:
        w = widths[r["width_idx"]]
        b = out[r["dm_idx"], r["t"]:r["t"] + w].sum()
        assert abs(r["value"] - b) < 1e-9
        assert abs(r["snr"] - (b - w * mu) / (sg * math.sqrt(w))) < 1e-9
    # integer path, exact
    oi = np.rint(out * 100).astype(np.int64)
    mu, sg = oracle.stats(oi)
    got = oracle.search(oi, widths, mu, sg, k)
    ref = _search_by_convolution(oi, widths, mu, sg, k)
    assert {(int(r["dm_idx"]), int(r["t"]), int(r["width_idx"])) for r in got} == ref


def test_strict_threshold_and_hand_example():
    # mu = 0.2, sigma = 0.4 for [0,0,0,0,1]; k = 2 -> T_1 = 1.0: 1.0 is NOT above it
    out = np.array([[0.0, 0.0, 0.0, 0.0, 1.0]])
    mu, sg = oracle.stats(out)
    assert abs(mu - 0.2) < 1e-15 and abs(sg - 0.4) < 1e-15
    assert len(oracle.search(out, [1], mu, sg, 2.0)) == 0
    got = oracle.search(out, [1], mu, sg, 1.999)
    assert [(int(r["dm_idx"]), int(r["t"])) for r in got] == [(0, 4)]


# ------------------------------------------------------- injected pulses (Sec. 4)

def test_small_workload_pulse_recovered():
    wl = synth.workload("small_f32")
    data = synth.noise_f32(wl.nchans, wl.nsamp, seed=wl.seed)
    dms = wl.dm_list
    d, m = oracle.delays(wl.nchans, wl.fch1, wl.foff, wl.tsamp, dms)
    pulse = synth.Pulse(dm=float(dms[30]), t0=4000, width=4, amp=5.0)
    synth.inject_pulses(data, [pulse], lambda dm: oracle.delays(
        wl.nchans, wl.fch1, wl.foff, wl.tsamp, [dm])[0][0], wl.nsamp)
    nout = wl.nsamp - m
    out = oracle.dedisperse(data, d, nout)
    mu, sg = oracle.stats(out)
    # the mean: the pulse's samples each enter every DM row whose window holds
    # them (counted exactly here), plus noise whose mean over a row's window
    # of one channel has spread 1/sqrt(nout), summed over C channels
    dp = oracle.delays(wl.nchans, wl.fch1, wl.foff, wl.tsamp, [pulse.dm])[0][0]
    hits = 0
    for i in range(len(dms)):
        for j in range(pulse.width):
            t = pulse.t0 + dp + j - d[i]
            hits += int(np.sum((t >= 0) & (t < nout)))
    mu_pulse = pulse.amp * hits / (len(dms) * nout)
    assert abs(mu - mu_pulse) < 4 * math.sqrt(wl.nchans / nout), (mu, mu_pulse)
    assert abs(sg - math.sqrt(wl.nchans)) < 0.1 * math.sqrt(wl.nchans)
    cands = oracle.search(out, list(wl.widths), mu, sg, wl.sigma)
    best = cands[np.argmax(cands["snr"])]
    assert (int(best["dm_idx"]), int(best["t"]), int(best["width_idx"])) == (30, 4000, 2)
    expect = 4 * wl.nchans * 5.0 / (sg * 2.0)       # B_4 signal over sigma*sqrt(4)
    assert abs(best["snr"] - expect) < 0.05 * expect


def test_table2_fake_pulsar_snr(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "e1_fake_pulsar.json")))
    nch, ftop, bw, ts = g["nchans"], g["ftop_mhz"], g["chan_bw_mhz"], g["tsamp_s"]
    foff = -bw
    dms = 72.0 + np.arange(61, dtype=np.float64) * g["dm_step"]     # 72.0 .. 78.0
    d, m = oracle.delays(nch, ftop, foff, ts, dms)
    dpsr, _ = oracle.delays(nch, ftop, foff, ts, [g["pulsar_dm"]])
    assert int(dpsr[0].max()) == g["delay_bottom_channel_at_dm75_samples"]
    # the stored value is Eq. 1 worked by hand; re-derive it in exact rationals
    exact = _exact_delay(ftop, foff, nch, ts, g["pulsar_dm"], nch - 1)
    assert _round_half_away(exact) == g["delay_bottom_channel_at_dm75_samples"]
    width = int(round(g["period_ms"] * g["duty_cycle"] / (ts * 1e3)))      # ~61 samples
    nsamp = m + 2048
    data = synth.noise_f32(nch, nsamp, seed=75)
    synth.inject_pulses(data, [synth.Pulse(dm=g["pulsar_dm"], t0=900, width=width,
                                           amp=g["pulse_height"])],
                        lambda dm: dpsr[0], nsamp)
    out = oracle.dedisperse(data, d, nsamp - m)
    i75 = int(np.argmin(np.abs(dms - g["pulsar_dm"])))
    seg = out[i75, 900:900 + width]
    snr_per_sample = seg.mean() / math.sqrt(nch)
    assert abs(snr_per_sample - g["integrated_snr_per_sample"]) < 0.8
    mu, sg = oracle.stats(out)
    cands = oracle.search(out, [1, 16, 64], mu, sg, g["detect_snr"])
    best = cands[np.argmax(cands["snr"])]
    assert abs(int(best["dm_idx"]) - i75) <= 1
    assert 900 - 64 <= int(best["t"]) <= 900 + width
