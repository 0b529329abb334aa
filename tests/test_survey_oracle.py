"""Pins of the binning and survey-pass oracle (Section 3.2 binning, Table 1 /
Table 4 survey plans): closed forms of the bin average, a numpy restatement,
the Table 4 plan's pass sizes from its printed columns, and the reduction of a
bin-1 pass to the subband oracle."""
import json
import os

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def test_bin_one_is_identity():
    x = synth.noise_f32(5, 301, 1)
    assert np.array_equal(oracle.bin_samples(x, 1), x.astype(np.float64))


def test_bin_constant_and_ramp_closed_forms():
    c = np.full((3, 100), 2.5, np.float32)
    assert np.all(oracle.bin_samples(c, 7) == 2.5)
    ramp = np.tile(np.arange(1000, dtype=np.float32), (2, 1))
    for nb in (2, 3, 4, 16):
        got = oracle.bin_samples(ramp, nb)
        i = np.arange(1000 // nb)
        assert got.shape == (2, 1000 // nb)
        assert np.array_equal(got[1], nb * i + (nb - 1) / 2.0)      # mean of nb*i .. nb*i+nb-1


@pytest.mark.parametrize("dtype", ["f32", "u8", "f16"])
def test_bin_numpy_restatement(dtype):
    x = synth.noise_f32(4, 1003, 2)
    if dtype == "u8":
        x = synth.quantize_u8(x)
        ref_src = x.astype(np.float64)
    elif dtype == "f16":
        x = synth.to_f16_bits(x)
        ref_src = x.view(np.float16).astype(np.float64)
    else:
        ref_src = x.astype(np.float64)
    for nb in (2, 5):
        n = 1003 // nb
        ref = ref_src[:, :n * nb].reshape(4, n, nb).sum(axis=2) / nb
        assert np.max(np.abs(oracle.bin_samples(x, nb) - ref)) <= 1e-12


def test_table4_plan_reading():
    plan = json.load(open(os.path.join(HERE, "golden", "survey_plan_table4.json")))
    passes = oracle.survey_passes(plan["passes"])
    # (high - low) / step and sub step / step of the printed columns
    assert [len(d) for d, _, _ in passes] == [1782, 696, 624]
    assert [b for _, b, _ in passes] == [1, 2, 4]
    assert [g for _, _, g in passes] == [22, 24, 24]
    for (d0, _, _), (d1, _, _), p in zip(passes, passes[1:], plan["passes"][1:]):
        assert abs(d0[-1] + (d0[1] - d0[0]) - p[0]) < 1e-9          # passes tile the DM range
    assert abs(passes[-1][0][-1] - (150.66 - 0.10)) < 1e-9


def test_bin_one_pass_is_the_subband_oracle():
    nch, fch1, foff, tsamp = 64, 150.0, -0.1953125, 327.68e-6
    dms = [0.1 * i for i in range(20)]
    nom, d1, d2, m = oracle.subband_tables(nch, fch1, foff, tsamp, dms, 5, 8)
    x = synth.noise_f32(nch, 800, 3)
    nout = 800 - m
    via_bin = oracle.subband_dedisperse(oracle.bin_samples(x, 1), d1, d2, 5, nout)
    direct = oracle.subband_dedisperse(x, d1, d2, 5, nout)
    assert np.array_equal(via_bin, direct)


def test_binned_pulse_energy_within_one_bin_of_its_delay():
    # a unit square pulse 2*nb raw samples wide per channel, starting on a bin
    # boundary at the raw delays of DM dm: binned at nb it is two bins of 1.0
    # per channel; de-dispersed at tsamp*nb (G = 1, one channel per subband:
    # brute force) each channel lands within one bin of t0/nb (the rounded
    # binned delay vs the raw delay), so the 4 bins around t0/nb hold exactly
    # 2*nchans and no other bin holds anything
    nch, fch1, foff, tsamp, nb = 32, 150.0, -0.390625, 163.84e-6, 4
    dm = 12.0
    draw, _ = oracle.delays(nch, fch1, foff, tsamp, [dm])
    x = np.zeros((nch, 4096), np.float32)
    t0 = 400
    for c in range(nch):
        s = (t0 + draw[0, c]) // nb * nb
        x[c, s:s + 2 * nb] = 1.0
    xb = oracle.bin_samples(x, nb)
    nom, d1, d2, m = oracle.subband_tables(nch, fch1, foff, tsamp * nb, [dm], 1, nch)
    out = oracle.subband_dedisperse(xb, d1, d2, 1, xb.shape[1] - m)[0]
    b0 = t0 // nb
    assert out[b0 - 1:b0 + 3].sum() == 2 * nch
    assert out.sum() == 2 * nch
