"""Pins of the subband oracle (Section 3.2) to things other than itself: the
brute-force oracle (already pinned to Eq. 1 and the Section 3.1 definition) in
the special cases where the two-stage method is exact, a numpy restatement of
the two stages on tiny inputs, the smearing bound on the effective per-channel
delay, and the S/N loss of a noise-free pulse implied by that bound."""
import math

import numpy as np
import pytest

import oracle
import synth

FCH1, FOFF, TSAMP = 150.0, -0.1953125, 327.68e-6


def _data(nch, nsamp, seed, dtype="f32"):
    x = synth.noise_f32(nch, nsamp, seed)
    if dtype == "u8":
        return synth.quantize_u8(x)
    return x


def _brute(data, dms, fch1=FCH1, foff=FOFF, nout=None):
    d, m = oracle.delays(data.shape[0], fch1, foff, TSAMP, dms)
    return oracle.dedisperse(data, d, nout if nout is not None else data.shape[1] - m)


@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_one_channel_per_subband_is_brute_force(dtype):
    # nsub = nchans: every subband is its own reference channel, d1 = 0 and
    # d2 = the brute-force delay, so the two stages are the Section 3.1 sum
    nch, dms = 32, [0.37 * i for i in range(15)]
    nom, d1, d2, m = oracle.subband_tables(nch, FCH1, FOFF, TSAMP, dms, 4, nch)
    assert not d1.any()
    x = _data(nch, 1500, 3, dtype)
    nout = x.shape[1] - m
    sub = oracle.subband_dedisperse(x, d1, d2, 4, nout)
    ref = _brute(x, dms, nout=nout)
    assert np.array_equal(sub, ref)


@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_one_dm_per_group_is_brute_force(dtype):
    # G = 1: the nominal DM is the fine DM, d2 + d1 = d(c, dm) exactly
    nch, dms = 48, [0.21 * i for i in range(11)]
    nom, d1, d2, m = oracle.subband_tables(nch, FCH1, FOFF, TSAMP, dms, 1, 6)
    assert np.array_equal(nom, np.asarray(dms))
    x = _data(nch, 1800, 4, dtype)
    nout = x.shape[1] - m
    sub = oracle.subband_dedisperse(x, d1, d2, 1, nout)
    ref = _brute(x, dms, nout=nout)
    if dtype == "u8":
        assert np.array_equal(sub, ref)
    else:
        assert np.max(np.abs(sub - ref)) <= 1e-9


def test_single_subband_repeats_the_nominal_row():
    # nsub = 1: the reference is the top channel (delay 0), so every fine DM of
    # a group gives the brute-force row of the group's nominal DM
    nch, G, dms = 40, 5, [0.13 * i for i in range(14)]
    nom, d1, d2, m = oracle.subband_tables(nch, FCH1, FOFF, TSAMP, dms, G, 1)
    assert not d2.any()
    x = _data(nch, 1200, 5, "u8")
    nout = x.shape[1] - m
    sub = oracle.subband_dedisperse(x, d1, d2, G, nout)
    dn, _ = oracle.delays(nch, FCH1, FOFF, TSAMP, nom)
    ref = oracle.dedisperse(x, dn, nout)
    for j in range(len(dms)):
        assert np.array_equal(sub[j], ref[j // G])


def test_fine_dm_at_the_nominal_delays_is_exact():
    # a fine DM whose delays equal the nominal DM's (the group centre, G odd)
    nch, G, nsub = 64, 5, 8
    dms = [0.1 * i for i in range(25)]
    nom, d1, d2, m = oracle.subband_tables(nch, FCH1, FOFF, TSAMP, dms, G, nsub)
    df, _ = oracle.delays(nch, FCH1, FOFF, TSAMP, dms)
    dn, _ = oracle.delays(nch, FCH1, FOFF, TSAMP, nom)
    x = _data(nch, 2000, 6, "u8")
    nout = x.shape[1] - max(m, int(df.max()))
    sub = oracle.subband_dedisperse(x, d1, d2, G, nout)
    bf = oracle.dedisperse(x, df, nout)
    hits = 0
    for j in range(len(dms)):
        if np.array_equal(df[j], dn[j // G]):
            assert np.array_equal(sub[j], bf[j])
            hits += 1
    assert hits >= len(dms) // G          # every group's centre


@pytest.mark.parametrize("sign", [-1, 1])
def test_numpy_restatement_of_the_two_stages(sign):
    # stage 1 and stage 2 re-done with numpy fancy indexing from the pinned
    # brute-force delay tables (both band orientations)
    nch, G, nsub = 24, 3, 4
    foff = sign * 0.1953125
    fch1 = FCH1 if sign < 0 else FCH1 - (nch - 1) * 0.1953125
    dms = [0.45 * i for i in range(8)]
    nom, d1, d2, m = oracle.subband_tables(nch, fch1, foff, TSAMP, dms, G, nsub)
    df, _ = oracle.delays(nch, fch1, foff, TSAMP, dms)
    dn, _ = oracle.delays(nch, fch1, foff, TSAMP, nom)
    cs = nch // nsub
    freqs = fch1 + np.arange(nch) * foff
    ref_ch = [int(s * cs + np.argmax(freqs[s * cs:(s + 1) * cs])) for s in range(nsub)]
    K = len(nom)
    assert np.allclose(nom, [(dms[k * G] + dms[min(k * G + G, len(dms)) - 1]) / 2 for k in range(K)])
    x = _data(nch, 700, 7)
    nout = x.shape[1] - m
    exp = np.zeros((len(dms), nout))
    t = np.arange(nout)
    for j in range(len(dms)):
        k = j // G
        for s in range(nsub):
            r = ref_ch[s]
            sub = np.zeros(nout)
            for c in range(s * cs, (s + 1) * cs):
                sub += x[c, t + df[j, r] + dn[k, c] - dn[k, r]].astype(np.float64)
            exp[j] += sub
    got = oracle.subband_dedisperse(x, d1, d2, G, nout)
    assert np.max(np.abs(got - exp)) <= 1e-9


def test_effective_delay_within_the_smearing_bound():
    # effective delay of channel c at fine DM j: d2(j, s(c)) + d1(k(j), c).
    # Exact fractional delays are linear in DM: x(c, dm) = dm * x(c, 1), so
    #   eff - d(c, dm) = d(ref, dm) + d(c, D_k) - d(ref, D_k) - d(c, dm)
    #   |eff - d(c, dm)| <= |dm - D_k| * (x(c,1) - x(ref,1)) + 2
    # (four rounded delays, each within 1/2 of its exact value).
    lw = synth.workload("lofar_f32")
    nch, G, nsub = 1024, 24, 32
    dms = lw.dm_list
    nom, d1, d2, m = oracle.subband_tables(nch, lw.fch1, lw.foff, lw.tsamp, dms, G, nsub)
    df, mf = oracle.delays(nch, lw.fch1, lw.foff, lw.tsamp, dms)
    cs = nch // nsub
    per = np.array([oracle.delay_exact(lw.fch1, lw.foff, nch, lw.tsamp, 1.0, c) for c in range(nch)])
    ref = np.arange(nch) // cs * cs                       # foff < 0: first channel of the subband
    slope = per - per[ref]
    worst, worst_bound = 0, 0.0
    for j in range(0, len(dms), 7):
        k = j // G
        eff = d2[j][np.arange(nch) // cs] + d1[k]
        err = np.abs(eff - df[j])
        bound = abs(dms[j] - nom[k]) * slope + 2.0
        assert np.all(err <= bound + 1e-9), (j, int(np.argmax(err - bound)))
        worst = max(worst, int(err.max()))
        worst_bound = max(worst_bound, float(bound.max()))
    # half a 1.2 pc/cm3 group x the bottom subband's slope spread + rounding
    assert 0 < worst <= worst_bound < 6.5
    assert abs(m - mf) <= worst_bound


def test_pulse_snr_loss_bounded_by_the_smearing():
    # noise-free square pulse of width w at an off-nominal fine DM: the best
    # width-w boxcar of the subband output keeps at least 1 - mean|e_c|/w of
    # the brute-force peak, e_c = each channel's effective-delay error
    nch, G, nsub, w = 256, 9, 16, 8
    dms = [0.5 * i for i in range(36)]
    foff = -0.046875
    nom, d1, d2, m = oracle.subband_tables(nch, FCH1, foff, TSAMP, dms, G, nsub)
    df, mf = oracle.delays(nch, FCH1, foff, TSAMP, dms)
    cs = nch // nsub
    nsamp = max(m, mf) + 600
    for j in (3, 17, 31):                                 # off-centre trials of three groups
        x = np.zeros((nch, nsamp), np.float32)
        t0 = 200
        for c in range(nch):
            x[c, t0 + df[j, c]:t0 + df[j, c] + w] = 1.0
        nout = nsamp - max(m, mf)
        sub = oracle.subband_dedisperse(x, d1, d2, G, nout)[j]
        bf = oracle.dedisperse(x, df[j:j + 1], nout)[0]
        box = lambda r: max(float(np.sum(r[t:t + w])) for t in range(nout - w + 1))
        e = np.abs(d2[j][np.arange(nch) // cs] + d1[j // G] - df[j])
        assert box(bf) == nch * w
        assert box(sub) >= box(bf) * (1.0 - e.mean() / w) - 1e-9
        assert box(sub) <= box(bf)


def test_tables_reject_bad_arguments():
    with pytest.raises(ValueError):
        oracle.subband_tables(30, FCH1, FOFF, TSAMP, [0.0, 1.0], 2, 7)    # 30 % 7 != 0
    with pytest.raises(ValueError):
        oracle.subband_tables(32, FCH1, FOFF, TSAMP, [0.0, 1.0], 0, 4)
