"""GPU parity of survey plans (binning + subband passes, Section 3.2 and the
Table 1 / Table 4 plans) through the C ABI against the oracle: each pass =
oracle binning (FP64) then the subband oracle at the binned sampling time."""
import numpy as np
import pytest

import oracle
import synth
from ddhelpers import compare_candidates, fp_tol, make_input

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1107_2516_gb300 as dd
from paper_1107_2516_gb300 import build as ddbuild

DTYPES = {"f32": dd.DD_F32, "u8": dd.DD_U8, "f16": dd.DD_F16}
SMALL = synth.workload("small_f32")
SMALL_PLAN = ((0.0, 2.0, 0.1, 1, 0.5), (2.0, 4.0, 0.2, 2, 1.0), (4.0, 6.4, 0.4, 4, 1.6))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ddbuild.build()
    dd.load()


def _dev(arr):
    if arr.dtype == np.uint16:
        arr = arr.view(np.int16)
    return torch.from_numpy(np.ascontiguousarray(arr)).cuda()


def _pass_oracle(arr, nsamp, wl, plan_row, nsub, t_lo=0, n=None):
    """Oracle output of one pass for output times [t_lo, t_lo + n)."""
    dms, nb, G = oracle.survey_passes([plan_row])[0]
    xb = oracle.bin_samples(arr, nb, nsamp)
    nom, d1, d2, m = oracle.subband_tables(wl.nchans, wl.fch1, wl.foff, wl.tsamp * nb, dms, G, nsub)
    nout = xb.shape[1] - m
    n = nout - t_lo if n is None else n
    return oracle.subband_dedisperse(np.ascontiguousarray(xb[:, t_lo:]), d1, d2, G, n), nout, m


@pytest.mark.parametrize("dtype", ["f32", "u8", "f16"])
def test_small_survey_all_passes(dtype):
    wl, nsub = SMALL, 16
    pulse = [synth.Pulse(dm=2.5, t0=3000, width=8, amp=4.0)]
    arr, _ = make_input(wl.nchans, wl.nsamp, wl.fch1, wl.foff, wl.tsamp, wl.seed, pulse, dtype)
    sp = dd.SurveyPlan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, SMALL_PLAN, nsub, wl.widths, wl.sigma,
                       DTYPES[dtype], wl.nsamp)
    outs = []
    for i, (ndm, nb, G, m, nout) in enumerate(sp.passes):
        dms, nb_o, G_o = oracle.survey_passes([SMALL_PLAN[i]])[0]
        assert (ndm, nb, G) == (len(dms), nb_o, G_o)
        assert np.array_equal(sp.dm_list(i), np.asarray(dms))
        int_out = dtype == "u8" and nb == 1
        outs.append(torch.empty(ndm * nout, device="cuda", dtype=torch.int32 if int_out else torch.float32))
    sp.execute(_dev(arr), wl.nsamp, outs)
    for i, (ndm, nb, G, m, nout) in enumerate(sp.passes):
        cands, total = sp.search(i, outs[i], capacity=1 << 18)
        torch.cuda.synchronize()
        ora, nout_o, m_o = _pass_oracle(arr, wl.nsamp, wl, SMALL_PLAN[i], nsub)
        assert (m, nout) == (m_o, nout_o)
        got = outs[i].cpu().numpy().reshape(ndm, nout)
        if dtype == "u8" and nb == 1:
            assert np.array_equal(got.astype(np.int64), ora.astype(np.int64))
            eps = 0.0
        else:
            if dtype == "u8":
                # binned 8-bit data are averages near 128, not unit-variance:
                # FP32 rounding bound of bin + two summation stages, each
                # partial sum at most nchans * 255
                eps = (wl.nchans // nsub + nsub + nb) * 2.0 ** -24 * wl.nchans * 255
            else:
                eps = fp_tol(wl.nchans)
            err = np.max(np.abs(got.astype(np.float64) - ora))
            assert err <= eps, (i, err)
        mu_g, sg_g = sp.stats(i)
        mu_o, sg_o = oracle.stats(ora)
        assert abs(mu_g - mu_o) <= max(eps, 1e-9 * abs(mu_o) + 1e-12)
        assert abs(sg_g - sg_o) <= 1e-5 * max(1.0, sg_o)
        res = compare_candidates(cands, ora, list(wl.widths), mu_g, sg_g, mu_o, sg_o, wl.sigma, eps)
        assert res[1] <= 2
    sp.close()


def test_table4_plan_on_the_survey_beam_sampled():
    # the paper's survey plan (Table 4) on a 60 s, 300 MHz, 16 MHz, 1024-channel
    # beam: every pass checked on output windows at the start, middle and end
    wl, nsub = synth.workload("survey_f32"), 32
    x = synth.noise_f32(wl.nchans, wl.nsamp, seed=wl.seed)
    sp = dd.SurveyPlan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, synth.SURVEY_PLAN, nsub, wl.widths, wl.sigma,
                       dd.DD_F32, wl.nsamp)
    assert [p[0] for p in sp.passes] == [1782, 696, 624] and [p[1] for p in sp.passes] == [1, 2, 4]
    outs = [torch.empty(p[0] * p[4], device="cuda") for p in sp.passes]
    sp.execute(torch.from_numpy(x).cuda(), wl.nsamp, outs)
    torch.cuda.synchronize()
    for i, (ndm, nb, G, m, nout) in enumerate(sp.passes):
        got = outs[i].view(ndm, nout)
        for t_lo in (0, nout // 2, nout - 48):
            ora, nout_o, _ = _pass_oracle(x, wl.nsamp, wl, synth.SURVEY_PLAN[i], nsub, t_lo, 48)
            assert nout_o == nout
            g = got[:, t_lo:t_lo + 48].cpu().numpy().astype(np.float64)
            assert np.max(np.abs(g - ora)) <= fp_tol(wl.nchans), (i, t_lo)
    sp.close()


def test_rejects_bad_passes():
    wl = SMALL
    for bad in (((1.0, 0.5, 0.1, 1, 0.5),), ((0.0, 1.0, 0.0, 1, 0.5),), ((0.0, 1.0, 0.1, 0, 0.5),)):
        with pytest.raises(dd.DDError):
            dd.SurveyPlan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, bad, 16, wl.widths, wl.sigma, dd.DD_F32,
                          wl.nsamp)
