"""GPU parity of subband de-dispersion (Section 3.2) through the C ABI against
the subband oracle: plan tables bit-equal; uint8 output bit-exact; float
output within 1e-5 * nchans; mu/sigma; candidates identical outside the gray
zone.  Plus the cases where the method is exact against the brute-force GPU
path, edge shapes, and sampled points of the full LOFAR-like beam."""
import math

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


def run_subband(nch, fch1, foff, tsamp, nsamp, dms, G, nsub, widths, sigma, dtype="f32", seed=0,
                pulses=(), pitch=None, check_cands=True, max_gray=0):
    arr, _ = make_input(nch, nsamp, fch1, foff, tsamp, seed, pulses, dtype, pitch)
    pitch = arr.shape[1]
    plan = dd.SubbandPlan(nch, fch1, foff, tsamp, dms, G, nsub, widths, sigma, DTYPES[dtype], nsamp)
    nom_o, d1_o, d2_o, m_o = oracle.subband_tables(nch, fch1, foff, tsamp, dms, G, nsub)
    nom, d1, d2 = plan.tables()
    assert np.array_equal(nom, nom_o)
    assert np.array_equal(d1.astype(np.int64), d1_o) and np.array_equal(d2.astype(np.int64), d2_o)
    assert plan.maxshift == m_o and plan.nsamp_out == nsamp - m_o
    nout = plan.nsamp_out
    out = torch.empty(len(dms) * nout, dtype=torch.int32 if dtype == "u8" else torch.float32,
                      device="cuda")
    plan.execute(_dev(arr), pitch, out)
    cands, total = plan.search(out, capacity=1 << 18)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(len(dms), nout)
    ora = oracle.subband_dedisperse(arr, d1_o, d2_o, G, nout)
    if dtype == "u8":
        assert np.array_equal(got.astype(np.int64), ora)
    else:
        err = np.max(np.abs(got.astype(np.float64) - ora))
        assert err <= fp_tol(nch), err
    mu_g, sg_g = plan.stats()
    mu_o, sg_o = oracle.stats(ora)
    if dtype == "u8":
        assert abs(mu_g - mu_o) <= 1e-12 * max(1.0, abs(mu_o))
        assert abs(sg_g - sg_o) <= 1e-12 * max(1.0, sg_o)
    else:
        assert abs(mu_g - mu_o) <= fp_tol(nch)
        assert abs(sg_g - sg_o) <= 1e-5 * max(1.0, sg_o)
    assert total == len(cands)
    if check_cands:
        eps = 0.0 if dtype == "u8" else fp_tol(nch)
        res = compare_candidates(cands, ora, list(widths), mu_g, sg_g, mu_o, sg_o, sigma, eps)
        assert res[1] <= max_gray, f"{res[1]} gray-zone points"
    plan.close()
    return cands, got, ora


@pytest.mark.parametrize("G,nsub", [(5, 16), (8, 4), (3, 32)])
@pytest.mark.parametrize("dtype", ["f32", "u8", "f16"])
def test_small_workload(dtype, G, nsub):
    wl = SMALL
    pulse = [synth.Pulse(dm=float(wl.dm_list[32]), t0=4000, width=4, amp=5.0)]
    cands, got, ora = run_subband(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.nsamp, wl.dm_list, G, nsub,
                                  wl.widths, wl.sigma, dtype, seed=wl.seed, pulses=pulse)
    # the pulse is recovered near its DM and time; off its nominal DM the
    # channels are misaligned by up to e samples, which can move the peak
    _, d1, d2, _ = oracle.subband_tables(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list, G, nsub)
    df, _ = oracle.delays(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list)
    cs = wl.nchans // nsub
    e = int(np.abs(d2[32][np.arange(wl.nchans) // cs] + d1[32 // G] - df[32]).max())
    best = cands[np.argmax(cands["snr"])]
    assert abs(int(best["dm_idx"]) - 32) <= G and abs(int(best["t"]) - 4000) <= e + 4


@pytest.mark.parametrize("dtype", ["u8", "f32"])
def test_exact_cases_match_brute_force_gpu(dtype):
    # one channel per subband, and one DM per group: the GPU subband output is
    # the GPU brute-force output (bit for bit for uint8)
    wl = SMALL
    arr, _ = make_input(wl.nchans, wl.nsamp, wl.fch1, wl.foff, wl.tsamp, 9, (), dtype)
    bf = dd.Plan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list, wl.widths, wl.sigma, DTYPES[dtype],
                 wl.nsamp)
    tdt = torch.int32 if dtype == "u8" else torch.float32
    ob = torch.empty(wl.ndm * bf.nsamp_out, dtype=tdt, device="cuda")
    x = _dev(arr)
    bf.execute(x, wl.nsamp, ob)
    ref = ob.view(wl.ndm, -1)
    for G, nsub in ((4, wl.nchans), (1, 8)):
        sp = dd.SubbandPlan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list, G, nsub, wl.widths,
                            wl.sigma, DTYPES[dtype], wl.nsamp)
        assert sp.maxshift == bf.maxshift
        os_ = torch.empty(wl.ndm * sp.nsamp_out, dtype=tdt, device="cuda")
        sp.execute(x, wl.nsamp, os_)
        torch.cuda.synchronize()
        got = os_.view(wl.ndm, -1)
        if dtype == "u8":
            assert bool(torch.equal(got, ref))
        else:
            assert float((got - ref).abs().max()) <= fp_tol(wl.nchans)
        sp.close()
    bf.close()


EDGE = [
    # nchans, nsamp beyond maxshift, dms, G, nsub, foff sign, pitch pad (elements)
    (64, 700, [0.05 * i for i in range(70)], 7, 8, -1, 0),        # ragged DM blocks and groups
    (96, 333, [0.25 * i for i in range(40)], 6, 12, 1, 4),        # ascending band, padded pitch
    (32, 100, [0.4 * i for i in range(9)], 4, 1, -1, 0),          # one subband
    (128, 1500, [0.1 * i for i in range(33)], 33, 8, -1, 0),      # one group, 33 trials
    (48, 50, [0.0, 0.0, 0.3, 0.3, 0.9], 2, 6, -1, 0),              # repeated DMs, tiny output
]


@pytest.mark.parametrize("case", range(len(EDGE)))
@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_edge_shapes(case, dtype):
    nch, extra, dms, G, nsub, sgn, pad = EDGE[case]
    foff = sgn * 0.1953125
    fch1 = 150.0 if sgn < 0 else 150.0 - (nch - 1) * 0.1953125
    _, _, _, m = oracle.subband_tables(nch, fch1, foff, 327.68e-6, dms, G, nsub)
    nsamp = m + extra
    al = 16 if dtype == "u8" else 4
    pitch = (nsamp + pad + al - 1) // al * al
    run_subband(nch, fch1, foff, 327.68e-6, nsamp, dms, G, nsub, [1, 2, 4], 3.0, dtype, seed=case + 50,
                pitch=pitch, max_gray=2)


def test_rejects_bad_arguments():
    wl = SMALL
    with pytest.raises(dd.DDError):
        dd.SubbandPlan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list, 4, 7, wl.widths, wl.sigma,
                       dd.DD_F32, wl.nsamp)                       # 128 % 7 != 0
    with pytest.raises(dd.DDError):
        dd.SubbandPlan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list, 0, 8, wl.widths, wl.sigma,
                       dd.DD_F32, wl.nsamp)
    sp = dd.SubbandPlan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list, 4, 8, wl.widths, wl.sigma,
                        dd.DD_F32, wl.nsamp)
    x = torch.zeros(wl.nchans * wl.nsamp + 1, device="cuda")
    out = torch.empty(wl.ndm * sp.nsamp_out, device="cuda")
    with pytest.raises(dd.DDError):
        sp.execute(x[1:], wl.nsamp, out)                          # misaligned rows
    sp.close()


def test_lofar_full_size_sampled():
    # the benchmark's subband configuration: 1024 channels in 32 subbands,
    # 2000 fine DMs in groups of 24 (1.2 pc/cm3 per nominal DM)
    wl = synth.workload("lofar_f32")
    G, nsub = 24, 32
    x = synth.noise_f32(wl.nchans, wl.nsamp, seed=wl.seed)
    sp = dd.SubbandPlan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list, G, nsub, wl.widths, wl.sigma,
                        dd.DD_F32, wl.nsamp)
    nom_o, d1_o, d2_o, m_o = oracle.subband_tables(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list,
                                                   G, nsub)
    assert sp.maxshift == m_o
    nout = sp.nsamp_out
    out = torch.empty(wl.ndm * nout, dtype=torch.float32, device="cuda")
    sp.execute(torch.from_numpy(x).cuda(), wl.nsamp, out)
    cands, total = sp.search(out, capacity=1 << 20)
    torch.cuda.synchronize()
    out = out.view(wl.ndm, nout)
    rng = np.random.default_rng(99)
    js = list(rng.integers(0, wl.ndm, 1500)) + [0, 23, 24, 31, 32, 1999, 1999]
    ts = list(rng.integers(0, nout, 1500)) + [0, 511, 512, nout - 1, 0, nout - 512, nout - 1]
    got = out[torch.tensor(js, device="cuda"), torch.tensor(ts, device="cuda")].cpu().numpy()
    for k, (j, t) in enumerate(zip(js, ts)):
        ref = oracle.subband_point_f32(x, d1_o, d2_o, G, int(j), int(t))
        assert abs(float(got[k]) - ref) <= fp_tol(wl.nchans), (j, t, float(got[k]), ref)
    mu, sg = sp.stats()
    assert abs(sg - math.sqrt(wl.nchans)) <= 0.05 * math.sqrt(wl.nchans)
    sp.close()
