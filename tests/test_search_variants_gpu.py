"""GPU parity of the per-DM-row search variant through the C ABI against the
oracle's per-row search (row statistics and candidates, gray-zone rule per
row), with a DM-dependent baseline that the whole-buffer statistics would
mistake for signal."""
import numpy as np
import pytest

import oracle
import synth
from ddhelpers import compare_candidates, fp_tol, make_input

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1107_2516_gb300 as dd
from paper_1107_2516_gb300 import build as ddbuild

SMALL = synth.workload("small_f32")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ddbuild.build()
    dd.load()


@pytest.mark.parametrize("dtype", ["f32", "u8"])
@pytest.mark.parametrize("widths", [(1, 2, 4, 8), (1, 3, 7)])
def test_per_row_statistics_match_oracle(dtype, widths):
    wl = SMALL
    pulse = [synth.Pulse(dm=float(wl.dm_list[30]), t0=4000, width=4, amp=5.0)]
    arr, _ = make_input(wl.nchans, wl.nsamp, wl.fch1, wl.foff, wl.tsamp, wl.seed, pulse, dtype)
    # a baseline ramp along the channels shifts low-DM and high-DM rows
    # differently (the rows sum different sample ranges of a ramp in time)
    ramp = (np.arange(wl.nsamp) / wl.nsamp)[None, :]
    if dtype == "f32":
        arr = (arr + 0.5 * ramp).astype(np.float32)
    else:
        arr = np.clip(arr.astype(np.int32) + (8 * ramp).astype(np.int32), 0, 255).astype(np.uint8)
    plan = dd.Plan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list, widths, wl.sigma,
                   dd.DD_U8 if dtype == "u8" else dd.DD_F32, wl.nsamp)
    plan.set_search_stats(True)
    nout = plan.nsamp_out
    out = torch.empty(wl.ndm * nout, dtype=torch.int32 if dtype == "u8" else torch.float32, device="cuda")
    plan.execute(torch.from_numpy(arr).cuda(), wl.nsamp, out)
    cands, total = plan.search(out, capacity=1 << 18)
    mu_g, sg_g = plan.row_stats()
    d, m = oracle.delays(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list)
    ora = oracle.dedisperse(arr, d, nout)
    c_o, mu_o, sg_o = oracle.search_per_row(ora, list(widths), wl.sigma)
    eps = 0.0 if dtype == "u8" else fp_tol(wl.nchans)
    tol_mu = 1e-12 if dtype == "u8" else fp_tol(wl.nchans)
    assert np.max(np.abs(mu_g - mu_o)) <= tol_mu * max(1.0, np.abs(mu_o).max())
    assert np.max(np.abs(sg_g - sg_o) / sg_o) <= 1e-5
    gray = 0
    for j in range(wl.ndm):
        cj = cands[cands["dm_idx"] == j].copy()
        cj["dm_idx"] = 0
        res = compare_candidates(cj, ora[j:j + 1], list(widths), mu_g[j], sg_g[j], mu_o[j], sg_o[j],
                                 wl.sigma, eps)
        gray += res[1]
        if len(cj):
            # per-row S/N
            w = np.asarray(widths)[cj["width_idx"]]
            snr = (cj["value"] - w * mu_g[j]) / (sg_g[j] * np.sqrt(w))
            assert np.allclose(cj["snr"], snr, rtol=1e-5, atol=1e-4)
    assert gray <= 2
    best = cands[np.argmax(cands["snr"])]
    assert (int(best["dm_idx"]), int(best["t"])) == (30, 4000)
    # whole-buffer statistics are restored
    plan.set_search_stats(False)
    c2, n2 = plan.search(out, capacity=1 << 18)
    mu, sg = plan.stats()
    mu_all, sg_all = oracle.stats(ora)
    assert abs(mu - mu_all) <= max(tol_mu * max(1.0, abs(mu_all)), 1e-9)
    plan.close()
