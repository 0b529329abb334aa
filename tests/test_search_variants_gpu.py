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
    # the strongest candidate is the oracle's, on the pulse's DM and
    # overlapping it (with widths 3 and 7 several windows of the 4-sample
    # pulse hold the same signal; the noise decides between them)
    best = cands[np.argmax(cands["snr"])]
    best_o = c_o[np.argmax(c_o["snr"])]
    key = (int(best["dm_idx"]), int(best["t"]), int(best["width_idx"]))
    assert key == (int(best_o["dm_idx"]), int(best_o["t"]), int(best_o["width_idx"]))
    w = widths[key[2]]
    assert key[0] == 30 and key[1] <= 4000 + 3 and key[1] + w - 1 >= 4000
    # whole-buffer statistics are restored
    plan.set_search_stats(False)
    c2, n2 = plan.search(out, capacity=1 << 18)
    mu, sg = plan.stats()
    mu_all, sg_all = oracle.stats(ora)
    assert abs(mu - mu_all) <= max(tol_mu * max(1.0, abs(mu_all)), 1e-9)
    plan.close()


@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_server_boundary_search_matches_oracle(dtype):
    # a beam streamed in 512-sample chunks with a pulse straddling a chunk
    # boundary; per searched chunk: in-chunk and boundary candidates against
    # the oracle's streaming search (gray-zone rule)
    nch, fch1, foff, tsamp = 64, 150.0, -0.390625, 327.68e-6
    dms = [0.1 * i for i in range(40)]
    widths = (1, 2, 4, 8, 16)
    chunk, K = 512, 9
    d, M = oracle.delays(nch, fch1, foff, tsamp, dms)
    total = K * chunk
    x = synth.noise_f32(nch, total, 21)
    nprime = (M + chunk - 1) // chunk
    # stream time of the first output of chunk k is k*chunk - M; put the pulse
    # across the boundary between searched chunks nprime+2 and nprime+3
    tb = (nprime + 3) * chunk - M
    synth.inject_pulses(x, [synth.Pulse(dm=dms[20], t0=tb - 5, width=10, amp=1.2)],
                        lambda dm: oracle.delays(nch, fch1, foff, tsamp, [dm])[0][0], total)
    if dtype == "u8":
        x = synth.quantize_u8(x)
    srv = dd.Server(1 << 30, nworkers=1)
    bid = srv.add_beam(nch, fch1, foff, tsamp, dms, widths, 5.0, dd.DD_U8 if dtype == "u8" else dd.DD_F32, chunk)
    srv.set_boundary_search(bid, True)
    got = {}
    for k in range(K):
        ck = torch.from_numpy(np.ascontiguousarray(x[:, k * chunk:(k + 1) * chunk])).pin_memory()
        srv.submit(bid, ck, chunk, k)
        r = None
        for _ in range(300):
            hit = [q for q in srv.poll(wait_ms=50) if q["seq"] == k]
            if hit:
                r = hit[0]
                break
        assert r is not None and r["status"] in (0, dd.DD_PRIMING)
        if r["status"] == 0:
            got[k] = (srv.candidates(bid, k), r["mu"], r["sigma"])
    ora_full = oracle.dedisperse(x, d, total - M)
    ks = sorted(got)
    assert ks[0] == nprime
    chunks = [ora_full[:, k * chunk - M:(k + 1) * chunk - M] for k in ks]
    ora = oracle.search_stream(chunks, widths, 5.0, carry=True)
    eps = 0.0 if dtype == "u8" else fp_tol(nch)
    L = max(widths) - 1
    crossing = 0
    for ci, k in enumerate(ks):
        g, mu_g, sg_g = got[k]
        mu_o, sg_o = oracle.stats(chunks[ci])
        inside = g[g["t"] >= 0]
        res = compare_candidates(inside, chunks[ci], list(widths), mu_g, sg_g, mu_o, sg_o, 5.0, eps)
        assert res[1] <= 2
        gb = {(int(c["dm_idx"]), int(c["t"]), int(c["width_idx"])) for c in g if c["t"] < 0}
        ob = {(int(c["dm_idx"]), int(c["t"]), int(c["width_idx"])): float(c["value"]) for c in ora[ci] if c["t"] < 0}
        if ci == 0:
            assert not gb                              # no previous searched chunk
            continue
        prev = chunks[ci - 1]
        for j in range(len(dms)):
            xx = np.concatenate([prev[j, -L:], chunks[ci][j, :L]])
            for p, w in enumerate(widths):
                for i in range(max(0, L - w + 1), L):
                    b = float(np.sum(xx[i:i + w]))
                    T = oracle.threshold(w, mu_o, sg_o, 5.0)
                    key = (j, i - L, p)
                    if abs(b - T) <= w * eps + abs(w * (mu_g - mu_o)) + 5.0 * abs(sg_g - sg_o) * np.sqrt(w) + 1e-9:
                        continue                       # gray zone
                    assert (key in gb) == (b > T), (k, key, b, T)
                    assert (key in ob) == (b > T)
        crossing += len(gb)
        for c in g[g["t"] < 0]:                        # S/N of boundary candidates
            w = widths[int(c["width_idx"])]
            assert abs(float(c["snr"]) - (float(c["value"]) - w * mu_g) / (sg_g * np.sqrt(w))) <= 1e-4
    assert crossing > 0
    srv.close()
