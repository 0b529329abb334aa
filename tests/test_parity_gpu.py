"""GPU parity: libdd (through its C ABI) against the CPU oracle.

Criteria: delay tables bit-equal; uint8 -> int32 output bit-exact; FP32 and
FP16 -> FP32 output within 1e-5 * nchans (unit-variance data); mu/sigma
consistent; candidate lists identical outside the gray zone (points whose
oracle boxcar lies within the FP error bound of the threshold).
"""
import math

import numpy as np
import pytest

import oracle
import synth
from ddhelpers import compare_candidates, fp_tol, keys, make_input

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1107_2516_gb300 as dd
from paper_1107_2516_gb300 import build as ddbuild
from paper_1107_2516_gb300 import dd as ddc

DTYPES = {"f32": dd.DD_F32, "u8": dd.DD_U8, "f16": dd.DD_F16}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ddbuild.build()
    dd.load()


def to_device(arr: np.ndarray):
    if arr.dtype == np.uint16:
        arr = arr.view(np.int16)
    return torch.from_numpy(np.ascontiguousarray(arr)).cuda()


def run_case(nchans, fch1, foff, tsamp, nsamp, dm_list, widths, sigma, dtype="f32", seed=0,
             pulses=(), pitch=None, kernel=0, check_cands=True, max_gray=0, tile=None):
    arr, _ = make_input(nchans, nsamp, fch1, foff, tsamp, seed, pulses, dtype, pitch)
    pitch = arr.shape[1]
    plan = dd.Plan(nchans, fch1, foff, tsamp, dm_list, widths, sigma, DTYPES[dtype], nsamp)
    if kernel:
        plan.set_kernel(kernel)
    if tile is not None:
        plan.set_tile(*tile)
    used_kernel = plan.kernel
    d_o, m_o = oracle.delays(nchans, fch1, foff, tsamp, dm_list)
    assert plan.maxshift == m_o
    assert np.array_equal(plan.delays().astype(np.int64), d_o)
    nout = nsamp - m_o
    assert plan.nsamp_out == nout
    in_dev = to_device(arr)
    out_dev = torch.empty(len(dm_list) * nout, dtype=torch.int32 if dtype == "u8" else torch.float32,
                          device="cuda")
    plan.execute(in_dev, pitch, out_dev)
    cands, total = plan.search(out_dev, capacity=1 << 18)
    torch.cuda.synchronize()
    out = out_dev.cpu().numpy().reshape(len(dm_list), nout)
    ora = oracle.dedisperse(arr, d_o, nout)
    if dtype == "u8":
        assert np.array_equal(out.astype(np.int64), ora)
    else:
        err = np.max(np.abs(out.astype(np.float64) - ora))
        assert err <= fp_tol(nchans), err
    mu_g, sg_g = plan.stats()
    mu_o, sg_o = oracle.stats(ora)
    if dtype == "u8":
        assert abs(mu_g - mu_o) <= 1e-12 * max(1.0, abs(mu_o))
        assert abs(sg_g - sg_o) <= 1e-12 * max(1.0, sg_o)
    else:
        assert abs(mu_g - mu_o) <= fp_tol(nchans)
        assert abs(sg_g - sg_o) <= 1e-5 * max(1.0, sg_o)
    assert total == len(cands)
    res = None
    if check_cands:
        eps = 0.0 if dtype == "u8" else fp_tol(nchans)
        res = compare_candidates(cands, ora, list(widths), mu_g, sg_g, mu_o, sg_o, sigma, eps)
        assert res[1] <= max_gray, f"{res[1]} gray-zone points"
    plan.close()
    return cands, out, ora, res, used_kernel


SMALL = synth.workload("small_f32")


def small_pulse():
    return [synth.Pulse(dm=float(SMALL.dm_list[30]), t0=4000, width=4, amp=5.0)]


@pytest.mark.parametrize("kernel", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("dtype", ["f32", "u8", "f16"])
def test_small_workload_parity(dtype, kernel):
    wl = SMALL
    cands, out, ora, res, used = run_case(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.nsamp,
                                          wl.dm_list, wl.widths, wl.sigma, dtype, seed=wl.seed,
                                          pulses=small_pulse(), kernel=kernel)
    assert used == (kernel or 3)           # default: kernel 5 cannot run this plan, so kernel 3
    best = cands[np.argmax(cands["snr"])]
    assert (int(best["dm_idx"]), int(best["t"]), int(best["width_idx"])) == (30, 4000, 2)


@pytest.mark.parametrize("tile", [(0, 1), (0, 3), (1, 8), (1, 2), (2, 16), (3, 8), (3, 1), (4, 4),
                                  (5, 8), (5, 3), (6, 16), (6, 2), (7, 8), (7, 3), (8, 16), (8, 1),
                                  (9, 8), (9, 1), (10, 4), (11, 8), (11, 1), (12, 8)])
@pytest.mark.parametrize("dtype", ["f32", "u8", "f16"])
def test_small_workload_tile_configs(dtype, tile):
    # every compiled tile configuration of kernels 2-4 and several raster
    # groups (incl. a ragged last group) give the oracle's result
    wl = SMALL
    try:
        cands, out, ora, res, used = run_case(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.nsamp,
                                              wl.dm_list, wl.widths, wl.sigma, dtype, seed=wl.seed,
                                              pulses=small_pulse(), kernel=2, tile=tile)
    except dd.DDError as e:
        # kernel 4 windows must fit the warp's TMEM buffer (config 8 does not
        # at this plan's ~25 samples per DM step); kernel 5 needs at most 16
        # delay patterns per block and 4-channel subband (this plan has 29)
        assert tile[0] in (8, 9, 10, 11, 12) and e.code == 1
        pytest.skip("configuration unavailable for this plan")
    assert used == (2 if tile[0] < 3 else 3 if tile[0] < 7 else 4 if tile[0] < 9 else 5)


@pytest.mark.parametrize("tile", [(7, 8), (8, 4), (8, 1)])
@pytest.mark.parametrize("dtype", ["f32", "u8", "f16"])
def test_kernel4_lofar_geometry(dtype, tile):
    # LOFAR-band geometry (a few samples per DM step) where every kernel 4
    # configuration runs: 256 of the 1024 channels, 2^15 samples, 100 trials
    # with a ragged last DM block, two pulses
    lw = synth.workload("lofar_f32")
    nch, foff = 256, lw.foff * 4
    dms = [0.05 * i for i in range(100)]
    _, m = oracle.delays(nch, lw.fch1, foff, lw.tsamp, dms)
    nsamp = (1 << 15) + 17
    pulses = [synth.Pulse(dm=dms[61], t0=5000, width=8, amp=0.6),
              synth.Pulse(dm=dms[97], t0=9001, width=3, amp=0.9)]
    cands, out, ora, res, used = run_case(nch, lw.fch1, foff, lw.tsamp, nsamp, dms, [1, 2, 4, 8, 16],
                                          6.0, dtype, seed=77, pulses=pulses, kernel=4, tile=tile,
                                          max_gray=2)
    assert used == 4


@pytest.mark.parametrize("tile", [(9, 8), (9, 1), (10, 16), (11, 8), (11, 1), (12, 8), (12, 1), (12, 64)])
@pytest.mark.parametrize("dtype", ["f32", "u8", "f16"])
def test_kernel5_lofar_full_band(dtype, tile):
    # the shared-subband kernel on the full LOFAR band (1024 channels: at most
    # 10 delay patterns per block of 32, 48 or 64 trials and 4-channel subband), 100
    # trials (ragged last block), 2^15 samples, two pulses
    lw = synth.workload("lofar_f32")
    dms = [0.05 * i for i in range(100)]
    pulses = [synth.Pulse(dm=dms[61], t0=5000, width=8, amp=0.3),
              synth.Pulse(dm=dms[97], t0=9001, width=3, amp=0.5)]
    cands, out, ora, res, used = run_case(lw.nchans, lw.fch1, lw.foff, lw.tsamp, (1 << 15) + 17, dms,
                                          [1, 2, 4, 8, 16], 6.0, dtype, seed=78, pulses=pulses, kernel=5,
                                          tile=tile, max_gray=2)
    assert used == 5


@pytest.mark.parametrize("tile", [(9, 8), (9, 1), (10, 1), (10, 16)])
@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_kernel5_quarter_band(dtype, tile):
    # 256 of the LOFAR band's channels (4x wider): up to 13 delay patterns per
    # 32-trial block and subband, so many patterns per subband; ragged last
    # block and sample tile
    lw = synth.workload("lofar_f32")
    nch, foff = 256, lw.foff * 4
    dms = [0.05 * i for i in range(100)]
    pulses = [synth.Pulse(dm=dms[61], t0=5000, width=8, amp=0.6),
              synth.Pulse(dm=dms[97], t0=9001, width=3, amp=0.9)]
    cands, out, ora, res, used = run_case(nch, lw.fch1, foff, lw.tsamp, (1 << 15) + 17, dms, [1, 2, 4, 8, 16],
                                          6.0, dtype, seed=79, pulses=pulses, kernel=5, tile=tile,
                                          max_gray=2)
    assert used == 5


def test_autotune_keeps_parity():
    wl = SMALL
    arr, _ = make_input(wl.nchans, wl.nsamp, wl.fch1, wl.foff, wl.tsamp, wl.seed, small_pulse())
    plan = dd.Plan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list, wl.widths, wl.sigma,
                   dd.DD_F32, wl.nsamp)
    x = to_device(arr)
    out = torch.empty(wl.ndm * plan.nsamp_out, dtype=torch.float32, device="cuda")
    plan.autotune(x, wl.nsamp, out)
    cfg, group, tr, nw = plan.tile
    assert cfg in (0, 1, 2, 3, 4, 5, 6, 9, 10, 11, 12) and group in (4, 8, 16, 64) and tr in (8, 16, 20, 28, 36) \
        and nw in (4, 6, 8, 12)
    plan.execute(x, wl.nsamp, out)
    torch.cuda.synchronize()
    d_o, m_o = oracle.delays(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list)
    ora = oracle.dedisperse(arr, d_o, plan.nsamp_out)
    err = np.max(np.abs(out.cpu().numpy().reshape(wl.ndm, -1) - ora))
    assert err <= fp_tol(wl.nchans)
    # a second plan of the same shape starts from the cached choice
    plan2 = dd.Plan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list, wl.widths, wl.sigma,
                    dd.DD_F32, wl.nsamp)
    assert plan2.tile[:2] == (cfg, group)
    plan.close()
    plan2.close()


EDGE = [
    # nchans, nsamp extra beyond maxshift, dm_list, widths, pitch_pad, foff sign
    (1, 1, [0.0], [1], 0, -1),
    (3, 31, [0.0, 1.0, 2.0], [1, 2], 0, -1),
    (3, 32, [0.0, 1.0, 2.0], [1, 32], 0, -1),
    (128, 33, [0.5 * i for i in range(17)], [1, 2, 4, 8], 1, -1),
    (128, 1000, [0.0] * 5, [1, 3, 7], 0, -1),                       # maxshift 0
    (64, 777, [3.1, 0.2, 5.5, 1.0, 0.0, 2.2], [2, 1, 4], 3, -1),    # unsorted DMs
    (96, 600, [0.25 * i for i in range(40)], [1, 2, 4, 8, 16], 0, 1),  # ascending band
    (200, 2049, [0.1 * i for i in range(33)], [1, 5], 5, -1),
]


@pytest.mark.parametrize("case", range(len(EDGE)))
@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_edge_shapes(case, dtype):
    nch, extra, dms, widths, pad, sgn = EDGE[case]
    foff = sgn * 0.1953125
    fch1 = 150.0 if sgn < 0 else 150.0 - (nch - 1) * 0.1953125
    tsamp = 327.68e-6
    _, m = oracle.delays(nch, fch1, foff, tsamp, dms)
    nsamp = m + extra
    d_o, _ = oracle.delays(nch, fch1, foff, tsamp, dms)
    k5_tables = any(ddc.dd_share_tables(np.asarray(d_o), foff, DTYPES[dtype], c) is not None for c in range(9, 13))
    al = 4 if dtype == "f32" else 16
    # the shape's own pitch (often not 16-byte aligned: the tiled kernels then
    # fall back to kernel 1) and the next aligned one (the tiled kernels run)
    for pitch in sorted({nsamp + pad, synth.aligned_pitch(nsamp + pad, 4 if dtype == "f32" else 1)}):
        ran = {}
        for kernel in (0, 1, 3, 4, 5):
            try:
                *_, used = run_case(nch, fch1, foff, tsamp, nsamp, dms, widths, 3.0, dtype, seed=case + 100,
                                    pitch=pitch, kernel=kernel, max_gray=2)
            except dd.DDError as e:
                assert kernel >= 3 and e.code == 1      # kernel unavailable for this plan
                ran[kernel] = None
                continue
            # the tiled kernels need 16-byte aligned rows; other pitches run kernel 1
            ran[kernel] = used if used == 1 or pitch % al == 0 else 1
            assert kernel == 0 or used == kernel, (kernel, used)
        assert ran[1] == 1 and ran[0] in (1, 2, 3, 5)
        if pitch % al == 0:
            assert ran[3] == 3                           # every edge shape has kernel-3 tables
        if not k5_tables:
            assert ran[5] is None                        # more delay patterns than a record holds
        print(f"edge case {case} {dtype} pitch {pitch}: kernels run {ran} "
              f"(kernel-5 tables {'yes' if k5_tables else 'no'})")



def test_constant_input_gives_nchans_times_value():
    # Section 4: "all the elements initialized to the same value"
    nch, nsamp = 256, 4096
    dms = [0.2 * i for i in range(24)]
    plan = dd.Plan(nch, 150.0, -0.1953125, 327.68e-6, dms, [1, 2], 6.0, dd.DD_F32, nsamp)
    x = torch.full((nch, nsamp), 0.75, dtype=torch.float32, device="cuda")
    out = torch.empty(len(dms) * plan.nsamp_out, dtype=torch.float32, device="cuda")
    plan.execute(x, nsamp, out)
    torch.cuda.synchronize()
    assert bool(torch.all(out == nch * 0.75))
    plan.close()


def test_plans_of_different_geometry_coexist():
    # a later, smaller plan must not break launches of an earlier, larger one
    wl = SMALL
    arr, _ = make_input(wl.nchans, wl.nsamp, wl.fch1, wl.foff, wl.tsamp, wl.seed, small_pulse())
    big = dd.Plan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list, wl.widths, wl.sigma,
                  dd.DD_F32, wl.nsamp)
    small = dd.Plan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list[:3], [1], wl.sigma,
                    dd.DD_F32, wl.nsamp)
    x = to_device(arr)
    for plan in (big, small, big):
        out = torch.empty(plan.ndm * plan.nsamp_out, dtype=torch.float32, device="cuda")
        plan.execute(x, wl.nsamp, out)
        cands, total = plan.search(out)
        if plan is big:
            best = cands[np.argmax(cands["snr"])]
            assert (int(best["dm_idx"]), int(best["t"])) == (30, 4000)
    big.close()
    small.close()


def test_search_overflow_reports_true_count():
    wl = SMALL
    arr, _ = make_input(wl.nchans, wl.nsamp, wl.fch1, wl.foff, wl.tsamp, 5)
    plan = dd.Plan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list, wl.widths, 1.0, dd.DD_F32,
                   wl.nsamp)
    out = torch.empty(wl.ndm * plan.nsamp_out, dtype=torch.float32, device="cuda")
    plan.execute(to_device(arr), wl.nsamp, out)
    cands, total = plan.search(out, capacity=100, allow_overflow=True)
    assert total > 100 and len(cands) == 100
    k = [(int(r["dm_idx"]), int(r["t"]), int(r["width_idx"])) for r in cands]
    assert k == sorted(k)
    with pytest.raises(dd.DDError) as e:
        plan.search(out, capacity=100)
    assert e.value.code == dd.dd.DD_ERR_OVERFLOW
    plan.close()


def test_process_host_matches_device_path():
    wl = SMALL
    arr, _ = make_input(wl.nchans, wl.nsamp, wl.fch1, wl.foff, wl.tsamp, wl.seed, small_pulse())
    plan = dd.Plan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list, wl.widths, wl.sigma,
                   dd.DD_F32, wl.nsamp)
    host = torch.from_numpy(arr).pin_memory()
    c1, n1 = plan.process_host(host, wl.nsamp)
    out = torch.empty(wl.ndm * plan.nsamp_out, dtype=torch.float32, device="cuda")
    plan.execute(to_device(arr), wl.nsamp, out)
    c2, n2 = plan.search(out)
    assert n1 == n2 and keys(c1) == keys(c2)
    plan.close()


@pytest.mark.parametrize("kernel,tile", [(3, (5, 8)), (3, (6, 1)), (5, (9, 4)), (5, (11, 16)), (5, (12, 64))])
@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_process_host_pipelined(dtype, kernel, tile):
    # dd_process_host with kernels 3 and 5 copies the input in 8 column chunks
    # and de-disperses each chunk's output tiles as separate launches: same
    # candidates and statistics as one device-resident execute + search (the
    # partial statistics are combined in another order: FP32 path to 1e-12).
    # Full LOFAR band, 100 trials, 2^15 + 17 samples, padded pitch, 4 sigma.
    lw = synth.workload("lofar_f32")
    dms = [0.05 * i for i in range(100)]
    nsamp = (1 << 15) + 17
    pitch = synth.aligned_pitch(nsamp + 40, 4 if dtype == "f32" else 1)
    pulses = [synth.Pulse(dm=dms[61], t0=5000, width=8, amp=0.3),
              synth.Pulse(dm=dms[97], t0=30001, width=3, amp=0.5)]
    arr, _ = make_input(lw.nchans, nsamp, lw.fch1, lw.foff, lw.tsamp, 91, pulses, dtype, pitch)
    plan = dd.Plan(lw.nchans, lw.fch1, lw.foff, lw.tsamp, dms, [1, 2, 4, 8, 16], 4.0, DTYPES[dtype], nsamp)
    plan.set_kernel(kernel)
    plan.set_tile(*tile)
    host = torch.from_numpy(arr).pin_memory()
    c1, n1 = plan.process_host(host, pitch, capacity=1 << 16)
    mu1, sg1 = plan.stats()
    out = torch.empty(len(dms) * plan.nsamp_out, dtype=torch.int32 if dtype == "u8" else torch.float32,
                      device="cuda")
    plan.execute(to_device(arr), pitch, out)
    c2, n2 = plan.search(out, capacity=1 << 16)
    mu2, sg2 = plan.stats()
    assert plan.tile[0] == tile[0]
    assert n1 == n2 and n1 > 100 and keys(c1) == keys(c2)
    if dtype == "u8":
        assert (mu1, sg1) == (mu2, sg2)
        assert np.array_equal(c1["value"], c2["value"])
    else:
        assert abs(mu1 - mu2) <= 1e-12 * max(1.0, abs(mu2)) and abs(sg1 - sg2) <= 1e-12 * sg2
        assert np.max(np.abs(c1["snr"].astype(np.float64) - c2["snr"])) <= 1e-4
    # and the host path against the oracle: statistics and candidate list
    d_o, m_o = oracle.delays(lw.nchans, lw.fch1, lw.foff, lw.tsamp, dms)
    ora = oracle.dedisperse(arr, d_o, plan.nsamp_out)
    mu_o, sg_o = oracle.stats(ora)
    if dtype == "u8":
        assert abs(mu1 - mu_o) <= 1e-12 * max(1.0, abs(mu_o)) and abs(sg1 - sg_o) <= 1e-12 * sg_o
    else:
        assert abs(mu1 - mu_o) <= fp_tol(lw.nchans) and abs(sg1 - sg_o) <= 1e-5 * sg_o
    eps = 0.0 if dtype == "u8" else fp_tol(lw.nchans)
    n_match, n_gray = compare_candidates(c1, ora, [1, 2, 4, 8, 16], mu1, sg1, mu_o, sg_o, 4.0, eps)
    assert n_match > 100 and n_gray <= 2, (n_match, n_gray)
    plan.close()


def test_measured_precision_errors(capsys):
    """The precision variants' measured error against the FP64 oracle on the
    config-1 shape (128 channels, 64 DM trials, 8192 samples, noise + the
    amplitude-5 pulse): float32 input, the same data rounded to FP16 (oracle
    on the rounded values) and quantised to uint8 (exact integers), for every
    kernel that runs this plan.  Bound: 1e-5 * nchans = 1.28e-3."""
    wl = SMALL
    d_o, m_o = oracle.delays(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list)
    nout = wl.nsamp - m_o
    rows = []
    for dtype in ("f32", "f16", "u8"):
        arr, _ = make_input(wl.nchans, wl.nsamp, wl.fch1, wl.foff, wl.tsamp, wl.seed, small_pulse(), dtype)
        ora = oracle.dedisperse(arr, d_o, nout)
        for kernel in (1, 2, 3, 4):
            plan = dd.Plan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list, wl.widths, wl.sigma,
                           DTYPES[dtype], wl.nsamp)
            plan.set_kernel(kernel)
            out_dev = torch.empty(wl.ndm * nout, dtype=torch.int32 if dtype == "u8" else torch.float32,
                                  device="cuda")
            plan.execute(to_device(arr), arr.shape[1], out_dev)
            torch.cuda.synchronize()
            out = out_dev.cpu().numpy().reshape(wl.ndm, nout).astype(np.float64)
            err = float(np.max(np.abs(out - ora)))
            rows.append((dtype, kernel, err, float(np.sqrt(np.mean((out - ora) ** 2)))))
            plan.close()
    msg = "; ".join(f"{dt} kernel {k}: max|err| {e:.3g} rms {r:.3g}" for dt, k, e, r in rows)
    with capsys.disabled():
        print(f"\nprecision (config 1/3 shape, bound {fp_tol(wl.nchans):.3g}): {msg}")
    for dt, k, e, _ in rows:
        if dt == "u8":
            assert e == 0.0, msg
        else:
            assert e <= fp_tol(wl.nchans), msg
