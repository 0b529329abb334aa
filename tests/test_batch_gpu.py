"""Batched beams (one persistent launch for uneven beams, mixed float32/uint8):
every beam's output and candidate list equal what its plan alone produces, the
CUDA-graph replay equals the direct launch, and small beams match the oracle."""
import numpy as np
import pytest

import oracle
import synth
from ddhelpers import compare_candidates, fp_tol, keys

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1107_2516_gb300 as dd
from paper_1107_2516_gb300 import build as ddbuild

WIDTHS = (1, 2, 4, 8)
SIGMA = 5.0


def maxshift_of(c, f1, fo, ts, dm):
    return oracle.delays(c, f1, fo, ts, [dm])[1]


@pytest.fixture(scope="module")
def beams():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ddbuild.build()
    bs = synth.batch_beams(6, 4, maxshift_of, mini=True)
    data = []
    for b in bs:
        pitch = synth.aligned_pitch(b.nsamp, 4 if b.dtype == "f32" else 1)
        x = synth.noise_f32(b.nchans, b.nsamp, b.seed, pitch=pitch)
        d1, _ = oracle.delays(b.nchans, b.fch1, b.foff, b.tsamp, [float(b.dm_list[b.ndm // 2])])
        p = synth.Pulse(dm=float(b.dm_list[b.ndm // 2]), t0=b.nsamp // 4, width=4,
                        amp=synth.pulse_amplitude(15.0, b.nchans, 4))
        synth.inject_pulses(x, [p], lambda dm: d1[0], b.nsamp)
        arr = x if b.dtype == "f32" else synth.quantize_u8(x)
        data.append((b, arr, pitch))
    return data


def _plans(data, cfg=None):
    plans = []
    for b, arr, pitch in data:
        p = dd.Plan(b.nchans, b.fch1, b.foff, b.tsamp, b.dm_list, WIDTHS, SIGMA,
                    dd.DD_F32 if b.dtype == "f32" else dd.DD_U8, b.nsamp)
        if cfg is not None:
            p.set_tile(cfg, 8)
        plans.append(p)
    return plans


def _bufs(data, plans):
    ins = [torch.from_numpy(arr).cuda() for _, arr, _ in data]
    outs = [torch.empty(p.ndm * p.nsamp_out, dtype=torch.int32 if p.out_is_int else torch.float32,
                        device="cuda") for p in plans]
    return ins, [pitch for _, _, pitch in data], outs


@pytest.mark.parametrize("config,per_beam", [(None, False), (1, False), (5, False), (3, False), (9, False),
                                             (9, True), (5, True)])
def test_batch_matches_single_plans_and_graph(beams, config, per_beam):
    # default configuration (the mixed kernel 5 / kernel 3 one), a kernel 2
    # shape, kernel 3 shapes; one persistent grid or each beam's own launch
    plans = _plans(beams)
    batch = dd.Batch(plans)
    if config is not None:
        batch.set_config(config)
    if per_beam:
        batch.set_launch_mode(True)
    assert batch.per_beam == per_beam
    cfg, nitems, nsep = batch.info
    assert cfg == (9 if config is None else config) and nitems > 0 and nsep == 0
    for i, p in enumerate(plans):
        bc = batch.beam_config(i)
        if cfg == 9:
            # mixed: kernel 3's shape 5, or kernel 5 (own launches: the beam's first available kernel 5 shape)
            assert bc in ((5, 9, 10, 11, 12) if per_beam else (5, 9))
        else:
            assert bc == cfg
        p.set_tile(bc, 8)
    ins, pitches, outs = _bufs(beams, plans)
    # each plan alone
    single = []
    for p, x, pitch, o in zip(plans, ins, pitches, outs):
        p.execute(x, pitch, o)
        c, n = p.search(o)
        single.append((o.clone(), c, n))
    # one persistent launch for all beams
    for o in outs:
        o.zero_()
    batch.execute(ins, pitches, outs)
    for i, (o_ref, c_ref, n_ref) in enumerate(single):
        c, n = batch.results(i)
        assert torch.equal(outs[i], o_ref), f"beam {i} output differs"
        assert n == n_ref and keys(c) == keys(c_ref)
    # CUDA graph capture + replay
    s = torch.cuda.Stream()
    for o in outs:
        o.zero_()
    batch.capture(ins, pitches, outs, s)
    for rep in range(2):
        batch.launch(s)
        for i, (o_ref, c_ref, n_ref) in enumerate(single):
            c, n = batch.results(i, stream=s)
            assert torch.equal(outs[i], o_ref)
            assert n == n_ref and keys(c) == keys(c_ref)
    batch.close()
    for p in plans:
        p.close()


def test_batch_beams_match_oracle(beams):
    plans = _plans(beams)
    batch = dd.Batch(plans)
    ins, pitches, outs = _bufs(beams, plans)
    batch.autotune(ins, pitches, outs)
    batch.execute(ins, pitches, outs)
    torch.cuda.synchronize()
    for i, ((b, arr, pitch), p) in enumerate(zip(beams, plans)):
        d, m = oracle.delays(b.nchans, b.fch1, b.foff, b.tsamp, b.dm_list)
        nout = b.nsamp - m
        assert p.nsamp_out == nout
        ora = oracle.dedisperse(arr, d, nout)
        got = outs[i].cpu().numpy().reshape(b.ndm, nout)
        if b.dtype == "u8":
            assert np.array_equal(got.astype(np.int64), ora)
        else:
            assert np.max(np.abs(got - ora)) <= fp_tol(b.nchans)
        c, n = batch.results(i)
        mu_g, sg_g = p.stats()
        mu_o, sg_o = oracle.stats(ora)
        res = compare_candidates(c, ora, list(WIDTHS), mu_g, sg_g, mu_o, sg_o, SIGMA,
                                 0.0 if b.dtype == "u8" else fp_tol(b.nchans))
        assert res[1] <= 2
    batch.close()
    for p in plans:
        p.close()


def test_mixed_batch_kernel5_and_kernel3():
    # the mixed configuration with beams on both kernels in one persistent
    # launch: three small beams on kernel 5, and the 128-channel plan of the
    # small workload (29 delay patterns per 4-channel subband: kernel 3) as
    # float32 and uint8; every beam bit-identical to its plan alone on the
    # same configuration, graph replay included, and to the oracle
    data = []
    for b, arr, pitch in synth_beams_mini(3):
        data.append((b.nchans, b.fch1, b.foff, b.tsamp, b.dm_list, b.nsamp, b.dtype, arr, pitch))
    wl = synth.workload("small_f32")
    x = synth.noise_f32(wl.nchans, wl.nsamp, wl.seed)
    for dt, arr in (("f32", x), ("u8", synth.quantize_u8(x))):
        data.append((wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list, wl.nsamp, dt, arr, arr.shape[1]))
    plans = [dd.Plan(c, f1, fo, ts, dms, WIDTHS, SIGMA, dd.DD_F32 if dt == "f32" else dd.DD_U8, n)
             for c, f1, fo, ts, dms, n, dt, _, _ in data]
    batch = dd.Batch(plans)
    batch.set_config(9)
    assert [batch.beam_config(i) for i in range(len(plans))] == [9, 9, 9, 5, 5]
    ins = [torch.from_numpy(d[7]).cuda() for d in data]
    pitches = [d[8] for d in data]
    outs = [torch.empty(p.ndm * p.nsamp_out, dtype=torch.int32 if p.out_is_int else torch.float32,
                        device="cuda") for p in plans]
    single = []
    for i, (p, xi, pitch, o) in enumerate(zip(plans, ins, pitches, outs)):
        p.set_tile(batch.beam_config(i), 8)
        p.execute(xi, pitch, o)
        c, n = p.search(o)
        single.append((o.clone(), c, n))
    for o in outs:
        o.zero_()
    batch.execute(ins, pitches, outs)
    for i, (o_ref, c_ref, n_ref) in enumerate(single):
        c, n = batch.results(i)
        assert torch.equal(outs[i], o_ref), f"beam {i} output differs"
        assert n == n_ref and keys(c) == keys(c_ref)
    s = torch.cuda.Stream()
    for o in outs:
        o.zero_()
    batch.capture(ins, pitches, outs, s)
    batch.launch(s)
    for i, (o_ref, c_ref, n_ref) in enumerate(single):
        c, n = batch.results(i, stream=s)
        assert torch.equal(outs[i], o_ref)
        assert n == n_ref and keys(c) == keys(c_ref)
    torch.cuda.synchronize()
    for (c, f1, fo, ts, dms, n, dt, arr, pitch), p, o in zip(data, plans, outs):
        d, m = oracle.delays(c, f1, fo, ts, dms)
        ora = oracle.dedisperse(arr, d, n - m)
        got = o.cpu().numpy().reshape(len(dms), n - m)
        if dt == "u8":
            assert np.array_equal(got.astype(np.int64), ora)
        else:
            assert np.max(np.abs(got - ora)) <= fp_tol(c)
    batch.close()
    for p in plans:
        p.close()


def synth_beams_mini(n):
    bs = synth.batch_beams(6, 4, maxshift_of, mini=True)[:n]
    out = []
    for b in bs:
        pitch = synth.aligned_pitch(b.nsamp, 4 if b.dtype == "f32" else 1)
        x = synth.noise_f32(b.nchans, b.nsamp, b.seed, pitch=pitch)
        out.append((b, x if b.dtype == "f32" else synth.quantize_u8(x), pitch))
    return out
