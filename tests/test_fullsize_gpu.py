"""Parity at the batching and serving workloads' full sizes, in the launch
configurations the benchmark times: the 24 uneven beams of the batch (one
persistent launch, autotuned tile shape) and streamed beams of the serving
workload (uint8, 1024 and 4096 channels, 65536-sample chunks).  The oracle
cannot recompute these outputs whole, so sampled outputs are checked one by
one: the input samples each output needs are gathered with the ORACLE's delay
table and summed by the oracle."""
import numpy as np
import pytest

import oracle
import synth
from ddhelpers import compare_candidates, fp_tol, keys

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1107_2516_gb300 as dd
from paper_1107_2516_gb300 import build as ddbuild


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ddbuild.build()
    dd.load()


def _oracle_points(column_values, is_int):
    """The oracle's sum over channels of gathered values [npoints][C]."""
    v = np.ascontiguousarray(column_values.T)                      # [C][npoints]
    zero = np.zeros((1, v.shape[0]), np.int64)
    out = np.empty(v.shape[1], np.int64 if is_int else np.float64)
    for k in range(v.shape[1]):
        out[k] = oracle.dedisperse(np.ascontiguousarray(v[:, k:k + 1]), zero, 1)[0, 0]
    return out


def _device_input(b, pitch, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    x = torch.randn(b.nchans, pitch, device="cuda", generator=g)
    if b.dtype == "u8":
        x = (x * 16.0 + 128.0).round_().clamp_(0, 255).to(torch.uint8)
    return x


# beams of the 24-beam batch checked whole against the oracle: the smallest
# float32 beam (20: 256 channels, 500 trials) and the smallest uint8 beam
# (5: 512 channels, 2830 trials); their inputs come from the seeded host
# generator with one injected pulse each, the others' from the device RNG
ORACLE_BEAMS = (5, 20)


def _host_input(b, pitch):
    x = synth.noise_f32(b.nchans, b.nsamp, b.seed, pitch=pitch)
    dm = float(b.dm_list[b.ndm // 3])
    d1, _ = oracle.delays(b.nchans, b.fch1, b.foff, b.tsamp, [dm])
    p = synth.Pulse(dm=dm, t0=b.nsamp // 5, width=8, amp=synth.pulse_amplitude(14.0, b.nchans, 8))
    synth.inject_pulses(x, [p], lambda _: d1[0], b.nsamp)
    return x if b.dtype == "f32" else synth.quantize_u8(x)


def test_batch_full_size():
    beams = synth.batch_beams(24, 4, lambda c, f1, fo, ts, dm: oracle.delays(c, f1, fo, ts, [dm])[1])
    widths = (1, 2, 4, 8, 16, 32)
    plans, ins, pitches, outs, host = [], [], [], [], {}
    for i, b in enumerate(beams):
        p = dd.Plan(b.nchans, b.fch1, b.foff, b.tsamp, b.dm_list, widths, 6.0,
                    dd.DD_F32 if b.dtype == "f32" else dd.DD_U8, b.nsamp)
        pitch = synth.aligned_pitch(b.nsamp, 4 if b.dtype == "f32" else 1)
        plans.append(p)
        pitches.append(pitch)
        if i in ORACLE_BEAMS:
            host[i] = _host_input(b, pitch)
            ins.append(torch.from_numpy(host[i]).cuda())
        else:
            ins.append(_device_input(b, pitch, b.seed))
        outs.append(torch.empty(p.ndm * p.nsamp_out, device="cuda",
                                dtype=torch.int32 if p.out_is_int else torch.float32))
    batch = dd.Batch(plans)
    s = torch.cuda.Stream()
    batch.autotune(ins, pitches, outs, s)          # the benchmark's launch configuration
    batch.capture(ins, pitches, outs, s)
    batch.launch(s)
    res = [batch.results(i, capacity=1 << 20, stream=s) for i in range(len(plans))]
    assert batch.info[2] == 0
    rng = np.random.default_rng(44)
    for i, (b, p) in enumerate(zip(beams, plans)):
        d, m = oracle.delays(b.nchans, b.fch1, b.foff, b.tsamp, b.dm_list)
        assert p.maxshift == m
        nout = b.nsamp - m
        got = outs[i].view(b.ndm, nout)
        if i in ORACLE_BEAMS:
            # the whole beam: every output, the statistics, the whole candidate list
            ref = oracle.dedisperse(host[i][:, :b.nsamp].copy(), d, nout)
            g = got.cpu().numpy()
            if b.dtype == "u8":
                assert np.array_equal(g.astype(np.int64), ref), i
            else:
                err = np.max(np.abs(g.astype(np.float64) - ref))
                assert err <= fp_tol(b.nchans), (i, err)
            mu_o, sg_o = oracle.stats(ref)
            mu_g, sg_g = p.stats()
            assert abs(mu_g - mu_o) <= 1e-6 * np.sqrt(b.nchans) and abs(sg_g - sg_o) <= 1e-6 * sg_o, i
            eps = 0.0 if b.dtype == "u8" else fp_tol(b.nchans)
            n_match, n_gray = compare_candidates(res[i][0], ref, widths, mu_g, sg_g, mu_o, sg_o, 6.0, eps)
            assert n_match > 0 and n_gray == 0, (i, n_match, n_gray)
            assert res[i][1] == len(res[i][0])
        else:
            # sampled outputs against the oracle on the gathered input samples
            js = np.concatenate([rng.integers(0, b.ndm, 40), [0, b.ndm - 1]])
            ts = np.concatenate([rng.integers(0, nout, 40), [nout - 1, 0]])
            idx_c = torch.arange(b.nchans, device="cuda")
            cols = torch.stack([ins[i][idx_c, torch.from_numpy(t + d[j]).cuda()] for j, t in zip(js, ts)])
            ref = _oracle_points(cols.cpu().numpy(), b.dtype == "u8")
            gs = got[torch.from_numpy(js).cuda(), torch.from_numpy(ts).cuda()].cpu().numpy()
            if b.dtype == "u8":
                assert np.array_equal(gs.astype(np.int64), ref), i
            else:
                assert np.max(np.abs(gs.astype(np.float64) - ref)) <= fp_tol(b.nchans), i
    # every beam equals its plan alone on the beam's batch configuration: the
    # whole output bit for bit, the candidate count and list
    for i, p in enumerate(plans):
        bc = batch.beam_config(i)
        if bc >= 0:
            p.set_tile(bc, 8)
        ref_out = outs[i].clone()
        outs[i].zero_()
        p.execute(ins[i], pitches[i], outs[i])
        c, n = p.search(outs[i], capacity=1 << 20)
        torch.cuda.synchronize()
        assert torch.equal(outs[i], ref_out), f"beam {i}: batched output differs from its plan alone"
        assert n == res[i][1] and keys(c) == keys(res[i][0]), i
        del ref_out
    batch.close()
    for p in plans:
        p.close()


@pytest.mark.parametrize("which", [0, 1])
def test_serving_beam_full_size_sampled(which):
    # the serving workload's beams 0 (1024 channels) and 1 (4096 channels)
    b = synth.serve_beams(64, 5)[which]
    srv = dd.Server(1 << 36, nworkers=2)
    bid = srv.add_beam(b.nchans, b.fch1, b.foff, b.tsamp, b.dm_list, (1, 2, 4, 8, 16, 32, 64), 6.0,
                       dd.DD_U8, b.chunk)
    info = srv.beam_info(bid)
    d, M = oracle.delays(b.nchans, b.fch1, b.foff, b.tsamp, b.dm_list)
    assert info["maxshift"] == M
    nprime = (M + b.chunk - 1) // b.chunk
    nchunks = nprime + 2
    x = synth.quantize_u8(synth.noise_f32(b.nchans, nchunks * b.chunk, b.seed))
    rng = np.random.default_rng(which)
    checked = 0
    for k in range(nchunks):
        ck = torch.from_numpy(np.ascontiguousarray(x[:, k * b.chunk:(k + 1) * b.chunk])).pin_memory()
        srv.submit(bid, ck, b.chunk, k)
        got_r = None
        for _ in range(600):
            res = srv.poll(wait_ms=100)
            hit = [r for r in res if r["beam"] == bid and r["seq"] == k]
            if hit:
                got_r = hit[0]
                break
        assert got_r is not None
        if k < nprime:
            assert got_r["status"] == dd.DD_PRIMING
            continue
        assert got_r["status"] == 0
        cls = type("V", (), {"__cuda_array_interface__": {"shape": (b.ndm * b.chunk,), "typestr": "<i4",
                                                          "data": (info["out_dev"], False), "version": 3}})
        cur = torch.as_tensor(cls(), device="cuda").view(b.ndm, b.chunk)
        lo = k * b.chunk - M                         # stream time of this chunk's first output
        js = np.concatenate([rng.integers(0, b.ndm, 60), [0, b.ndm - 1]])
        us = np.concatenate([rng.integers(0, b.chunk, 60), [b.chunk - 1, 0]])
        cols = np.stack([x[np.arange(b.nchans), lo + u + d[j]] for j, u in zip(js, us)])
        ref = _oracle_points(cols, True)
        got = cur[torch.from_numpy(js).cuda(), torch.from_numpy(us).cuda()].cpu().numpy().astype(np.int64)
        assert np.array_equal(got, ref), k
        # the chunk's mean, exactly, from per-channel prefix sums of the input
        P = np.concatenate([np.zeros((b.nchans, 1), np.int64), np.cumsum(x[:, lo:lo + b.chunk + M], axis=1,
                                                                          dtype=np.int64)], axis=1)
        tot = 0
        cidx = np.arange(b.nchans)
        for j in range(b.ndm):
            tot += int(np.sum(P[cidx, d[j] + b.chunk] - P[cidx, d[j]]))
        assert abs(got_r["mu"] - tot / (b.ndm * b.chunk)) <= 1e-9 * abs(tot / (b.ndm * b.chunk))
        checked += 1
    assert checked == 2
    srv.close()


def test_serving_whole_chunks_oracle():
    # serving beam 2 (1024 channels, 1151 DM trials to DM 500, uint8, maxshift
    # 7978 samples): every output of two searched 65536-sample chunks bit for
    # bit, the chunk statistics, and the complete candidate list of each chunk
    # against the oracle run over the stream (kernel 5 serves this beam)
    b = synth.serve_beams(64, 5)[2]
    widths = (1, 2, 4, 8, 16, 32, 64)
    srv = dd.Server(1 << 36, nworkers=2)
    bid = srv.add_beam(b.nchans, b.fch1, b.foff, b.tsamp, b.dm_list, widths, 6.0, dd.DD_U8, b.chunk)
    assert srv.beam_kernel(bid)[0] == 5
    info = srv.beam_info(bid)
    d, M = oracle.delays(b.nchans, b.fch1, b.foff, b.tsamp, b.dm_list)
    assert info["maxshift"] == M
    nprime = (M + b.chunk - 1) // b.chunk
    nchunks = nprime + 2
    x = synth.noise_f32(b.nchans, nchunks * b.chunk, b.seed)
    dm = float(b.dm_list[b.ndm // 2])
    d1, _ = oracle.delays(b.nchans, b.fch1, b.foff, b.tsamp, [dm])
    t_pulse = (nprime + 1) * b.chunk + 1000 - M          # stream output time inside the last chunk
    synth.inject_pulses(x, [synth.Pulse(dm=dm, t0=t_pulse, width=16,
                                        amp=synth.pulse_amplitude(12.0, b.nchans, 16))],
                        lambda _: d1[0], nchunks * b.chunk)
    x = synth.quantize_u8(x)
    stream = np.concatenate([np.zeros((b.nchans, M), np.uint8), x], axis=1)   # zero history first
    found_pulse = False
    for k in range(nchunks):
        ck = torch.from_numpy(np.ascontiguousarray(x[:, k * b.chunk:(k + 1) * b.chunk])).pin_memory()
        assert srv.submit(bid, ck, b.chunk, k) == 0
        r = None
        for _ in range(600):
            hit = [q for q in srv.poll(wait_ms=100) if q["beam"] == bid and q["seq"] == k]
            if hit:
                r = hit[0]
                break
        assert r is not None
        if k < nprime:
            assert r["status"] == dd.DD_PRIMING
            continue
        assert r["status"] == 0
        # chunk k's window: stream samples [k*chunk - M, (k+1)*chunk), i.e. stream[:, k*chunk : ...]
        win = np.ascontiguousarray(stream[:, k * b.chunk:k * b.chunk + M + b.chunk])
        ref = oracle.dedisperse(win, d, b.chunk)
        cls = type("V", (), {"__cuda_array_interface__": {"shape": (b.ndm * b.chunk,), "typestr": "<i4",
                                                          "data": (info["out_dev"], False), "version": 3}})
        got = torch.as_tensor(cls(), device="cuda").view(b.ndm, b.chunk).cpu().numpy().astype(np.int64)
        assert np.array_equal(got, ref), k
        mu_o, sg_o = oracle.stats(ref)
        assert abs(r["mu"] - mu_o) <= 1e-12 * abs(mu_o) and abs(r["sigma"] - sg_o) <= 1e-9 * sg_o, k
        cands = srv.candidates(bid, k, capacity=1 << 20)
        assert len(cands) == r["n_candidates"]
        n_match, n_gray = compare_candidates(cands, ref, widths, r["mu"], r["sigma"], mu_o, sg_o, 6.0, 0.0)
        assert n_gray == 0, (k, n_gray)
        found_pulse |= any(abs(int(c["t"]) - (t_pulse - (k * b.chunk - M))) < 64 for c in cands)
    assert found_pulse
    srv.close()
