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
from ddhelpers import fp_tol

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


def test_batch_full_size_sampled():
    beams = synth.batch_beams(24, 4, lambda c, f1, fo, ts, dm: oracle.delays(c, f1, fo, ts, [dm])[1])
    widths = (1, 2, 4, 8, 16, 32)
    plans, ins, pitches, outs = [], [], [], []
    for b in beams:
        p = dd.Plan(b.nchans, b.fch1, b.foff, b.tsamp, b.dm_list, widths, 6.0,
                    dd.DD_F32 if b.dtype == "f32" else dd.DD_U8, b.nsamp)
        pitch = synth.aligned_pitch(b.nsamp, 4 if b.dtype == "f32" else 1)
        plans.append(p)
        pitches.append(pitch)
        ins.append(_device_input(b, pitch, b.seed))
        outs.append(torch.empty(p.ndm * p.nsamp_out, device="cuda",
                                dtype=torch.int32 if p.out_is_int else torch.float32))
    batch = dd.Batch(plans)
    s = torch.cuda.Stream()
    batch.autotune(ins, pitches, outs, s)
    batch.capture(ins, pitches, outs, s)
    batch.launch(s)
    totals = [batch.results(i, stream=s, allow_overflow=True)[1] for i in range(len(plans))]
    assert batch.info[2] == 0
    rng = np.random.default_rng(44)
    for i, (b, p) in enumerate(zip(beams, plans)):
        d, m = oracle.delays(b.nchans, b.fch1, b.foff, b.tsamp, b.dm_list)
        assert p.maxshift == m
        nout = b.nsamp - m
        js = np.concatenate([rng.integers(0, b.ndm, 40), [0, b.ndm - 1]])
        ts = np.concatenate([rng.integers(0, nout, 40), [nout - 1, 0]])
        idx_c = torch.arange(b.nchans, device="cuda")
        cols = torch.stack([ins[i][idx_c, torch.from_numpy(t + d[j]).cuda()] for j, t in zip(js, ts)])
        ref = _oracle_points(cols.cpu().numpy(), b.dtype == "u8")
        got = outs[i].view(b.ndm, nout)[torch.from_numpy(js).cuda(), torch.from_numpy(ts).cuda()].cpu().numpy()
        if b.dtype == "u8":
            assert np.array_equal(got.astype(np.int64), ref), i
        else:
            assert np.max(np.abs(got.astype(np.float64) - ref)) <= fp_tol(b.nchans), i
    assert sum(totals) >= 0
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
