"""Streaming server: chunk-boundary continuity against one-shot de-dispersion of
the concatenated stream, identical results for a beam alone and in a mix of
concurrently served beams, device-memory admission, and oracle parity."""
import numpy as np
import pytest

import oracle
import synth
from ddhelpers import fp_tol, keys

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1107_2516_gb300 as dd
from paper_1107_2516_gb300 import build as ddbuild

WIDTHS = (1, 2, 4, 8)
BEAM = dict(nchans=64, fch1=150.0, foff=-0.390625, tsamp=327.68e-6,
            dm_list=[0.1 * i for i in range(40)], widths=WIDTHS, sigma=5.0)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ddbuild.build()


def stream_data(nchans, total, seed, dtype="f32", pulses=()):
    x = synth.noise_f32(nchans, total, seed)
    if pulses:
        synth.inject_pulses(x, list(pulses), lambda dm: oracle.delays(
            nchans, BEAM["fch1"], BEAM["foff"], BEAM["tsamp"], [dm])[0][0], total)
    return x if dtype == "f32" else synth.quantize_u8(x)


def chunks_of(x, chunk):
    return [torch.from_numpy(np.ascontiguousarray(x[:, k * chunk:(k + 1) * chunk])).pin_memory()
            for k in range(x.shape[1] // chunk)]


def wait_for(srv, beam, seq, timeout_ms=20000):
    got = []
    waited = 0
    while waited < timeout_ms:
        for r in srv.poll(wait_ms=100):
            got.append(r)
        hit = [r for r in got if r["beam"] == beam and r["seq"] == seq]
        if hit:
            return hit[0]
        waited += 100
    raise TimeoutError(f"chunk {(beam, seq)} not reported")


@pytest.mark.parametrize("chunk", [2048, 512])
def test_stream_matches_one_shot(chunk):
    K = 10
    total = K * chunk
    dms = BEAM["dm_list"]
    pulse = synth.Pulse(dm=dms[25], t0=total // 2, width=4, amp=2.0)
    x = stream_data(BEAM["nchans"], total, seed=11, pulses=[pulse])
    srv = dd.Server(1 << 30, nworkers=2)
    bid = srv.add_beam(BEAM["nchans"], BEAM["fch1"], BEAM["foff"], BEAM["tsamp"], dms, WIDTHS,
                       BEAM["sigma"], dd.DD_F32, chunk)
    info = srv.beam_info(bid)
    M = info["maxshift"]
    assert M == oracle.delays(BEAM["nchans"], BEAM["fch1"], BEAM["foff"], BEAM["tsamp"], dms)[1]
    one = dd.Plan(BEAM["nchans"], BEAM["fch1"], BEAM["foff"], BEAM["tsamp"], dms, WIDTHS, BEAM["sigma"],
                  dd.DD_F32, total)
    full = torch.empty(len(dms) * one.nsamp_out, dtype=torch.float32, device="cuda")
    one.execute(torch.from_numpy(x).cuda(), total, full)
    torch.cuda.synchronize()
    full = full.view(len(dms), one.nsamp_out)
    d_o, _ = oracle.delays(BEAM["nchans"], BEAM["fch1"], BEAM["foff"], BEAM["tsamp"], dms)
    ora = oracle.dedisperse(x, d_o, total - M)
    n_real = 0
    for k, ck in enumerate(chunks_of(x, chunk)):
        srv.submit(bid, ck, chunk, k)
        r = wait_for(srv, bid, k)
        if k * chunk < M:
            assert r["status"] == dd.DD_PRIMING
            continue
        assert r["status"] == 0
        n_real += 1
        # this chunk's outputs are stream times [k*chunk - M, (k+1)*chunk - M)
        cur = _device_view(info["out_dev"], len(dms) * chunk).view(len(dms), chunk).clone()
        lo = k * chunk - M
        assert torch.equal(cur, full[:, lo:lo + chunk]), f"chunk {k} differs from one-shot"
        err = np.max(np.abs(cur.cpu().numpy().astype(np.float64) - ora[:, lo:lo + chunk]))
        assert err <= fp_tol(BEAM["nchans"])
    assert n_real == K - ((M + chunk - 1) // chunk)
    srv.close()
    one.close()


def _device_view(ptr, n):
    """A float32 torch view of n elements at a device address owned by the server."""
    class _Cuda:
        __cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (ptr, False), "version": 3}
    return torch.as_tensor(_Cuda(), device="cuda")


def _serve(srv, streams, order_alone=None):
    """Submit every beam's chunks as fast as possible; return {beam: [(status, mu, sigma, keys)]}."""
    ids, data = [], []
    for spec, x in streams:
        bid = srv.add_beam(spec["nchans"], BEAM["fch1"], BEAM["foff"], BEAM["tsamp"], spec["dm_list"],
                           WIDTHS, BEAM["sigma"], spec["dtype_code"], spec["chunk"])
        ids.append(bid)
        data.append(chunks_of(x, spec["chunk"]))
    nk = max(len(c) for c in data)
    for k in range(nk):
        for bid, cks in zip(ids, data):
            if k < len(cks):
                srv.submit(bid, cks[k], cks[k].shape[1], k)
    expect = sum(len(c) for c in data)
    res = []
    while len(res) < expect:
        res.extend(srv.poll(wait_ms=200))
    out = {}
    for bid in ids:
        rows = sorted([r for r in res if r["beam"] == bid], key=lambda r: r["seq"])
        out[bid] = [(int(r["status"]), float(r["mu"]), float(r["sigma"]),
                     sorted((int(c["dm_idx"]), int(c["t"]), int(c["width_idx"]), float(c["value"]))
                            for c in srv.candidates(bid, int(r["seq"]))))
                    for r in rows]
    return ids, out


def test_beam_same_alone_and_in_mix():
    X = dict(nchans=64, dm_list=BEAM["dm_list"], dtype_code=dd.DD_F32, chunk=1024)
    pulse = synth.Pulse(dm=X["dm_list"][20], t0=5000, width=2, amp=3.0)
    xs = stream_data(64, 8 * 1024, 21, pulses=[pulse])
    srv = dd.Server(1 << 31, nworkers=1)
    (bx,), alone = _serve(srv, [(X, xs)])
    srv.close()
    others = []
    for j, (nch, dt) in enumerate([(128, "u8"), (64, "f32"), (256, "u8"), (96, "f32")]):
        spec = dict(nchans=nch, dm_list=[0.05 * i for i in range(30 + 10 * j)],
                    dtype_code=dd.DD_U8 if dt == "u8" else dd.DD_F32, chunk=768 + 256 * j)
        others.append((spec, stream_data(nch, 8 * spec["chunk"], 100 + j, dtype=dt)))
    srv = dd.Server(1 << 31, nworkers=4)
    ids, mix = _serve(srv, others[:2] + [(X, xs)] + others[2:])
    srv.close()
    got = mix[ids[2]]
    assert len(got) == len(alone[bx])
    assert any(st == 0 and c for st, _, _, c in got)          # the pulse is found
    assert got == alone[bx]                                    # bit-identical, chunk by chunk


def test_admission_by_device_budget():
    srv = dd.Server(1 << 30, nworkers=1)
    spec = dict(nchans=256, dm_list=[0.1 * i for i in range(64)])
    a = srv.add_beam(256, 150.0, -0.1, 327.68e-6, spec["dm_list"], WIDTHS, 6.0, dd.DD_F32, 1 << 16)
    need = srv.beam_info(a)["device_bytes"]
    srv.close()
    srv = dd.Server(int(2.5 * need), nworkers=1)
    b1 = srv.add_beam(256, 150.0, -0.1, 327.68e-6, spec["dm_list"], WIDTHS, 6.0, dd.DD_F32, 1 << 16)
    b2 = srv.add_beam(256, 150.0, -0.1, 327.68e-6, spec["dm_list"], WIDTHS, 6.0, dd.DD_F32, 1 << 16)
    with pytest.raises(dd.DDError) as e:
        srv.add_beam(256, 150.0, -0.1, 327.68e-6, spec["dm_list"], WIDTHS, 6.0, dd.DD_F32, 1 << 16)
    assert e.value.code == dd.dd.DD_ERR_BUDGET
    used, budget = srv.memory()
    assert used == 2 * need and budget == int(2.5 * need)
    srv.remove_beam(b1)
    b3 = srv.add_beam(256, 150.0, -0.1, 327.68e-6, spec["dm_list"], WIDTHS, 6.0, dd.DD_F32, 1 << 16)
    assert srv.memory()[0] == 2 * need and b3 not in (b1, b2)
    srv.close()
