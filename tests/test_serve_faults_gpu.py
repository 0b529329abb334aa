"""Streaming server under host-injected faults: a missing chunk (gap in seq),
a repeated chunk, a late chunk, and a beam removed mid-stream.  No GPU fault
is caused: every failure is made on the host (chunks the test drops, reorders
or repeats).  After a gap the beam's stream restarts at the new chunk, so its
outputs must equal the oracle's de-dispersion of the restarted stream (zeros
before it); refused chunks produce no result; a removed beam leaves the other
beams' results unchanged and its memory returns to the budget."""
import numpy as np
import pytest

import oracle
import synth
from ddhelpers import fp_tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1107_2516_gb300 as dd
from paper_1107_2516_gb300 import build as ddbuild

WIDTHS = (1, 2, 4, 8)
NCH, FCH1, FOFF, TSAMP = 64, 150.0, -0.390625, 327.68e-6
DMS = [0.1 * i for i in range(40)]
CHUNK = 512


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ddbuild.build()


def _view(ptr, n, typestr):
    class _Cuda:
        __cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3}
    return torch.as_tensor(_Cuda(), device="cuda")


def _poll_until(srv, want, timeout_polls=400):
    """Poll until every (beam, seq) in `want` has reported; return {(beam, seq): record}."""
    got = {}
    for _ in range(timeout_polls):
        for r in srv.poll(wait_ms=50):
            got[(int(r["beam"]), int(r["seq"]))] = r
        if all(w in got for w in want):
            return got
    raise TimeoutError(f"missing results {[w for w in want if w not in got]}")


def _chunk(x, k):
    return torch.from_numpy(np.ascontiguousarray(x[:, k * CHUNK:(k + 1) * CHUNK])).pin_memory()


@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_gap_restarts_the_stream(dtype):
    nk = 14
    x = synth.noise_f32(NCH, nk * CHUNK, seed=31)
    if dtype == "u8":
        x = synth.quantize_u8(x)
    code = dd.DD_F32 if dtype == "f32" else dd.DD_U8
    srv = dd.Server(1 << 30, nworkers=2)
    bid = srv.add_beam(NCH, FCH1, FOFF, TSAMP, DMS, WIDTHS, 6.0, code, CHUNK)
    info = srv.beam_info(bid)
    M = info["maxshift"]
    d, m_o = oracle.delays(NCH, FCH1, FOFF, TSAMP, DMS)
    assert M == m_o
    nprime = (M + CHUNK - 1) // CHUNK
    lost = 5                                       # chunk 5 never arrives
    restart_at = lost + 1
    seen = 0
    for k in range(nk):
        if k == lost:
            continue
        rc = srv.submit(bid, _chunk(x, k), CHUNK, k)
        assert rc == (dd.DD_SEQ_GAP if k == restart_at else 0), k
        r = _poll_until(srv, [(bid, k)])[(bid, k)]
        j = k if k < lost else k - restart_at       # chunk index within its stream
        if j < nprime:
            assert r["status"] == dd.DD_PRIMING, k
            continue
        assert r["status"] == 0, k
        # the restarted stream: zeros, then the samples from chunk restart_at on
        first = 0 if k < lost else restart_at
        s = np.zeros((NCH, M + (j + 1) * CHUNK), dtype=x.dtype)
        s[:, M:] = x[:, first * CHUNK:(k + 1) * CHUNK]
        ref = oracle.dedisperse(s, d, (j + 1) * CHUNK)[:, j * CHUNK:(j + 1) * CHUNK]
        typ = "<f4" if dtype == "f32" else "<i4"
        got = _view(info["out_dev"], len(DMS) * CHUNK, typ).view(len(DMS), CHUNK).cpu().numpy()
        if dtype == "u8":
            assert np.array_equal(got.astype(np.int64), ref), k
        else:
            assert np.max(np.abs(got.astype(np.float64) - ref)) <= fp_tol(NCH), k
        seen += 1
    assert seen == (lost - nprime) + (nk - restart_at - nprime)
    srv.close()


def test_repeated_and_late_chunks_are_refused():
    x = synth.noise_f32(NCH, 8 * CHUNK, seed=32)
    srv = dd.Server(1 << 30, nworkers=1)
    bid = srv.add_beam(NCH, FCH1, FOFF, TSAMP, DMS, WIDTHS, 6.0, dd.DD_F32, CHUNK)
    for k in (0, 1):
        assert srv.submit(bid, _chunk(x, k), CHUNK, k) == 0
    with pytest.raises(dd.DDError) as e:
        srv.submit(bid, _chunk(x, 1), CHUNK, 1)          # repeated
    assert e.value.code == dd.DD_ERR_SEQ
    assert srv.submit(bid, _chunk(x, 3), CHUNK, 3) == dd.DD_SEQ_GAP
    with pytest.raises(dd.DDError) as e:
        srv.submit(bid, _chunk(x, 2), CHUNK, 2)          # late: after 3
    assert e.value.code == dd.DD_ERR_SEQ
    assert srv.submit(bid, _chunk(x, 4), CHUNK, 4) == 0
    got = _poll_until(srv, [(bid, k) for k in (0, 1, 3, 4)])
    assert sorted(s for (b, s) in got) == [0, 1, 3, 4]     # the refused chunks left no result
    for _ in range(5):
        assert not [r for r in srv.poll(wait_ms=20) if int(r["seq"]) == 2]
    srv.close()


def _run_beam(srv, bid, x, nk, remove_other=None):
    res = {}
    for k in range(nk):
        srv.submit(bid, _chunk(x, k), CHUNK, k)
        if remove_other is not None and k == nk // 2:
            remove_other()
    res = _poll_until(srv, [(bid, k) for k in range(nk)])
    out = []
    for k in range(nk):
        r = res[(bid, k)]
        c = srv.candidates(bid, k) if r["status"] == 0 else []
        out.append((int(r["status"]), float(r["mu"]), float(r["sigma"]),
                    sorted((int(a["dm_idx"]), int(a["t"]), int(a["width_idx"]), float(a["value"])) for a in c)))
    return out


def test_beam_removed_mid_stream():
    nk = 10
    xa = synth.noise_f32(NCH, nk * CHUNK, seed=41)
    xb = synth.noise_f32(NCH, nk * CHUNK, seed=42)
    xb[:, 3000:3004] += 2.0
    srv = dd.Server(1 << 30, nworkers=1)
    b = srv.add_beam(NCH, FCH1, FOFF, TSAMP, DMS, WIDTHS, 5.0, dd.DD_F32, CHUNK)
    alone = _run_beam(srv, b, xb, nk)
    srv.close()

    srv = dd.Server(1 << 30, nworkers=2)
    a = srv.add_beam(NCH, FCH1, FOFF, TSAMP, DMS, WIDTHS, 5.0, dd.DD_F32, CHUNK)
    b = srv.add_beam(NCH, FCH1, FOFF, TSAMP, DMS, WIDTHS, 5.0, dd.DD_F32, CHUNK)
    need_b = srv.beam_info(b)["device_bytes"]
    for k in range(nk):                      # beam a's chunks queued ahead of b's
        srv.submit(a, _chunk(xa, k), CHUNK, k)
    removed = []

    def remove_a():
        srv.remove_beam(a)
        removed.append(True)
    mixed = _run_beam(srv, b, xb, nk, remove_other=remove_a)
    assert removed
    assert mixed == alone                    # the other beam is unaffected, chunk by chunk
    with pytest.raises(dd.DDError) as e:
        srv.submit(a, _chunk(xa, 0), CHUNK, nk)
    assert e.value.code == dd.dd.DD_ERR_ARG
    for _ in range(50):                      # a's running chunk (if any) finishes, then its memory returns
        srv.poll(wait_ms=20)
        if srv.memory()[0] == need_b:
            break
    assert srv.memory()[0] == need_b
    srv.close()


def test_serving_beam_uses_kernel5_where_it_fits():
    b = synth.serve_beams(64, 5)[2]          # 1024 channels, uint8: kernel 5's tables fit
    srv = dd.Server(1 << 36, nworkers=1)
    bid = srv.add_beam(b.nchans, b.fch1, b.foff, b.tsamp, b.dm_list, (1, 2, 4, 8, 16, 32, 64), 6.0,
                       dd.DD_U8, b.chunk)
    k, cfg = srv.beam_kernel(bid)
    assert k == 5 and cfg in range(9, 13)
    small = srv.add_beam(NCH, FCH1, FOFF, TSAMP, DMS, WIDTHS, 6.0, dd.DD_F32, CHUNK)
    assert srv.beam_kernel(small)[0] == 3    # kernel 5 unavailable (too many delay patterns): default
    srv.close()
