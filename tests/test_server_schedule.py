"""The streaming server's host-side schedule, checked without a GPU.

dd_server_ring_schedule runs the same sequence check and ring steps the
server applies to a beam's device buffers.  Here a ring of stream-sample
indices is simulated on the CPU from that schedule: every searched chunk's
window must hold exactly the stream samples its outputs need
([k*chunk - maxshift, (k+1)*chunk) for the k-th chunk of the stream, with the
samples before the stream's start read as zeros), history moves must never
overlap their destination, and repeated, late and missing chunks must be
refused or restart the stream (Section 3, "Maximum shift"; serving)."""
import numpy as np
import pytest

import paper_1107_2516_gb300 as dd
from paper_1107_2516_gb300.dd import DD_OK

ZERO = -(1 << 40)      # marks a column that holds a zero (no stream sample)


def _simulate(M, chunk, seqs):
    sch = dd.dd_server_ring_schedule(M, chunk, seqs)
    span = sch["span"]
    K = 2 + M // chunk
    assert span == M + K * chunk
    ring = np.full(span + chunk, ZERO, dtype=np.int64)
    ring[:M] = np.arange(-M, 0)                 # the stream's zero history
    j = -1                                      # chunks since the stream (re)started
    last_move = None
    expect_next = None
    for i, seq in enumerate(seqs):
        st = int(sch["status"][i])
        # the sequence rule
        if expect_next is None or seq == expect_next:
            assert st == DD_OK, (i, seq)
        elif seq < expect_next:
            assert st == dd.DD_ERR_SEQ, (i, seq)
            assert sch["write_col"][i] == sch["window_col"][i] == sch["move_src"][i] == -1
            continue
        else:
            assert st == dd.DD_SEQ_GAP and sch["restart"][i] == 1, (i, seq)
        expect_next = seq + 1
        if sch["restart"][i]:
            ring[:M] = np.arange(-M, 0)
            j = -1
        j += 1
        src = int(sch["move_src"][i])
        if src >= 0:
            assert src >= M                    # source and destination disjoint
            assert src + M <= span
            ring[:M] = ring[src:src + M].copy()
            if last_move is not None:
                assert i - last_move >= K      # at most one move per K chunks
            last_move = i
        w, win = int(sch["write_col"][i]), int(sch["window_col"][i])
        assert w == win + M and 0 <= win and w + chunk <= span
        ring[w:w + chunk] = np.arange(j * chunk, (j + 1) * chunk)
        assert int(sch["priming"][i]) == (j * chunk < M), (i, j)
        if not sch["priming"][i]:
            got = ring[win:win + M + chunk]
            want = np.arange(j * chunk - M, (j + 1) * chunk)
            assert np.array_equal(got, want), (i, j)
    return sch


@pytest.mark.parametrize("M,chunk", [(0, 64), (5, 64), (63, 64), (64, 64), (65, 64), (256, 64),
                                     (257, 64), (3746, 65536), (35761, 65536), (1000, 7)])
def test_in_order_stream_windows(M, chunk):
    _simulate(M, chunk, list(range(40)))


@pytest.mark.parametrize("M,chunk", [(5, 64), (100, 64), (257, 64), (0, 16)])
def test_gaps_duplicates_and_late_chunks(M, chunk):
    seqs = [10, 11, 12, 12, 11, 14, 15, 13, 16, 17, 30, 31, 29, 32, 33, 34, 35, 36, 37]
    sch = _simulate(M, chunk, seqs)
    # the first chunk may carry any seq; 12 repeated and 11, 13, 29 late: refused
    refused = [s for s, st in zip(seqs, sch["status"]) if st == dd.DD_ERR_SEQ]
    assert refused == [12, 11, 13, 29]
    restarts = [s for s, r in zip(seqs, sch["restart"]) if r]
    assert restarts == [14, 30]


def test_schedule_rejects_bad_arguments():
    with pytest.raises(dd.DDError):
        dd.dd_server_ring_schedule(-1, 64, [0])
    with pytest.raises(dd.DDError):
        dd.dd_server_ring_schedule(10, 0, [0])
