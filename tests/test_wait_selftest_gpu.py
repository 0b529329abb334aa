"""Failure detection without a GPU fault: the bounded mbarrier wait that every
staged kernel uses gives up after its limit, reports DD_ERR_TIMEOUT to the
host, and leaves the context usable.  The wait is made to run out by arming an
mbarrier for a copy that is never issued (nothing is in flight), with the
limit shortened to 50 ms."""
import time

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1107_2516_gb300 as dd
from paper_1107_2516_gb300 import build as ddbuild
from paper_1107_2516_gb300.dd import DD_ERR_ARG, DD_ERR_TIMEOUT, dd_wait_selftest


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ddbuild.build()


def test_wait_runs_out_and_context_stays_usable():
    assert dd_wait_selftest(50_000_000, True) == (0, 0)           # the copy arrives: no timeout
    t0 = time.time()
    rc, st = dd_wait_selftest(50_000_000, False)                  # nothing arrives
    dt = time.time() - t0
    assert rc == DD_ERR_TIMEOUT and st == DD_ERR_TIMEOUT
    assert 0.05 <= dt < 2.0, dt
    assert "gave up" in dd.dd_last_error()
    assert dd_wait_selftest(0, False)[0] == DD_ERR_ARG
    # the context still runs the de-dispersion correctly
    wl = synth.workload("small_f32")
    x = synth.noise_f32(wl.nchans, wl.nsamp, wl.seed)
    d, m = oracle.delays(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list)
    plan = dd.Plan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list, wl.widths, wl.sigma, dd.DD_F32, wl.nsamp)
    out = torch.empty(wl.ndm * plan.nsamp_out, dtype=torch.float32, device="cuda")
    plan.execute(torch.from_numpy(x).cuda(), wl.nsamp, out)
    torch.cuda.synchronize()
    ref = oracle.dedisperse(x, d, wl.nsamp - m)
    assert np.max(np.abs(out.cpu().numpy().reshape(wl.ndm, -1) - ref)) <= 1e-5 * wl.nchans
    plan.close()
