"""The allocation-free statistics entry point (dd_stats_f32_noalloc).

It serves callers that cannot allocate device memory once running (a real-time
pipeline with a fixed memory budget, or code whose allocator belongs to
another runtime).  This file is collected last so that a run stopping at the
first failure has already run every other test.  The test calls the entry
point through the C ABI twice in a row on the same buffer and compares each
result with the statistics the plan-based path (dd_execute + dd_search)
reports, within the tolerance the parity tests use, and with the FP64
oracle's statistics of the same float32 values.
"""
import numpy as np
import pytest

import oracle
import synth
from ddhelpers import fp_tol, make_input

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1107_2516_gb300 as dd
from paper_1107_2516_gb300 import build as ddbuild


def test_noalloc_stats_match_plan_stats_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ddbuild.build()
    wl = synth.workload("small_f32")
    arr, _ = make_input(wl.nchans, wl.nsamp, wl.fch1, wl.foff, wl.tsamp, wl.seed)
    plan = dd.Plan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list, wl.widths, wl.sigma,
                   dd.DD_F32, wl.nsamp)
    x = torch.from_numpy(arr).cuda()
    out = torch.empty(wl.ndm * plan.nsamp_out, dtype=torch.float32, device="cuda")
    plan.execute(x, wl.nsamp, out)
    plan.search(out)
    mu_ref, sg_ref = plan.stats()
    res = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    # the FP64 oracle's two-pass statistics of exactly these float32 values
    mu_o, sg_o = oracle.stats(out.cpu().numpy().astype(np.float64))
    for _ in range(2):
        res.fill_(float("nan"))
        dd.dd_stats_f32_noalloc(out, out.numel(), res)
        torch.cuda.synchronize()
        mu, sg = (float(v) for v in res.cpu())
        assert abs(mu - mu_ref) <= fp_tol(wl.nchans)
        assert abs(sg - sg_ref) <= 1e-5 * sg_ref
        # per-thread partials of 16 values are FP32: relative error ~1e-7 each
        assert abs(mu - mu_o) <= 1e-6 * sg_o and abs(sg - sg_o) <= 1e-6 * sg_o
    # a buffer beyond the fixed scratch is refused before any launch
    with pytest.raises(dd.DDError) as e:
        dd.dd_stats_f32_noalloc(out, (1 << 28) + 1, res)
    assert e.value.code == dd.dd.DD_ERR_ARG
    plan.close()
