"""Run one de-dispersion case of the LOFAR-like beam for profiling.

    python -m paper_1107_2516_gb300.profile_case --dm-lo 1744 --ndm 256 --tile 1 16

A contiguous slice of the 2000 DM trials (0..99.95 step 0.05) over 1024
channels and 2^20 samples, random N(0,1) input generated on the device,
two warm-up executions and one timed execution (CUDA events).  Small slices
keep ncu captures inside a few GB of device memory.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    import torch

    import synth
    import paper_1107_2516_gb300 as dd
    from paper_1107_2516_gb300 import build as ddbuild

    ap = argparse.ArgumentParser()
    ap.add_argument("--dm-lo", type=int, default=1744)
    ap.add_argument("--ndm", type=int, default=256)
    ap.add_argument("--nsamp", type=int, default=1 << 20)
    ap.add_argument("--tile", type=int, nargs=2, default=None, metavar=("CONFIG", "GROUP"))
    ap.add_argument("--kernel", type=int, default=0)
    ap.add_argument("--search", action="store_true", help="also run dd_search")
    a = ap.parse_args(argv)
    ddbuild.build()
    wl = synth.workload("lofar_f32")
    dms = wl.dm_list[a.dm_lo:a.dm_lo + a.ndm]
    plan = dd.Plan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, dms, wl.widths, wl.sigma, dd.DD_F32, a.nsamp)
    if a.kernel:
        plan.set_kernel(a.kernel)
    if a.tile and plan.kernel in (2, 3, 4, 5):
        plan.set_tile(*a.tile)
    g = torch.Generator(device="cuda")
    g.manual_seed(1)
    x = torch.randn(wl.nchans, a.nsamp, device="cuda", generator=g)
    out = torch.empty(len(dms) * plan.nsamp_out, device="cuda")
    for _ in range(2):
        plan.execute(x, a.nsamp, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    plan.execute(x, a.nsamp, out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if a.search:
        plan.search(out)
    units = len(dms) * plan.nsamp_out
    tile = plan.tile if plan.kernel in (2, 3, 4, 5) else None
    print(f"kernel {plan.kernel} tile {tile} dms {a.dm_lo}+{len(dms)} nsamp {a.nsamp}: {ms:.2f} ms, "
          f"{units / (ms / 1e3):.3e} DM-trial.samples/s, {units * wl.nchans / ms / 1e9:.2f} Tadd/s")
    plan.close()


if __name__ == "__main__":
    main()
