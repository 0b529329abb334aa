"""Write the oracle's complete result for the LOFAR-like beam as a golden file.

Runs the FP64 CPU oracle (and nothing else: only ``oracle`` and ``synth`` are
imported) over the whole benchmark workload -- 1024 channels, 2^20 samples,
2000 DM trials 0-99.95 step 0.05, N(0,1) noise (seed 2) plus 16 pulses placed
with the oracle's own delay table -- and stores the population mean and
standard deviation of the full de-dispersed buffer (Section 3, output stage)
and the complete candidate list of the boxcar search (widths 1..32, 6 sigma),
sorted by (dm, t, width).  The input's SHA-256 is stored too, so a reader can
check that the seeded generator reproduced the same samples.

About 2.1e12 double additions: a few minutes on 8 host cores, and 21 GB of
memory (the input and the float64 output plane).

    python tests/golden/make_lofar_golden.py [--threads N]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT_NPZ = os.path.join(HERE, "lofar_f32_oracle.npz")
OUT_JSON = os.path.join(HERE, "lofar_f32_oracle.json")


def lofar_input():
    """The workload's input exactly as the GPU test builds it: (x, delays, maxshift, nout, pulses)."""
    wl = synth.workload("lofar_f32")
    d, m = oracle.delays(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list)
    nout = wl.nsamp - m
    x = synth.noise_f32(wl.nchans, wl.nsamp, seed=wl.seed)
    pulses = synth.draw_pulses(16, 0.0, float(wl.dm_list[-1]), 1, 32, 8.0, 20.0, nout - 64,
                               wl.nchans, seed=wl.seed)
    synth.inject_pulses(x, pulses, lambda dm: oracle.delays(wl.nchans, wl.fch1, wl.foff, wl.tsamp,
                                                            [dm])[0][0], wl.nsamp)
    return x, d, m, nout, pulses


def sha256(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count())
    args = ap.parse_args()
    oracle.set_threads(args.threads)
    wl = synth.workload("lofar_f32")
    t0 = time.time()
    x, d, m, nout, pulses = lofar_input()
    digest = sha256(x)
    t1 = time.time()
    out = oracle.dedisperse(x, d, nout)
    t2 = time.time()
    mu, sg = oracle.stats(out)
    cands = oracle.search(out, list(wl.widths), mu, sg, wl.sigma, cap=1 << 22)
    t3 = time.time()
    np.savez_compressed(
        OUT_NPZ,
        dm_idx=cands["dm_idx"].astype(np.int32), t=cands["t"].astype(np.int32),
        width_idx=cands["width_idx"].astype(np.int8), value=cands["value"], snr=cands["snr"])
    meta = {
        "_source": "written by tests/golden/make_lofar_golden.py: the FP64 CPU oracle over the whole "
                   "LOFAR-like beam (Section 3.1 sum, Section 3 output-stage statistics over the whole "
                   "buffer, boxcar n-sigma search); no value comes from the GPU library",
        "workload": "lofar_f32: 1024 ch, fch1 150 MHz, foff -0.01171875 MHz, tsamp 163.84 us, 2^20 "
                    "samples, 2000 DMs 0-99.95 step 0.05, N(0,1) seed 2 + 16 pulses (seed 2)",
        "input_sha256": digest,
        "maxshift": int(m), "nsamp_out": int(nout),
        "widths": list(wl.widths), "sigma_k": wl.sigma,
        "mu": mu, "sigma": sg,
        "n_candidates": int(len(cands)),
        "pulses": [{"dm": p.dm, "t0": p.t0, "width": p.width, "amp": p.amp} for p in pulses],
        "threads": args.threads,
        "seconds": {"input": round(t1 - t0, 1), "dedisperse": round(t2 - t1, 1),
                    "stats_search": round(t3 - t2, 1)},
    }
    with open(OUT_JSON, "w") as f:
        json.dump(meta, f, indent=1)
        f.write("\n")
    print(json.dumps({k: v for k, v in meta.items() if k != "pulses"}))


if __name__ == "__main__":
    main()
