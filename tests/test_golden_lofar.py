"""The LOFAR-like beam's golden file (the oracle's full run, written by
tests/golden/make_lofar_golden.py), checked without a GPU: the seeded input
regenerates to the recorded SHA-256; the list is sorted and complete in form
(every record above its threshold, S/N consistent with mu and sigma); a
sample of its boxcar values, and the strongest candidate of every injected
pulse, are recomputed here by the oracle's one-point helper; and the
injected pulses are found near their DM and time (Section 4: a pulse of
known S/N is recovered)."""
import hashlib
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "lofar_f32_oracle")
WL = synth.workload("lofar_f32")


@pytest.fixture(scope="module")
def golden():
    if not os.path.exists(GOLDEN + ".npz"):
        pytest.skip("golden file not generated")
    with open(GOLDEN + ".json") as f:
        meta = json.load(f)
    return meta, np.load(GOLDEN + ".npz")


@pytest.fixture(scope="module")
def lofar_input():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_lofar_golden",
                                                  os.path.join(HERE, "golden", "make_lofar_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.lofar_input()


def test_golden_form(golden):
    meta, c = golden
    n = meta["n_candidates"]
    assert len(c["dm_idx"]) == len(c["t"]) == len(c["width_idx"]) == len(c["value"]) == n > 0
    key = np.lexsort((c["width_idx"], c["t"], c["dm_idx"]))
    assert np.array_equal(key, np.arange(n))                   # sorted by (dm, t, width)
    w = np.asarray(meta["widths"])[c["width_idx"].astype(np.int64)]
    mu, sg, k = meta["mu"], meta["sigma"], meta["sigma_k"]
    assert np.all(c["value"] > w * mu + k * sg * np.sqrt(w))
    np.testing.assert_allclose(c["snr"], (c["value"] - w * mu) / (sg * np.sqrt(w)), rtol=1e-12)
    assert np.all((c["t"] >= 0) & (c["t"] + w <= meta["nsamp_out"]))
    # unit-variance noise summed over C channels: sigma close to sqrt(C)
    assert abs(sg - math.sqrt(WL.nchans)) < 0.01 * math.sqrt(WL.nchans)


def test_golden_reproduced_by_the_oracle(golden, lofar_input):
    meta, c = golden
    x, d, m, nout, pulses = lofar_input
    assert m == meta["maxshift"] and nout == meta["nsamp_out"]
    assert hashlib.sha256(x.tobytes()).hexdigest() == meta["input_sha256"]
    rng = np.random.default_rng(3)
    pick = list(rng.choice(len(c["t"]), size=min(200, len(c["t"])), replace=False))
    # plus the strongest record near every injected pulse
    for p in pulses:
        near = np.nonzero(np.abs(c["t"].astype(np.int64) - p.t0) < 64)[0]
        if near.size:
            pick.append(int(near[np.argmax(c["snr"][near])]))
    for r in pick:
        i, t, wi = int(c["dm_idx"][r]), int(c["t"][r]), int(c["width_idx"][r])
        w = meta["widths"][wi]
        b = sum(oracle.point_f32(x, d[i], t + j) for j in range(w))
        assert abs(b - c["value"][r]) <= 1e-9 * max(1.0, abs(b)), (i, t, wi)
    # most pulses (S/N 8-20, some at off-grid DMs and narrow widths) are found
    # within a few DM steps and samples of where they were injected
    found = 0
    for p in pulses:
        i0 = int(round(p.dm / WL.dm_step))
        hit = (np.abs(c["dm_idx"].astype(np.int64) - i0) <= 3) & (np.abs(c["t"].astype(np.int64) - p.t0) < 48)
        found += bool(hit.any())
    assert found >= 12
