"""Shared test helpers: build seeded inputs, run the library through its C ABI,
and compare with the CPU oracle (candidate lists with the gray-zone rule)."""
from __future__ import annotations

import math

import numpy as np

import oracle
import synth

# FP32 bound on unit-variance data: max |out_gpu - out_oracle| <= 1e-5 * nchans.
def fp_tol(nchans: int) -> float:
    return 1e-5 * nchans


def oracle_offsets(wl_or_params):
    """Per-channel pulse offsets from the ORACLE's delay law for any DM."""
    nchans, fch1, foff, tsamp = wl_or_params

    def f(dm):
        return oracle.delays(nchans, fch1, foff, tsamp, [dm])[0][0]
    return f


def make_input(nchans, nsamp, fch1, foff, tsamp, seed, pulses=(), dtype="f32", pitch=None):
    """Seeded N(0,1) float data (+ pulses placed with oracle delays), converted to
    the requested input type.  Returns (array [nchans][pitch], float32 source)."""
    x = synth.noise_f32(nchans, nsamp, seed, pitch=pitch)
    if pulses:
        synth.inject_pulses(x, list(pulses), oracle_offsets((nchans, fch1, foff, tsamp)), nsamp)
    if dtype == "f32":
        return x, x
    if dtype == "u8":
        return synth.quantize_u8(x), x
    if dtype == "f16":
        return synth.to_f16_bits(x), x
    raise ValueError(dtype)


def keys(c):
    return {(int(r["dm_idx"]), int(r["t"]), int(r["width_idx"])) for r in c}


def boxcar(out_row: np.ndarray, t: int, w: int):
    seg = out_row[t:t + w]
    return int(seg.sum()) if out_row.dtype == np.int64 else float(np.sum(seg, dtype=np.float64))


def compare_candidates(gpu_c, ora_out, widths, mu_g, sg_g, mu_o, sg_o, k, eps_elem):
    """Gray-zone identity check of two candidate lists.

    ora_out: the oracle's full de-dispersed buffer.  A point whose oracle boxcar
    lies within w*eps_elem + |T_w(gpu) - T_w(oracle)| of the oracle threshold
    may legitimately fall on either side; it is excluded from the identity
    check and counted.  Everything else must match exactly.
    Returns (n_matched, n_gray).
    """
    ora_c = oracle.search(ora_out, widths, mu_o, sg_o, k)
    G, O = keys(gpu_c), keys(ora_c)
    gray = 0
    diff = G ^ O
    for (i, t, wi) in diff:
        w = widths[wi]
        b = boxcar(ora_out[i], t, w)
        to = w * mu_o + k * sg_o * math.sqrt(w)
        tg = w * mu_g + k * sg_g * math.sqrt(w)
        slack = w * eps_elem + abs(tg - to) + 1e-9 * abs(to)
        assert abs(b - to) <= slack, f"candidate mismatch at {(i, t, wi)}: B={b} T={to} slack={slack}"
        gray += 1
    # values of matched GPU candidates agree with the oracle boxcar
    for r in gpu_c:
        key = (int(r["dm_idx"]), int(r["t"]), int(r["width_idx"]))
        if key in O:
            w = widths[key[2]]
            b = boxcar(ora_out[key[0]], key[1], w)
            assert abs(r["value"] - b) <= w * eps_elem + 1e-9 * abs(b), (key, r["value"], b)
    return len(G & O), gray
