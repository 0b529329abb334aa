"""Pins of the front-end oracle (Section 5: channeliser, intensity, corner
turn) to things other than itself: a brute-force DFT written out with
cos/sin, Parseval's identity, pure tones landing in one channel of the
descending-frequency order, and the polarisation sum."""
import math

import numpy as np
import pytest

import oracle


def _volts(npol, nsub, n, seed):
    r = np.random.default_rng(seed)
    return (r.standard_normal((npol, nsub, n)) + 1j * r.standard_normal((npol, nsub, n))).astype(np.complex64)


def test_brute_force_dft_on_tiny_input():
    nfft, v = 8, _volts(1, 3, 32, 1)
    got = oracle.channelise_power(v, nfft)
    for s in range(3):
        for b in range(4):
            blk = v[0, s, b * nfft:(b + 1) * nfft].astype(np.complex128)
            for k in range(nfft):
                X = sum(blk[q] * complex(math.cos(-2 * math.pi * k * q / nfft), math.sin(-2 * math.pi * k * q / nfft))
                        for q in range(nfft))
                j = (nfft // 2 - 1 - k) % nfft          # channel of bin k (descending frequency)
                assert abs(got[s * nfft + j, b] - abs(X) ** 2) <= 1e-9 * max(1.0, abs(X) ** 2)


@pytest.mark.parametrize("nfft", [2, 4, 8, 16])
def test_parseval(nfft):
    v = _volts(2, 4, 64 * nfft, 2)
    got = oracle.channelise_power(v, nfft)
    for s in range(4):
        for b in range(64):
            e = sum(np.sum(np.abs(v[p, s, b * nfft:(b + 1) * nfft].astype(np.complex128)) ** 2) for p in range(2))
            assert abs(got[s * nfft:(s + 1) * nfft, b].sum() - nfft * e) <= 1e-9 * nfft * e


def test_tone_lands_in_one_channel_descending():
    # a tone at bin offset m (positive m: above the subband's reference
    # frequency) lands in channel nfft/2 - 1 - m (mod nfft): higher frequency,
    # lower channel index
    nfft, n = 8, 8 * 16
    t = np.arange(n)
    for m in range(-nfft // 2, nfft // 2):
        v = np.exp(2j * math.pi * m * t / nfft)[None, None, :]
        got = oracle.channelise_power(v, nfft)
        j = (nfft // 2 - 1 - m) % nfft
        assert np.allclose(got[j], nfft ** 2) and np.allclose(np.delete(got, j, axis=0), 0.0, atol=1e-18)


def test_polarisations_add_and_leftover_dropped():
    v = _volts(2, 2, 8 * 10 + 5, 3)
    both = oracle.channelise_power(v, 8)
    assert both.shape == (16, 10)
    a = oracle.channelise_power(v[:1], 8)
    b = oracle.channelise_power(v[1:], 8)
    assert np.allclose(both, a + b, rtol=1e-12)
