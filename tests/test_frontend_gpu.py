"""GPU parity of the front end (Section 5: channeliser, intensity, corner
turn) through the C ABI against the oracle, and the whole real-time chain
(voltages -> filterbank -> de-dispersion -> search) recovering a dispersed
pulse injected into the voltages."""
import math

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1107_2516_gb300 as dd
from paper_1107_2516_gb300 import build as ddbuild


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ddbuild.build()
    dd.load()


def _volts(npol, nsub, n, seed):
    r = np.random.default_rng(seed)
    return (r.standard_normal((npol, nsub, n)) + 1j * r.standard_normal((npol, nsub, n))).astype(np.complex64)


def _channelise(v, nfft, pitch_pad=0):
    npol, nsub, n = v.shape
    nb = n // nfft
    pitch = nb + pitch_pad
    x = torch.from_numpy(v.view(np.float32).copy()).cuda()
    out = torch.zeros(nsub * nfft * pitch, device="cuda")
    dd.dd_channelise(x, npol, nsub, n, nfft, out, pitch)
    torch.cuda.synchronize()
    return out.view(nsub * nfft, pitch)[:, :nb].cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("nfft", [2, 4, 8, 16, 32])
@pytest.mark.parametrize("npol", [1, 2])
def test_channelise_matches_oracle(nfft, npol):
    v = _volts(npol, 12, nfft * 700 + 2, 10 + nfft)
    got = _channelise(v, nfft, pitch_pad=3)
    ora = oracle.channelise_power(v, nfft)
    # FP32 transform: error of |X|^2 within a few ulps of the block energy
    scale = ora.max()
    assert np.max(np.abs(got - ora)) <= 1e-6 * nfft * scale


def test_channelise_rejects_bad_arguments():
    x = torch.zeros(2 * 4 * 64, device="cuda")
    out = torch.zeros(32 * 8, device="cuda")
    with pytest.raises(dd.DDError):
        dd.dd_channelise(x, 1, 4, 64, 6, out, 8)          # nfft not a power of two
    with pytest.raises(dd.DDError):
        dd.dd_channelise(x, 3, 4, 64, 8, out, 8)          # npol
    with pytest.raises(dd.DDError):
        dd.dd_channelise(x, 1, 4, 64, 8, out, 4)          # pitch too small
    with pytest.raises(dd.DDError):
        dd.dd_channelise(x[1:], 1, 4, 62, 8, out, 8)      # misaligned voltages


def test_pipeline_recovers_a_dispersed_pulse():
    # 32 subbands of 0.625 MHz from 620 MHz down (1.6 us voltage sampling),
    # 8 channels each -> 256 channels of 78.125 kHz at 12.8 us; a pulse at
    # DM 30 injected into the voltages with each subband's centre delay
    nsub, nfft, nb = 32, 8, 8192
    fbw, ftop, tv = 0.625, 620.0, 1.6e-6
    dm, t0, w, gain = 30.0, 3000, 6, 1.8
    v = _volts(1, nsub, nfft * nb, 5)
    fch1 = ftop - 0.5 * fbw / nfft                     # top channel centre
    delay = lambda f: 4.15e6 * dm * (1.0 / f ** 2 - 1.0 / fch1 ** 2) / (nfft * tv * 1e3)
    for s in range(nsub):
        # the voltages of a subband carry the pulse at the subband centre's
        # delay: all its channels see it there (smearing of a few samples at
        # the bottom of the band)
        d = int(round(delay(ftop - (s + 0.5) * fbw)))
        v[0, s, (t0 + d) * nfft:(t0 + d + w) * nfft] *= gain
    t_top = t0 + round(delay(ftop - 0.5 * fbw))        # arrival at the top channel
    x = torch.from_numpy(v.view(np.float32).copy()).cuda()
    nchans = nsub * nfft
    fil = torch.empty(nchans * nb, device="cuda")
    dd.dd_channelise(x, 1, nsub, nfft * nb, nfft, fil, nb)
    dms = [1.0 * i for i in range(61)]
    plan = dd.Plan(nchans, fch1, -fbw / nfft, nfft * tv, dms, [1, 2, 4, 8], 6.0, dd.DD_F32, nb)
    out = torch.empty(len(dms) * plan.nsamp_out, device="cuda")
    plan.execute(fil, nb, out)
    cands, total = plan.search(out, capacity=1 << 16)
    best = cands[np.argmax(cands["snr"])]
    assert abs(int(best["dm_idx"]) - 30) <= 1 and abs(int(best["t"]) - t_top) <= 3, best
    assert float(best["snr"]) > 10
    # the filterbank the de-dispersion saw is the oracle's front end
    ora = oracle.channelise_power(v, nfft)
    got = fil.view(nchans, nb).cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ora)) <= 1e-6 * nfft * ora.max()
    plan.close()
