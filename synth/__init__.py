"""Seeded synthetic filterbank inputs shared by the tests, the benchmark and smoke().

This module holds no de-dispersion arithmetic.  It draws noise, quantises it, and
adds square pulses at per-channel sample offsets that the CALLER supplies (the
tests take those offsets from the CPU oracle's delay table, the benchmark from
the library's plan).  The workloads mirror the paper's test data: Gaussian noise
of mean 0 and standard deviation 1 per channel plus square pulses whose height
per channel sets the frequency-integrated S/N (Section 4, the fake-pulsar test
of Table 2).

Every generator is deterministic in its seed (numpy PCG64).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional, Sequence

import numpy as np

__all__ = [
    "Workload", "Pulse", "WORKLOADS", "workload", "noise_f32", "quantize_u8",
    "to_f16_bits", "inject_pulses", "draw_pulses", "pulse_amplitude",
    "aligned_pitch",
]


@dataclasses.dataclass(frozen=True)
class Workload:
    """Plan parameters of one synthetic search, in the paper's units.

    fch1/foff in MHz (foff < 0: descending band, channel 0 is the top), tsamp in
    seconds, DM in pc cm^-3.  dm_list is built as i*dm_step in double, exactly
    as the pulse injection reads it back.
    """
    name: str
    nchans: int
    fch1: float
    foff: float
    tsamp: float
    nsamp: int
    ndm: int
    dm_step: float
    widths: tuple
    sigma: float = 6.0
    seed: int = 0
    dm_start: float = 0.0

    @property
    def dm_list(self) -> np.ndarray:
        i = np.arange(self.ndm, dtype=np.float64)
        return self.dm_start + i * self.dm_step


# Small FP32 case (fits the oracle in seconds), the LOFAR-like single beam,
# and the uint8 / FP16 precision cases share the first shape.
WORKLOADS = {
    "small_f32": Workload("small_f32", nchans=128, fch1=150.0, foff=-0.1953125,
                          tsamp=327.68e-6, nsamp=8192, ndm=64, dm_step=0.1,
                          widths=(1, 2, 4, 8), seed=1),
    "lofar_f32": Workload("lofar_f32", nchans=1024, fch1=150.0, foff=-0.01171875,
                          tsamp=163.84e-6, nsamp=1 << 20, ndm=2000, dm_step=0.05,
                          widths=(1, 2, 4, 8, 16, 32), seed=2),
    # the survey-plan comparison's beam (Table 4: 60 s at 300 MHz, 16 MHz in
    # 1024 channels); the sampling time is not stated, 64 us is taken.  Its
    # DM trials come from SURVEY_PLAN (3102 over three passes), not dm_list.
    "survey_f32": Workload("survey_f32", nchans=1024, fch1=308.0 - 0.0078125, foff=-0.015625,
                           tsamp=64e-6, nsamp=937500, ndm=3102, dm_step=0.03,
                           widths=(1, 2, 4, 8, 16, 32), seed=6),
}

# The survey plan of Table 1 / Table 4: (low DM, high DM, DM step, bin,
# subband DM step) per pass.
SURVEY_PLAN = ((0.00, 53.46, 0.03, 1, 0.66), (53.46, 88.26, 0.05, 2, 1.2), (88.26, 150.66, 0.10, 4, 2.4))


def workload(name: str) -> Workload:
    return WORKLOADS[name]


def aligned_pitch(nsamp: int, elem_bytes: int, align: int = 16) -> int:
    """Smallest row pitch (in elements) >= nsamp whose byte size is a multiple of align."""
    per = max(1, align // elem_bytes)
    return ((nsamp + per - 1) // per) * per


def noise_f32(nchans: int, nsamp: int, seed: int, pitch: Optional[int] = None) -> np.ndarray:
    """Channel-major float32 N(0,1) noise, shape [nchans][pitch]; padding columns are 0.

    Drawn as float64 normals and rounded to float32: numpy's float32 normal
    sampler takes accept/reject decisions in single precision with the
    platform's exp, and one decision that rounds differently on another
    machine shifts the whole rest of the stream; the float64 sampler's
    decisions agree across machines, so the same seed gives the same samples
    on the x86 build host and the Arm GPU host."""
    pitch = nsamp if pitch is None else pitch
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.zeros((nchans, pitch), dtype=np.float32)
    for c in range(nchans):
        out[c, :nsamp] = rng.standard_normal(nsamp)
    return out


def quantize_u8(x: np.ndarray, mean: float = 128.0, std: float = 16.0) -> np.ndarray:
    """q = clip(rint(mean + std*x), 0, 255) as uint8 (the 8-bit digitiser model)."""
    return np.clip(np.rint(mean + std * x.astype(np.float64)), 0, 255).astype(np.uint8)


def to_f16_bits(x: np.ndarray) -> np.ndarray:
    """Round float32 data to IEEE binary16 and return the raw 16-bit patterns."""
    return x.astype(np.float16).view(np.uint16)


@dataclasses.dataclass
class Pulse:
    dm: float        # the DM value the offsets were computed for
    t0: int          # arrival sample in the top (reference) channel
    width: int       # samples
    amp: float       # height per channel per sample


def pulse_amplitude(snr: float, nchans: int, width: int) -> float:
    """Per-channel height giving boxcar S/N `snr` for unit-variance noise.

    A square pulse of height a and width w summed over C channels gives a
    signal a*C*w against noise sqrt(C*w): S/N = a*sqrt(C*w).  (The paper's
    fake-pulsar file uses height 8/sqrt(1024) = 0.25 for a per-sample S/N of 8.)
    """
    return snr / math.sqrt(nchans * width)


def inject_pulses(data: np.ndarray, pulses: Sequence[Pulse],
                  offsets_for: Callable[[float], np.ndarray], nsamp: int) -> None:
    """Add square pulses in place.

    offsets_for(dm) must return the per-channel integer arrival offsets (int64,
    length nchans) of a pulse at that DM; the pulse covers samples
    t0 + offsets[c] + j for j < width in channel c.  Samples past nsamp are
    dropped.
    """
    nchans = data.shape[0]
    for p in pulses:
        off = np.asarray(offsets_for(p.dm), dtype=np.int64)
        assert off.shape == (nchans,)
        for c in range(nchans):
            s = p.t0 + int(off[c])
            e = min(s + p.width, nsamp)
            if s < nsamp and e > s:
                data[c, s:e] += np.asarray(p.amp, dtype=data.dtype)


def draw_pulses(n: int, dm_lo: float, dm_hi: float, width_lo: int, width_hi: int,
                snr_lo: float, snr_hi: float, t_hi: int, nchans: int,
                seed: int, min_sep: int = 64) -> List[Pulse]:
    """Draw n non-overlapping pulses: DM ~ U(dm_lo, dm_hi) (off-grid allowed),
    width ~ U{width_lo..width_hi}, S/N ~ U(snr_lo, snr_hi), t0 ~ U[0, t_hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out: List[Pulse] = []
    taken: List[int] = []
    while len(out) < n:
        dm = float(rng.uniform(dm_lo, dm_hi))
        w = int(rng.integers(width_lo, width_hi + 1))
        snr = float(rng.uniform(snr_lo, snr_hi))
        t0 = int(rng.integers(0, t_hi + 1))
        if any(abs(t0 - u) < min_sep + w for u in taken):
            continue
        taken.append(t0)
        out.append(Pulse(dm=dm, t0=t0, width=w, amp=pulse_amplitude(snr, nchans, w)))
    return out


@dataclasses.dataclass(frozen=True)
class Beam:
    """One beam of a batched or served workload (units as Workload)."""
    nchans: int
    fch1: float
    foff: float
    tsamp: float
    nsamp: int
    ndm: int
    dm_step: float
    dtype: str          # "f32" or "u8"
    seed: int

    @property
    def dm_list(self) -> np.ndarray:
        return np.arange(self.ndm, dtype=np.float64) * self.dm_step


def batch_beams(n: int, seed: int, maxshift_of: Callable[[int, float, float, float, float], int],
                mini: bool = False) -> List[Beam]:
    """Uneven beams for the batched workload.

    Full recipe: channels cycle {256, 512, 1024, 4096}; nsamp = 2^(16 + (7i mod 5));
    fch1 ~ U(120, 1500) MHz; bandwidth ~ U(6, 300) MHz capped at fch1/2;
    tsamp in {64, 81.92, 163.84, 327.68} us; DM trials ~ U{500..4000} with a
    log-uniform step in [0.01, 0.5]; the number of trials is reduced (not
    below 500) and then the step, until the maximum delay fits in half the
    input.  Even beams float32, odd beams uint8.  `mini` shrinks every size for
    tests (channels {64, 128, 256, 512}, nsamp 2^(13 + (7i mod 3)), 40..200 trials).
    maxshift_of(nchans, fch1, foff, tsamp, dm_max) must return the plan's
    maximum delay in samples (the caller supplies the delay law).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    chans = (64, 128, 256, 512) if mini else (256, 512, 1024, 4096)
    tsamps = (64e-6, 81.92e-6, 163.84e-6, 327.68e-6)
    out: List[Beam] = []
    for i in range(n):
        c = chans[i % len(chans)]
        nsamp = 1 << ((13 + (7 * i) % 3) if mini else (16 + (7 * i) % 5))
        fch1 = float(rng.uniform(120.0, 1500.0))
        bw = min(float(rng.uniform(6.0, 300.0)), 0.5 * fch1)
        ts = float(tsamps[int(rng.integers(0, 4))])
        lo, hi = (40, 200) if mini else (500, 4000)
        ndm = int(rng.integers(lo, hi + 1))
        step = float(np.exp(rng.uniform(np.log(0.01), np.log(0.5))))
        foff = -bw / c
        while maxshift_of(c, fch1, foff, ts, (ndm - 1) * step) > nsamp // 2:
            if ndm > lo:
                ndm = max(lo, int(ndm * 0.8))
            else:
                step *= 0.8
        out.append(Beam(nchans=c, fch1=fch1, foff=foff, tsamp=ts, nsamp=nsamp, ndm=ndm, dm_step=step,
                        dtype="f32" if i % 2 == 0 else "u8", seed=seed * 1000 + i))
    return out


@dataclasses.dataclass(frozen=True)
class ServedBeam:
    """One streaming beam: plan parameters, chunk size and arrival schedule."""
    nchans: int
    fch1: float
    foff: float
    tsamp: float
    ndm: int
    dm_max: float
    chunk: int
    dtype: str
    phase: float        # first arrival, fraction of a chunk period
    seed: int

    @property
    def dm_list(self) -> np.ndarray:
        return np.arange(self.ndm, dtype=np.float64) * (self.dm_max / self.ndm)

    @property
    def period(self) -> float:
        """Seconds of sky time per chunk (the real-time arrival interval)."""
        return self.chunk * self.tsamp


def serve_beams(n: int, seed: int) -> List[ServedBeam]:
    """Streaming beams: channels alternate 1024/4096, uint8 samples; tsamp in
    {64, 81.92, 163.84, 327.68} us; fch1 ~ U(300, 1500) MHz, bandwidth
    ~ U(0.10, 0.25) fch1; 1000..4096 DM trials over [0, 500); chunks of 65536
    samples with a random arrival phase."""
    rng = np.random.Generator(np.random.PCG64(seed))
    tsamps = (64e-6, 81.92e-6, 163.84e-6, 327.68e-6)
    out: List[ServedBeam] = []
    for i in range(n):
        c = 1024 if i % 2 == 0 else 4096
        ts = float(tsamps[int(rng.integers(0, 4))])
        fch1 = float(rng.uniform(300.0, 1500.0))
        bw = float(rng.uniform(0.10, 0.25)) * fch1
        ndm = int(rng.integers(1000, 4097))
        out.append(ServedBeam(nchans=c, fch1=fch1, foff=-bw / c, tsamp=ts, ndm=ndm, dm_max=500.0,
                              chunk=65536, dtype="u8", phase=float(rng.uniform(0.0, 1.0)),
                              seed=seed * 1000 + i))
    return out


def arrival_times(beam: ServedBeam, nchunks: int, seed: int, jitter: float = 0.1) -> np.ndarray:
    """Arrival time of each chunk (seconds from the start): one chunk period
    apart, each interval scaled by U(1 - jitter, 1 + jitter)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = beam.period * rng.uniform(1.0 - jitter, 1.0 + jitter, size=nchunks)
    t = beam.phase * beam.period + np.concatenate([[0.0], np.cumsum(gaps[:-1])])
    return t
