"""CPU oracle (FP64 / exact integer) for brute-force de-dispersion and the
boxcar threshold search -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product library never loads it and shares
no code with it.  The arithmetic lives in ``dd_oracle.c`` (plain loops, built
with FMA contraction off); this module builds it with gcc and marshals numpy
arrays through ctypes.

Paper passages followed (Magro et al. 2011):
  Eq. 1 (Section 1)        dispersion delay          -> delays()
  Section 3, Eq. 2         maximum shift             -> delays(), maxshift_eq2()
  Section 3.1              brute-force sum           -> dedisperse()
  Section 3 (output thread) mean, sigma, n-sigma test -> stats(), search()
  Section 3.2              subband de-dispersion     -> subband_tables(), subband_dedisperse()
  Section 3.2, Table 1     binning, survey passes    -> bin_samples(), survey_passes()
  Section 5, Tables 5-6    channelise, power, corner turn -> channelise_power()
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dd_oracle.c")
_LIB = os.path.join(_HERE, "libdd_oracle.so")
_lock = threading.Lock()
_lib = None

CAND_DTYPE = np.dtype([("dm_idx", np.int64), ("t", np.int64), ("width_idx", np.int64),
                       ("snr", np.float64), ("value", np.float64)])


def build(force: bool = False) -> str:
    """Compile dd_oracle.c into libdd_oracle.so (gcc, -O2, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = C.CDLL(_LIB)
        i64, f64, vp = C.c_int64, C.c_double, C.c_void_p
        lib.oracle_num_threads.restype = C.c_int
        lib.oracle_set_threads.argtypes = [C.c_int]
        lib.oracle_delay_exact.restype = f64
        lib.oracle_delay_exact.argtypes = [f64, f64, i64, f64, f64, i64]
        lib.oracle_delays.restype = C.c_int
        lib.oracle_delays.argtypes = [i64, f64, f64, f64, vp, i64, vp, C.POINTER(i64)]
        lib.oracle_maxshift_eq2.restype = f64
        lib.oracle_maxshift_eq2.argtypes = [i64, f64, f64, f64, f64]
        lib.oracle_half_to_double.restype = f64
        lib.oracle_half_to_double.argtypes = [C.c_uint16]
        for name in ("oracle_dedisperse_f32", "oracle_dedisperse_f16", "oracle_dedisperse_u8"):
            getattr(lib, name).restype = None
            getattr(lib, name).argtypes = [vp, i64, i64, vp, i64, i64, vp]
        lib.oracle_point_f32.restype = f64
        lib.oracle_point_f32.argtypes = [vp, i64, i64, vp, i64]
        lib.oracle_row_f32.restype = None
        lib.oracle_row_f32.argtypes = [vp, i64, i64, vp, i64, vp]
        lib.oracle_stats_f64.argtypes = [vp, i64, C.POINTER(f64), C.POINTER(f64)]
        lib.oracle_stats_i64.argtypes = [vp, i64, C.POINTER(f64), C.POINTER(f64)]
        lib.oracle_threshold.restype = f64
        lib.oracle_threshold.argtypes = [i64, f64, f64, f64]
        for name in ("oracle_search_f64", "oracle_search_i64"):
            getattr(lib, name).restype = i64
            getattr(lib, name).argtypes = [vp, i64, i64, vp, i64, f64, f64, f64, vp, i64]
        lib.oracle_subband_tables.restype = C.c_int
        lib.oracle_subband_tables.argtypes = [i64, f64, f64, f64, vp, i64, i64, i64, vp, vp, vp,
                                              C.POINTER(i64)]
        for name in ("oracle_subband_f32", "oracle_subband_f16", "oracle_subband_u8"):
            getattr(lib, name).restype = None
            getattr(lib, name).argtypes = [vp, i64, i64, i64, vp, vp, i64, i64, i64, vp]
        lib.oracle_bin.restype = None
        lib.oracle_bin.argtypes = [vp, C.c_int, i64, i64, i64, i64, vp, i64]
        lib.oracle_subband_f64.restype = None
        lib.oracle_subband_f64.argtypes = [vp, i64, i64, i64, vp, vp, i64, i64, i64, vp]
        lib.oracle_subband_point_f32.restype = f64
        lib.oracle_subband_point_f32.argtypes = [vp, i64, i64, i64, vp, vp, i64, i64, i64]
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def delay_exact(fch1, foff, nchans, tsamp, dm, c) -> float:
    """Fractional delay in samples of channel c at DM dm (Eq. 1 / tsamp)."""
    return float(_load().oracle_delay_exact(fch1, foff, nchans, tsamp, dm, c))


def delays(nchans: int, fch1: float, foff: float, tsamp: float, dm_list) -> tuple:
    """Integer delay table [ndm][nchans] (int64) and maxshift (Eq. 1, rounded)."""
    dm = np.ascontiguousarray(np.asarray(dm_list, dtype=np.float64))
    d = np.empty((dm.size, nchans), dtype=np.int64)
    m = C.c_int64(0)
    rc = _load().oracle_delays(nchans, fch1, foff, tsamp, _p(dm), dm.size, _p(d), C.byref(m))
    if rc != 0:
        raise ValueError("oracle_delays: invalid arguments")
    return d, int(m.value)


def maxshift_eq2(nchans, fch1, foff, tsamp, dm_max) -> float:
    """Eq. 2 derivative approximation of the maximum shift (sanity bound only)."""
    return float(_load().oracle_maxshift_eq2(nchans, fch1, foff, tsamp, dm_max))


def half_to_double(bits: int) -> float:
    return float(_load().oracle_half_to_double(int(bits)))


def dedisperse(data: np.ndarray, delay_table: np.ndarray, nout: int) -> np.ndarray:
    """Brute-force sum (Section 3.1).

    data: [nchans][pitch] float32, uint16 (binary16 bit patterns) or uint8.
    Returns [ndm][nout] float64 for float input, int64 for uint8.
    """
    lib = _load()
    data = np.ascontiguousarray(data)
    dl = np.ascontiguousarray(delay_table, dtype=np.int64)
    nchans, pitch = data.shape
    ndm = dl.shape[0]
    assert dl.shape[1] == nchans
    if nout < 0 or (nout > 0 and int(dl.max()) + nout > pitch):
        raise ValueError("input too short for nout + maxshift")
    if data.dtype == np.float32:
        out = np.empty((ndm, nout), np.float64)
        lib.oracle_dedisperse_f32(_p(data), pitch, nchans, _p(dl), ndm, nout, _p(out))
    elif data.dtype == np.uint16:
        out = np.empty((ndm, nout), np.float64)
        lib.oracle_dedisperse_f16(_p(data), pitch, nchans, _p(dl), ndm, nout, _p(out))
    elif data.dtype == np.uint8:
        out = np.empty((ndm, nout), np.int64)
        lib.oracle_dedisperse_u8(_p(data), pitch, nchans, _p(dl), ndm, nout, _p(out))
    else:
        raise TypeError(f"unsupported input dtype {data.dtype}")
    return out


def point_f32(data: np.ndarray, delay_row: np.ndarray, t: int) -> float:
    data = np.ascontiguousarray(data, dtype=np.float32)
    row = np.ascontiguousarray(delay_row, dtype=np.int64)
    return float(_load().oracle_point_f32(_p(data), data.shape[1], data.shape[0], _p(row), int(t)))


def row_f32(data: np.ndarray, delay_row: np.ndarray, nout: int) -> np.ndarray:
    data = np.ascontiguousarray(data, dtype=np.float32)
    row = np.ascontiguousarray(delay_row, dtype=np.int64)
    out = np.empty(nout, np.float64)
    _load().oracle_row_f32(_p(data), data.shape[1], data.shape[0], _p(row), int(nout), _p(out))
    return out


def stats(out: np.ndarray) -> tuple:
    """(mu, sigma): population mean and std over the whole buffer, two-pass double."""
    lib = _load()
    x = np.ascontiguousarray(out)
    mu, sg = C.c_double(0), C.c_double(0)
    if x.dtype == np.int64:
        lib.oracle_stats_i64(_p(x), x.size, C.byref(mu), C.byref(sg))
    else:
        x = np.ascontiguousarray(x, dtype=np.float64)
        lib.oracle_stats_f64(_p(x), x.size, C.byref(mu), C.byref(sg))
    return float(mu.value), float(sg.value)


def threshold(w: int, mu: float, sigma: float, k: float) -> float:
    return float(_load().oracle_threshold(int(w), mu, sigma, k))


def search(out: np.ndarray, widths, mu: float, sigma: float, k: float,
           cap: int = 1 << 20) -> np.ndarray:
    """Boxcar threshold search; returns a structured array sorted by (dm, t, width_idx)."""
    lib = _load()
    x = np.ascontiguousarray(out)
    ndm, nout = x.shape
    w = np.ascontiguousarray(np.asarray(widths, dtype=np.int32))
    cands = np.empty(cap, dtype=CAND_DTYPE)
    if x.dtype == np.int64:
        n = lib.oracle_search_i64(_p(x), ndm, nout, _p(w), w.size, mu, sigma, k, _p(cands), cap)
    else:
        x = np.ascontiguousarray(x, dtype=np.float64)
        n = lib.oracle_search_f64(_p(x), ndm, nout, _p(w), w.size, mu, sigma, k, _p(cands), cap)
    if n > cap:
        raise OverflowError(f"oracle search found {n} candidates > cap {cap}")
    return cands[:n].copy()


def subband_tables(nchans: int, fch1: float, foff: float, tsamp: float, dm_list, G: int,
                   nsub: int) -> tuple:
    """Section 3.2 subband plan: (nominal DMs [K], d1 [K][nchans], d2 [ndm][nsub], maxshift).

    Fine DMs in consecutive groups of G around nominal DM k (the midpoint of
    the group's first and last DM); nsub equal subbands of consecutive
    channels; d1 = stage-1 delay of each channel at the nominal DM relative to
    its subband's highest-frequency channel; d2 = stage-2 delay of each
    subband (its highest-frequency channel) at each fine DM."""
    dm = np.ascontiguousarray(np.asarray(dm_list, dtype=np.float64))
    if G < 1 or nsub < 1:
        raise ValueError("oracle_subband_tables: invalid arguments")
    K = (dm.size + G - 1) // G
    nominal = np.empty(K, np.float64)
    d1 = np.empty((K, nchans), np.int64)
    d2 = np.empty((dm.size, nsub), np.int64)
    m = C.c_int64(0)
    rc = _load().oracle_subband_tables(nchans, fch1, foff, tsamp, _p(dm), dm.size, G, nsub,
                                       _p(nominal), _p(d1), _p(d2), C.byref(m))
    if rc != 0:
        raise ValueError("oracle_subband_tables: invalid arguments")
    return nominal, d1, d2, int(m.value)


def subband_dedisperse(data: np.ndarray, d1: np.ndarray, d2: np.ndarray, G: int,
                       nout: int) -> np.ndarray:
    """Two-stage subband sum (Section 3.2); [ndm][nout] float64 (int64 for uint8)."""
    lib = _load()
    data = np.ascontiguousarray(data)
    d1 = np.ascontiguousarray(d1, dtype=np.int64)
    d2 = np.ascontiguousarray(d2, dtype=np.int64)
    nchans, pitch = data.shape
    ndm, nsub = d2.shape
    assert d1.shape[1] == nchans and nchans % nsub == 0
    cs = nchans // nsub
    need = 0
    for j in range(ndm):
        e = d2[j][np.arange(nchans) // cs] + d1[j // G]
        need = max(need, int(e.max()))
    if nout < 0 or (nout > 0 and need + nout > pitch):
        raise ValueError("input too short for nout + maxshift")
    if data.dtype == np.float64:
        out = np.empty((ndm, nout), np.float64)
        lib.oracle_subband_f64(_p(data), pitch, nchans, nsub, _p(d1), _p(d2), G, ndm, nout, _p(out))
    elif data.dtype == np.float32:
        out = np.empty((ndm, nout), np.float64)
        lib.oracle_subband_f32(_p(data), pitch, nchans, nsub, _p(d1), _p(d2), G, ndm, nout, _p(out))
    elif data.dtype == np.uint16:
        out = np.empty((ndm, nout), np.float64)
        lib.oracle_subband_f16(_p(data), pitch, nchans, nsub, _p(d1), _p(d2), G, ndm, nout, _p(out))
    elif data.dtype == np.uint8:
        out = np.empty((ndm, nout), np.int64)
        lib.oracle_subband_u8(_p(data), pitch, nchans, nsub, _p(d1), _p(d2), G, ndm, nout, _p(out))
    else:
        raise TypeError(f"unsupported input dtype {data.dtype}")
    return out


def subband_point_f32(data: np.ndarray, d1: np.ndarray, d2: np.ndarray, G: int, j: int,
                      t: int) -> float:
    data = np.ascontiguousarray(data, dtype=np.float32)
    d1 = np.ascontiguousarray(d1, dtype=np.int64)
    d2 = np.ascontiguousarray(d2, dtype=np.int64)
    return float(_load().oracle_subband_point_f32(_p(data), data.shape[1], data.shape[0],
                                                  d2.shape[1], _p(d1), _p(d2), G, int(j), int(t)))


def bin_samples(data: np.ndarray, nb: int, nsamp: int = None) -> np.ndarray:
    """Binning (Section 3.2): mean of nb adjacent samples per channel, in double.

    data: [nchans][pitch] float32, uint8 or uint16 (binary16 bits); the first
    nsamp samples (default: all) give floor(nsamp / nb) binned samples."""
    data = np.ascontiguousarray(data)
    nchans, pitch = data.shape
    nsamp = pitch if nsamp is None else int(nsamp)
    code = {np.dtype(np.float32): 0, np.dtype(np.uint8): 1, np.dtype(np.uint16): 2}[data.dtype]
    n = nsamp // nb
    out = np.empty((nchans, max(n, 1)), np.float64)
    _load().oracle_bin(_p(data), code, pitch, nchans, nsamp, int(nb), _p(out), out.shape[1])
    return out[:, :n]


def survey_passes(passes) -> list:
    """Reading of a Table 1 survey plan: each pass (low DM, high DM, DM step,
    bin, subband DM step) gives round((high - low) / step) fine DMs
    low + i * step and round(subband step / step) fine DMs per nominal DM.
    Returns [(dm_list, bin, dms_per_nominal)]."""
    out = []
    for lo, hi, step, nb, sub in passes:
        n = int(round((hi - lo) / step))
        out.append(([lo + i * step for i in range(n)], int(nb), int(round(sub / step))))
    return out


def channelise_power(volts: np.ndarray, nfft: int) -> np.ndarray:
    """Front end of the real-time pipeline (Section 5, Tables 5-6):
    channelisation, intensity, corner turn.

    volts: complex [npol][nsub][n] baseband voltages (upper sideband).  Each
    subband's stream is cut into blocks of nfft samples and transformed (the
    FFT is the channeliser); the intensity is |X|^2 summed over polarisations;
    the result is written channel-major ("corner turn") as
    out[s*nfft + j][b], j ordering the subband's nfft channels by DEScending
    frequency: FFT bin k has offset k (k < nfft/2) or k - nfft (k >= nfft/2),
    so channel j holds bin (nfft/2 - 1 - j) mod nfft.  Float64."""
    v = np.asarray(volts)
    npol, nsub, n = v.shape
    nb = n // nfft
    x = v[:, :, :nb * nfft].astype(np.complex128).reshape(npol, nsub, nb, nfft)
    p = (np.abs(np.fft.fft(x, axis=-1)) ** 2).sum(axis=0)          # [nsub][nb][nfft]
    order = [(nfft // 2 - 1 - j) % nfft for j in range(nfft)]
    p = p[:, :, order]                                               # descending frequency
    return np.ascontiguousarray(p.transpose(0, 2, 1).reshape(nsub * nfft, nb))


def search_per_row(out: np.ndarray, widths, k: float, cap: int = 1 << 20):
    """Search variant with per-DM-row statistics: each row's population mean
    and standard deviation (stats() of the row) set its thresholds
    T_w = w*mu_row + k*sigma_row*sqrt(w); otherwise search().  Returns
    (candidates sorted by (dm, t, width_idx), mu [ndm], sigma [ndm])."""
    x = np.ascontiguousarray(out)
    ndm = x.shape[0]
    mus, sgs, parts = np.empty(ndm), np.empty(ndm), []
    for j in range(ndm):
        mus[j], sgs[j] = stats(x[j:j + 1])
        c = search(x[j:j + 1], widths, mus[j], sgs[j], k, cap)
        c["dm_idx"] = j
        parts.append(c)
    cands = np.concatenate(parts) if parts else np.empty(0, CAND_DTYPE)
    return cands, mus, sgs


def cluster(cands: np.ndarray, dm_link: int, t_link: int):
    """Friends-of-friends clustering of candidates (search variant): pairs with
    |d dm_idx| <= dm_link and |d t| <= t_link are linked; clusters are the
    connected components.  Every pair is tested (plain O(n^2)).  Returns a list
    of (strongest member index, member indices, dm range, t range) sorted by the
    strongest member's (dm_idx, t, width_idx); the strongest member has the
    largest snr, ties to the smallest (dm_idx, t, width_idx)."""
    n = len(cands)
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            a = parent[a]
        return a

    for i in range(n):
        for j in range(i + 1, n):
            if (abs(int(cands[i]["dm_idx"]) - int(cands[j]["dm_idx"])) <= dm_link and
                    abs(int(cands[i]["t"]) - int(cands[j]["t"])) <= t_link):
                a, b = find(i), find(j)
                if a != b:
                    parent[max(a, b)] = min(a, b)
    groups = {}
    for i in range(n):
        groups.setdefault(find(i), []).append(i)
    key = lambda i: (int(cands[i]["dm_idx"]), int(cands[i]["t"]), int(cands[i]["width_idx"]))
    out = []
    for members in groups.values():
        best = min(members, key=lambda i: (-float(cands[i]["snr"]),) + key(i))
        dms = [int(cands[i]["dm_idx"]) for i in members]
        ts = [int(cands[i]["t"]) for i in members]
        out.append((best, sorted(members), (min(dms), max(dms)), (min(ts), max(ts))))
    out.sort(key=lambda g: key(g[0]))
    return out


def search_stream(chunks, widths, k: float, carry: bool = True):
    """Streaming search (serving; search variant with boundary carry): each
    chunk's outputs [ndm][chunk] are searched with the chunk's own mu, sigma;
    with `carry`, windows that start in the previous chunk's last wmax - 1
    outputs and end in this chunk are also tested, against this chunk's
    thresholds, and reported with t = start - chunk_start < 0.  Returns one
    candidate array per chunk, sorted by (dm, t, width_idx)."""
    widths = list(widths)
    L = max(widths) - 1
    res = []
    for c, cur in enumerate(chunks):
        cur = np.ascontiguousarray(cur)
        mu, sg = stats(cur)
        part = [search(cur, widths, mu, sg, k)]
        if carry and c > 0 and L > 0:
            prev = np.ascontiguousarray(chunks[c - 1])
            isint = cur.dtype == np.int64
            rows = []
            for j in range(cur.shape[0]):
                x = np.concatenate([prev[j, -L:], cur[j, :L]])
                for p, w in enumerate(widths):
                    for i in range(max(0, L - w + 1), L):
                        b = int(np.sum(x[i:i + w])) if isint else float(np.sum(x[i:i + w], dtype=np.float64))
                        if b > threshold(w, mu, sg, k):
                            rows.append((j, i - L, p, (b - w * mu) / (sg * math.sqrt(w)), float(b)))
            extra = np.array(rows, dtype=CAND_DTYPE) if rows else np.empty(0, CAND_DTYPE)
            part.append(extra)
        allc = np.concatenate(part)
        order = np.lexsort((allc["width_idx"], allc["t"], allc["dm_idx"]))
        res.append(allc[order])
    return res
