"""ctypes binding of libdd (include/dd.h): argument marshalling only.

Every step of de-dispersion and search runs in the CUDA kernels of libdd.so;
this module converts Python/numpy/torch arguments to the C ABI and raises on
any non-zero status.  There is no CPU fallback: if libdd.so is missing or
cannot be loaded, loading raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdd.so")

DD_F32, DD_U8, DD_F16 = 0, 1, 2
DD_OK, DD_ERR_ARG, DD_ERR_NOMEM, DD_ERR_CUDA, DD_ERR_OVERFLOW, DD_ERR_TIMEOUT, DD_ERR_BUDGET = range(7)

CANDIDATE_DTYPE = np.dtype([("dm_idx", np.int32), ("width_idx", np.int32), ("t", np.int64),
                            ("snr", np.float32), ("reserved", np.float32), ("value", np.float64)])
assert CANDIDATE_DTYPE.itemsize == 32

# Names of every function declared in include/dd.h.
EXPORTS = ("dd_plan_create", "dd_plan_destroy", "dd_plan_info", "dd_execute", "dd_search",
           "dd_last_stats", "dd_process_host", "dd_plan_set_kernel", "dd_plan_get_kernel",
           "dd_plan_autotune", "dd_plan_set_tile", "dd_plan_get_tile",
           "dd_stats_f32_noalloc", "dd_last_error", "dd_version",
           "dd_batch_create", "dd_batch_destroy", "dd_batch_execute", "dd_batch_capture",
           "dd_batch_launch", "dd_batch_results", "dd_batch_autotune", "dd_batch_info", "dd_batch_set_config", "dd_batch_beam_config",
           "dd_batch_set_launch_mode", "dd_batch_launch_mode", "dd_share_tables",
           "dd_host_chunk_schedule",
           "dd_server_create", "dd_server_destroy", "dd_server_add_beam", "dd_server_remove_beam",
           "dd_server_submit", "dd_server_poll", "dd_server_candidates", "dd_server_beam_info",
           "dd_server_memory", "dd_subband_plan_create", "dd_subband_plan_destroy",
           "dd_subband_plan_info", "dd_subband_execute", "dd_subband_search", "dd_subband_last_stats",
           "dd_survey_plan_create", "dd_survey_plan_destroy", "dd_survey_pass_info", "dd_survey_execute",
           "dd_survey_search", "dd_survey_last_stats", "dd_channelise",
           "dd_plan_set_search_stats", "dd_last_row_stats", "dd_cluster_candidates",
           "dd_server_set_boundary_search", "dd_server_set_autotune", "dd_server_beam_kernel",
           "dd_server_ring_schedule", "dd_wait_selftest")

DD_PRIMING, DD_ERR_SEQ, DD_SEQ_GAP = 7, 8, 9

CLUSTER_DTYPE = np.dtype([("dm_idx", np.int32), ("width_idx", np.int32), ("t", np.int64),
                          ("snr", np.float32), ("n_members", np.int32), ("dm_lo", np.int32),
                          ("dm_hi", np.int32), ("t_lo", np.int64), ("t_hi", np.int64)])
assert CLUSTER_DTYPE.itemsize == 48

CHUNK_RESULT_DTYPE = np.dtype([("beam", np.int32), ("status", np.int32), ("seq", np.int64),
                               ("n_candidates", np.int64), ("t_submit", np.float64),
                               ("t_start", np.float64), ("t_done", np.float64),
                               ("mu", np.float64), ("sigma", np.float64)])
assert CHUNK_RESULT_DTYPE.itemsize == 64


class DDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libdd status {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def load(path: Optional[str] = None):
    """Load libdd.so (once) and declare the C signatures."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libdd.so not found at {p}: build it with "
                               "paper_1107_2516_gb300.build.build() (nvcc, sm_103a)")
        lib = C.CDLL(p)
        vp, i32, i64, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        P64 = C.POINTER(C.c_int64)
        sig = {
            "dd_plan_create": (C.c_int, [i32, f64, f64, f64, vp, i32, vp, i32, f64, i32, i64,
                                         C.POINTER(vp)]),
            "dd_plan_destroy": (C.c_int, [vp]),
            "dd_plan_info": (C.c_int, [vp, P64, P64, vp]),
            "dd_execute": (C.c_int, [vp, vp, i64, vp, vp]),
            "dd_search": (C.c_int, [vp, vp, vp, i64, P64, vp]),
            "dd_last_stats": (C.c_int, [vp, C.POINTER(f64), C.POINTER(f64)]),
            "dd_process_host": (C.c_int, [vp, vp, i64, vp, i64, P64, vp]),
            "dd_plan_set_kernel": (C.c_int, [vp, i32]),
            "dd_plan_get_kernel": (C.c_int, [vp, C.POINTER(i32)]),
            "dd_plan_autotune": (C.c_int, [vp, vp, i64, vp, vp]),
            "dd_plan_set_tile": (C.c_int, [vp, i32, i32]),
            "dd_stats_f32_noalloc": (C.c_int, [vp, i64, vp, vp]),
            "dd_batch_create": (C.c_int, [vp, i32, C.POINTER(vp)]),
            "dd_batch_destroy": (C.c_int, [vp]),
            "dd_batch_execute": (C.c_int, [vp, vp, vp, vp, vp]),
            "dd_batch_capture": (C.c_int, [vp, vp, vp, vp, vp]),
            "dd_batch_launch": (C.c_int, [vp, vp]),
            "dd_batch_results": (C.c_int, [vp, i32, vp, i64, P64, vp]),
            "dd_batch_autotune": (C.c_int, [vp, vp, vp, vp, vp]),
            "dd_batch_info": (C.c_int, [vp, C.POINTER(i32), P64, C.POINTER(i32)]),
            "dd_batch_set_config": (C.c_int, [vp, i32]),
            "dd_batch_beam_config": (C.c_int, [vp, i32, C.POINTER(i32)]),
            "dd_batch_set_launch_mode": (C.c_int, [vp, i32]),
            "dd_batch_launch_mode": (C.c_int, [vp, C.POINTER(i32)]),
            "dd_share_tables": (C.c_int, [vp, i32, i32, f64, i32, i32, vp, vp, i64, vp, i64]),
            "dd_host_chunk_schedule": (C.c_int, [i64, i64, i32, i64, vp, vp, C.POINTER(i32)]),
            "dd_server_create": (C.c_int, [i64, i32, i64, C.POINTER(vp)]),
            "dd_server_destroy": (C.c_int, [vp]),
            "dd_server_add_beam": (C.c_int, [vp, i32, f64, f64, f64, vp, i32, vp, i32, f64, i32, i64,
                                             C.POINTER(i32)]),
            "dd_server_remove_beam": (C.c_int, [vp, i32]),
            "dd_server_submit": (C.c_int, [vp, i32, vp, i64, i64]),
            "dd_server_poll": (C.c_int, [vp, vp, i32, C.POINTER(i32), i32]),
            "dd_server_candidates": (C.c_int, [vp, i32, i64, vp, i64, P64]),
            "dd_server_beam_info": (C.c_int, [vp, i32, P64, P64, P64, C.POINTER(vp), P64]),
            "dd_server_memory": (C.c_int, [vp, P64, P64]),
            "dd_plan_get_tile": (C.c_int, [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32),
                                           C.POINTER(i32)]),
            "dd_subband_plan_create": (C.c_int, [i32, f64, f64, f64, vp, i32, i32, i32, vp, i32, f64,
                                                 i32, i64, C.POINTER(vp)]),
            "dd_subband_plan_destroy": (C.c_int, [vp]),
            "dd_subband_plan_info": (C.c_int, [vp, C.POINTER(i32), P64, P64, vp, vp, vp, P64]),
            "dd_subband_execute": (C.c_int, [vp, vp, i64, vp, vp]),
            "dd_subband_search": (C.c_int, [vp, vp, vp, i64, P64, vp]),
            "dd_subband_last_stats": (C.c_int, [vp, C.POINTER(f64), C.POINTER(f64)]),
            "dd_survey_plan_create": (C.c_int, [i32, f64, f64, f64, vp, i32, i32, vp, i32, f64, i32, i64,
                                                C.POINTER(vp)]),
            "dd_survey_plan_destroy": (C.c_int, [vp]),
            "dd_survey_pass_info": (C.c_int, [vp, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), P64,
                                              P64, vp]),
            "dd_survey_execute": (C.c_int, [vp, vp, i64, vp, vp]),
            "dd_survey_search": (C.c_int, [vp, i32, vp, vp, i64, P64, vp]),
            "dd_survey_last_stats": (C.c_int, [vp, i32, C.POINTER(f64), C.POINTER(f64)]),
            "dd_channelise": (C.c_int, [vp, i32, i32, i64, i32, vp, i64, vp]),
            "dd_plan_set_search_stats": (C.c_int, [vp, i32]),
            "dd_cluster_candidates": (C.c_int, [vp, i64, i32, i64, vp, i64, P64, vp]),
            "dd_server_set_boundary_search": (C.c_int, [vp, i32, i32]),
            "dd_server_set_autotune": (C.c_int, [vp, i32]),
            "dd_wait_selftest": (C.c_int, [i64, i32, C.POINTER(i32)]),
            "dd_server_beam_kernel": (C.c_int, [vp, i32, C.POINTER(i32), C.POINTER(i32)]),
            "dd_server_ring_schedule": (C.c_int, [i64, i64, i32, vp, P64, vp, vp, vp, vp, vp, vp]),
            "dd_last_row_stats": (C.c_int, [vp, vp, vp]),
            "dd_last_error": (C.c_char_p, []),
            "dd_version": (C.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype, f.argtypes = res, args
        if path is None:
            _lib = lib
        return lib


def _check(rc: int, allow=()):
    if rc != DD_OK and rc not in allow:
        raise DDError(rc, load().dd_last_error().decode())
    return rc


def _ptr(x) -> int:
    """Raw address of a torch tensor / numpy array / int."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        return int(x.ctypes.data)
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream) -> int:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return int(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# ------------------------------------------------------------------ C-named calls

def dd_version() -> str:
    return load().dd_version().decode()


def dd_last_error() -> str:
    return load().dd_last_error().decode()


def dd_plan_create(nchans: int, fch1: float, foff: float, tsamp: float, dm_list: Sequence[float],
                   boxcar_widths: Sequence[int], sigma: float, in_dtype: int, nsamp_in: int) -> int:
    dm = np.ascontiguousarray(np.asarray(dm_list, dtype=np.float64))
    w = np.ascontiguousarray(np.asarray(boxcar_widths, dtype=np.int32))
    out = C.c_void_p()
    _check(load().dd_plan_create(int(nchans), float(fch1), float(foff), float(tsamp),
                                 dm.ctypes.data, int(dm.size), w.ctypes.data, int(w.size),
                                 float(sigma), int(in_dtype), int(nsamp_in), C.byref(out)))
    return int(out.value)


def dd_plan_destroy(plan: int) -> None:
    _check(load().dd_plan_destroy(plan))


def dd_plan_info(plan: int, ndm: int = 0, nchans: int = 0, delays: bool = False):
    m, n = C.c_int64(), C.c_int64()
    tab = np.empty((ndm, nchans), np.int32) if delays else None
    _check(load().dd_plan_info(plan, C.byref(m), C.byref(n), _ptr(tab) if delays else None))
    return (int(m.value), int(n.value), tab) if delays else (int(m.value), int(n.value))


def dd_execute(plan: int, in_dev, in_pitch: int, out_dev, stream=None) -> None:
    _check(load().dd_execute(plan, _ptr(in_dev), int(in_pitch), _ptr(out_dev), _stream(stream)))


def dd_search(plan: int, out_dev, capacity: int = 1 << 16, stream=None, allow_overflow=False):
    """Returns (candidates structured array sorted by (dm, t, width), true count)."""
    cands = np.zeros(max(capacity, 1), dtype=CANDIDATE_DTYPE)
    n = C.c_int64()
    rc = _check(load().dd_search(plan, _ptr(out_dev), cands.ctypes.data, int(capacity), C.byref(n),
                                 _stream(stream)), allow=(DD_ERR_OVERFLOW,) if allow_overflow else ())
    total = int(n.value)
    return cands[:min(total, capacity)].copy(), total


def dd_last_stats(plan: int):
    mu, sg = C.c_double(), C.c_double()
    _check(load().dd_last_stats(plan, C.byref(mu), C.byref(sg)))
    return float(mu.value), float(sg.value)


def dd_process_host(plan: int, in_host, in_pitch: int, capacity: int = 1 << 16, stream=None,
                    allow_overflow=False):
    cands = np.zeros(max(capacity, 1), dtype=CANDIDATE_DTYPE)
    n = C.c_int64()
    _check(load().dd_process_host(plan, _ptr(in_host), int(in_pitch), cands.ctypes.data,
                                  int(capacity), C.byref(n), _stream(stream)),
           allow=(DD_ERR_OVERFLOW,) if allow_overflow else ())
    total = int(n.value)
    return cands[:min(total, capacity)].copy(), total


def dd_plan_set_kernel(plan: int, kernel: int) -> None:
    _check(load().dd_plan_set_kernel(plan, int(kernel)))


def dd_plan_get_kernel(plan: int) -> int:
    k = C.c_int32()
    _check(load().dd_plan_get_kernel(plan, C.byref(k)))
    return int(k.value)


def dd_plan_autotune(plan: int, in_dev, in_pitch: int, out_dev, stream=None) -> None:
    _check(load().dd_plan_autotune(plan, _ptr(in_dev), int(in_pitch), _ptr(out_dev), _stream(stream)))


def dd_plan_set_tile(plan: int, config: int, raster_group: int) -> None:
    _check(load().dd_plan_set_tile(plan, int(config), int(raster_group)))


def dd_plan_get_tile(plan: int):
    """(config, raster_group, samples_per_thread, warps_per_block) of kernel 2."""
    v = [C.c_int32() for _ in range(4)]
    _check(load().dd_plan_get_tile(plan, *[C.byref(x) for x in v]))
    return tuple(int(x.value) for x in v)


def dd_stats_f32_noalloc(x_dev, n: int, mu_sigma_dev, stream=None) -> None:
    """Mean and standard deviation of n float32 device values into mu_sigma_dev[0:2]
    (device, float64) without any allocation; for callers that cannot allocate
    device memory after start-up.  At most 2**28 values; see include/dd.h."""
    _check(load().dd_stats_f32_noalloc(_ptr(x_dev), int(n), _ptr(mu_sigma_dev), _stream(stream)))


def _ptr_array(xs):
    arr = (C.c_void_p * len(xs))(*[_ptr(x) for x in xs])
    return arr


def dd_batch_create(plans) -> int:
    handles = (C.c_void_p * len(plans))(*[p.handle if isinstance(p, Plan) else int(p) for p in plans])
    out = C.c_void_p()
    _check(load().dd_batch_create(handles, len(plans), C.byref(out)))
    return int(out.value)


def dd_batch_destroy(batch: int) -> None:
    _check(load().dd_batch_destroy(batch))


def _batch_bufs(ins, pitches, outs):
    p = (C.c_int64 * len(pitches))(*[int(v) for v in pitches])
    return _ptr_array(ins), p, _ptr_array(outs)


def dd_batch_execute(batch: int, ins, pitches, outs, stream=None) -> None:
    a, p, o = _batch_bufs(ins, pitches, outs)
    _check(load().dd_batch_execute(batch, a, p, o, _stream(stream)))


def dd_batch_capture(batch: int, ins, pitches, outs, stream) -> None:
    a, p, o = _batch_bufs(ins, pitches, outs)
    _check(load().dd_batch_capture(batch, a, p, o, _stream(stream)))


def dd_batch_launch(batch: int, stream) -> None:
    _check(load().dd_batch_launch(batch, _stream(stream)))


def dd_batch_results(batch: int, beam: int, capacity: int = 1 << 16, stream=None, allow_overflow=False):
    cands = np.zeros(max(capacity, 1), dtype=CANDIDATE_DTYPE)
    n = C.c_int64()
    _check(load().dd_batch_results(batch, int(beam), cands.ctypes.data, int(capacity), C.byref(n),
                                   _stream(stream)), allow=(DD_ERR_OVERFLOW,) if allow_overflow else ())
    total = int(n.value)
    return cands[:min(total, capacity)].copy(), total


def dd_batch_autotune(batch: int, ins, pitches, outs, stream=None) -> None:
    a, p, o = _batch_bufs(ins, pitches, outs)
    _check(load().dd_batch_autotune(batch, a, p, o, _stream(stream)))


def dd_batch_info(batch: int):
    """(tile configuration of the persistent launch, work items, beams run separately)."""
    c, n, s = C.c_int32(), C.c_int64(), C.c_int32()
    _check(load().dd_batch_info(batch, C.byref(c), C.byref(n), C.byref(s)))
    return int(c.value), int(n.value), int(s.value)


def dd_batch_set_config(batch: int, config: int) -> None:
    _check(load().dd_batch_set_config(batch, int(config)))


def dd_host_chunk_schedule(nsamp_out: int, pitch: int, tile: int, reach: int):
    """dd_process_host's pipeline schedule: (col_end, tile_end) arrays, one entry per chunk."""
    col = np.zeros(8, np.int64)
    til = np.zeros(8, np.int64)
    n = C.c_int32()
    _check(load().dd_host_chunk_schedule(int(nsamp_out), int(pitch), int(tile), int(reach), _ptr(col),
                                         _ptr(til), C.byref(n)))
    return col[:n.value].copy(), til[:n.value].copy()


def dd_wait_selftest(limit_ns: int, issue_copy: bool):
    """Bounded-wait self-test: (return status, device status); never raises."""
    st = C.c_int32(-1)
    rc = load().dd_wait_selftest(int(limit_ns), 1 if issue_copy else 0, C.byref(st))
    return int(rc), int(st.value)


def dd_server_ring_schedule(maxshift: int, chunk: int, seqs):
    """The server's host-side schedule for one beam (no device work): dict of
    span and, per submission, status, restart, move_src, write_col, window_col,
    priming (numpy arrays)."""
    sq = np.ascontiguousarray(np.asarray(seqs, dtype=np.int64))
    n = sq.size
    st, rs, pr = (np.zeros(max(n, 1), np.int32) for _ in range(3))
    mv, wc, wn = (np.zeros(max(n, 1), np.int64) for _ in range(3))
    span = C.c_int64()
    _check(load().dd_server_ring_schedule(int(maxshift), int(chunk), int(n), _ptr(sq), C.byref(span), _ptr(st),
                                          _ptr(rs), _ptr(mv), _ptr(wc), _ptr(wn), _ptr(pr)))
    return {"span": int(span.value), "status": st[:n], "restart": rs[:n], "move_src": mv[:n],
            "write_col": wc[:n], "window_col": wn[:n], "priming": pr[:n]}


def dd_share_tables(delays: np.ndarray, foff: float, dtype: int, config: int):
    """Kernel 5's tables (host only) for a delay table [ndm][nchans]: None if the
    shape cannot run it, else dict(rec [blocks][subbands][kLen], base
    [blocks][nchans] staged row starts, rlen [blocks][nchans] staged row
    lengths, rs, pmax, klen)."""
    d = np.ascontiguousarray(delays, dtype=np.int32)
    ndm, nch = d.shape
    info = np.zeros(6, np.int32)
    _check(load().dd_share_tables(_ptr(d), ndm, nch, float(foff), int(dtype), int(config), _ptr(info), None, 0,
                                  None, 0))
    if not info[0]:
        return None
    nblk, nsub, rs, pmax, klen = (int(v) for v in info[1:])
    rec = np.empty((nblk, nsub, klen), np.int32)
    base = np.empty((2, nblk, nch), np.int32)
    _check(load().dd_share_tables(_ptr(d), ndm, nch, float(foff), int(dtype), int(config), _ptr(info), _ptr(rec),
                                  rec.size, _ptr(base), base.size))
    return {"rec": rec, "base": base[0], "rlen": base[1], "rs": rs, "pmax": pmax, "klen": klen}


def dd_batch_beam_config(batch: int, beam: int) -> int:
    c = C.c_int32()
    _check(load().dd_batch_beam_config(batch, int(beam), C.byref(c)))
    return int(c.value)


class Server:
    """Owning wrapper around a dd_server handle (marshalling only)."""

    def __init__(self, hbm_budget_bytes: int, nworkers: int = 4, max_candidates: int = 1 << 16):
        out = C.c_void_p()
        _check(load().dd_server_create(int(hbm_budget_bytes), int(nworkers), int(max_candidates),
                                       C.byref(out)))
        self.handle = int(out.value)
        self._keep = {}

    def add_beam(self, nchans, fch1, foff, tsamp, dm_list, widths, sigma, in_dtype, chunk) -> int:
        """Beam id; raises DDError(DD_ERR_BUDGET) if its memory does not fit the budget."""
        dm = np.ascontiguousarray(np.asarray(dm_list, dtype=np.float64))
        w = np.ascontiguousarray(np.asarray(widths, dtype=np.int32))
        bid = C.c_int32()
        _check(load().dd_server_add_beam(self.handle, int(nchans), float(fch1), float(foff),
                                         float(tsamp), dm.ctypes.data, int(dm.size), w.ctypes.data,
                                         int(w.size), float(sigma), int(in_dtype), int(chunk),
                                         C.byref(bid)))
        return int(bid.value)

    def remove_beam(self, beam: int) -> None:
        _check(load().dd_server_remove_beam(self.handle, int(beam)))

    def set_boundary_search(self, beam: int, on: bool = True) -> None:
        """Also search boxcars crossing from the previous chunk (reported with t < 0)."""
        _check(load().dd_server_set_boundary_search(self.handle, int(beam), 1 if on else 0))

    def submit(self, beam: int, chunk_host, host_pitch: int, seq: int) -> int:
        """chunk_host must stay alive and unchanged until poll() reports (beam, seq).
        Returns DD_OK, or DD_SEQ_GAP when the beam's stream restarts at this
        chunk; raises DDError(DD_ERR_SEQ) for a repeated or late seq (nothing queued)."""
        rc = load().dd_server_submit(self.handle, int(beam), _ptr(chunk_host), int(host_pitch), int(seq))
        _check(rc, allow=(DD_SEQ_GAP,))
        self._keep[(int(beam), int(seq))] = chunk_host
        return rc

    def set_autotune(self, on: bool = True) -> None:
        """Autotune beams admitted from now on (on their own buffers, cached per plan shape)."""
        _check(load().dd_server_set_autotune(self.handle, 1 if on else 0))

    def beam_kernel(self, beam: int):
        """(kernel, tile configuration) the beam runs."""
        k, c = C.c_int32(), C.c_int32()
        _check(load().dd_server_beam_kernel(self.handle, int(beam), C.byref(k), C.byref(c)))
        return int(k.value), int(c.value)

    def poll(self, max_results: int = 256, wait_ms: int = 0) -> np.ndarray:
        res = np.zeros(max_results, dtype=CHUNK_RESULT_DTYPE)
        n = C.c_int32()
        _check(load().dd_server_poll(self.handle, res.ctypes.data, int(max_results), C.byref(n),
                                     int(wait_ms)))
        res = res[:n.value].copy()
        for r in res:
            self._keep.pop((int(r["beam"]), int(r["seq"])), None)
        return res

    def candidates(self, beam: int, seq: int, capacity: int = 1 << 16):
        cands = np.zeros(max(capacity, 1), dtype=CANDIDATE_DTYPE)
        n = C.c_int64()
        _check(load().dd_server_candidates(self.handle, int(beam), int(seq), cands.ctypes.data,
                                           int(capacity), C.byref(n)))
        return cands[:min(int(n.value), capacity)].copy()

    def beam_info(self, beam: int) -> dict:
        m, ch, nd, nb = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        outp = C.c_void_p()
        _check(load().dd_server_beam_info(self.handle, int(beam), C.byref(m), C.byref(ch),
                                          C.byref(nd), C.byref(outp), C.byref(nb)))
        return {"maxshift": int(m.value), "chunk": int(ch.value), "ndm": int(nd.value),
                "out_dev": int(outp.value or 0), "device_bytes": int(nb.value)}

    def memory(self):
        u, b = C.c_int64(), C.c_int64()
        _check(load().dd_server_memory(self.handle, C.byref(u), C.byref(b)))
        return int(u.value), int(b.value)

    def close(self):
        if self.handle:
            load().dd_server_destroy(self.handle)
            self.handle = 0
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owning wrapper around a dd_batch handle; keeps its plans alive."""

    def __init__(self, plans):
        self.plans = list(plans)
        self.handle = dd_batch_create(self.plans)

    def execute(self, ins, pitches, outs, stream=None):
        dd_batch_execute(self.handle, ins, pitches, outs, stream)

    def capture(self, ins, pitches, outs, stream):
        dd_batch_capture(self.handle, ins, pitches, outs, stream)

    def launch(self, stream):
        dd_batch_launch(self.handle, stream)

    def results(self, beam, capacity=1 << 16, stream=None, allow_overflow=False):
        return dd_batch_results(self.handle, beam, capacity, stream, allow_overflow)

    def autotune(self, ins, pitches, outs, stream=None):
        dd_batch_autotune(self.handle, ins, pitches, outs, stream)

    @property
    def info(self):
        return dd_batch_info(self.handle)

    def set_config(self, config):
        dd_batch_set_config(self.handle, config)

    @property
    def per_beam(self):
        """True if the batch runs each beam's own launch instead of one persistent grid."""
        c = C.c_int32()
        _check(load().dd_batch_launch_mode(self.handle, C.byref(c)))
        return bool(c.value)

    def set_launch_mode(self, per_beam: bool):
        _check(load().dd_batch_set_launch_mode(self.handle, 1 if per_beam else 0))

    def beam_config(self, beam):
        """Tile configuration beam `beam` runs in the persistent launch (-1: its own launch)."""
        return dd_batch_beam_config(self.handle, beam)

    def close(self):
        if self.handle:
            dd_batch_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------- convenience object

class Plan:
    """Owning wrapper around a dd_plan handle (marshalling only)."""

    def __init__(self, nchans, fch1, foff, tsamp, dm_list, boxcar_widths, sigma, in_dtype, nsamp_in):
        self.nchans, self.ndm = int(nchans), len(dm_list)
        self.in_dtype = int(in_dtype)
        self.handle = dd_plan_create(nchans, fch1, foff, tsamp, dm_list, boxcar_widths, sigma,
                                     in_dtype, nsamp_in)
        self.maxshift, self.nsamp_out = dd_plan_info(self.handle)

    @property
    def out_is_int(self) -> bool:
        return self.in_dtype == DD_U8

    def delays(self) -> np.ndarray:
        return dd_plan_info(self.handle, self.ndm, self.nchans, delays=True)[2]

    def execute(self, in_dev, in_pitch, out_dev, stream=None):
        dd_execute(self.handle, in_dev, in_pitch, out_dev, stream)

    def search(self, out_dev, capacity=1 << 16, stream=None, allow_overflow=False):
        return dd_search(self.handle, out_dev, capacity, stream, allow_overflow)

    def stats(self):
        return dd_last_stats(self.handle)

    def process_host(self, in_host, in_pitch, capacity=1 << 16, stream=None, allow_overflow=False):
        return dd_process_host(self.handle, in_host, in_pitch, capacity, stream, allow_overflow)

    def set_kernel(self, k):
        dd_plan_set_kernel(self.handle, k)

    def set_search_stats(self, per_row: bool):
        """Search variant: per-DM-row (True) or whole-buffer (False) statistics."""
        _check(load().dd_plan_set_search_stats(self.handle, 1 if per_row else 0))

    def row_stats(self):
        """(mu [ndm], sigma [ndm]) of the last per-row search."""
        mu = np.empty(self.ndm, np.float64)
        sg = np.empty(self.ndm, np.float64)
        _check(load().dd_last_row_stats(self.handle, _ptr(mu), _ptr(sg)))
        return mu, sg

    def autotune(self, in_dev, in_pitch, out_dev, stream=None):
        dd_plan_autotune(self.handle, in_dev, in_pitch, out_dev, stream)

    def set_tile(self, config, raster_group=8):
        dd_plan_set_tile(self.handle, config, raster_group)

    @property
    def tile(self):
        return dd_plan_get_tile(self.handle)

    @property
    def kernel(self):
        return dd_plan_get_kernel(self.handle)

    def close(self):
        if self.handle:
            dd_plan_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ subband (Section 3.2)

def dd_subband_plan_create(nchans, fch1, foff, tsamp, dm_list, dms_per_nominal, nsub, boxcar_widths,
                           sigma, in_dtype, nsamp_in) -> int:
    dm = np.ascontiguousarray(np.asarray(dm_list, dtype=np.float64))
    w = np.ascontiguousarray(np.asarray(boxcar_widths, dtype=np.int32))
    out = C.c_void_p()
    _check(load().dd_subband_plan_create(int(nchans), float(fch1), float(foff), float(tsamp),
                                         dm.ctypes.data, int(dm.size), int(dms_per_nominal), int(nsub),
                                         w.ctypes.data, int(w.size), float(sigma), int(in_dtype),
                                         int(nsamp_in), C.byref(out)))
    return int(out.value)


def dd_subband_plan_destroy(plan: int) -> None:
    _check(load().dd_subband_plan_destroy(plan))


def dd_subband_plan_info(plan: int, ndm: int = 0, nchans: int = 0, nsub: int = 0, tables=False):
    """(n_nominal, maxshift, nsamp_out, work_bytes[, nominal, stage1 [K][nchans], stage2 [ndm][nsub]])."""
    k, m, n, wb = C.c_int32(), C.c_int64(), C.c_int64(), C.c_int64()
    lib = load()
    _check(lib.dd_subband_plan_info(plan, C.byref(k), C.byref(m), C.byref(n), None, None, None,
                                    C.byref(wb)))
    base = (int(k.value), int(m.value), int(n.value), int(wb.value))
    if not tables:
        return base
    nom = np.empty(base[0], np.float64)
    d1 = np.empty((base[0], nchans), np.int32)
    d2 = np.empty((ndm, nsub), np.int32)
    _check(lib.dd_subband_plan_info(plan, None, None, None, _ptr(nom), _ptr(d1), _ptr(d2), None))
    return base + (nom, d1, d2)


def dd_subband_execute(plan: int, in_dev, in_pitch: int, out_dev, stream=None) -> None:
    _check(load().dd_subband_execute(plan, _ptr(in_dev), int(in_pitch), _ptr(out_dev), _stream(stream)))


def dd_subband_search(plan: int, out_dev, capacity: int = 1 << 16, stream=None, allow_overflow=False):
    cands = np.zeros(max(capacity, 1), dtype=CANDIDATE_DTYPE)
    n = C.c_int64()
    _check(load().dd_subband_search(plan, _ptr(out_dev), cands.ctypes.data, int(capacity), C.byref(n),
                                    _stream(stream)), allow=(DD_ERR_OVERFLOW,) if allow_overflow else ())
    total = int(n.value)
    return cands[:min(total, capacity)].copy(), total


def dd_subband_last_stats(plan: int):
    mu, sg = C.c_double(), C.c_double()
    _check(load().dd_subband_last_stats(plan, C.byref(mu), C.byref(sg)))
    return float(mu.value), float(sg.value)


class SubbandPlan:
    """Owning wrapper around a dd_subband_plan handle (marshalling only)."""

    def __init__(self, nchans, fch1, foff, tsamp, dm_list, dms_per_nominal, nsub, boxcar_widths, sigma,
                 in_dtype, nsamp_in):
        self.nchans, self.ndm, self.nsub = int(nchans), len(dm_list), int(nsub)
        self.in_dtype = int(in_dtype)
        self.handle = dd_subband_plan_create(nchans, fch1, foff, tsamp, dm_list, dms_per_nominal, nsub,
                                             boxcar_widths, sigma, in_dtype, nsamp_in)
        self.n_nominal, self.maxshift, self.nsamp_out, self.work_bytes = dd_subband_plan_info(self.handle)

    def tables(self):
        """(nominal DMs, stage-1 delays [K][nchans], stage-2 delays [ndm][nsub])."""
        return dd_subband_plan_info(self.handle, self.ndm, self.nchans, self.nsub, tables=True)[4:]

    def execute(self, in_dev, in_pitch, out_dev, stream=None):
        dd_subband_execute(self.handle, in_dev, in_pitch, out_dev, stream)

    def search(self, out_dev, capacity=1 << 16, stream=None, allow_overflow=False):
        return dd_subband_search(self.handle, out_dev, capacity, stream, allow_overflow)

    def stats(self):
        return dd_subband_last_stats(self.handle)

    def close(self):
        if self.handle:
            dd_subband_plan_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ survey plans (Table 1)

class SurveyPass(C.Structure):
    """One row of a survey plan (Table 1): DM range, DM step, binning factor,
    subband DM step."""
    _fields_ = [("low_dm", C.c_double), ("high_dm", C.c_double), ("dm_step", C.c_double),
                ("bin", C.c_int32), ("reserved", C.c_int32), ("sub_dm_step", C.c_double)]


def dd_survey_plan_create(nchans, fch1, foff, tsamp, passes, nsub, boxcar_widths, sigma, in_dtype,
                          nsamp_in) -> int:
    arr = (SurveyPass * len(passes))(*[SurveyPass(float(lo), float(hi), float(st), int(b), 0, float(sub))
                                       for lo, hi, st, b, sub in passes])
    w = np.ascontiguousarray(np.asarray(boxcar_widths, dtype=np.int32))
    out = C.c_void_p()
    _check(load().dd_survey_plan_create(int(nchans), float(fch1), float(foff), float(tsamp), C.cast(arr, C.c_void_p),
                                        len(passes), int(nsub), w.ctypes.data, int(w.size), float(sigma),
                                        int(in_dtype), int(nsamp_in), C.byref(out)))
    return int(out.value)


def dd_survey_plan_destroy(plan: int) -> None:
    _check(load().dd_survey_plan_destroy(plan))


def dd_survey_pass_info(plan: int, pass_idx: int, dm_list=False):
    """(ndm, bin, dms_per_nominal, maxshift, nsamp_out[, dm_list])."""
    nd, b, g = C.c_int32(), C.c_int32(), C.c_int32()
    m, n = C.c_int64(), C.c_int64()
    lib = load()
    _check(lib.dd_survey_pass_info(plan, int(pass_idx), C.byref(nd), C.byref(b), C.byref(g), C.byref(m),
                                   C.byref(n), None))
    base = (int(nd.value), int(b.value), int(g.value), int(m.value), int(n.value))
    if not dm_list:
        return base
    dms = np.empty(base[0], np.float64)
    _check(lib.dd_survey_pass_info(plan, int(pass_idx), None, None, None, None, None, _ptr(dms)))
    return base + (dms,)


def dd_survey_execute(plan: int, in_dev, in_pitch: int, out_devs, stream=None) -> None:
    ptrs = (C.c_void_p * len(out_devs))(*[_ptr(o) for o in out_devs])
    _check(load().dd_survey_execute(plan, _ptr(in_dev), int(in_pitch), C.cast(ptrs, C.c_void_p),
                                    _stream(stream)))


def dd_survey_search(plan: int, pass_idx: int, out_dev, capacity: int = 1 << 16, stream=None,
                     allow_overflow=False):
    cands = np.zeros(max(capacity, 1), dtype=CANDIDATE_DTYPE)
    n = C.c_int64()
    _check(load().dd_survey_search(plan, int(pass_idx), _ptr(out_dev), cands.ctypes.data, int(capacity),
                                   C.byref(n), _stream(stream)),
           allow=(DD_ERR_OVERFLOW,) if allow_overflow else ())
    total = int(n.value)
    return cands[:min(total, capacity)].copy(), total


def dd_survey_last_stats(plan: int, pass_idx: int):
    mu, sg = C.c_double(), C.c_double()
    _check(load().dd_survey_last_stats(plan, int(pass_idx), C.byref(mu), C.byref(sg)))
    return float(mu.value), float(sg.value)


class SurveyPlan:
    """Owning wrapper around a dd_survey_plan handle (marshalling only).
    passes: rows (low_dm, high_dm, dm_step, bin, sub_dm_step)."""

    def __init__(self, nchans, fch1, foff, tsamp, passes, nsub, boxcar_widths, sigma, in_dtype, nsamp_in):
        self.npass = len(passes)
        self.handle = dd_survey_plan_create(nchans, fch1, foff, tsamp, passes, nsub, boxcar_widths, sigma,
                                            in_dtype, nsamp_in)
        self.passes = [dd_survey_pass_info(self.handle, i) for i in range(self.npass)]

    def dm_list(self, i):
        return dd_survey_pass_info(self.handle, i, dm_list=True)[5]

    def execute(self, in_dev, in_pitch, out_devs, stream=None):
        dd_survey_execute(self.handle, in_dev, in_pitch, out_devs, stream)

    def search(self, i, out_dev, capacity=1 << 16, stream=None, allow_overflow=False):
        return dd_survey_search(self.handle, i, out_dev, capacity, stream, allow_overflow)

    def stats(self, i):
        return dd_survey_last_stats(self.handle, i)

    def close(self):
        if self.handle:
            dd_survey_plan_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ front end (Section 5)

def dd_channelise(volt_dev, npol: int, nsub: int, nsamp: int, nfft: int, out_dev, out_pitch: int,
                  stream=None) -> None:
    """Channeliser + intensity + corner turn: complex64 [npol][nsub][nsamp] ->
    float32 [nsub*nfft][out_pitch] (descending frequency within each subband)."""
    _check(load().dd_channelise(_ptr(volt_dev), int(npol), int(nsub), int(nsamp), int(nfft), _ptr(out_dev),
                                int(out_pitch), _stream(stream)))


# ------------------------------------------------------------------ candidate clustering

def dd_cluster_candidates(cands: np.ndarray, dm_link: int, t_link: int):
    """Friends-of-friends clusters of a candidate array (CANDIDATE_DTYPE).
    Returns (clusters CLUSTER_DTYPE sorted by strongest member, labels [n])."""
    c = np.ascontiguousarray(cands, dtype=CANDIDATE_DTYPE)
    n = len(c)
    out = np.zeros(max(n, 1), dtype=CLUSTER_DTYPE)
    labels = np.zeros(max(n, 1), dtype=np.int64)
    m = C.c_int64()
    _check(load().dd_cluster_candidates(c.ctypes.data if n else None, n, int(dm_link), int(t_link),
                                        out.ctypes.data, n, C.byref(m), labels.ctypes.data))
    return out[:m.value].copy(), labels[:n].copy()
