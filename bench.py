#!/usr/bin/env python3
"""Benchmark: brute-force de-dispersion + boxcar search on the LOFAR-like
single beam (1024 channels, 150 MHz top, 12 MHz band, 163.84 us, 2^20
samples, 2000 DM trials 0..99.95 step 0.05, 16 injected pulses), one GB300.

One step = dd_execute (Section 3.1 sum, fused partial statistics) + dd_search
(statistics finalisation, boxcar sums, threshold, compaction, candidate
readback) on device-resident input.  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (FP64, plain loops, all host cores) on a
bounded sample of the same workload.  Under torchrun every rank processes its
own beam of the same shape (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "DM-trial·samples/s"
WORKLOAD = "lofar_f32"
# ncu DRAM bytes (read + write) per de-dispersion launch, keyed by the
# (tile configuration, raster group) the capture used, with the digest of the
# kernel's source files at capture time (kernel_source_digest): the figure is
# reported only while the sources are unchanged.  Kernel 5 was captured on a
# slice of the benchmark plan (all 2000 DM trials, 2^17 input samples: 217 of
# the full plan's 2009 time tiles, 0.54 GB in, 0.89 GB out) and scaled to the
# full launch: reads by the tile count (9.2581x), writes by the output count
# (9.2901x); profiles/dedisp_kernel5_lofar_f32.md has the capture.
PROFILED_TRAFFIC = {
    (12, 64): (13982494111, "88eaa72c6d055f3e6e4d616657b71096ac879d87a0ffec8976a576ca6db5e24b"),
    (11, 64): (14441256410, "88eaa72c6d055f3e6e4d616657b71096ac879d87a0ffec8976a576ca6db5e24b"),
}
# the kernel's device sources (a change to the host tables that alters the
# staged row lengths, i.e. the bytes each copy moves, needs a new capture too)
KERNEL_SOURCES = {3: ("dd_lane_impl.cuh", "dd_lane_c2.cu", "dd_device.cuh", "dd_fast_impl.cuh"),
                  5: ("dd_share_impl.cuh", "dd_share.cu", "dd_lane_impl.cuh", "dd_device.cuh", "dd_fast_impl.cuh")}


def kernel_source_digest(kernel_id: int) -> str:
    """sha256 over the source files that define a de-dispersion kernel."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1107_2516_gb300", "csrc")
    for f in KERNEL_SOURCES.get(kernel_id, ()):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()


def profiled_traffic(kernel_id: int, tile):
    """The recorded ncu traffic of this launch configuration, or None if there
    is none or the kernel's sources changed since it was captured."""
    if not tile:
        return None
    rec = PROFILED_TRAFFIC.get(tuple(tile[:2]))
    if rec is None or rec[1] != kernel_source_digest(kernel_id):
        return None
    return rec[0]

# tile configurations of dd_plan_set_tile: (kernel, samples per thread or lane,
# DM trials per thread or warp, warps per block)
TILE_CONFIGS = {0: (2, 36, 4, 8), 1: (2, 20, 4, 12), 2: (2, 28, 4, 8), 3: (3, 16, 4, 8),
                4: (3, 16, 8, 8), 5: (3, 16, 8, 4), 6: (3, 8, 16, 4), 7: (4, 20, 4, 8),
                8: (4, 12, 8, 8), 9: (5, 16, 8, 4), 10: (5, 8, 8, 4), 11: (5, 16, 8, 6),
                12: (5, 16, 8, 8)}
# warp-specialised kernel 5 shapes: their stage-1 warps (beside the warps above)
STAGE1_WARPS = {12: 8}


# ------------------------------------------------------------------ replicas (N > 1)
# Under torchrun each rank is an independent replica: its own beam of the
# workload's shape (its own seed), no data-path collective; the step time is
# the maximum over ranks and the value counts every rank's units.

def replica_seed(base_seed: int, rank: int) -> int:
    """Seed of rank `rank`'s beam (distinct per rank)."""
    return base_seed + 1000 * rank


def max_over_ranks(x: float, world: int, device: str) -> float:
    """Maximum of x over the ranks of the default process group (x if alone)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, seconds: float) -> float:
    """Units per second of the whole job: every rank's units over the slowest rank's time."""
    return units_per_rank * world / seconds


def share_words(d: np.ndarray, foff: float, db: int, tile: int, cs: int = 4) -> int:
    """Shared-memory words one kernel 5 launch moves, from the plan's delay
    table d [ndm][nchans]: per (DM block of db trials, subband of cs channels,
    time tile) stage 1 reads cs words and writes one for every partial sum
    (each delay pattern's sums cover its trials' reference-delay span plus the
    tile), and stage 2 reads one word per trial and sample."""
    ndm, nch = d.shape
    nblk, nsub = -(-ndm // db), nch // cs
    rows = np.minimum(np.arange(nblk * db), ndm - 1)      # the ragged last block repeats the last trial
    dd = d[rows].astype(np.int64).reshape(nblk, db, nsub, cs)
    ref = dd[..., 0] if foff < 0 else dd[..., cs - 1]      # the subband's highest frequency
    rel = dd - ref[..., None]
    key = np.zeros(ref.shape, np.int64)
    for c in range(cs):                                   # relative delays as one key (each < 2^15)
        key = key * (1 << 15) + rel[..., c]
    b = np.broadcast_to(np.arange(nblk)[:, None, None], key.shape).ravel()
    s = np.broadcast_to(np.arange(nsub)[None, None, :], key.shape).ravel()
    k, r = key.ravel(), ref.ravel()
    order = np.lexsort((r, k, s, b))
    b, s, k, r = b[order], s[order], k[order], r[order]
    start = np.ones(len(k), bool)
    start[1:] = (b[1:] != b[:-1]) | (s[1:] != s[:-1]) | (k[1:] != k[:-1])
    first = np.flatnonzero(start)
    last = np.append(first[1:], len(k)) - 1
    stage1 = int(np.sum(r[last] - r[first] + tile)) * (cs + 1)
    stage2 = nblk * nsub * db * tile
    return stage1 + stage2


def _pulses(wl, nout, seed):
    return synth.draw_pulses(16, 0.0, wl.dm_list[-1], 1, 32, 8.0, 20.0, nout - 32, wl.nchans, seed)


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampler for the timed region (SM clock, throttle reasons)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_sample(ndm_s, nt_s):
    """Inputs for one bounded oracle sample of the LOFAR-like workload: ndm_s DM
    rows spread evenly over the 2000 trials, nt_s output samples."""
    import oracle
    wl = synth.workload(WORKLOAD)
    oracle.build()
    d_all, m = oracle.delays(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list)
    rows = np.linspace(0, wl.ndm - 1, ndm_s).astype(np.int64)
    d = np.ascontiguousarray(d_all[rows])
    x = synth.noise_f32(wl.nchans, nt_s + m, seed=wl.seed)
    return wl, x, d


def _oracle_step(wl, x, d, nt_s):
    """One oracle pass over the sample: de-dispersion, statistics, search."""
    import oracle
    t0 = time.perf_counter()
    out = oracle.dedisperse(x, d, nt_s)
    mu, sg = oracle.stats(out)
    oracle.search(out, list(wl.widths), mu, sg, wl.sigma)
    return time.perf_counter() - t0


REF_SAMPLE = (64, 131072)        # per --impl reference step (about 1 s on 16 cores)
BASELINE_SAMPLE = (256, 262144)  # the GPU line's cpu_baseline (about 10-30 s)


def run_reference(args, rank, world):
    """CPU oracle on a bounded sample of the same workload (rank 0 only)."""
    import oracle
    if rank != 0:
        return
    ndm_s, nt_s = REF_SAMPLE
    wl, x, d = _oracle_sample(ndm_s, nt_s)
    cores = oracle.num_threads()
    times = []
    for i in range(args.warmup + args.steps):
        dt = _oracle_step(wl, x, d, nt_s)
        if i >= args.warmup:
            times.append(dt)
    tm = statistics.median(times)
    value = ndm_s * nt_s / tm
    sample = (f"{ndm_s} of 2000 DM rows x {nt_s} of 1028179 samples per step: "
              "dedisperse + stats + search")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tm * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "lofar_f32: 1024 ch, 150 MHz top, foff -0.01171875 MHz, "
                   "tsamp 163.84 us, 2^20 samples, 2000 DMs 0-99.95 step 0.05",
                   "sample": sample},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_sample():
    """Oracle on a bounded sample (about 10-30 s of CPU work), for the GPU line:
    on all host cores, and on one core (the paper's CPU comparison) over a
    sixteenth of the DM rows."""
    import oracle
    ndm_s, nt_s = BASELINE_SAMPLE
    wl, x, d = _oracle_sample(ndm_s, nt_s)
    dt = _oracle_step(wl, x, d, nt_s)
    cores = oracle.num_threads()
    d1 = np.ascontiguousarray(d[::16])
    oracle.set_threads(1)
    try:
        dt1 = _oracle_step(wl, x, d1, nt_s)
    finally:
        oracle.set_threads(cores)
    return {"value": ndm_s * nt_s / dt, "unit": METRIC, "cores": cores,
            "kind": "oracle", "seconds": dt,
            "sample": f"{ndm_s} of 2000 DM rows x {nt_s} of 1028179 samples: "
                      "dedisperse + stats + search, FP64, all host cores",
            "single_core": {"value": d1.shape[0] * nt_s / dt1, "unit": METRIC, "cores": 1, "seconds": dt1,
                            "sample": f"{d1.shape[0]} of those DM rows x {nt_s} samples, one thread"}}


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    import paper_1107_2516_gb300 as dd
    from paper_1107_2516_gb300 import build as ddbuild

    torch.cuda.set_device(local_rank)
    if rank == 0 or world == 1:
        ddbuild.build()
    if world > 1:
        dist.barrier()
    dd.load()
    wl = synth.workload(WORKLOAD)
    plan = dd.Plan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list, wl.widths, wl.sigma,
                   dd.DD_F32, wl.nsamp)
    if args.kernel:
        plan.set_kernel(args.kernel)
    nout, M = plan.nsamp_out, plan.maxshift
    # input: seeded noise + 16 pulses placed with the plan's own delay law
    x = synth.noise_f32(wl.nchans, wl.nsamp, seed=replica_seed(wl.seed, rank))
    pulses = _pulses(wl, nout, seed=replica_seed(wl.seed, rank))
    pplan = dd.Plan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, [p.dm for p in pulses], [1], 6.0,
                    dd.DD_F32, wl.nsamp)
    ptab = pplan.delays().astype(np.int64)
    pplan.close()
    lookup = {p.dm: ptab[i] for i, p in enumerate(pulses)}
    synth.inject_pulses(x, pulses, lambda dm: lookup[dm], wl.nsamp)
    host = torch.from_numpy(x)
    xin = host.cuda()
    out = torch.empty(wl.ndm * nout, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        plan.execute(xin, wl.nsamp, out, stream)
        if ev is not None:
            ev[1].record(stream)
        return plan.search(out, capacity=1 << 16, stream=stream)

    if not args.kernel and not args.no_autotune:
        plan.autotune(xin, wl.nsamp, out, stream)      # picks tile shape + raster (cached per shape)
    for _ in range(args.warmup):
        cands, total = step()
    torch.cuda.synchronize()
    ev_steps = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)]
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(torch.cuda.current_device())
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    g0.record(stream)
    for i in range(args.steps):
        cands, total = step(ev_steps[i])
    g1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    total_ms = g0.elapsed_time(g1)
    ker_ms = statistics.mean(a.elapsed_time(b) for a, b in ev_steps)
    total_ms = max_over_ranks(total_ms, world, "cuda")
    ms_per_step = total_ms / args.steps
    units_per_rank = wl.ndm * nout
    value = whole_job_rate(units_per_rank, world, ms_per_step / 1e3)

    # end to end through the C ABI with host input (H2D + execute + search + readback)
    pinned = host.pin_memory()
    for _ in range(max(1, args.warmup // 2)):
        plan.process_host(pinned, wl.nsamp, capacity=1 << 16, stream=stream)
    torch.cuda.synchronize()
    e2e_t = []
    for _ in range(max(3, args.steps)):
        e0 = time.perf_counter()
        c2, n2 = plan.process_host(pinned, wl.nsamp, capacity=1 << 16, stream=stream)
        e2e_t.append(time.perf_counter() - e0)
    e2e_s = max_over_ranks(statistics.median(e2e_t), world, "cuda")
    e2e_value = whole_job_rate(units_per_rank, world, e2e_s)

    kernel_id = plan.kernel
    tile = plan.tile if kernel_id in (2, 3, 4, 5) else None
    d_plan = plan.delays() if kernel_id == 5 else None
    plan.close()
    del out, xin
    if rank != 0:
        return
    peaks = _peaks()
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    adds = float(wl.ndm) * nout * wl.nchans
    achieved = adds / (ker_ms / 1e3) / 1e9             # G channel-adds / s
    peak = sm * 128 * sm_max * 1e6 / 1e9               # FP32 lanes x max clock
    tile_s = ""
    if tile:
        k, ns, nd, nw = TILE_CONFIGS[tile[0]]
        per = "thread" if k == 2 else "lane"
        tile_s = (f", tile config {tile[0]}: {ns} samples per {per} x {nd} DM trials per "
                  f"{'thread' if k == 2 else 'warp'}, {nw} warps"
                  + (f" + {STAGE1_WARPS[tile[0]]} stage-1 warps" if tile[0] in STAGE1_WARPS else "")
                  + f", raster group {tile[1]}")
    roof = {"bound": "alu", "kernel": f"dd kernel {kernel_id} (de-dispersion{tile_s})",
            "achieved": achieved, "peak": peak, "unit": "Gadd/s", "frac": achieved / peak,
            "peak_basis": f"{sm} SMs x 128 FP32 lanes x {sm_max:.0f} MHz (max clock)",
            # dram__bytes_read.sum + dram__bytes_write.sum of one launch from an ncu
            # capture of this tile with these kernel sources (null otherwise)
            "traffic": profiled_traffic(kernel_id, tile),
            "traffic_unit": "bytes per launch",
            "kernel_ms": ker_ms}
    if kernel_id == 5:
        # kernel 5 shares each 4-channel subband's partial sums between the DM
        # trials of a block with the same relative delays: `achieved` counts
        # the brute-force-equivalent channel-adds of the exact result; the
        # bound it meets is the shared-memory data path, here against the words
        # its two stages move
        roof["note"] = ("kernel 5: exact shared subband partial sums; achieved = brute-force-equivalent "
                        "channel-adds (the sum is identical; fewer adds are executed)")
        _, ns, nd, nw = TILE_CONFIGS[tile[0]]
        ntile = -(-nout // (32 * ns))
        words = share_words(d_plan, wl.foff, nd * nw, 32 * ns) * ntile
        lds_peak = sm * 32 * sm_max * 1e6 / 1e9
        aw = words / (ker_ms / 1e3) / 1e9
        roof["secondary"] = {"bound": "shared-memory words", "achieved": aw, "peak": lds_peak,
                             "unit": "Gword/s", "frac": aw / lds_peak,
                             "words_per_output": words / (wl.ndm * nout),
                             "peak_basis": f"{sm} SMs x 32 banks x {sm_max:.0f} MHz"}
    if kernel_id == 3:
        # kernel 3 loads one shared-memory word per add: the shared-memory data
        # path (32 words/clk/SM, 4 B x 32 banks) caps it at a quarter of the add peak
        lds_peak = sm * 32 * sm_max * 1e6 / 1e9
        roof["secondary"] = {"bound": "shared-memory words", "achieved": achieved, "peak": lds_peak,
                             "unit": "Gword/s", "frac": achieved / lds_peak,
                             "peak_basis": f"{sm} SMs x 32 banks x {sm_max:.0f} MHz"}
    if clk.get("sm_mhz"):
        roof["frac_at_measured_clock"] = achieved / (sm * 128 * clk["sm_mhz"] * 1e6 / 1e9)
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "lofar_f32: 1024 ch, fch1 150 MHz, foff -0.01171875 MHz, "
                   "tsamp 163.84 us, nsamp 2^20, 2000 DMs 0-99.95 step 0.05, widths 1..32, 6 sigma",
                   "nsamp_out": nout, "maxshift": M, "l2": "inputs larger than L2 (4.3 GB in, 8.2 GB out)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "real_time_factor": (nout * wl.tsamp) / (ms_per_step / 1e3),
        "dedisp_ms": ker_ms, "search_ms": ms_per_step - ker_ms,
        "candidates": int(total),
        "e2e": {"value": e2e_value, "unit": METRIC,
                "h2d_bytes_per_step": int(wl.nchans * wl.nsamp * 4),
                "d2h_bytes_per_step": int(8 + 32 * min(total, 1 << 16) + 272)},
        # per step: the de-dispersion kernel, finalize_kernel (statistics),
        # the boxcar search kernel and cand_snr_kernel
        "gpu_launches": 4 * args.steps,
        "clocks": clk,
        "roofline": roof,
    }
    if world == 1 and not args.no_batch_serve:
        # the batched and the serving forms on the same GPU, beside the plain
        # single-beam line: 24 uneven beams in one CUDA graph, and 64 streaming
        # beams under real-time arrival (latency) and a burst (capacity)
        del host, pinned
        torch.cuda.empty_cache()
        bt = batch_measure(torch, dd, steps=3, warmup=1)
        sv = serve_measure(torch, dd, args.serve_window, args.speed, args.workers, args.budget_frac, args.burst)
        line["batched"] = bt
        line["serving"] = sv
        line["plain_vs_batched_serving"] = {
            "plain_single_beam_f32": {"value": value, "latency_s": ms_per_step / 1e3,
                                      "buffer_duration_s": nout * wl.tsamp},
            "batched_24_beams": {"value": bt["value"], "latency_s": bt["ms_per_step"] / 1e3},
            "serving_64_beams": {"capacity_value": sv["value"],
                                 "realtime_p50_s": sv["realtime"]["latency_s"]["p50"],
                                 "realtime_p99_s": sv["realtime"]["latency_s"]["p99"],
                                 "realtime_rtf_min": sv["realtime"]["real_time_factor"]["min"]},
            "unit": METRIC,
        }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample()
    print(json.dumps(line), flush=True)


def _device_beam_input(torch, b, pitch, seed):
    """N(0,1) float32 (or 8-bit quantised) channel-major input generated on the device."""
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    x = torch.randn(b.nchans, pitch, device="cuda", generator=g)
    if b.dtype == "u8":
        x = (x * 16.0 + 128.0).round_().clamp_(0, 255).to(torch.uint8)
    return x


def batch_measure(torch, dd, steps, warmup, full_autotune=False, sequential=True):
    """The 24-beam batched workload (float32/uint8 mix, 256-4096 channels,
    2^16-2^20 samples, 500-4000 DM trials): the whole batch (every beam's
    de-dispersion + search) replayed from one CUDA graph, against the same
    beams run one after another through dd_execute + dd_search.  The launch
    configuration is the batch autotuner's choice (full_autotune), or else the
    faster of the two launch modes of the default mixed configuration (kernel 5
    where its tables fit, kernel 3 otherwise), each timed once.  Returns a dict."""
    def maxshift_of(c, f1, fo, ts, dm):
        p = dd.Plan(c, f1, fo, ts, [dm], [1], 6.0, dd.DD_F32, 1 << 30)
        m = p.maxshift
        p.close()
        return m

    t_setup = time.perf_counter()
    beams = synth.batch_beams(24, 4, maxshift_of)
    widths = (1, 2, 4, 8, 16, 32)
    plans, ins, pitches, outs = [], [], [], []
    for i, b in enumerate(beams):
        p = dd.Plan(b.nchans, b.fch1, b.foff, b.tsamp, b.dm_list, widths, 6.0,
                    dd.DD_F32 if b.dtype == "f32" else dd.DD_U8, b.nsamp)
        pitch = synth.aligned_pitch(b.nsamp, 4 if b.dtype == "f32" else 1)
        plans.append(p)
        pitches.append(pitch)
        ins.append(_device_beam_input(torch, b, pitch, b.seed))
        outs.append(torch.empty(p.ndm * p.nsamp_out, device="cuda",
                                dtype=torch.int32 if p.out_is_int else torch.float32))
    units = sum(p.ndm * p.nsamp_out for p in plans)
    adds = sum(p.ndm * p.nsamp_out * p.nchans for p in plans)
    stream = torch.cuda.Stream()
    batch = dd.Batch(plans)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    if full_autotune:
        batch.autotune(ins, pitches, outs, stream)
        how = "the batch autotuner's choice over every configuration and both launch modes"
    else:
        best = None
        for per_beam in (True, False):
            batch.set_launch_mode(per_beam)
            batch.execute(ins, pitches, outs, stream)            # warm-up
            ev[0].record(stream)
            batch.execute(ins, pitches, outs, stream)
            ev[1].record(stream)
            torch.cuda.synchronize()
            ms = ev[0].elapsed_time(ev[1])
            if best is None or ms < best[0]:
                best = (ms, per_beam)
        batch.set_launch_mode(best[1])
        how = "default mixed configuration (kernel 5 / kernel 3), the faster launch mode of one timed run each"
    batch.capture(ins, pitches, outs, stream)
    # the sequential reference runs each plan with the tile shape it has in the batch
    beam_cfg = [batch.beam_config(i) for i in range(len(plans))]
    for p, c in zip(plans, beam_cfg):
        if c >= 0:
            p.set_tile(c, 8)
    setup_s = time.perf_counter() - t_setup

    def run_batch_once():
        batch.launch(stream)
        tot = 0
        for i in range(len(plans)):
            tot += batch.results(i, stream=stream, allow_overflow=True)[1]
        return tot

    def run_sequential_once():
        tot = 0
        for p, x, pitch, o in zip(plans, ins, pitches, outs):
            p.execute(x, pitch, o, stream)
            tot += p.search(o, stream=stream, allow_overflow=True)[1]
        return tot

    for _ in range(warmup):
        run_batch_once()
    if sequential:
        run_sequential_once()
    torch.cuda.synchronize()
    tb, ts_ = [], []
    for _ in range(steps):
        ev[0].record(stream)
        nb = run_batch_once()
        ev[1].record(stream)
        torch.cuda.synchronize()
        tb.append(ev[0].elapsed_time(ev[1]))
        if sequential:
            ev[2].record(stream)
            run_sequential_once()
            ev[3].record(stream)
            torch.cuda.synchronize()
            ts_.append(ev[2].elapsed_time(ev[3]))
    mb = statistics.median(tb)
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    peak = sm * 128 * 2070e6 / 1e9
    cfg, nitems, nsep = batch.info
    res = {
        "value": units / (mb / 1e3), "unit": METRIC, "ms_per_step": mb, "steps": steps, "warmup": warmup,
        "workload": "24 uneven beams: 256-4096 ch, 2^16-2^20 samples, 500-4000 DMs, fp32 + uint8, "
                    "widths 1..32, 6 sigma", "units": units, "adds": adds,
        "tile_config": cfg, "work_items": nitems, "separate_beams": nsep,
        "beams_on_kernel5": sum(1 for c in beam_cfg if c >= 9),
        "launch": ("each beam's own de-dispersion launch" if batch.per_beam else "one persistent kernel")
                  + " + per-beam search, CUDA graph replay",
        "how_chosen": how, "candidates": int(nb),
        "achieved_gadd_s": adds / (mb / 1e3) / 1e9, "alu_frac_of_peak": adds / (mb / 1e3) / 1e9 / peak,
        "setup_s": setup_s,
    }
    if sequential:
        ms = statistics.median(ts_)
        res["sequential"] = {"value": units / (ms / 1e3), "ms_per_step": ms,
                             "how": "each beam through dd_execute + dd_search in turn, its batch tile shape"}
        res["speedup_vs_sequential"] = ms / mb
    batch.close()
    for p in plans:
        p.close()
    del ins, outs
    torch.cuda.synchronize()
    return res


def run_batch(args):
    """The batched workload alone: prints one JSON line (mode "batch")."""
    import torch
    import paper_1107_2516_gb300 as dd
    from paper_1107_2516_gb300 import build as ddbuild

    ddbuild.build()
    dd.load()
    r = batch_measure(torch, dd, args.steps, args.warmup, full_autotune=not args.no_autotune)
    line = {"mode": "batch", "metric": METRIC, "value": r.pop("value"), "unit": METRIC, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r.pop("ms_per_step"),
            "higher_is_better": True, "dtype": "f32/u8", "data": "synthetic", "config": r}
    print(json.dumps(line), flush=True)


def serve_measure(torch, dd, window_s, speed, workers, budget_frac, burst):
    """The 64-beam streaming workload (uint8, 1024/4096 channels, 1000-4096 DM
    trials to DM 500, chunks of 65536 samples) on one server, in steady state.
    Admission: every beam is admitted against budget_frac of free device
    memory (a beam that does not fit waits for one to leave) and streams its
    priming chunks at once (the history a live stream holds already).  Then
    (1) real-time window: each beam's chunks arrive at `speed` x its real-time
    rate (+-10% jitter, random phase) for window_s seconds: chunk latency
    (submit -> candidates on the host) p50/p99 and the real-time factor (chunk
    duration / processing time); (2) capacity: every served beam submits
    `burst` chunks at once and the server runs them with its worker streams
    (continuous batching): DM-trial.samples/s over the burst.  Returns a dict."""
    beams = synth.serve_beams(64, 5)
    free, _ = torch.cuda.mem_get_info()
    budget = int(budget_frac * free)
    t_setup = time.perf_counter()
    srv = dd.Server(budget, nworkers=workers, max_candidates=1 << 16)
    data = {c: torch.from_numpy(synth.quantize_u8(synth.noise_f32(c, 65536, seed=c))).pin_memory()
            for c in (1024, 4096)}
    widths = (1, 2, 4, 8, 16, 32, 64)
    st = {}
    refused = []
    kernels = {}
    for i, b in enumerate(beams):
        try:
            bid = srv.add_beam(b.nchans, b.fch1, b.foff, b.tsamp, b.dm_list, widths, 6.0, dd.DD_U8, b.chunk)
        except dd.DDError as e:
            if e.code != dd.dd.DD_ERR_BUDGET:
                raise
            refused.append(i)
            continue
        info = srv.beam_info(bid)
        k = srv.beam_kernel(bid)[0]
        kernels[k] = kernels.get(k, 0) + 1
        prime = -(-info["maxshift"] // b.chunk)
        st[bid] = dict(i=i, next=0, prime=prime, ndm=b.ndm, period=b.period, chunk=b.chunk)
    for bid, s in st.items():
        for q in range(s["prime"]):
            srv.submit(bid, data[beams[s["i"]].nchans], s["chunk"], q)
        s["next"] = s["prime"]
    npr = sum(s["prime"] for s in st.values())
    got = 0
    while got < npr:
        for r in srv.poll(max_results=256, wait_ms=100):
            if int(r["status"]) != dd.DD_PRIMING:
                raise RuntimeError(f"priming chunk status {int(r['status'])}")
            got += 1
    setup_s = time.perf_counter() - t_setup

    # (1) real-time window
    for bid, s in st.items():
        b = beams[s["i"]]
        s["times"] = synth.arrival_times(b, 64, b.seed) / speed
    lat, proc, rtf, units_rt = [], [], [], 0
    t0 = time.perf_counter()
    outstanding = 0
    while True:
        now = time.perf_counter() - t0
        nxt = None
        if now < window_s:
            for bid, s in st.items():
                j = s["next"] - s["prime"]
                while j < len(s["times"]) and s["times"][j] <= now:
                    srv.submit(bid, data[beams[s["i"]].nchans], s["chunk"], s["next"])
                    s["next"] += 1
                    outstanding += 1
                    j += 1
                if j < len(s["times"]):
                    nxt = s["times"][j] if nxt is None else min(nxt, s["times"][j])
        elif outstanding == 0:
            break
        wait = 50 if nxt is None else max(1, min(50, int((nxt - now) * 1000)))
        for r in srv.poll(max_results=256, wait_ms=wait):
            s = st[int(r["beam"])]
            if int(r["status"]) != 0:
                raise RuntimeError(f"chunk status {int(r['status'])}")
            outstanding -= 1
            lat.append(float(r["t_done"] - r["t_submit"]))
            pt = float(r["t_done"] - r["t_start"])
            proc.append(pt)
            rtf.append(s["period"] / pt)
            units_rt += s["ndm"] * s["chunk"]
            srv.candidates(int(r["beam"]), int(r["seq"]), capacity=1 << 16)   # fetched (and freed)
        if time.perf_counter() - t0 > window_s + 120:
            raise RuntimeError("serving window did not drain")
    wall_rt = time.perf_counter() - t0

    # (2) capacity: `burst` chunks per beam submitted at once
    units_b, lat_b = 0, []
    t1 = time.perf_counter()
    for bid, s in st.items():
        for _ in range(burst):
            srv.submit(bid, data[beams[s["i"]].nchans], s["chunk"], s["next"])
            s["next"] += 1
    left = burst * len(st)
    while left:
        for r in srv.poll(max_results=256, wait_ms=100):
            if int(r["status"]) != 0:
                raise RuntimeError(f"chunk status {int(r['status'])}")
            s = st[int(r["beam"])]
            units_b += s["ndm"] * s["chunk"]
            lat_b.append(float(r["t_done"] - r["t_submit"]))
            left -= 1
        if time.perf_counter() - t1 > 600:
            raise RuntimeError("burst did not drain")
    wall_b = time.perf_counter() - t1
    srv.close()
    lat_a, rtf_a = np.array(lat), np.array(rtf)
    periods = [beams[s["i"]].period for s in st.values()]
    return {
        "value": units_b / wall_b, "unit": METRIC,
        "workload": "64 streaming uint8 beams, 1024/4096 ch, 1000-4096 DMs to DM 500, chunks of 65536 "
                    "samples, widths 1..64, 6 sigma",
        "hbm_budget_bytes": budget, "workers": workers, "beams_admitted": len(st),
        "beams_refused_by_budget": len(refused), "beam_kernels": {str(k): v for k, v in sorted(kernels.items())},
        "setup_s": setup_s,
        "realtime": {"arrival": f"{speed}x real-time rate, +-10% jitter, random phase", "window_s": window_s,
                     "chunks_searched": len(lat), "chunk_duration_s": [min(periods), max(periods)],
                     "latency_s": {"p50": float(np.percentile(lat_a, 50)) if len(lat) else None,
                                   "p99": float(np.percentile(lat_a, 99)) if len(lat) else None},
                     "processing_s": {"p50": float(np.percentile(proc, 50)) if proc else None},
                     "real_time_factor": {"median": float(np.median(rtf_a)) if len(rtf) else None,
                                          "min": float(rtf_a.min()) if len(rtf) else None},
                     "rate": units_rt / wall_rt, "wall_s": wall_rt},
        "capacity": {"how": f"{burst} chunks per served beam submitted at once", "chunks": burst * len(st),
                     "wall_s": wall_b, "value": units_b / wall_b,
                     "latency_s": {"p50": float(np.percentile(lat_b, 50)), "p99": float(np.percentile(lat_b, 99))},
                     "real_time_factor": (sum(burst * p for p in periods)) / wall_b},
    }


def run_serve(args):
    """The streaming workload alone: prints one JSON line (mode "serve")."""
    import torch
    import paper_1107_2516_gb300 as dd
    from paper_1107_2516_gb300 import build as ddbuild

    ddbuild.build()
    dd.load()
    r = serve_measure(torch, dd, args.serve_window, args.speed, args.workers, args.budget_frac, args.burst)
    line = {"mode": "serve", "metric": METRIC, "value": r.pop("value"), "unit": METRIC, "n_gpus": 1,
            "higher_is_better": True, "dtype": "u8", "data": "synthetic", "config": r}
    print(json.dumps(line), flush=True)


def run_subband(args):
    """Section 3.2 subband de-dispersion of the LOFAR-like beam (1024 channels
    in 32 subbands, 2000 fine DMs in groups of 24 = 1.2 pc/cm3 per nominal DM)
    against the brute-force path on the same input: throughput, adds, and the
    S/N of the 16 injected pulses found by each.  Prints one JSON line (mode
    "subband")."""
    import torch
    import paper_1107_2516_gb300 as dd
    from paper_1107_2516_gb300 import build as ddbuild

    ddbuild.build()
    dd.load()
    wl = synth.workload(WORKLOAD)
    G, nsub = args.dms_per_nominal, args.nsub
    sp = dd.SubbandPlan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list, G, nsub, wl.widths, wl.sigma,
                        dd.DD_F32, wl.nsamp)
    bf = dd.Plan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, wl.dm_list, wl.widths, wl.sigma, dd.DD_F32,
                 wl.nsamp)
    x = synth.noise_f32(wl.nchans, wl.nsamp, seed=wl.seed + 7)
    pulses = _pulses(wl, min(sp.nsamp_out, bf.nsamp_out), seed=wl.seed + 7)
    ptab = dd.Plan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, [p.dm for p in pulses], [1], 6.0, dd.DD_F32,
                   wl.nsamp)
    lookup = {p.dm: ptab.delays().astype(np.int64)[i] for i, p in enumerate(pulses)}
    ptab.close()
    synth.inject_pulses(x, pulses, lambda dm: lookup[dm], wl.nsamp)
    xin = torch.from_numpy(x).cuda()
    stream = torch.cuda.current_stream()
    out_s = torch.empty(wl.ndm * sp.nsamp_out, device="cuda")
    out_b = torch.empty(wl.ndm * bf.nsamp_out, device="cuda")
    bf.autotune(xin, wl.nsamp, out_b, stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

    def step(plan, out):
        ev[0].record(stream)
        plan.execute(xin, wl.nsamp, out, stream)
        ev[1].record(stream)
        c, n = plan.search(out, capacity=1 << 18, stream=stream)
        ev[2].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]), ev[0].elapsed_time(ev[2]), c

    for _ in range(args.warmup):
        step(sp, out_s)
        step(bf, out_b)
    ts, tb = [], []
    for _ in range(args.steps):
        ts.append(step(sp, out_s))
        tb.append(step(bf, out_b))
    ex_s = statistics.median(t[0] for t in ts)
    st_s = statistics.median(t[1] for t in ts)
    ex_b = statistics.median(t[0] for t in tb)
    st_b = statistics.median(t[1] for t in tb)

    def best_snr(cands, p):
        i0 = int(round(p.dm / 0.05))
        sel = cands[(np.abs(cands["dm_idx"] - i0) <= G) & (np.abs(cands["t"] - p.t0) <= 64)]
        return float(sel["snr"].max()) if len(sel) else 0.0

    snr = [(best_snr(ts[-1][2], p), best_snr(tb[-1][2], p)) for p in pulses]
    K = sp.n_nominal
    L = sp.work_bytes // (4 * nsub * K)
    adds_sub = K * wl.nchans * L + wl.ndm * nsub * sp.nsamp_out
    adds_bf = wl.ndm * wl.nchans * bf.nsamp_out
    units = wl.ndm * sp.nsamp_out
    line = {
        "mode": "subband", "metric": METRIC, "value": units / (st_s / 1e3), "unit": METRIC,
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": st_s,
        "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "lofar_f32 (1024 ch, 2^20 samples, 2000 DMs 0-99.95) + 16 pulses",
                   "dms_per_nominal": G, "nsub": nsub, "n_nominal": K, "maxshift": sp.maxshift,
                   "series_bytes": sp.work_bytes},
        "subband": {"execute_ms": ex_s, "step_ms": st_s, "adds": adds_sub,
                    "tadd_s": adds_sub / (ex_s / 1e3) / 1e12},
        "brute_force": {"execute_ms": ex_b, "step_ms": st_b, "adds": adds_bf,
                        "tadd_s": adds_bf / (ex_b / 1e3) / 1e12, "tile": bf.tile},
        "speedup_execute": ex_b / ex_s, "speedup_step": st_b / st_s,
        "pulse_snr": {"subband": [round(a, 2) for a, _ in snr], "brute_force": [round(b, 2) for _, b in snr],
                      "mean_ratio": float(np.mean([a / b for a, b in snr if b > 0]))},
    }
    sp.close()
    bf.close()
    print(json.dumps(line), flush=True)


def run_survey(args):
    """The survey plan of Table 1 / Table 4 (three passes: DM 0-53.46 step 0.03
    unbinned, 53.46-88.26 step 0.05 binned x2, 88.26-150.66 step 0.10 binned
    x4; 32 subbands) on a 60 s beam at 300 MHz, 16 MHz in 1024 channels
    (64 us sampling): binning + subband de-dispersion + search of every pass.
    The paper's GPU code took 90 s for its 60 s file (Table 4 comparison,
    C1060).  Prints one JSON line (mode "survey")."""
    import torch
    import paper_1107_2516_gb300 as dd
    from paper_1107_2516_gb300 import build as ddbuild

    ddbuild.build()
    dd.load()
    wl = synth.workload("survey_f32")
    sp = dd.SurveyPlan(wl.nchans, wl.fch1, wl.foff, wl.tsamp, synth.SURVEY_PLAN, args.nsub, wl.widths, wl.sigma,
                       dd.DD_F32, wl.nsamp)
    x = synth.noise_f32(wl.nchans, wl.nsamp, seed=wl.seed + 11)
    xin = torch.from_numpy(x).cuda()
    outs = [torch.empty(p[0] * p[4], device="cuda") for p in sp.passes]
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

    def step():
        ev[0].record(stream)
        sp.execute(xin, wl.nsamp, outs, stream)
        ev[1].record(stream)
        n = sum(sp.search(i, outs[i], capacity=1 << 18, stream=stream, allow_overflow=True)[1]
                for i in range(sp.npass))
        ev[2].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]), ev[0].elapsed_time(ev[2]), n

    for _ in range(args.warmup):
        step()
    res = [step() for _ in range(args.steps)]
    ex = statistics.median(r[0] for r in res)
    st = statistics.median(r[1] for r in res)
    units = sum(p[0] * p[4] for p in sp.passes)
    obs_s = wl.nsamp * wl.tsamp
    line = {
        "mode": "survey", "metric": METRIC, "value": units / (st / 1e3), "unit": METRIC,
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": st,
        "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "survey_f32: 60 s, 1024 ch, 300 MHz centre, 16 MHz, tsamp 64 us; "
                   "Table 4 plan (3 passes, 3102 DM trials to 150.66), nsub 32",
                   "passes": [{"ndm": p[0], "bin": p[1], "dms_per_nominal": p[2], "maxshift": p[3],
                               "nsamp_out": p[4]} for p in sp.passes]},
        "execute_ms": ex, "step_ms": st, "candidates": res[-1][2],
        "observation_s": obs_s, "real_time_factor": obs_s / (st / 1e3),
        "paper_gpu_s_per_observation": 90.0,
    }
    sp.close()
    print(json.dumps(line), flush=True)


def run_realtime(args):
    """The real-time pipeline of Section 5 (Table 5 toy observation: 610 MHz
    centre, 20 MHz in 256 subbands sampled at 12.8 us, 8 channels per subband,
    500 DM trials to 60 pc/cm3; buffers of 2^19 spectra = 6.7 s): per buffer,
    H2D copy of the complex voltages from pinned memory, the fused front end
    (channeliser + intensity + corner turn), brute-force de-dispersion and
    search with candidate readback.  Stage times beside Table 6 (C1060: 475,
    458 + 20 + 112, 4500 and 220 ms of 5785 ms).  Prints one JSON line (mode
    "realtime")."""
    import torch
    import paper_1107_2516_gb300 as dd
    from paper_1107_2516_gb300 import build as ddbuild

    ddbuild.build()
    dd.load()
    nsub, nfft, tv, spectra = 256, 8, 12.8e-6, 1 << 19
    fbw = 20.0 / nsub
    ftop = 610.0 + 10.0
    nchans, nb = nsub * nfft, spectra // nfft
    dms = [0.12 * i for i in range(500)]
    fch1 = ftop - 0.5 * fbw / nfft
    plan = dd.Plan(nchans, fch1, -fbw / nfft, nfft * tv, dms, (1, 2, 4, 8, 16, 32), 6.0, dd.DD_F32, nb)
    r = np.random.default_rng(7)
    v = (r.standard_normal((nsub, spectra), dtype=np.float32) +
         1j * r.standard_normal((nsub, spectra), dtype=np.float32)).astype(np.complex64)
    host = torch.from_numpy(v.view(np.float32)).pin_memory()
    volt = torch.empty_like(host, device="cuda")
    fil = torch.empty(nchans * nb, device="cuda")
    out = torch.empty(len(dms) * plan.nsamp_out, device="cuda")
    stream = torch.cuda.current_stream()
    plan.autotune(fil, nb, out, stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]

    def buffer():
        ev[0].record(stream)
        volt.copy_(host, non_blocking=True)
        ev[1].record(stream)
        dd.dd_channelise(volt, 1, nsub, spectra, nfft, fil, nb, stream)
        ev[2].record(stream)
        plan.execute(fil, nb, out, stream)
        ev[3].record(stream)
        c, n = plan.search(out, capacity=1 << 16, stream=stream, allow_overflow=True)
        ev[4].record(stream)
        torch.cuda.synchronize()
        return [ev[i].elapsed_time(ev[i + 1]) for i in range(4)], n

    for _ in range(args.warmup):
        buffer()
    res = [buffer() for _ in range(args.steps)]
    med = [statistics.median(x[0][i] for x in res) for i in range(4)]
    total = sum(med)
    buf_s = spectra * tv
    fe_bytes = nsub * spectra * 8 + nchans * nb * 4
    peaks = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6784.5))
    line = {
        "mode": "realtime", "metric": "real-time factor", "value": buf_s / (total / 1e3),
        "unit": "buffer seconds / processing seconds", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "Table 5: 610 MHz, 20 MHz, 256 subbands x 8 channels, 12.8 us, 2^19 spectra "
                   "per buffer, 500 DMs to 59.88, brute force", "nchans": nchans, "nsamp": nb,
                   "nsamp_out": plan.nsamp_out, "maxshift": plan.maxshift, "tile": plan.tile},
        "stages_ms": {"h2d": med[0], "channelise_intensity_corner_turn": med[1], "dedisperse": med[2],
                      "search_and_readback": med[3]},
        "paper_stages_ms": {"h2d": 475, "channelise_intensity_corner_turn": 458 + 20 + 112, "dedisperse": 4500,
                            "search_and_readback": 220, "total": 5785},
        "buffer_s": buf_s, "candidates": res[-1][1],
        "frontend_roofline": {"bound": "hbm", "achieved": fe_bytes / (med[1] / 1e3) / 1e9, "peak": hbm,
                              "unit": "GB/s", "frac": fe_bytes / (med[1] / 1e3) / 1e9 / hbm,
                              "bytes": fe_bytes},
    }
    plan.close()
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="lofar", choices=["lofar", "batch", "serve", "subband", "survey", "realtime"],
                    help="lofar: the benchmark line; batch: the 24-beam batched workload; "
                         "serve: the 64-beam streaming workload; subband: Section 3.2 "
                         "subband de-dispersion of the lofar workload vs brute force; survey: "
                         "the Table 4 survey plan (binning + subband passes) on a 60 s beam; "
                         "realtime: the Section 5 pipeline (voltages -> front end -> de-dispersion)")
    ap.add_argument("--dms-per-nominal", type=int, default=24, help="subband: fine DMs per nominal DM")
    ap.add_argument("--nsub", type=int, default=32, help="subband: number of subbands")
    ap.add_argument("--speed", type=float, default=1.0, help="serve: arrival rate / real-time rate")
    ap.add_argument("--workers", type=int, default=4, help="serve: server worker streams")
    ap.add_argument("--serve-window", type=float, default=25.0, help="serve: real-time window (s)")
    ap.add_argument("--burst", type=int, default=2, help="serve: chunks per beam in the capacity burst")
    ap.add_argument("--no-batch-serve", action="store_true",
                    help="lofar: skip the batched and serving measurements")
    ap.add_argument("--budget-frac", type=float, default=0.6, help="serve: HBM budget / free memory")
    ap.add_argument("--kernel", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.mode == "batch":
        run_batch(args)
        return
    if args.mode == "serve":
        run_serve(args)
        return
    if args.mode == "subband":
        run_subband(args)
        return
    if args.mode == "survey":
        run_survey(args)
        return
    if args.mode == "realtime":
        run_realtime(args)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
