"""The multi-GPU form is replicas (one independent beam per rank, no
data-path collective): its host logic -- distinct per-rank beams, the step
time as the maximum over ranks, the whole-job rate -- run as two gloo ranks
on the CPU through the same functions bench.py uses under torchrun."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seed = bench.replica_seed(2, rank)
        t = 10.0 + 5.0 * rank                                  # this rank's step time
        tmax = bench.max_over_ranks(t, world, "cpu")
        rate = bench.whole_job_rate(1000, world, tmax)
        seeds = [None] * world
        dist.all_gather_object(seeds, seed)
        q.put((rank, tmax, rate, seeds))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tmax, rate, seeds in res:
        assert tmax == 15.0                                    # slowest rank's time on every rank
        assert rate == 1000 * world / 15.0
        assert len(set(seeds)) == world                        # every rank its own beam


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0
