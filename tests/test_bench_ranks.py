"""The benchmark's N-replica timing on two gloo ranks on the CPU: every rank learns the slowest
rank's timed-region length (all_reduce MAX), and the whole-job rate is all ranks' units over that
length. The library path itself has no data-parallel split (one independent replica per GPU).
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms_max = bench.max_over_ranks(times[rank], world, "cpu")
        out[rank] = (ms_max, bench.whole_job_rate(11, world, ms_max))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_sets_the_job_time():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    world, port = 2, _free_port()
    times = [8.0, 12.5]
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, times, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    for r in range(world):
        ms_max, rate = res[r]
        assert ms_max == 12.5
        assert rate == pytest.approx(11 * 2 / 0.0125)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.25, 1, "cpu") == 7.25
    assert bench.whole_job_rate(10, 1, 7.25) == pytest.approx(10 / 0.00725)
