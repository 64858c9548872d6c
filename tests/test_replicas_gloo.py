"""The multi-GPU combination of the benchmark (replicas, no data-path
collective), run as two gloo ranks on the CPU: every rank gets the slowest
rank's time, the job rate counts the units of all ranks, only rank 0 prints.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2310_17864_gb300 import replicas


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = [2.5, 4.0, 3.0][rank]
        ms = replicas.slowest(ms_local, dist)
        rate = replicas.job_rate(1000.0, world, ms)
        q.put((rank, ms_local, ms, rate, replicas.prints(rank)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slowest_rank_and_job_rate(world):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    want_ms = max([2.5, 4.0, 3.0][:world])
    for rank, ms_local, ms, rate, prints in got:
        assert ms == want_ms
        assert rate == pytest.approx(world * 1000.0 / (want_ms / 1e3))
        assert prints == (rank == 0)


def test_single_process_needs_no_group():
    assert replicas.slowest(1.25) == 1.25
    assert replicas.job_rate(10.0, 1, 2.0) == pytest.approx(5000.0)
    with pytest.raises(ValueError):
        replicas.job_rate(1.0, 1, 0.0)
