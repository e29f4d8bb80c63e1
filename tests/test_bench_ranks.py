"""The multi-GPU form of the benchmark is N independent replicas (the path
does not shard): each rank renders the whole frame, the job time is the
slowest rank's and the job rate counts every rank's samples.  The reduction
is checked here with world-size-2 gloo process groups on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.reduce_max(times[rank], world, "cpu")
        dist.barrier()
        out.put((rank, ms, bench.job_rate(1_000_000_000, world, ms)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("times", [(10.0, 12.5), (7.0, 3.0)])
def test_replicas_take_the_slowest_rank(times):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    slow = max(times)
    assert [g[1] for g in got] == [slow, slow]
    assert got[0][2] == pytest.approx(2 * 1e9 / (slow * 1e-3) / 1e9)


def test_single_rank_is_local():
    assert bench.reduce_max(4.5, 1, "cpu") == 4.5
    assert bench.job_rate(1.59e9, 1, 9.15) == pytest.approx(173.77, rel=1e-3)
