"""The multi-rank path of bench.py (replicas, weak scaling) on CPU with the
gloo backend: the step time is the maximum over ranks and the reported value
is the units of all ranks over that time."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [10.0 + rank, 5.0 * (rank + 1), 1.0]
    got = bench.reduce_max(ms, world, "cpu")
    val = bench.whole_job_value(1000.0, got[0], world)
    dist.barrier()
    q.put((rank, got, val))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_reduce_max_and_value(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, val in res:
        assert got == [10.0 + world - 1, 5.0 * world, 1.0]
        assert val == pytest.approx(world * 1000.0 / ((10.0 + world - 1) * 1e-3))


def test_single_rank_needs_no_collective():
    import bench
    assert bench.reduce_max([1.0, 2.0], 1, "cpu") == [1.0, 2.0]
    assert bench.whole_job_value(500.0, 2.0, 1) == pytest.approx(250000.0)
