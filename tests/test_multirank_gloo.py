"""The N > 1 path of bench.py on CPU: two gloo ranks (one replica each) agree on
the slowest rank's time and report the whole-job throughput."""
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


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = 100.0 + 50.0 * rank     # rank 1 is the slow one
        units = 65536 * 1000
        ms, value = bench.aggregate(ms_local, units, world, "cpu")
        q.put((rank, ms, value))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ms, value in res:
        assert ms == pytest.approx(150.0)                       # max over ranks
        assert value == pytest.approx(world * 65536 * 1000 / 0.150)  # all ranks' units / max time


def test_single_rank_aggregation_is_local():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.aggregate(200.0, 1000.0, 1)
    assert ms == 200.0 and value == pytest.approx(5000.0)
