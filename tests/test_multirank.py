"""Multi-rank path of bench.py on CPU ranks (gloo, world size 2): the whole-job rate
uses the slowest rank's time and every rank agrees on it."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [120.0, 150.0][rank]
    ms_max, value = bench.aggregate(ms_local, 10, world, None)
    out.put((rank, ms_max, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _rank_id, ms_max, value in res:
        assert ms_max == 150.0
        assert value == pytest.approx(2 * 10 / 0.150)


def test_single_rank_aggregation():
    import bench
    ms_max, value = bench.aggregate(200.0, 5, 1, None)
    assert ms_max == 200.0 and value == pytest.approx(25.0)
