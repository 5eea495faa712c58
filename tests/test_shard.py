"""The sharded cross (A partitioned by rows over P ranks) on CPU ranks.

The driver in paper_2502_11017_gb300.shard strings the per-rank steps together with the
collectives between them; here each rank's steps are done by tests/shard_numpy_ops.py
(FP64 NumPy in the kernels' contract), and the ranks are gloo processes or threads. The
sharded cross must return the single-process oracle's I, J and log-volume: the partition,
the merge tree across ranks, the agreement on each swap (MAXLOC) and the reductions of the
residual change where the work is done, not what is computed. A rank that leaves between
steps makes the others' next collective fail, and they report a timeout status.
"""
import datetime
import math
import os
import socket
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import cur_oracle as orc
from paper_2502_11017_gb300 import shard
from paper_2502_11017_gb300 import workloads as wl

from shard_numpy_ops import NumpyRankOps

R, B_R, B_C = 16, 8, 8


def _lowrank():
    return wl.lowrank_haar(2000, 1500)


def test_slabs_partition_the_blocks():
    for m, nb, P in [(2000, 8, 1), (2000, 8, 2), (2000, 8, 4), (2003, 8, 8), (1501, 6, 3)]:
        bl = orc.balanced_blocks(m, nb)
        cover = []
        for k in range(P):
            s, e = shard.slab(m, nb, P, k)
            per = nb // P
            assert (s, e) == (bl[k * per][0], bl[(k + 1) * per - 1][1])
            # the slab's own balanced blocks are the global blocks it holds
            assert [(a + s, b + s) for a, b in orc.balanced_blocks(e - s, per)] == bl[k * per:(k + 1) * per]
            cover.append((s, e))
        assert cover[0][0] == 0 and cover[-1][1] == m
        assert all(cover[i][1] == cover[i + 1][0] for i in range(P - 1))
    for nb, P in [(8, 3), (12, 4), (6, 4), (8, 0)]:
        with pytest.raises(ValueError):
            shard.check_partition(nb, P)


def _run_threads(a, P, b_r, b_c, r=R):
    m, n = a.shape
    group = shard.ThreadGroup(P, timeout=120)
    out = [None] * P

    def rank(k):
        s, e = shard.slab(m, b_r, P, k)
        ops = NumpyRankOps(a[s:e], r)
        out[k] = shard.cross(group.transport(k), ops, m, n, r, b_r, b_c)

    ths = [threading.Thread(target=rank, args=(k,)) for k in range(P)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    return out


def _same_as_oracle(res, a, r, b_r, b_c):
    Io, Jo, info = orc.cross(a, r, b_r, b_c)
    assert res["status"] == info["status"]
    assert sorted(res["I"]) == sorted(Io) and sorted(res["J"]) == sorted(Jo)
    assert res["J0"] == info["J0"]
    assert res["logvol"] == pytest.approx(info["logvol"], abs=1e-9 * abs(info["logvol"]))
    assert res["sweeps"] == info["sweeps"] and res["sweep_swaps"] == info["sweep_swaps"]
    C, U, Rm, _rc, _p = orc.assemble(a, Io, Jo)
    cheb, fro = orc.residual(a, C, U, Rm)
    assert res["cheb"] == pytest.approx(cheb, rel=1e-9)
    assert res["fro_rel"] == pytest.approx(fro, rel=1e-9)


@pytest.mark.parametrize("P,b_r,b_c", [(1, 8, 8), (2, 8, 8), (4, 8, 8), (3, 6, 3)])
def test_thread_ranks_give_the_oracle_cross(P, b_r, b_c):
    a = _lowrank()
    out = _run_threads(a, P, b_r, b_c)
    for res in out:                      # every rank holds the same cross
        assert res["I"] == out[0]["I"] and res["J"] == out[0]["J"]
    _same_as_oracle(out[0], a, R, b_r, b_c)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_rank(k, P, port, b_r, b_c, leave_after_j0, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=k, world_size=P, timeout=datetime.timedelta(seconds=20))
    try:
        a = _lowrank()
        m, n = a.shape
        s, e = shard.slab(m, b_r, P, k)
        ops = NumpyRankOps(a[s:e], R)
        if leave_after_j0 and k == P - 1:
            # this rank takes part in Algorithm 3 and then leaves before the row selection
            class Leaving(NumpyRankOps):
                def gather_cols(self, J):
                    os._exit(0)
            ops = Leaving(a[s:e], R)
        res = shard.cross(shard.TorchTransport(), ops, m, n, R, b_r, b_c)
        q.put((k, res))
    finally:
        if not leave_after_j0:
            dist.destroy_process_group()


def _run_gloo(P, b_r, b_c, leave_after_j0=False):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_rank, args=(k, P, port, b_r, b_c, leave_after_j0, q)) for k in range(P)]
    for p in procs:
        p.start()
    expect = P - 1 if leave_after_j0 else P
    out = {}
    for _ in range(expect):
        k, res = q.get(timeout=300)
        out[k] = res
    for p in procs:
        p.join(timeout=120)
        if p.is_alive():
            p.kill()
    return out


@pytest.mark.parametrize("P", [2, 4])
def test_gloo_ranks_give_the_oracle_cross(P):
    out = _run_gloo(P, B_R, B_C)
    assert sorted(out) == list(range(P))
    for k in range(P):
        assert out[k]["I"] == out[0]["I"] and out[k]["J"] == out[0]["J"]
    _same_as_oracle(out[0], _lowrank(), R, B_R, B_C)


def test_gloo_rank_leaving_between_steps_gives_timeout_status():
    out = _run_gloo(2, B_R, B_C, leave_after_j0=True)
    assert list(out) == [0]
    assert out[0]["status"] == shard.CUR_ERR_TIMEOUT and "error" in out[0]


class _CountingTransport:
    """A rank's transport that counts the collectives it makes (by operation)."""

    def __init__(self, inner):
        self.inner = inner
        self.calls = []

    def allreduce(self, t, op):
        self.calls.append(("allreduce", op, int(t.numel())))
        return self.inner.allreduce(t, op)

    def send(self, t, dst):
        self.calls.append(("send", dst, int(t.numel())))
        return self.inner.send(t, dst)

    def recv(self, t, src):
        self.calls.append(("recv", src, int(t.numel())))
        return self.inner.recv(t, src)

    def broadcast(self, t, src):
        self.calls.append(("broadcast", src, int(t.numel())))
        return self.inner.broadcast(t, src)


def test_algorithm3_over_slabs_takes_two_allreduces_per_round():
    """J0 over row slabs: one allreduce of the squared norms, then per round an allreduce of
    the pick's r partials (Q^T v and ||v||^2 together) and, before every later round, one of
    the n partials of A^T q: 2 r collectives in all, and the oracle's J0."""
    a = _lowrank()
    m, n = a.shape
    P = 2
    group = shard.ThreadGroup(P, timeout=120)
    out = [None] * P
    cnt = [None] * P

    def rank(k):
        s, e = shard.slab(m, B_R, P, k)
        T = _CountingTransport(group.transport(k))
        out[k] = shard.aca_columns(T, NumpyRankOps(a[s:e], R), m, R)
        cnt[k] = T.calls

    ths = [threading.Thread(target=rank, args=(k,)) for k in range(P)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    for k in range(P):
        calls = cnt[k]
        assert all(c[0] == "allreduce" and c[1] == "sum" for c in calls)
        assert len(calls) == 2 * R
        assert [c[2] for c in calls] == [n] + [R, n] * (R - 1) + [R]
        assert out[k].tolist() == out[0].tolist()
    J0, _ = orc.aca_select(a, 1, R, 1)
    assert out[0].tolist()[:len(J0)] == list(J0)
