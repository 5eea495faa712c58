"""The sharded cross with its per-rank steps in libcur's kernels, ranks as threads on one GPU.

Each rank holds its row slab of A on the GPU and calls the cur_shard_* / cur_dmv_* /
cur_merge_pair entry points through the C ABI; the ranks agree through a host transport
(shard.ThreadGroup: reductions in rank order on the host). No kernel waits on another
rank's kernel: every exchange is a host collective between launches. The result must be
the single-process oracle's cross: identical sorted sets and log-volume on the FP64
low-rank workload (2000 x 1500, r = 16), and identical sets or a volume ratio of at
least 0.999 with the Chebyshev residual within 1e-5 of ||A||_C on an FP32 Gaussian-kernel
matrix.
"""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2502_11017_gb300 as cur
from paper_2502_11017_gb300 import shard
from paper_2502_11017_gb300 import workloads as wl
from oracle import cur_oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cur.load()
    return torch.device("cuda:0")


def _run(a, P, r, b_r, b_c, dev):
    m, n = a.shape
    group = shard.ThreadGroup(P, timeout=300)
    out, errs = [None] * P, []

    def rank(k):
        try:
            s, e = shard.slab(m, b_r, P, k)
            A_k = torch.from_numpy(np.ascontiguousarray(a[s:e])).to(dev)
            ops = shard.CudaRankOps(A_k, r, workspace_rows=max(m, n))
            out[k] = shard.cross(group.transport(k), ops, m, n, r, b_r, b_c)
            ops.close()
        except Exception as ex:          # reported by the main thread
            errs.append(ex)
            group._bar.abort()

    ths = [threading.Thread(target=rank, args=(k,)) for k in range(P)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    if errs:
        raise errs[0]
    for res in out:
        assert res["I"] == out[0]["I"] and res["J"] == out[0]["J"]
    return out[0]


@pytest.mark.parametrize("P", [1, 2, 4])
def test_sharded_lowrank_fp64_is_the_oracle_cross(dev, P):
    a = wl.lowrank_haar(2000, 1500)
    res = _run(a, P, 16, 8, 8, dev)
    Io, Jo, info = orc.cross(a, 16, 8, 8)
    assert res["status"] == info["status"] == cur.CUR_OK
    assert res["J0"] == info["J0"]
    assert sorted(res["I"]) == sorted(Io) and sorted(res["J"]) == sorted(Jo)
    assert res["logvol"] == pytest.approx(info["logvol"], abs=1e-9 * abs(info["logvol"]))
    C, U, Rm, _rc, _p = orc.assemble(a, Io, Jo)
    cheb, fro = orc.residual(a, C, U, Rm)
    assert res["cheb"] == pytest.approx(cheb, rel=1e-9, abs=1e-12)
    assert res["fro_rel"] == pytest.approx(fro, rel=1e-9)


@pytest.mark.parametrize("P", [1, 2, 4])
def test_sharded_gaussian_kernel_fp32_matches_oracle(dev, P):
    a = wl.gaussian_kernel(8192, 2048, 0.3, seed=515)
    r, b_r, b_c = 32, 8, 4
    res = _run(a, P, r, b_r, b_c, dev)
    Io, Jo, info = orc.cross(a, r, b_r, b_c)
    assert res["status"] == cur.CUR_OK
    I, J = res["I"], res["J"]
    lv = orc.logvol(a.astype(np.float64)[np.ix_(I, J)])
    if not (sorted(I) == sorted(Io) and sorted(J) == sorted(Jo)):
        assert lv >= info["logvol"] + np.log(0.999)
    assert res["logvol"] == pytest.approx(lv, abs=1e-6 * max(1.0, abs(lv)))
    dr, dc = orc.dominance(a, I, J)
    assert dr <= 1.01 * (1 + 1e-4) and dc <= 1.01 * (1 + 1e-4)
    C, U, Rm, _rc, _p = orc.assemble(a, I, J)
    cheb, fro = orc.residual(a, C, U, Rm)
    assert abs(res["cheb"] - cheb) <= 1e-5 * np.abs(a).max()
    assert res["fro_rel"] == pytest.approx(fro, rel=1e-3)
