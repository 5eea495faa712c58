"""Parity at full size, in the launch configuration the benchmark times: the 65536 x 8192
FP32 Gaussian-kernel matrix (h = 0.2, seed 11019), r = 64, 64 row blocks, 8 column
blocks, delta = 1e-2.

The whole FP64 oracle cross takes minutes, so it is stored: tests/golden/fullsize_crosses.json
is written by tests/golden/make_fullsize_crosses.py, which calls only the oracle and the
seeded generator. The GPU cross must give the oracle's sets (sorted) or a volume ratio of
at least 0.999 against the oracle's, and a Chebyshev residual within 1e-5 of ||A||_C of the
oracle's. Live, the oracle also computes what it can in seconds: the first Algorithm 3
picks, and the row and column stages from the same inputs as the GPU's. The cross is
further held to properties that hold at any size, evaluated in FP64 by the oracle on the
GPU's sets: two-sided (1 + delta)-dominance, the reported log-volume, and the Chebyshev
and Frobenius residuals of the assembled cross.
"""
import ctypes
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2502_11017_gb300 as cur
from paper_2502_11017_gb300 import workloads as wl
from oracle import cur_oracle as orc

pytestmark = pytest.mark.gpu

M, N, R, B_R, B_C, DELTA = 65536, 8192, 64, 64, 8, 1e-2


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cur.load()
    dev = torch.device("cuda:0")
    a32 = wl.gaussian_kernel(M, N, 0.2, seed=11019, chunk_rows=4096)
    A = torch.from_numpy(a32).to(dev)
    hd = cur.Handle(M, N, R, cur.CUR_F32)
    yield dev, a32, A, hd
    hd.close()


def _i32(x, dev):
    return torch.tensor(list(x), dtype=torch.int32, device=dev)


def test_algorithm3_first_picks_match_oracle(setup):
    dev, a32, A, hd = setup
    J0 = torch.empty(R, dtype=torch.int32, device=dev)
    cur.cur_aca_select(hd.h, A, 1, R, B_C, J0)
    assert cur.cur_sync_status(hd.h) == cur.CUR_OK
    Jo, st = orc.aca_select(a32, 1, 3, B_C)     # the first k picks do not depend on r
    assert st == orc.OK
    assert J0.tolist()[:3] == Jo


def test_row_and_column_stages_match_oracle(setup):
    """Both stages start from the oracle's inputs: the stored oracle J0 for the rows, the
    oracle's rows for the columns."""
    dev, a32, A, hd = setup
    J0l = _golden("gaussian_kernel_65536x8192_r64")["J0"]
    J0 = _i32(J0l, dev)
    I = torch.empty(R, dtype=torch.int32, device=dev)
    lv = torch.empty(1, dtype=torch.float64, device=dev)
    cur.cur_maxvol_rows(hd.h, A, J0, R, cur.opts(DELTA, nblocks=B_R), I, lv)
    assert cur.cur_sync_status(hd.h) == cur.CUR_OK
    Io, lvo, _sw, st, _ = orc.maxvol_rows(a32, J0l, B_R, DELTA)
    assert st == orc.OK
    if sorted(I.tolist()) == sorted(Io):
        assert lv.item() == pytest.approx(lvo, abs=1e-6 * max(1.0, abs(lvo)))
    else:
        C = a32[:, J0l].astype(np.float64)
        assert orc.logvol(C[I.tolist(), :]) >= lvo + np.log(0.999)
    J = torch.empty(R, dtype=torch.int32, device=dev)
    cur.cur_maxvol_cols(hd.h, A, _i32(Io, dev), R, cur.opts(DELTA, nblocks=B_C), J, lv)
    assert cur.cur_sync_status(hd.h) == cur.CUR_OK
    Jo, lvc, _sw, st, _ = orc.maxvol_cols(a32, Io, B_C, DELTA)
    assert st == orc.OK
    if sorted(J.tolist()) != sorted(Jo):
        Rt = a32[Io, :].astype(np.float64).T
        assert orc.logvol(Rt[J.tolist(), :]) >= lvc + np.log(0.999)


def test_cross_is_dominant_with_its_reported_volume_and_residual(setup):
    dev, a32, A, hd = setup
    I = torch.empty(R, dtype=torch.int32, device=dev)
    J = torch.empty(R, dtype=torch.int32, device=dev)
    info = torch.zeros(ctypes.sizeof(cur.CurCrossInfo), dtype=torch.uint8, device=dev)
    cur.cur_cross(hd.h, A, R, B_R, B_C, cur.opts(DELTA), I, J, info)
    C = torch.empty((M, R), dtype=torch.float32, device=dev)
    Rm = torch.empty((R, N), dtype=torch.float32, device=dev)
    U = torch.empty((R, R), dtype=torch.float64, device=dev)
    rc = torch.empty(1, dtype=torch.float64, device=dev)
    cheb = torch.empty(1, dtype=torch.float64, device=dev)
    fro = torch.empty(1, dtype=torch.float64, device=dev)
    cur.cur_assemble(hd.h, A, I, J, R, C, U, Rm, rc)
    cur.cur_residual_cheb(hd.h, A, C, U, Rm, R, cheb, fro)
    assert cur.cur_sync_status(hd.h) == cur.CUR_OK
    inf = cur.info_from_tensor(info)
    Il, Jl = I.tolist(), J.tolist()
    assert len(set(Il)) == R and len(set(Jl)) == R
    assert inf.sweeps >= 2 and inf.sweep_swaps[inf.sweeps - 1] == 0
    # two-sided dominance of the converged cross (FP32 B decides the swaps: 1e-4 slack)
    dr, dc = orc.dominance(a32, Il, Jl)
    assert dr <= (1 + DELTA) * (1 + 1e-4) and dc <= (1 + DELTA) * (1 + 1e-4)
    assert inf.logvol == pytest.approx(orc.logvol(a32[np.ix_(Il, Jl)].astype(np.float64)), abs=1e-6)
    Co, Uo, Ro, _rc, _p = orc.assemble(a32, Il, Jl)
    cheb_o, fro_o = orc.residual(a32, Co, Uo, Ro)
    assert abs(cheb.item() - cheb_o) <= 1e-5 * np.abs(a32).max()
    assert fro.item() == pytest.approx(fro_o, rel=1e-4)


GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fullsize_crosses.json")


def _golden(name):
    with open(GOLDEN) as f:
        return json.load(f)[name]


def test_algorithm3_columns_match_stored_oracle(setup):
    dev, a32, A, hd = setup
    g = _golden("gaussian_kernel_65536x8192_r64")
    J0 = torch.empty(R, dtype=torch.int32, device=dev)
    cur.cur_aca_select(hd.h, A, 1, R, B_C, J0)
    assert cur.cur_sync_status(hd.h) == cur.CUR_OK
    assert J0.tolist() == g["J0"]


def test_cross_matches_stored_oracle_cross(setup):
    dev, a32, A, hd = setup
    g = _golden("gaussian_kernel_65536x8192_r64")
    assert (g["m"], g["n"], g["r"], g["b_r"], g["b_c"]) == (M, N, R, B_R, B_C)
    I = torch.empty(R, dtype=torch.int32, device=dev)
    J = torch.empty(R, dtype=torch.int32, device=dev)
    info = torch.zeros(ctypes.sizeof(cur.CurCrossInfo), dtype=torch.uint8, device=dev)
    cur.cur_cross(hd.h, A, R, B_R, B_C, cur.opts(DELTA), I, J, info)
    C = torch.empty((M, R), dtype=torch.float32, device=dev)
    Rm = torch.empty((R, N), dtype=torch.float32, device=dev)
    U = torch.empty((R, R), dtype=torch.float64, device=dev)
    rc = torch.empty(1, dtype=torch.float64, device=dev)
    cheb = torch.empty(1, dtype=torch.float64, device=dev)
    fro = torch.empty(1, dtype=torch.float64, device=dev)
    cur.cur_assemble(hd.h, A, I, J, R, C, U, Rm, rc)
    cur.cur_residual_cheb(hd.h, A, C, U, Rm, R, cheb, fro)
    assert cur.cur_sync_status(hd.h) == cur.CUR_OK
    inf = cur.info_from_tensor(info)
    Il, Jl = I.tolist(), J.tolist()
    lv_gpu = orc.logvol(a32[np.ix_(Il, Jl)].astype(np.float64))
    if sorted(Il) == sorted(g["I"]) and sorted(Jl) == sorted(g["J"]):
        assert lv_gpu == pytest.approx(g["logvol"], abs=1e-9 * max(1.0, abs(g["logvol"])))
        assert inf.sweeps == g["sweeps"]
    else:
        assert lv_gpu >= g["logvol"] + np.log(0.999)
    assert abs(cheb.item() - g["cheb"]) <= 1e-5 * g["norm_cheb"]
    assert fro.item() == pytest.approx(g["fro_rel"], rel=1e-3)


def test_lowrank_haar_cross_matches_stored_oracle_cross():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cur.load()
    g = _golden("lowrank_haar_2000x1500_r16")
    a = wl.lowrank_haar(2000, 1500)
    A = torch.from_numpy(a).cuda()
    I, J, inf = cur.cross(A, g["r"], g["b_r"], g["b_c"], g["delta"])
    assert sorted(I.tolist()) == sorted(g["I"]) and sorted(J.tolist()) == sorted(g["J"])
    assert inf.logvol == pytest.approx(g["logvol"], abs=1e-9 * abs(g["logvol"]))
