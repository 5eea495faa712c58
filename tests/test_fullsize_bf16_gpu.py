"""The mixed-precision workload at full size: A = X diag(exp(-j/20)) Y^T + N(0, 1e-4)
noise, 262144 x 16384 stored as BF16 (8.6 GB), r = 128, 256 row blocks, 16 column blocks,
delta = 1e-2. BF16 data is read as FP32 by every kernel.

The FP64 oracle cannot run Algorithm 3 on this matrix (34 GB as FP64, tens of minutes),
so it checks the GPU's cross from its parts: two-sided (1 + delta)-dominance from A(:,J),
A(I,:) and A(I,J), the reported log-volume, and the residual kernels on sampled rows
against the oracle's residual of the same rows. The row and column stages are compared
with the oracle's directly: both start from the same seeded column set J (C = A(:,J) is
262144 x 128, 268 MB in FP64), and the column stage from the oracle's rows.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2502_11017_gb300 as cur
from paper_2502_11017_gb300 import workloads as wl
from oracle import cur_oracle as orc

pytestmark = pytest.mark.gpu

M, N, R, B_R, B_C, DELTA = 262144, 16384, 128, 256, 16, 1e-2


def test_bf16_rank128_cross_full_size():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cur.load()
    dev = torch.device("cuda:0")
    A = wl.bf16_factor_product(M, N, R, 1e-2, device=dev)
    hd = cur.Handle(M, N, R, cur.CUR_BF16)
    I = torch.empty(R, dtype=torch.int32, device=dev)
    J = torch.empty(R, dtype=torch.int32, device=dev)
    info = torch.zeros(ctypes.sizeof(cur.CurCrossInfo), dtype=torch.uint8, device=dev)
    cur.cur_cross(hd.h, A, R, B_R, B_C, cur.opts(DELTA), I, J, info)
    st = cur.cur_sync_status(hd.h)
    assert st == cur.CUR_OK, cur.cur_status_string(st)
    inf = cur.info_from_tensor(info)
    Il, Jl = I.tolist(), J.tolist()
    assert len(set(Il)) == R and len(set(Jl)) == R
    assert inf.sweeps >= 2 and inf.sweep_swaps[inf.sweeps - 1] == 0
    CJ = A[:, J.long()].float().cpu().numpy().astype(np.float64)
    RI = A[I.long(), :].float().cpu().numpy().astype(np.float64)
    MIJ = CJ[Il, :]
    dr, dc = orc.dominance_parts(CJ, RI, MIJ)
    assert dr <= (1 + DELTA) * (1 + 1e-4) and dc <= (1 + DELTA) * (1 + 1e-4)
    assert inf.logvol == pytest.approx(orc.logvol(MIJ), abs=1e-6 * max(1.0, abs(inf.logvol)))
    # the assembled cross on 256 sampled rows: the library's residual against the oracle's
    C = torch.empty((M, R), dtype=torch.bfloat16, device=dev)
    Rm = torch.empty((R, N), dtype=torch.bfloat16, device=dev)
    U = torch.empty((R, R), dtype=torch.float64, device=dev)
    rc = torch.empty(1, dtype=torch.float64, device=dev)
    cur.cur_assemble(hd.h, A, I, J, R, C, U, Rm, rc)
    rows = torch.from_numpy(np.sort(np.random.default_rng(1).choice(M, 256, replace=False))).to(dev)
    As, Cs = A[rows].contiguous(), C[rows].contiguous()
    cheb = torch.empty(1, dtype=torch.float64, device=dev)
    fro = torch.empty(1, dtype=torch.float64, device=dev)
    cur.cur_residual_cheb(hd.h, As, Cs, U, Rm, R, cheb, fro)
    assert cur.cur_sync_status(hd.h) == cur.CUR_OK
    a_s = As.float().cpu().numpy()
    cheb_o, fro_o = orc.residual(a_s, Cs.float().cpu().numpy(), U.cpu().numpy(), Rm.float().cpu().numpy())
    assert abs(cheb.item() - cheb_o) <= 1e-5 * np.abs(a_s).max()
    assert fro.item() == pytest.approx(fro_o, rel=1e-4)
    # a rank-128 product plus noise of std 1e-2: the cross leaves about the noise
    assert fro_o < 0.05
    hd.close()


def test_bf16_rank128_row_and_column_stages_match_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cur.load()
    dev = torch.device("cuda:0")
    A = wl.bf16_factor_product(M, N, R, 1e-2, device=dev)
    hd = cur.Handle(M, N, R, cur.CUR_BF16)
    Jl = sorted(np.random.default_rng(11021).choice(N, R, replace=False).tolist())
    Jd = torch.tensor(Jl, dtype=torch.int32, device=dev)
    I = torch.empty(R, dtype=torch.int32, device=dev)
    lv = torch.empty(1, dtype=torch.float64, device=dev)
    cur.cur_maxvol_rows(hd.h, A, Jd, R, cur.opts(DELTA, nblocks=B_R), I, lv)
    assert cur.cur_sync_status(hd.h) == cur.CUR_OK
    C = A[:, Jd.long()].float().cpu().numpy().astype(np.float64)
    Io, lvo, _sw, st, _ = orc.maxvol_basis_rows(C, B_R, DELTA)
    assert st == orc.OK
    if sorted(I.tolist()) == sorted(Io):
        assert lv.item() == pytest.approx(lvo, abs=1e-6 * max(1.0, abs(lvo)))
    else:
        assert orc.logvol(C[I.tolist(), :]) >= lvo + np.log(0.999)
    Jc = torch.empty(R, dtype=torch.int32, device=dev)
    Iod = torch.tensor(Io, dtype=torch.int32, device=dev)
    cur.cur_maxvol_cols(hd.h, A, Iod, R, cur.opts(DELTA, nblocks=B_C), Jc, lv)
    assert cur.cur_sync_status(hd.h) == cur.CUR_OK
    Rt = A[Iod.long(), :].float().cpu().numpy().astype(np.float64).T
    Jo, lvc, _sw, st, _ = orc.maxvol_basis_rows(Rt, B_C, DELTA)
    assert st == orc.OK
    if sorted(Jc.tolist()) == sorted(Jo):
        assert lv.item() == pytest.approx(lvc, abs=1e-6 * max(1.0, abs(lvc)))
    else:
        assert orc.logvol(Rt[Jc.tolist(), :]) >= lvc + np.log(0.999)
    hd.close()
