"""The swap coefficients B = C M^-1 on the tensor cores (3xTF32 tcgen05) against the oracle.

Each entry must lie within 1e-5 of sum_k |C_ik| |M^-1_kj| of the FP64 product: TF32 alone
(10-bit mantissa) would miss that bound by two orders of magnitude, so the test holds the
split into high and low parts to its FP32-level accuracy. Shapes span a ragged last tile,
both supported ranks and the 65536-row basis of the benchmarked workload.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2502_11017_gb300 as cur
from paper_2502_11017_gb300 import workloads as wl
from oracle import cur_oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cur.load()
    h = cur.Handle(65536, 64, 64, cur.CUR_F32)
    yield h
    h.close()


@pytest.mark.parametrize("p,r,seed", [(1000, 32, 1), (1000, 64, 2), (128, 64, 3), (65536, 64, 4), (4100, 32, 5)])
def test_coefficients_match_oracle(hd, p, r, seed):
    a = wl.gaussian_kernel(p, 4 * r, 0.3, seed=seed)
    C64 = a[:, :r].astype(np.float64)
    S, _ = orc.aca_select(C64, 0, r, 1)              # a well-conditioned start, as the engine's
    B_ref, Minv, _lv, sing = orc.coefficients(C64, S)
    assert not sing
    C = torch.from_numpy(np.ascontiguousarray(a[:, :r])).cuda()
    Mi = torch.from_numpy(Minv).cuda()
    B = torch.full((p, r), float("nan"), dtype=torch.float32, device="cuda")
    cur.cur_coef_tf32(hd.h, C, Mi, B)
    assert cur.cur_sync_status(hd.h) == cur.CUR_OK
    bound = np.abs(C64) @ np.abs(Minv)
    err = np.abs(B.cpu().numpy().astype(np.float64) - B_ref)
    assert np.all(err <= 1e-5 * bound + 1e-30), float((err / bound).max())
    # the selected rows give the identity (B(S,:) = I) to the same accuracy
    assert np.abs(B.cpu().numpy()[S] - np.eye(r)).max() <= 1e-5 * bound[S].max()


def test_rejects_other_ranks(hd):
    C = torch.zeros((300, 48), dtype=torch.float32, device="cuda")
    Mi = torch.zeros((48, 48), dtype=torch.float64, device="cuda")
    B = torch.empty((300, 48), dtype=torch.float32, device="cuda")
    with pytest.raises(cur.CurError):
        cur.cur_coef_tf32(hd.h, C, Mi, B)
