"""Failure handling on the GPU without faulting it: a device wait that runs out reports
CUR_ERR_TIMEOUT and leaves the context usable; host-made bad inputs give their status."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2502_11017_gb300 as cur
from paper_2502_11017_gb300 import workloads as wl
from oracle import cur_oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cur.load()
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def handle(dev):
    h = cur.Handle(4096, 2048, 32, cur.CUR_F32)
    yield h.h
    h.close()


def test_bounded_wait_times_out_and_context_survives(dev, handle):
    cur.cur_selftest_wait_timeout(handle)
    assert cur.cur_sync_status(handle) == cur.CUR_ERR_TIMEOUT
    assert cur.cur_sync_status(handle) == cur.CUR_OK          # read clears it
    a = wl.gaussian_kernel(600, 400, seed=3)
    ref, _ = orc.aca_select(a, 1, 6, 1)
    idx = torch.empty(6, dtype=torch.int32, device=dev)
    cur.cur_aca_select(handle, torch.from_numpy(a).to(dev), 1, 6, 1, idx)
    assert cur.cur_sync_status(handle) == cur.CUR_OK
    assert idx.cpu().tolist() == ref


def test_swap_cap_reports_noconv(dev, handle):
    rng = np.random.default_rng(5)
    c = rng.standard_normal((400, 6))
    c[[17, 111, 250, 390]] *= 50.0                  # the Algorithm 3 start needs swaps
    A = torch.from_numpy(c).to(dev)
    J = torch.arange(6, dtype=torch.int32, device=dev)
    I = torch.empty(6, dtype=torch.int32, device=dev)
    o = cur.opts(nblocks=1, max_swaps=1)
    cur.cur_maxvol_rows(handle, A, J, 6, o, I)
    st = cur.cur_sync_status(handle)
    _i, _lv, sw, st_ref, _ = orc.maxvol_rows(c, list(range(6)), 1, 1e-2)
    s0, _ = orc.aca_select(c, 0, 6, 1)
    needs = orc.maxvol(c, s0, 1e-2)[2]
    if needs > 1:
        assert st == cur.CUR_ERR_NOCONV
    else:
        assert st == cur.CUR_OK


def test_residual_of_nonfinite_data(dev, handle):
    a = wl.gaussian_kernel(300, 200, seed=6).astype(np.float64)
    I, J = [0, 5, 9], [1, 2, 3]
    A = torch.from_numpy(a).to(dev)
    C = torch.empty((300, 3), dtype=torch.float64, device=dev)
    R = torch.empty((3, 200), dtype=torch.float64, device=dev)
    U = torch.empty((3, 3), dtype=torch.float64, device=dev)
    rc = torch.empty(1, dtype=torch.float64, device=dev)
    cur.cur_assemble(handle, A, torch.tensor(I, dtype=torch.int32, device=dev),
                     torch.tensor(J, dtype=torch.int32, device=dev), 3, C, U, R, rc)
    assert cur.cur_sync_status(handle) == cur.CUR_OK
    A[100, 100] = float("nan")
    cheb = torch.empty(1, dtype=torch.float64, device=dev)
    cur.cur_residual_cheb(handle, A, C, U, R, 3, cheb)
    assert cur.cur_sync_status(handle) == cur.CUR_ERR_NONFINITE
    assert np.isnan(cheb.item())


def test_out_of_range_index_is_reported(dev, handle):
    a = torch.ones((100, 80), dtype=torch.float32, device=dev)
    I = torch.tensor([0, 1, 500], dtype=torch.int32, device=dev)     # 500 >= m
    J = torch.tensor([0, 1, 2], dtype=torch.int32, device=dev)
    U = torch.empty((3, 3), dtype=torch.float64, device=dev)
    rc = torch.empty(1, dtype=torch.float64, device=dev)
    cur.cur_assemble(handle, a, I, J, 3, None, U, None, rc)
    assert cur.cur_sync_status(handle) == cur.CUR_ERR_ARG
