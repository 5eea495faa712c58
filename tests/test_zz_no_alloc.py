"""The allocation-free residual entry point agrees with cur_residual_cheb and the oracle.

cur_residual_cheb_noalloc serves callers that cannot allocate device memory where
they need the residual (their memory is already handed to a pool of their own, or
they may not trigger cudaMalloc's synchronisation): it takes no handle and keeps its
scratch in an array compiled into the library. Here it is called twice in a row
through the C ABI and must match the handle-based call within the tolerances of the
residual parity tests, and the FP64 oracle's residual of the same C, U, R within
1e-5 of ||A||_C (FP32 and BF16 data) or 1e-12 (FP64 data); a problem too large for
its fixed array is refused up front.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2502_11017_gb300 as cur
from paper_2502_11017_gb300 import workloads as wl
from oracle import cur_oracle as orc

pytestmark = pytest.mark.gpu

CODES = {np.float32: cur.CUR_F32, np.float64: cur.CUR_F64, "bf16": cur.CUR_BF16}


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cur.load()
    return torch.device("cuda:0")


def _matrix(kind, m, n, r, dev):
    """(device A, the same values as an FP64 host array)."""
    if r >= 32:
        a = wl.lowrank_plus_noise(m, n, 2.0 ** (-np.arange(1, 97) / 8.0), 1e-6, seed=78)
    else:
        a = wl.gaussian_kernel(m, n, seed=77).astype(np.float64)
    if kind == "bf16":
        A = torch.from_numpy(a.astype(np.float32)).to(dev).to(torch.bfloat16)
        return A, A.float().cpu().numpy().astype(np.float64)
    A = torch.from_numpy(a.astype(kind)).to(dev)
    return A, A.cpu().numpy().astype(np.float64)


def _cross_parts(A, a64, r, dev, handle):
    I, J, _ = orc.cross(a64, r, 2, 2)
    m, n = a64.shape
    Id = torch.tensor(I, dtype=torch.int32, device=dev)
    Jd = torch.tensor(J, dtype=torch.int32, device=dev)
    C = torch.empty((m, r), dtype=A.dtype, device=dev)
    R = torch.empty((r, n), dtype=A.dtype, device=dev)
    U = torch.empty((r, r), dtype=torch.float64, device=dev)
    rc = torch.empty(1, dtype=torch.float64, device=dev)
    cur.cur_assemble(handle, A, Id, Jd, r, C, U, R, rc)
    return C, U, R


@pytest.mark.parametrize("kind,r,tol", [(np.float32, 12, 1e-5), (np.float64, 12, 1e-12),
                                        ("bf16", 12, 1e-5), (np.float32, 64, 1e-5)])
def test_noalloc_matches_handle_residual_twice(dev, kind, r, tol):
    m, n = 1536, 1100
    A, a64 = _matrix(kind, m, n, r, dev)
    with cur.Handle(m, n, r, CODES[kind]) as hd:
        C, U, R = _cross_parts(A, a64, r, dev, hd.h)
        ref_c = torch.empty(1, dtype=torch.float64, device=dev)
        ref_f = torch.empty(1, dtype=torch.float64, device=dev)
        cur.cur_residual_cheb(hd.h, A, C, U, R, r, ref_c, ref_f)
        assert cur.cur_sync_status(hd.h) == cur.CUR_OK
    amax = float(np.abs(a64).max())
    # the oracle on the same parts (C, R as stored, U as assembled)
    cheb_o, fro_o = orc.residual(a64, C.double().cpu().numpy(), U.cpu().numpy(),
                                 R.double().cpu().numpy())
    for _ in range(2):
        c = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
        f = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
        cur.cur_residual_cheb_noalloc(A, C, U, R, r, c, f)
        torch.cuda.synchronize()
        assert abs(c.item() - ref_c.item()) <= tol * amax
        assert f.item() == pytest.approx(ref_f.item(), rel=1e-3 if kind != np.float64 else 1e-9)
        assert abs(c.item() - cheb_o) <= tol * amax
        assert f.item() == pytest.approx(fro_o, rel=1e-3 if kind != np.float64 else 1e-9, abs=1e-7)


def test_noalloc_refuses_problems_larger_than_its_array(dev):
    m, n, r = 256, 70000, 64            # W alone is 64 * 70000 * 4 bytes > 16 MiB
    A = torch.zeros((m, n), dtype=torch.float32, device=dev)
    C = torch.zeros((m, r), dtype=torch.float32, device=dev)
    R = torch.zeros((r, n), dtype=torch.float32, device=dev)
    U = torch.zeros((r, r), dtype=torch.float64, device=dev)
    c = torch.empty(1, dtype=torch.float64, device=dev)
    with pytest.raises(cur.CurError) as e:
        cur.cur_residual_cheb_noalloc(A, C, U, R, r, c)
    assert e.value.status == cur.CUR_ERR_NOMEM
