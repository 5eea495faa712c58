"""Algorithm 1 (ACA with full pivoting, Section 1.3) on the GPU against the oracle.

FP64 data: the GPU runs the elimination in FP64 and must give the oracle's pivot
sequence, pivot values and residual. FP32/BF16 data: the residual is FP32, so picks
whose margin over the runner-up is below the FP32 error of R_k may go either way; the
test requires the oracle's sequence while the oracle's margins are clear, and beyond
that that every GPU pick be a maximum of the residual the oracle computes along the
GPU's own sequence (to the FP32 error), with the final residual matching that replay.
"""
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


def _run(A, r, hd=None):
    m, n = A.shape
    own = hd is None
    if own:
        hd = cur.Handle(m, n, 32, cur.CUR_F64 if A.dtype == torch.float64 else cur.CUR_F32)
    rt = torch.float64 if A.dtype == torch.float64 else torch.float32
    R = torch.empty((m, n), dtype=rt, device=A.device)
    I = torch.empty(r, dtype=torch.int32, device=A.device)
    J = torch.empty(r, dtype=torch.int32, device=A.device)
    piv = torch.empty(r, dtype=torch.float64, device=A.device)
    cur.cur_aca_full(hd.h, A, r, R, I, J, piv)
    st = cur.cur_sync_status(hd.h)
    if own:
        hd.close()
    return st, I.tolist(), J.tolist(), piv.tolist(), R


EPS32 = 2.0 ** -24


def _gaps(a, I, J):
    """Gap between the best and the second-best |R_k| at each oracle step."""
    R = np.array(a, dtype=np.float64)
    out = []
    for i, j in zip(I, J):
        v = np.partition(np.abs(R).ravel(), -2)[-2:]
        out.append(abs(v[1] - v[0]))
        R -= np.outer(R[:, j], R[i, :]) / R[i, j]
        R[i, :] = 0.0
        R[:, j] = 0.0
    return out


def _clear(gaps, amax):
    """Leading steps decided the same way on both sides: step 0 compares the same values
    of A (ties go to the lowest index on both), step k >= 1 needs a gap above twice a
    bound on the FP32 residual's error after k updates, 4 k eps32 max|A|."""
    k = 1
    while k < len(gaps) and gaps[k] > 2 * 4 * k * EPS32 * amax:
        k += 1
    return k


def test_fp64_is_the_oracles_elimination(dev):
    a = wl.lowrank_plus_noise(300, 257, 2.0 ** (-0.5 * np.arange(40)), 1e-6, seed=31)
    st, I, J, piv, R = _run(torch.from_numpy(a).to(dev), 24)
    Io, Jo, po, Ro, sto = orc.aca_full(a, 24)
    assert st == cur.CUR_OK and sto == orc.OK
    assert I == Io and J == Jo
    np.testing.assert_allclose(piv, po, rtol=1e-10)
    np.testing.assert_allclose(R.cpu().numpy(), Ro, atol=1e-12 * np.abs(a).max())


@pytest.mark.parametrize("m,n,r", [(1500, 1203, 32), (2048, 1024, 48)])
def test_fp32_follows_the_oracle_and_stays_valid(dev, m, n, r):
    a32 = wl.gaussian_kernel(m, n, 0.2, seed=77, dtype=np.float32)
    a = a32.astype(np.float64)
    st, I, J, piv, R = _run(torch.from_numpy(a32).to(dev), r)
    assert st == cur.CUR_OK
    Io, Jo, _po, _Ro, _sto = orc.aca_full(a, r)
    amax = np.abs(a).max()
    k = _clear(_gaps(a, Io, Jo), amax)
    assert k >= 4
    assert list(zip(I, J))[:k] == list(zip(Io, Jo))[:k]
    # every GPU pick is a maximum of the residual along the GPU's own sequence
    pr, mx, Rr = orc.aca_full_replay(a, I, J)
    for s in range(r):
        assert abs(pr[s]) >= mx[s] - 1e-5 * amax, s
    np.testing.assert_allclose(piv, pr, rtol=0, atol=1e-5 * amax)
    np.testing.assert_allclose(R.cpu().numpy(), Rr, rtol=0, atol=1e-5 * amax)
    Rg = R.cpu().numpy()
    assert np.all(Rg[I, :] == 0) and np.all(Rg[:, J] == 0)


def test_bf16_reads_the_rounded_values(dev):
    a32 = wl.gaussian_kernel(640, 384, 0.25, seed=5, dtype=np.float32)
    A = torch.from_numpy(a32).to(dev).to(torch.bfloat16)
    a = A.float().cpu().numpy().astype(np.float64)
    st, I, J, piv, R = _run(A, 8)
    assert st == cur.CUR_OK
    Io, Jo, _po, _Ro, _ = orc.aca_full(a, 8)
    amax = np.abs(a).max()
    k = _clear(_gaps(a, Io, Jo), amax)
    assert list(zip(I, J))[:k] == list(zip(Io, Jo))[:k]
    pr, mx, _Rr = orc.aca_full_replay(a, I, J)
    assert all(abs(p) >= x - 1e-5 * amax for p, x in zip(pr, mx))


def test_rank_deficient_stops_with_warning(dev):
    rng = np.random.default_rng(2)
    a = rng.standard_normal((200, 5)) @ rng.standard_normal((5, 150))
    st, I, J, piv, R = _run(torch.from_numpy(a).to(dev), 9)
    Io, Jo, _po, _Ro, sto = orc.aca_full(a, 9)
    assert st == cur.CUR_WARN_RANK and sto == orc.WARN_RANK
    assert I[:5] == Io and J[:5] == Jo and I[5:] == [-1] * 4 and J[5:] == [-1] * 4


def test_full_rank_square_and_strided_view(dev):
    a = np.random.default_rng(4).standard_normal((64, 80))
    A = torch.from_numpy(a).to(dev)[:, :64]          # ld = 80 > n = 64
    st, I, J, piv, R = _run(A, 64)
    Io, Jo, po, Ro, sto = orc.aca_full(a[:, :64], 64)
    assert st == cur.CUR_OK and I == Io and J == Jo
    np.testing.assert_allclose(piv, po, rtol=1e-9)


def test_bad_arguments_and_nonfinite(dev):
    a = torch.ones((16, 8), dtype=torch.float32, device=dev)
    hd = cur.Handle(16, 8, 8, cur.CUR_F32)
    R = torch.empty((16, 8), dtype=torch.float32, device=dev)
    I = torch.empty(9, dtype=torch.int32, device=dev)
    with pytest.raises(cur.CurError):
        cur.cur_aca_full(hd.h, a, 9, R, I, I)             # r > min(m, n)
    a[3, 2] = float("nan")
    cur.cur_aca_full(hd.h, a, 2, R, I, I)
    assert cur.cur_sync_status(hd.h) == cur.CUR_ERR_NONFINITE
    hd.close()


def test_full_size_residual_is_the_schur_complement_on_sampled_rows(dev):
    # 65536 x 8192 FP32 Gaussian kernel, r = 64: R_r(i,:) = A(i,:) - A(i,J) A(I,J)^-1 A(I,:)
    m, n, r = 65536, 8192, 64
    a32 = wl.gaussian_kernel(m, n, 0.2, seed=11019, dtype=np.float32, chunk_rows=4096)
    st, I, J, piv, R = _run(torch.from_numpy(a32).to(dev), r)
    assert st == cur.CUR_OK and len(set(I)) == r and len(set(J)) == r
    rows = np.random.default_rng(0).choice(m, 48, replace=False)
    a_IJ = a32[np.ix_(I, J)].astype(np.float64)
    X = np.linalg.solve(a_IJ, a32[I, :].astype(np.float64))
    ref = a32[rows, :].astype(np.float64) - a32[np.ix_(rows, J)].astype(np.float64) @ X
    got = R[torch.from_numpy(rows).to(dev)].cpu().numpy().astype(np.float64)
    amax = np.abs(a32).max()
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-4 * amax)
    # complete pivoting: |R_{k+1}| <= 2 max|R_k| = 2 |pivot_k| entrywise
    assert np.abs(got).max() <= 2 * abs(piv[-1]) + 1e-4 * amax
