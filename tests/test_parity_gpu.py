"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Index work (picks of Algorithm 3, maxvol sets, merges) must match exactly on
inputs whose decisions are well separated; floating-point outputs match within
the tolerances stated per test (1e-5 of ||A||_C for FP32 residuals).
"""
import ctypes
import math

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
    h = cur.Handle(70000, 9000, 64, cur.CUR_F32)
    yield h.h
    h.close()


def to_dev(a, dev, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(dev)


def sync(h):
    return cur.cur_sync_status(h)


def separated(m, n, seed, dtype=np.float64):
    """Gaussian m x n matrix whose columns carry distinct scales exp(-0.02 k)."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((m, n))
    scale = np.exp(-0.02 * np.arange(n))[rng.permutation(n)]
    return (a * scale[None, :]).astype(dtype)


# ---------------------------------------------------------------- Algorithm 3

@pytest.mark.parametrize("m,n,r,dtype,axis", [
    (3001, 700, 12, np.float64, 1), (3001, 700, 12, np.float32, 1),
    (700, 3001, 12, np.float32, 0), (517, 389, 9, np.float64, 0),
    (257, 1029, 20, np.float32, 1), (64, 33, 1, np.float32, 1)])
def test_aca_select_matches_oracle(dev, handle, m, n, r, dtype, axis):
    # separated norms along the selected axis
    a = separated(m, n, seed=m + n) if axis == 1 else separated(n, m, seed=m + n).T.copy()
    a = a.astype(dtype)
    ref, st = orc.aca_select(a, axis, r, 3)
    A = to_dev(a, dev)
    idx = torch.full((r,), -7, dtype=torch.int32, device=dev)
    cur.cur_aca_select(handle, A, axis, r, 3, idx)
    assert sync(handle) == cur.CUR_OK
    assert idx.cpu().tolist() == ref


def test_aca_select_on_lowrank_haar(dev, handle):
    a = wl.lowrank_haar()
    ref, _ = orc.aca_select(a, 1, 16, 8)
    idx = torch.empty(16, dtype=torch.int32, device=dev)
    cur.cur_aca_select(handle, to_dev(a, dev), 1, 16, 8, idx)
    assert sync(handle) == cur.CUR_OK
    assert idx.cpu().tolist() == ref


def test_aca_select_rank_deficient_warns(dev, handle):
    rng = np.random.default_rng(3)
    a = rng.standard_normal((400, 4)) @ rng.standard_normal((4, 300))
    ref, st = orc.aca_select(a, 1, 7, 2)
    assert st == orc.WARN_RANK and len(ref) == 4
    idx = torch.empty(7, dtype=torch.int32, device=dev)
    cur.cur_aca_select(handle, to_dev(a, dev), 1, 7, 2, idx)
    assert sync(handle) == cur.CUR_WARN_RANK
    got = idx.cpu().tolist()
    assert got[:4] == ref and got[4:] == [-1, -1, -1]


def test_aca_select_bf16(dev, handle):
    a = separated(1500, 600, seed=9, dtype=np.float32)
    t = torch.from_numpy(a).to(torch.bfloat16)
    a_bf = t.to(torch.float32).numpy().astype(np.float64)
    ref, _ = orc.aca_select(a_bf, 1, 10, 1)
    idx = torch.empty(10, dtype=torch.int32, device=dev)
    cur.cur_aca_select(handle, t.to(dev), 1, 10, 1, idx)
    assert sync(handle) == cur.CUR_OK
    assert idx.cpu().tolist() == ref


def test_aca_select_nonfinite(dev, handle):
    a = separated(300, 200, seed=4)
    a[17, 33] = np.nan
    idx = torch.empty(5, dtype=torch.int32, device=dev)
    cur.cur_aca_select(handle, to_dev(a, dev), 1, 5, 1, idx)
    assert sync(handle) == cur.CUR_ERR_NONFINITE


# ---------------------------------------------------------------- maxvol rows / cols / merge

@pytest.mark.parametrize("m,n,r,nb,dtype", [
    (1203, 300, 10, 5, np.float64), (1203, 300, 10, 5, np.float32),
    (2000, 1500, 16, 8, np.float64), (517, 211, 24, 3, np.float32), (90, 40, 1, 4, np.float32)])
def test_maxvol_rows_matches_oracle(dev, handle, m, n, r, nb, dtype):
    a = wl.lowrank_plus_noise(m, n, 0.8 ** np.arange(min(m, n, 60)), 1e-6, seed=m + r)
    a = a.astype(dtype)
    J, _ = orc.aca_select(a, 1, r, 1)
    I_ref, lv_ref, sw_ref, st_ref, _ = orc.maxvol_rows(a, J, nb)
    A = to_dev(a, dev)
    Jd = torch.tensor(J, dtype=torch.int32, device=dev)
    I = torch.empty(r, dtype=torch.int32, device=dev)
    lv = torch.empty(1, dtype=torch.float64, device=dev)
    sw = torch.empty(1, dtype=torch.int32, device=dev)
    cur.cur_maxvol_rows(handle, A, Jd, r, cur.opts(nblocks=nb), I, lv, sw)
    assert sync(handle) == cur.CUR_OK
    assert sorted(I.cpu().tolist()) == sorted(I_ref)
    assert lv.item() == pytest.approx(lv_ref, abs=1e-6 if dtype == np.float32 else 1e-9)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_maxvol_cols_matches_oracle(dev, handle, dtype):
    a = wl.lowrank_plus_noise(400, 1300, 0.75 ** np.arange(60), 1e-6, seed=44).astype(dtype)
    I, _ = orc.aca_select(a, 0, 12, 1)
    J_ref, lv_ref, _sw, _st, _ = orc.maxvol_cols(a, I, 4)
    A = to_dev(a, dev)
    J = torch.empty(12, dtype=torch.int32, device=dev)
    lv = torch.empty(1, dtype=torch.float64, device=dev)
    cur.cur_maxvol_cols(handle, A, torch.tensor(I, dtype=torch.int32, device=dev), 12,
                        cur.opts(nblocks=4), J, lv)
    assert sync(handle) == cur.CUR_OK
    assert sorted(J.cpu().tolist()) == sorted(J_ref)
    assert lv.item() == pytest.approx(lv_ref, abs=1e-6)


@pytest.mark.parametrize("nsets", [2, 3, 5, 8])
def test_merge_level_matches_oracle(dev, handle, nsets):
    r = 6
    rng = np.random.default_rng(50 + nsets)
    c = rng.standard_normal((30 * nsets, r))
    blocks = orc.balanced_blocks(c.shape[0], nsets)
    sets = []
    for (s, e) in blocks:
        S, _ = orc.aca_select(c[s:e], 0, r, 1)
        S, _lv, _sw, _st = orc.maxvol(c[s:e], S)
        sets.append([s + x for x in S])
    # one level of the oracle's tournament
    ref = []
    for t in range(0, nsets - 1, 2):
        U = sets[t] + sets[t + 1]
        S, _lv, _sw, _st = orc.maxvol(c[U], list(range(r)))
        ref.append(sorted(U[x] for x in S))
    if nsets % 2:
        ref.append(sorted(sets[-1]))
    basis = to_dev(c, dev)
    cand = torch.tensor(sets, dtype=torch.int32, device=dev)
    out = torch.empty(((nsets + 1) // 2, r), dtype=torch.int32, device=dev)
    cur.cur_merge(handle, basis, cand, nsets, r, cur.opts(), out)
    assert sync(handle) == cur.CUR_OK
    assert [sorted(x) for x in out.cpu().tolist()] == ref


def test_merge_singular_left_falls_back(dev, handle):
    r = 3
    rng = np.random.default_rng(61)
    c = rng.standard_normal((20, r))
    c[1] = c[0]
    c[2] = 2 * c[0]                      # left set {0,1,2} is singular
    sets = [[0, 1, 2], [10, 11, 12]]
    ref, _ = orc.merge(c, sets)
    out = torch.empty((1, r), dtype=torch.int32, device=dev)
    cur.cur_merge(handle, to_dev(c, dev), torch.tensor(sets, dtype=torch.int32, device=dev), 2, r,
                  cur.opts(), out)
    assert sync(handle) == cur.CUR_OK
    assert sorted(out.cpu().tolist()[0]) == sorted(ref)


# ---------------------------------------------------------------- assemble / residual

@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_assemble_and_residual_match_oracle(dev, handle, dtype):
    a = wl.lowrank_plus_noise(1100, 700, 0.7 ** np.arange(40), 1e-5, seed=70).astype(dtype)
    I, J, _ = orc.cross(a, 14, 3, 2)
    C_ref, U_ref, R_ref, rc_ref, _ = orc.assemble(a, I, J)
    cheb_ref, fro_ref = orc.residual(a, C_ref, U_ref, R_ref)
    A = to_dev(a, dev)
    td = A.dtype
    Id = torch.tensor(I, dtype=torch.int32, device=dev)
    Jd = torch.tensor(J, dtype=torch.int32, device=dev)
    C = torch.empty((1100, 14), dtype=td, device=dev)
    R = torch.empty((14, 700), dtype=td, device=dev)
    U = torch.empty((14, 14), dtype=torch.float64, device=dev)
    rc = torch.empty(1, dtype=torch.float64, device=dev)
    cur.cur_assemble(handle, A, Id, Jd, 14, C, U, R, rc)
    assert sync(handle) == cur.CUR_OK
    np.testing.assert_array_equal(C.cpu().double().numpy(), C_ref)
    np.testing.assert_array_equal(R.cpu().double().numpy(), R_ref)
    np.testing.assert_allclose(U.cpu().numpy(), U_ref, rtol=1e-9, atol=1e-9 * np.abs(U_ref).max())
    assert rc.item() == pytest.approx(rc_ref, rel=1e-9)
    cheb = torch.empty(1, dtype=torch.float64, device=dev)
    fro = torch.empty(1, dtype=torch.float64, device=dev)
    cur.cur_residual_cheb(handle, A, C, U, R, 14, cheb, fro)
    assert sync(handle) == cur.CUR_OK
    tol = 1e-5 if dtype == np.float32 else 1e-12
    assert abs(cheb.item() - cheb_ref) <= tol * np.abs(a).max()
    assert fro.item() == pytest.approx(fro_ref, rel=1e-3 if dtype == np.float32 else 1e-9)


def test_assemble_pinv_fallback(dev, handle):
    rng = np.random.default_rng(71)
    a = rng.standard_normal((50, 40))
    a[:, 4] = a[:, 2]
    I, J = [0, 1, 5, 9], [2, 4, 7, 11]
    _C, U_ref, _R, _rc, used = orc.assemble(a, I, J)
    assert used
    A = to_dev(a, dev)
    U = torch.empty((4, 4), dtype=torch.float64, device=dev)
    rc = torch.empty(1, dtype=torch.float64, device=dev)
    cur.cur_assemble(handle, A, torch.tensor(I, dtype=torch.int32, device=dev),
                     torch.tensor(J, dtype=torch.int32, device=dev), 4, None, U, None, rc)
    assert sync(handle) == cur.CUR_OK
    np.testing.assert_allclose(U.cpu().numpy(), U_ref, atol=1e-9)


# ---------------------------------------------------------------- whole cross

def test_cross_lowrank_haar_2000x1500_r16(dev, handle):
    """The FP64 workload at full size: identical index sets."""
    a = wl.lowrank_haar()
    I_ref, J_ref, info_ref = orc.cross(a, 16, 8, 8)
    I, J, info = cur.cross(to_dev(a, dev), 16, 8, 8)
    assert sorted(I.cpu().tolist()) == sorted(I_ref)
    assert sorted(J.cpu().tolist()) == sorted(J_ref)
    assert info.logvol == pytest.approx(info_ref["logvol"], abs=1e-9)
    assert info.sweeps == info_ref["sweeps"]


@pytest.mark.parametrize("m,n,r,b_r,b_c", [(4096, 1536, 24, 4, 2), (3001, 1100, 16, 3, 2),
                                           (1024, 640, 8, 8, 4)])
def test_cross_gaussian_kernel_fp32(dev, handle, m, n, r, b_r, b_c):
    a = wl.gaussian_kernel(m, n, seed=1000 + m)
    I_ref, J_ref, info_ref = orc.cross(a, r, b_r, b_c)
    A = to_dev(a, dev)
    I, J, info = cur.cross(A, r, b_r, b_c)
    Ig, Jg = I.cpu().tolist(), J.cpu().tolist()
    a64 = a.astype(np.float64)
    lv_gpu = orc.logvol(a64[np.ix_(Ig, Jg)])
    same = sorted(Ig) == sorted(I_ref) and sorted(Jg) == sorted(J_ref)
    assert same or math.exp(lv_gpu - info_ref["logvol"]) >= 0.999
    C_ref, U_ref, R_ref, _, _ = orc.assemble(a, I_ref, J_ref)
    cheb_ref, _ = orc.residual(a, C_ref, U_ref, R_ref)
    C_g, U_g, R_g, _, _ = orc.assemble(a, Ig, Jg)
    cheb_g, _ = orc.residual(a, C_g, U_g, R_g)
    assert same or abs(cheb_g - cheb_ref) <= 1e-5 * np.abs(a).max()
    rows, cols = orc.dominance(a, Ig, Jg)
    assert rows <= 1.01 + 1e-4 and cols <= 1.01 + 1e-4


def test_cross_rejects_bad_arguments(dev, handle):
    a = torch.ones((50, 40), dtype=torch.float32, device=dev)
    I = torch.empty(8, dtype=torch.int32, device=dev)
    J = torch.empty(8, dtype=torch.int32, device=dev)
    with pytest.raises(cur.CurError):
        cur.cur_cross(handle, a, 8, 8, 1, cur.opts(), I, J)     # 50 / 8 < 8 rows per block
    with pytest.raises(cur.CurError):
        cur.cur_cross(handle, a, 40, 1, 1, cur.opts(), I, J)    # r >= min(m, n)


def test_cross_nonfinite(dev, handle):
    a = wl.gaussian_kernel(600, 300, seed=5)
    a[10, 10] = np.inf
    A = to_dev(a, dev)
    I = torch.empty(8, dtype=torch.int32, device=dev)
    J = torch.empty(8, dtype=torch.int32, device=dev)
    # the call only enqueues; the device status word carries the error, and the stages after
    # Algorithm 3 do nothing (the index sets stay inside the matrix)
    cur.cur_cross(handle, A, 8, 2, 2, cur.opts(), I, J)
    assert sync(handle) == cur.CUR_ERR_NONFINITE
    assert 0 <= min(I.tolist()) and max(I.tolist()) < 600 and 0 <= min(J.tolist()) and max(J.tolist()) < 300


@pytest.mark.parametrize("m,n,r,tc", [(1000, 700, 32, True), (1000, 700, 64, True), (300, 2052, 64, True),
                                      (129, 132, 32, True), (300, 2050, 64, False), (129, 129, 32, False)])
def test_residual_tensor_core_path_matches_oracle(dev, handle, m, n, r, tc):
    """FP32 data with r = 32 or 64 and a row pitch of whole 16-byte units runs the tcgen05
    residual (3xTF32, A staged by TMA); other pitches run the CUDA-core kernel. Either is
    3 launches. Tiles are ragged in both directions."""
    a = wl.lowrank_plus_noise(m, n, 0.9 ** np.arange(min(m, n) - 1), 1e-3, seed=m + n + r).astype(np.float32)
    J, _ = orc.aca_select(a, 1, r, 1)
    I, _ = orc.aca_select(a[:, J], 0, r, 1)
    C_ref, U_ref, R_ref, _, _ = orc.assemble(a, I, J)
    cheb_ref, fro_ref = orc.residual(a, C_ref, U_ref, R_ref)
    A = to_dev(a, dev)
    C = torch.empty((m, r), dtype=torch.float32, device=dev)
    R = torch.empty((r, n), dtype=torch.float32, device=dev)
    U = torch.empty((r, r), dtype=torch.float64, device=dev)
    rc = torch.empty(1, dtype=torch.float64, device=dev)
    cur.cur_assemble(handle, A, torch.tensor(I, dtype=torch.int32, device=dev),
                     torch.tensor(J, dtype=torch.int32, device=dev), r, C, U, R, rc)
    cheb = torch.empty(1, dtype=torch.float64, device=dev)
    fro = torch.empty(1, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    cur.cur_prof_read(handle)
    cur.cur_residual_cheb(handle, A, C, U, R, r, cheb, fro)
    assert sync(handle) == cur.CUR_OK
    assert cur.cur_prof_read(handle)[2] == 3
    assert abs(cheb.item() - cheb_ref) <= 1e-5 * np.abs(a).max()
    assert fro.item() == pytest.approx(fro_ref, rel=1e-3)


@pytest.mark.parametrize("m,n,r,dtype", [(40, 30, 1, np.float64), (300, 1200, 12, np.float32),
                                         (25, 21, 4, np.float64)])
def test_cross_edge_shapes(dev, handle, m, n, r, dtype):
    """r = 1, a wide matrix, and a matrix barely larger than r (ragged single blocks)."""
    a = wl.lowrank_plus_noise(m, n, 0.7 ** np.arange(min(m, n) - 1), 1e-5, seed=m * n + r).astype(dtype)
    b_r, b_c = max(1, min(4, m // r)), max(1, min(2, n // r))
    I_ref, J_ref, info_ref = orc.cross(a, r, b_r, b_c)
    I, J, info = cur.cross(to_dev(a, dev), r, b_r, b_c)
    Ig, Jg = I.cpu().tolist(), J.cpu().tolist()
    same = sorted(Ig) == sorted(I_ref) and sorted(Jg) == sorted(J_ref)
    lv = orc.logvol(a.astype(np.float64)[np.ix_(Ig, Jg)])
    assert same or math.exp(lv - info_ref["logvol"]) >= 0.999


def test_cross_on_a_strided_view(dev, handle):
    """A with a leading dimension larger than its column count."""
    a = wl.gaussian_kernel(900, 700, seed=91)
    wide = np.zeros((900, 768), dtype=np.float32)
    wide[:, :700] = a
    W = to_dev(wide, dev)
    A = W[:, :700]
    assert A.stride(0) == 768
    I_ref, J_ref, _ = orc.cross(a, 10, 3, 2)
    I, J, _ = cur.cross(A, 10, 3, 2)
    lv = orc.logvol(a.astype(np.float64)[np.ix_(I.cpu().tolist(), J.cpu().tolist())])
    lv_ref = orc.logvol(a.astype(np.float64)[np.ix_(I_ref, J_ref)])
    assert math.exp(lv - lv_ref) >= 0.999


def test_cross_bf16(dev, handle):
    """BF16 data: the oracle reads the same BF16 values widened to FP64."""
    a = wl.gaussian_kernel(1200, 800, seed=93)
    t = torch.from_numpy(a).to(torch.bfloat16)
    a_bf = t.to(torch.float32).numpy()
    I_ref, J_ref, info_ref = orc.cross(a_bf, 12, 3, 2)
    I, J, _ = cur.cross(t.to(dev), 12, 3, 2)
    Ig, Jg = I.cpu().tolist(), J.cpu().tolist()
    lv = orc.logvol(a_bf.astype(np.float64)[np.ix_(Ig, Jg)])
    same = sorted(Ig) == sorted(I_ref) and sorted(Jg) == sorted(J_ref)
    assert same or math.exp(lv - info_ref["logvol"]) >= 0.999


def test_cross_replays_as_one_cuda_graph(dev):
    """cur_cross only enqueues work, so a whole cross (with its data-dependent merge fallbacks
    and sweeps decided on the device) is captured in a CUDA graph; replays give the eager
    call's sets and info."""
    a = wl.gaussian_kernel(3000, 1200, 0.25, seed=31).astype(np.float32)
    A = to_dev(a, dev)
    hd = cur.Handle(3000, 1200, 24, cur.CUR_F32)
    I = torch.empty(24, dtype=torch.int32, device=dev)
    J = torch.empty(24, dtype=torch.int32, device=dev)
    info = torch.zeros(ctypes.sizeof(cur.CurCrossInfo), dtype=torch.uint8, device=dev)
    cur.cur_cross(hd.h, A, 24, 6, 3, cur.opts(), I, J, info)
    assert cur.cur_sync_status(hd.h) == cur.CUR_OK
    ref = (I.clone(), J.clone(), info.clone())
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            cur.cur_cross(hd.h, A, 24, 6, 3, cur.opts(), I, J, info)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        I.fill_(-1)
        J.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(I, ref[0]) and torch.equal(J, ref[1]) and torch.equal(info, ref[2])
        assert cur.cur_sync_status(hd.h) == cur.CUR_OK
    hd.close()
