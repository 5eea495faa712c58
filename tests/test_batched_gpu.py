"""The batched cross (many matrices of uneven shapes and ranks, every stage shared by the
batch) against the oracle's cross of each matrix, and against the single-matrix path."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2502_11017_gb300 as cur
from paper_2502_11017_gb300 import workloads as wl
from oracle import cur_oracle as orc

pytestmark = pytest.mark.gpu

DELTA = 1e-2


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cur.load()
    return torch.device("cuda:0")


def _pack(mats, dev):
    offs, o = [], 0
    for a in mats:
        offs.append(o)
        o += a.size
    buf = np.concatenate([a.ravel() for a in mats]).astype(np.float32)
    return torch.from_numpy(buf).to(dev), offs


def _run(shapes, mats, dev):
    data, offs = _pack(mats, dev)
    items = cur.batch_items(shapes, offs)
    hd = cur.Handle(1, 1, 1, workspace_bytes=cur.cur_batch_workspace_size(items))
    total = sum(r for (_m, _n, r, _br, _bc) in shapes)
    IJ = torch.full((2 * total,), -7, dtype=torch.int32, device=dev)
    info = torch.zeros(len(shapes) * ctypes.sizeof(cur.CurCrossInfo), dtype=torch.uint8, device=dev)
    cur.cur_cross_batched(hd.h, data, items, cur.opts(DELTA), IJ, info)
    st = cur.cur_sync_status(hd.h)
    hd.close()
    ij = IJ.cpu().numpy()
    raw = info.cpu().numpy().tobytes()
    sz = ctypes.sizeof(cur.CurCrossInfo)
    infos = [cur.CurCrossInfo.from_buffer_copy(raw[t * sz:(t + 1) * sz]) for t in range(len(shapes))]
    out, o = [], 0
    for (_m, _n, r, _br, _bc) in shapes:
        out.append((list(ij[o:o + r]), list(ij[o + r:o + 2 * r])))
        o += 2 * r
    return st, out, infos


def _check_against_oracle(a, r, br, bc, I, J, inf):
    Io, Jo, oi = orc.cross(a, r, br, bc, DELTA)
    if sorted(I) == sorted(Io) and sorted(J) == sorted(Jo):
        return True
    # several crosses are correct: the GPU's must be dominant with the oracle's volume
    dr, dc = orc.dominance(a, I, J)
    assert dr <= (1 + DELTA) * (1 + 1e-4) and dc <= (1 + DELTA) * (1 + 1e-4)
    lv = orc.logvol(np.asarray(a, np.float64)[np.ix_(I, J)])
    assert lv >= oi["logvol"] + np.log(0.999)
    return False


def test_batch_matches_oracle_per_matrix(dev):
    shapes = wl.uneven_batch_shapes(24, m_range=(256, 1300), n_range=(128, 700), r_range=(4, 28))
    mats = [wl.uneven_batch_matrix(m, n, 11020 + 1 + t) for t, (m, n, _r, _br, _bc) in enumerate(shapes)]
    st, out, infos = _run(shapes, mats, dev)
    assert st in (cur.CUR_OK, cur.CUR_WARN_RANK)
    same = 0
    for t, ((m, n, r, br, bc), a, (I, J), inf) in enumerate(zip(shapes, mats, out, infos)):
        assert inf.status in (cur.CUR_OK, cur.CUR_WARN_RANK), t
        assert len(set(I)) == r and len(set(J)) == r and min(I) >= 0 and max(I) < m and max(J) < n
        same += _check_against_oracle(a, r, br, bc, I, J, inf)
        assert inf.logvol == pytest.approx(orc.logvol(a.astype(np.float64)[np.ix_(I, J)]), abs=1e-6)
        assert inf.sweeps >= 2 and inf.sweep_swaps[inf.sweeps - 1] == 0
    assert same >= len(shapes) // 2


def test_batch_of_one_is_the_single_matrix_cross(dev):
    shapes = [(1536, 640, 24, 3, 1)]
    a = wl.uneven_batch_matrix(1536, 640, 99)
    st, out, infos = _run(shapes, [a], dev)
    A = torch.from_numpy(a).to(dev)
    I, J, info = cur.cross(A, 24, 3, 1)
    assert sorted(out[0][0]) == sorted(I.tolist()) and sorted(out[0][1]) == sorted(J.tolist())
    assert infos[0].logvol == pytest.approx(info.logvol, abs=1e-9)
    assert list(infos[0].sweep_swaps) == list(info.sweep_swaps)


def test_batch_rank_deficient_member_warns(dev):
    # small integer factors: the product is exactly rank 3 in FP32 as well
    rng = np.random.default_rng(3)
    low = (rng.integers(-3, 4, (600, 3)) @ rng.integers(-3, 4, (3, 300))).astype(np.float32)
    ok = wl.uneven_batch_matrix(700, 320, 5)
    shapes = [(600, 300, 6, 1, 1), (700, 320, 10, 1, 1)]
    st, out, infos = _run(shapes, [low, ok], dev)
    assert st != cur.CUR_OK
    _Io, _Jo, oi = orc.cross(low, 6, 1, 1, DELTA)
    assert infos[0].aca_selected == 3 and len(oi["J0"]) == 6
    assert infos[0].status == oi["status"] and oi["status"] != orc.OK
    assert infos[1].status == cur.CUR_OK
    _check_against_oracle(ok, 10, 1, 1, out[1][0], out[1][1], infos[1])


def test_batch_rejects_bad_items(dev):
    a = torch.zeros(1000 * 100, dtype=torch.float32, device=dev)
    hd = cur.Handle(1, 1, 1, workspace_bytes=1 << 28)
    IJ = torch.empty(400, dtype=torch.int32, device=dev)
    for bad in ([(1000, 100, 65, 1, 1)], [(1000, 100, 20, 60, 1)], [(5000, 100, 8, 1, 1)]):
        with pytest.raises(cur.CurError):
            cur.cur_cross_batched(hd.h, a, cur.batch_items(bad, [0]), cur.opts(), IJ)
    with pytest.raises(cur.CurError):
        cur.cur_cross_batched(hd.h, a.double(), cur.batch_items([(100, 100, 8, 1, 1)], [0]), cur.opts(), IJ)
    hd.close()


def test_batch_extremes_match_oracle(dev):
    """Members at the batched workload's extremes (m = 4096, n = 1024, r = 64; m = 256,
    n = 128, r = 8; a tall-thin and a short-wide one), against the oracle's cross."""
    shapes = [(4096, 1024, 64, 8, 2), (256, 128, 8, 1, 1), (4096, 128, 40, 8, 1),
              (300, 1024, 64, 1, 2), (4000, 1000, 63, 8, 2)]
    mats = [wl.uneven_batch_matrix(m, n, 12100 + t) for t, (m, n, _r, _br, _bc) in enumerate(shapes)]
    st, out, infos = _run(shapes, mats, dev)
    assert st in (cur.CUR_OK, cur.CUR_WARN_RANK)
    for t, ((m, n, r, br, bc), a, (I, J), inf) in enumerate(zip(shapes, mats, out, infos)):
        assert inf.status in (cur.CUR_OK, cur.CUR_WARN_RANK), t
        assert len(set(I)) == r and len(set(J)) == r and max(I) < m and max(J) < n
        _check_against_oracle(a, r, br, bc, I, J, inf)
        assert inf.logvol == pytest.approx(orc.logvol(a.astype(np.float64)[np.ix_(I, J)]), abs=1e-6)


def test_batch_with_global_memory_coefficients_matches_oracle(dev):
    """A stage with more problems than twice the SM count puts the B of a problem too large
    for one CTA's shared memory in global memory, on one CTA. 330 small members plus three
    of 4096 rows at r = 64 make every polish stage such a stage; the large members and a
    sample of the small ones are checked against the oracle."""
    small = wl.uneven_batch_shapes(330, seed=12200, m_range=(256, 320), n_range=(128, 160),
                                   r_range=(8, 12))
    big = [(4096, 1024, 64, 8, 2), (3900, 900, 60, 8, 2), (4096, 700, 64, 8, 2)]
    shapes = big + small
    mats = [wl.uneven_batch_matrix(m, n, 12300 + t) for t, (m, n, _r, _br, _bc) in enumerate(shapes)]
    st, out, infos = _run(shapes, mats, dev)
    assert st in (cur.CUR_OK, cur.CUR_WARN_RANK)
    check = list(range(len(big))) + list(range(len(big), len(shapes), 37))
    for t in check:
        (m, n, r, br, bc), a, (I, J), inf = shapes[t], mats[t], out[t], infos[t]
        assert inf.status in (cur.CUR_OK, cur.CUR_WARN_RANK), t
        assert len(set(I)) == r and len(set(J)) == r
        _check_against_oracle(a, r, br, bc, I, J, inf)


def test_batch_replays_as_one_cuda_graph(dev):
    """After the first call of its class (which tunes the Algorithm 3 launch shape), the
    batched cross only enqueues work, so the whole batch is captured in one CUDA graph; a
    replay gives the eager call's sets, statuses and log-volumes."""
    shapes = wl.uneven_batch_shapes(40, seed=12400, m_range=(256, 1500), n_range=(128, 700), r_range=(4, 32))
    mats = [wl.uneven_batch_matrix(m, n, 12500 + t) for t, (m, n, _r, _br, _bc) in enumerate(shapes)]
    data, offs = _pack(mats, dev)
    items = cur.batch_items(shapes, offs)
    hd = cur.Handle(1, 1, 1, workspace_bytes=cur.cur_batch_workspace_size(items))
    total = sum(s[2] for s in shapes)
    IJ = torch.full((2 * total,), -7, dtype=torch.int32, device=dev)
    info = torch.zeros(len(shapes) * ctypes.sizeof(cur.CurCrossInfo), dtype=torch.uint8, device=dev)
    cur.cur_cross_batched(hd.h, data, items, cur.opts(DELTA), IJ, info)      # tunes, then runs
    st0 = cur.cur_sync_status(hd.h)
    ref_ij, ref_info = IJ.clone(), info.clone()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            cur.cur_cross_batched(hd.h, data, items, cur.opts(DELTA), IJ, info)
    torch.cuda.current_stream().wait_stream(s)
    IJ.fill_(-7)
    info.zero_()
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(IJ, ref_ij) and torch.equal(info, ref_info)
        assert cur.cur_sync_status(hd.h) == st0
    hd.close()
