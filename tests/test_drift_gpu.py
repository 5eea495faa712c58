"""The drift bound of the kept inverse (FP32 data), against the FP64 oracle.

For FP32/BF16 data the swap engine carries its double-float M^-1 across cycles and
factorises C(S,:) afresh only once the bound D = sum over swaps of kappa_inf(C(S,:)) exceeds
2^18 (CUR_FLAG_REFACTOR_ALWAYS factorises every cycle, as the iteration of Section 1.2 is
stated; the oracle does that in FP64). On a basis with a graded column space (sigma from 1
to 1e-4) the best 16 x 16 submatrices have kappa_inf ~ 6e4, so the first cycle's 16 swaps
take D past 2^18 (to ~1e6) and the engine must refactorise; on a flat spectrum kappa_inf is
~1e2 and it must not. Either way the swaps, the set and the log-volume are the oracle's.
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
        pytest.skip("no GPU")
    return torch.device("cuda:0")


def _run(dev, Cb, r, always):
    p = Cb.shape[0]
    hd = cur.Handle(p, r, r, cur.CUR_F32)
    C = torch.from_numpy(Cb).to(dev)
    S0 = torch.arange(r, dtype=torch.int32, device=dev)
    S = torch.empty(r, dtype=torch.int32, device=dev)
    lv = torch.empty(1, dtype=torch.float64, device=dev)
    sw = torch.zeros(2, dtype=torch.int32, device=dev)
    cur.cur_prof_refactors(hd.h)
    cur.cur_maxvol_global(hd.h, C, S0, r, cur.opts(refactor_always=always), S, lv, sw)
    st = cur.cur_sync_status(hd.h)
    n = cur.cur_prof_refactors(hd.h)
    hd.close()
    return st, S.tolist(), lv.item(), int(sw[0].item()), n


@pytest.mark.parametrize("seed", [9, 1])
def test_drift_bound_refactorises_and_matches_oracle(dev, seed):
    p, r = 1024, 16
    Cb = wl.graded_basis(p, r, 1e-4, seed)
    So, lvo, swo, sto = orc.maxvol(Cb.astype(np.float64), list(range(r)))
    assert sto == orc.OK
    st, S, lv, sw, n = _run(dev, Cb, r, always=False)
    assert st == cur.CUR_OK
    assert S == So and sw == swo
    assert lv == pytest.approx(lvo, abs=1e-9 * max(1.0, abs(lvo)))
    assert n >= 1, "the drift bound must have forced a refactorisation"
    st2, S2, lv2, sw2, n2 = _run(dev, Cb, r, always=True)
    assert st2 == cur.CUR_OK and S2 == So and sw2 == swo
    assert lv2 == pytest.approx(lvo, abs=1e-9 * max(1.0, abs(lvo)))
    assert n2 >= n   # every cycle with swaps refactorises now; the drift bound did so at least once


def test_flat_spectrum_keeps_the_carried_inverse(dev):
    p, r = 1024, 16
    Cb = wl.graded_basis(p, r, 1.0, 0)
    So, lvo, swo, sto = orc.maxvol(Cb.astype(np.float64), list(range(r)))
    st, S, lv, sw, n = _run(dev, Cb, r, always=False)
    assert st == cur.CUR_OK and sto == orc.OK
    assert S == So and sw == swo
    assert lv == pytest.approx(lvo, abs=1e-9 * max(1.0, abs(lvo)))
    assert n == 0
