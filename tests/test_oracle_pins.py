"""Pins of the FP64 oracle against facts fixed outside it (CPU only).

Each test ties one oracle function to something the oracle does not compute
itself: a LAPACK routine that the method reduces to (QR with column pivoting),
exact closed forms (Cauchy determinants of Hilbert submatrices), exhaustive
search on tiny inputs, invariants of the maximal-volume problem, and the error
bounds of Theorems 1 and 2.
"""
from fractions import Fraction
import itertools
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import cur_oracle as orc
from paper_2502_11017_gb300 import workloads as wl


def separated(m, n, seed):
    """Gaussian matrix whose columns carry clearly separated scales."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((m, n))
    return a * (1.5 ** -np.arange(n))[rng.permutation(n)][None, :]


def cauchy_logdet_hilbert(I, J):
    """log|det H(I,J)| for H_ij = 1/(i+j+1) (0-based), by the Cauchy determinant
    formula with x_i = i + 1, y_j = j, evaluated exactly in rationals."""
    num, den = Fraction(1), Fraction(1)
    for a, b in itertools.combinations(range(len(I)), 2):
        num *= (I[b] - I[a]) * (J[b] - J[a])
    for a in range(len(I)):
        for b in range(len(J)):
            den *= (I[a] + J[b] + 1)
    v = abs(num / den)
    return math.log(v.numerator) - math.log(v.denominator)


# ---------------------------------------------------------------- Algorithm 3

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_aca_columns_equal_qr_column_pivoting(seed):
    a = separated(70, 40, seed)
    r = 12
    sel, st = orc.aca_select(a, axis=1, r=r, nblocks=1)
    _q, _r, piv = scipy.linalg.qr(a, pivoting=True, mode="economic")
    assert st == orc.OK
    assert sel == list(piv[:r])


@pytest.mark.parametrize("seed", [3, 4])
def test_aca_rows_equal_qr_column_pivoting_of_transpose(seed):
    a = separated(40, 70, seed).T.copy()          # 70 x 40, separated rows
    r = 10
    sel, st = orc.aca_select(a, axis=0, r=r, nblocks=1)
    _q, _r, piv = scipy.linalg.qr(a.T, pivoting=True, mode="economic")
    assert st == orc.OK
    assert sel == list(piv[:r])


@pytest.mark.parametrize("axis", [0, 1])
def test_aca_independent_of_block_count(axis):
    a = separated(57, 43, 7)
    if axis == 0:
        a = a.T.copy()
    ref, _ = orc.aca_select(a, axis, 9, 1)
    for b in (2, 3, 8):
        got, _ = orc.aca_select(a, axis, 9, b)
        assert got == ref


def test_aca_first_pivot_is_max_norm():
    a = separated(30, 20, 9)
    sel, _ = orc.aca_select(a, 1, 1, 4)
    assert sel == [int(np.argmax((a * a).sum(axis=0)))]
    sel, _ = orc.aca_select(a, 0, 1, 4)
    assert sel == [int(np.argmax((a * a).sum(axis=1)))]


def test_aca_ties_go_to_lowest_index():
    rng = np.random.default_rng(5)
    x = rng.standard_normal(20)
    y = 0.5 * rng.standard_normal(20)
    a = np.stack([y, x, y, x], axis=1)             # columns 1 and 3 tie
    sel, st = orc.aca_select(a, 1, 2, 2)
    assert sel[0] == 1
    assert sel[1] == 0                              # 2 and 3 are dependent
    assert st == orc.OK


def test_aca_rank_deficient_stops_with_warning():
    rng = np.random.default_rng(6)
    a = rng.standard_normal((30, 3)) @ rng.standard_normal((3, 25))
    sel, st = orc.aca_select(a, 1, 5, 3)
    assert st == orc.WARN_RANK
    assert len(sel) == 3
    assert np.linalg.matrix_rank(a[:, sel]) == 3


def test_aca_residual_is_projection():
    """After the r rounds the selected columns span what was removed: the
    volume of the Gram matrix of the selection equals the product of the pivot
    norms (Gram-Schmidt)."""
    a = separated(40, 25, 11)
    sel, _ = orc.aca_select(a, 1, 6, 2)
    q, rr = np.linalg.qr(a[:, sel])
    pivot_norms = []
    for t, j in enumerate(sel):
        proj = a[:, j] - q[:, :t] @ (q[:, :t].T @ a[:, j])
        pivot_norms.append(np.linalg.norm(proj))
    np.testing.assert_allclose(np.abs(np.diag(rr)), pivot_norms, rtol=1e-12)


# ---------------------------------------------------------------- LU, logvol

@pytest.mark.parametrize("r", [1, 3, 8, 17])
def test_lu_matches_lapack(r):
    rng = np.random.default_rng(r)
    m = rng.standard_normal((r, r))
    lu, perm, sing = orc.lu_factor(m)
    lu_ref, piv_ref = scipy.linalg.lu_factor(m)
    assert not sing
    np.testing.assert_allclose(lu, lu_ref, rtol=1e-12, atol=1e-12)
    lower = np.tril(lu, -1) + np.eye(r)
    np.testing.assert_allclose(m[perm], lower @ np.triu(lu), rtol=1e-10, atol=1e-10)
    inv = orc.lu_inverse(lu, perm)
    np.testing.assert_allclose(inv, np.linalg.inv(m), rtol=1e-9, atol=1e-9)


def test_lu_flags_singular():
    rng = np.random.default_rng(1)
    m = rng.standard_normal((6, 6))
    m[:, 4] = m[:, 1] + m[:, 2]
    _lu, _perm, sing = orc.lu_factor(m)
    assert sing


@pytest.mark.parametrize("I,J", [([0, 1, 2], [0, 1, 2]), ([3, 7, 11, 20], [0, 5, 9, 30]),
                                 ([1, 4], [2, 3]), ([0, 10, 20, 30, 40], [1, 2, 3, 4, 5])])
def test_logvol_equals_cauchy_closed_form(I, J):
    h = wl.hilbert(48)
    got = orc.logvol(h[np.ix_(I, J)])
    assert got == pytest.approx(cauchy_logdet_hilbert(I, J), rel=1e-9, abs=1e-9)


# ---------------------------------------------------------------- maxvol

def _swap_gain(cb, S, i, j):
    m = cb[S, :].copy()
    m2 = m.copy()
    m2[j] = cb[i]
    return abs(np.linalg.det(m2)) / abs(np.linalg.det(m))


@pytest.mark.parametrize("seed,p,r", [(0, 10, 2), (1, 12, 3), (2, 9, 3), (3, 11, 1),
                                      (4, 12, 2), (5, 8, 3)])
def test_maxvol_against_bruteforce(seed, p, r):
    rng = np.random.default_rng(seed)
    cb = rng.standard_normal((p, r))
    delta = 1e-2
    start, _ = orc.aca_select(cb, 0, r, 1)
    S, lv, sw, st = orc.maxvol(cb, start, delta)
    assert st == orc.OK
    # (i) no single swap gains more than 1 + delta (determinants, not B)
    for i in set(range(p)) - set(S):
        for j in range(r):
            assert _swap_gain(cb, S, i, j) <= (1 + delta) * (1 + 1e-12)
    # (ii) Hadamard bound against the exhaustive maximum
    _best_s, best = orc.bruteforce_rows(cb, r)
    vol = abs(np.linalg.det(cb[S, :]))
    assert vol >= best / ((1 + delta) * math.sqrt(r)) ** r * (1 - 1e-12)
    # (v) logvol is log|det| of the selected rows
    assert lv == pytest.approx(np.linalg.slogdet(cb[S, :])[1], abs=1e-10)


def test_maxvol_coefficients_identity_on_selected_rows():
    rng = np.random.default_rng(8)
    cb = rng.standard_normal((40, 6))
    S = [3, 9, 17, 22, 30, 38]
    B, Minv, lv, sing = orc.coefficients(cb, S)
    assert not sing
    np.testing.assert_allclose(B[S, :], np.eye(6), atol=1e-12)
    np.testing.assert_allclose(B, np.linalg.solve(cb[S, :].T, cb.T).T, rtol=1e-10, atol=1e-10)


def test_sherman_morrison_equals_recompute():
    rng = np.random.default_rng(9)
    cb = rng.standard_normal((50, 7))
    S = list(range(7))
    B, Minv, lv, _ = orc.coefficients(cb, S)
    i, j = orc.argmax_abs(B)
    assert abs(B[i, j]) > 1.5
    b = orc.sm_swap(B, Minv, i, j)
    S2 = list(S)
    S2[j] = i
    B2, Minv2, lv2, _ = orc.coefficients(cb, S2)
    np.testing.assert_allclose(B, B2, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(Minv, Minv2, rtol=1e-10, atol=1e-10)
    assert lv + math.log(abs(b)) == pytest.approx(lv2, abs=1e-10)


def test_maxvol_finds_planted_rows_from_any_start():
    rng = np.random.default_rng(10)
    cb = rng.standard_normal((30, 3))
    planted = [4, 17, 25]
    cb[planted] *= 1e3
    for start in ([0, 1, 2], [5, 6, 7], [29, 28, 4], [17, 0, 9]):
        S, _lv, _sw, st = orc.maxvol(cb, start)
        assert st == orc.OK
        assert sorted(S) == planted


def test_maxvol_square_and_errors():
    rng = np.random.default_rng(11)
    cb = rng.standard_normal((5, 5))
    S, _lv, sw, st = orc.maxvol(cb, [4, 2, 0, 1, 3])
    assert (sw, st) == (0, orc.OK)
    tall = rng.standard_normal((20, 4))
    tall[7] = tall[3]
    assert orc.maxvol(tall, [3, 7, 1, 2])[3] == orc.ERR_SINGULAR
    assert orc.maxvol(tall, [3, 3, 1, 2])[3] == orc.ERR_ARG
    tall[12] *= 1e3
    assert orc.maxvol(tall, [0, 1, 2, 4], max_swaps=0)[3] == orc.ERR_NOCONV


def test_maxvol_on_hilbert_matches_exhaustive_search():
    h = wl.hilbert(12)[:, :3]
    start, _ = orc.aca_select(h, 0, 3, 1)
    S, lv, _sw, _st = orc.maxvol(h, start, delta=0.0)
    best_s, _best = orc.bruteforce_rows(h, 3)
    assert sorted(S) == best_s
    assert lv == pytest.approx(cauchy_logdet_hilbert(sorted(S), [0, 1, 2]), abs=1e-9)


# ---------------------------------------------------------------- merge

def test_merge_single_set_and_self_merge_are_identity():
    rng = np.random.default_rng(12)
    c = rng.standard_normal((40, 4))
    s = [5, 9, 20, 33]
    assert orc.merge(c, [s])[0] == s
    out, sw = orc.merge(c, [s, s])
    assert out == s and sw == 0


@pytest.mark.parametrize("nsets", [2, 3, 5, 8])
def test_merge_finds_planted_set(nsets):
    rng = np.random.default_rng(13 + nsets)
    p, r = 16 * nsets, 3
    c = rng.standard_normal((p, r))
    planted = [2, p // 2 + 1, p - 3]
    c[planted] *= 1e3
    blocks = orc.balanced_blocks(p, nsets)
    sets = [list(range(s, s + r)) for (s, e) in blocks]
    out, _sw = orc.merge(c, sets)
    # every planted row lives in some set only if it was started there; merge then
    # polish (maxvol on all rows) must recover the planted set
    S, _lv, _sw2, st = orc.maxvol(c, out)
    assert sorted(S) == planted


def test_merge_node_is_dominant_on_union():
    rng = np.random.default_rng(14)
    c = rng.standard_normal((24, 3))
    left, right = [0, 1, 2], [12, 13, 14]
    out, _ = orc.merge(c, [left, right])
    union = left + right
    m = c[out]
    for i in union:
        for j in range(3):
            m2 = m.copy()
            m2[j] = c[i]
            assert abs(np.linalg.det(m2)) <= 1.01 * abs(np.linalg.det(m)) * (1 + 1e-12)


# ---------------------------------------------------------------- rows / cols

def test_block_rows_polish_is_globally_dominant():
    a = wl.lowrank_plus_noise(300, 80, 0.7 ** np.arange(30), 1e-6, seed=15)
    J, _ = orc.aca_select(a, 1, 8, 2)
    I, lv, _sw, st, info = orc.maxvol_rows(a, J, 5)
    assert st == orc.OK
    c = a[:, J]
    coef = np.linalg.solve(c[I].T, c.T).T
    assert np.abs(coef).max() <= 1.01 + 1e-9
    assert lv == pytest.approx(np.linalg.slogdet(c[I])[1], abs=1e-9)
    assert len(info["block_sets"]) == 5


def test_block_rows_rejects_small_blocks():
    a = np.random.default_rng(16).standard_normal((40, 30))
    assert orc.maxvol_rows(a, list(range(8)), 6)[3] == orc.ERR_ARG


def test_cols_are_rows_of_transpose():
    a = wl.lowrank_plus_noise(120, 90, 0.6 ** np.arange(20), 1e-7, seed=17)
    I = [3, 50, 77, 101, 9]
    J1 = orc.maxvol_cols(a, I, 3)[0]
    J2 = orc.maxvol_rows(a.T.copy(), I, 3)[0]
    assert J1 == J2


# ---------------------------------------------------------------- cross

@pytest.mark.parametrize("seed,m,n,r", [(20, 7, 6, 2), (21, 6, 7, 2), (22, 6, 6, 3),
                                        (23, 8, 5, 1)])
def test_theorems_hold_for_bruteforce_maximiser(seed, m, n, r):
    a = np.random.default_rng(seed).standard_normal((m, n))
    I, J, _best = orc.bruteforce_cross(a, r)
    C, U, R, _rc, _p = orc.assemble(a, I, J)
    cheb, _ = orc.residual(a, C, U, R)
    s = np.linalg.svd(a, compute_uv=False)
    assert cheb <= orc.theorem2_bound(s, r) * (1 + 1e-10)
    assert orc.theorem2_bound(s, r) <= orc.theorem1_bound(s, r)


def test_cross_finds_planted_submatrix():
    rng = np.random.default_rng(24)
    a = rng.standard_normal((9, 8)) * 0.1
    a[np.ix_([1, 6], [2, 5])] = np.array([[9.0, 1.0], [-2.0, 8.0]])
    I, J, info = orc.cross(a, 2, 2, 2)
    Ib, Jb, _ = orc.bruteforce_cross(a, 2)
    assert (sorted(I), sorted(J)) == (Ib, Jb)
    assert info["status"] == orc.OK


@pytest.mark.parametrize("seed", [25, 26, 27])
def test_cross_two_sided_dominance_and_sweeps(seed):
    a = wl.lowrank_plus_noise(200, 150, 0.8 ** np.arange(40), 1e-8, seed=seed)
    I, J, info = orc.cross(a, 10, 4, 3)
    assert info["status"] == orc.OK
    M = a[np.ix_(I, J)]
    rows = np.abs(np.linalg.solve(M.T, a[:, J].T)).max()
    cols = np.abs(np.linalg.solve(M, a[I, :])).max()
    assert rows <= 1.01 + 1e-9 and cols <= 1.01 + 1e-9
    assert info["sweep_swaps"][-1] == 0
    assert orc.dominance(a, I, J) == pytest.approx((rows, cols), rel=1e-9)


def test_cross_rank_one_is_rook_pivot():
    a = np.random.default_rng(28).standard_normal((30, 20))
    I, J, _ = orc.cross(a, 1, 3, 2)
    v = abs(a[I[0], J[0]])
    assert v * 1.01 >= np.abs(a[:, J[0]]).max()
    assert v * 1.01 >= np.abs(a[I[0], :]).max()


def test_cross_rejects_bad_input():
    a = np.ones((10, 8))
    assert orc.cross(a, 8, 1, 1)[2]["status"] == orc.ERR_ARG
    a[3, 3] = np.nan
    assert orc.cross(a, 2, 1, 1)[2]["status"] == orc.ERR_NONFINITE


# ---------------------------------------------------------------- assemble / residual

def test_exact_rank_r_reconstruction():
    rng = np.random.default_rng(29)
    a = rng.standard_normal((60, 6)) @ rng.standard_normal((6, 45))
    I, J, _ = orc.cross(a, 6, 2, 2)
    C, U, R, rc, used_pinv = orc.assemble(a, I, J)
    cheb, fro = orc.residual(a, C, U, R)
    assert not used_pinv
    assert cheb <= 1e3 * orc.EPS * np.abs(a).max()
    assert fro <= 1e3 * orc.EPS


def test_residual_vanishes_on_the_cross():
    a = wl.lowrank_plus_noise(70, 50, 0.5 ** np.arange(20), 1e-3, seed=30)
    I, J = [1, 20, 33, 60], [0, 7, 19, 44]
    C, U, R, _rc, _p = orc.assemble(a, I, J)
    e = a - C @ U @ R
    assert np.abs(e[I, :]).max() < 1e-10 and np.abs(e[:, J]).max() < 1e-10
    cheb, fro = orc.residual(a, C, U, R)
    assert cheb == pytest.approx(np.abs(e).max(), rel=1e-12)
    assert fro == pytest.approx(np.linalg.norm(e) / np.linalg.norm(a), rel=1e-10)


def test_jacobi_svd_and_pinv_match_lapack():
    rng = np.random.default_rng(31)
    m = rng.standard_normal((9, 9))
    m[:, 8] = m[:, 0] - 2 * m[:, 3]          # rank 8
    u, s, v = orc.jacobi_svd(m)
    np.testing.assert_allclose(s, np.linalg.svd(m, compute_uv=False), atol=1e-12)
    np.testing.assert_allclose((u * s) @ v.T, m, atol=1e-12)
    np.testing.assert_allclose(orc.pinv(m), np.linalg.pinv(m, rcond=9 * orc.EPS), atol=1e-9)


def test_assemble_falls_back_to_pinv_when_singular():
    rng = np.random.default_rng(32)
    a = rng.standard_normal((12, 10))
    a[:, 4] = a[:, 2]
    C, U, R, rc, used = orc.assemble(a, [0, 1, 5], [2, 4, 7])
    assert used
    np.testing.assert_allclose(U, np.linalg.pinv(a[np.ix_([0, 1, 5], [2, 4, 7])], rcond=3 * orc.EPS),
                               atol=1e-9)


def test_balanced_blocks():
    assert orc.balanced_blocks(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert orc.balanced_blocks(8, 8) == [(k, k + 1) for k in range(8)]


# ---------------------------------------------------------------- Section 3.1 behaviour

def test_hilbert_error_decreases_with_rank():
    """Qualitative only: the paper's Hilbert figure prints no values."""
    h = wl.hilbert(128)
    errs = []
    for r in (2, 4, 6, 8, 10):
        I, J, _ = orc.cross(h, r, 2, 2)
        C, U, R, _rc, _p = orc.assemble(h, I, J)
        errs.append(orc.residual(h, C, U, R)[1])
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-5


def test_cauchy_product_is_recovered_at_its_rank():
    """Qualitative only: near-zero error once r reaches the rank (Section 3.1)."""
    hm = wl.cauchy_product(128, 5)
    I, J, _ = orc.cross(hm, 5, 2, 2)
    C, U, R, _rc, _p = orc.assemble(hm, I, J)
    assert orc.residual(hm, C, U, R)[1] < 1e-6     # cond(A(I,J)) ~ 1e10


# ---------------------------------------------------------------- Algorithm 1 (ACA, full pivoting)

def _gecp_pivots(a):
    """Pivot positions (original row, column) and values of LAPACK's LU with complete
    pivoting (dgetc2), step by step (SciPy returns the interchanges 0-based)."""
    lu, ipiv, jpiv, info = scipy.linalg.lapack.dgetc2(np.array(a, dtype=np.float64, order="F"))
    assert info == 0
    n = a.shape[0]
    rows, cols = list(range(n)), list(range(n))
    out = []
    for k in range(n):
        p, q = ipiv[k], jpiv[k]
        rows[k], rows[p] = rows[p], rows[k]
        cols[k], cols[q] = cols[q], cols[k]
        out.append((rows[k], cols[k], lu[k, k]))
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_aca_full_equals_lapack_complete_pivoting(seed):
    a = np.random.default_rng(seed).standard_normal((12, 12))
    I, J, piv, _R, st = orc.aca_full(a, 8)
    assert st == orc.OK
    ref = _gecp_pivots(a)[:8]
    assert I == [x[0] for x in ref] and J == [x[1] for x in ref]
    np.testing.assert_allclose(piv, [x[2] for x in ref], rtol=1e-12)


def test_aca_full_residual_is_schur_complement():
    # R_k = A - A(:,J) A(I,J)^-1 A(I,:), the k-th Schur complement, at every k
    a = wl.lowrank_plus_noise(40, 30, 2.0 ** -np.arange(8), 1e-6, seed=5)
    for k in (1, 3, 5, 7):
        I, J, _p, R, st = orc.aca_full(a, k)
        assert st == orc.OK
        schur = a - a[:, J] @ np.linalg.solve(a[np.ix_(I, J)], a[I, :])
        np.testing.assert_allclose(R, schur, atol=1e-10 * np.abs(a).max())
        assert np.all(R[I, :] == 0.0) and np.all(R[:, J] == 0.0)


def test_aca_full_first_pivot_and_ties():
    a = np.random.default_rng(3).standard_normal((9, 7))
    I, J, _p, _R, _st = orc.aca_full(a, 1)
    assert (I[0], J[0]) == np.unravel_index(np.argmax(np.abs(a)), a.shape)
    t = np.zeros((5, 5))
    t[3, 1] = t[1, 4] = t[1, 2] = -2.0   # equal magnitudes: smallest row, then column
    I, J, _p, _R, _st = orc.aca_full(t, 1)
    assert (I[0], J[0]) == (1, 2)


def test_aca_full_rank_r_exact_and_early_stop():
    rng = np.random.default_rng(7)
    a = rng.standard_normal((30, 4)) @ rng.standard_normal((4, 25))
    I, J, _p, R, st = orc.aca_full(a, 4)
    assert st == orc.OK and np.abs(R).max() <= 1e-12 * np.abs(a).max()
    I, J, _p, R, st = orc.aca_full(a, 6)
    assert st == orc.WARN_RANK and len(I) == 4


def test_aca_full_replay_reproduces_its_own_run():
    a = np.random.default_rng(11).standard_normal((20, 15))
    I, J, piv, R, _st = orc.aca_full(a, 6)
    piv2, mx, R2 = orc.aca_full_replay(a, I, J)
    assert piv2 == piv and np.array_equal(R, R2)
    assert all(abs(p) == m for p, m in zip(piv, mx))   # each pivot is the step's maximum


def test_cross_batched_is_the_cross_of_each_matrix():
    shapes = [(60, 40, 3, 2, 1), (50, 45, 4, 1, 2)]
    mats = [wl.uneven_batch_matrix(m, n, 7 + t) for t, (m, n, _r, _b, _c) in enumerate(shapes)]
    out = orc.cross_batched(mats, [s[2] for s in shapes], [(s[3], s[4]) for s in shapes])
    for a, (m, n, r, br, bc), (I, J, info) in zip(mats, shapes, out):
        I2, J2, info2 = orc.cross(a, r, br, bc)
        assert I == I2 and J == J2 and info["logvol"] == info2["logvol"]


# ---------------------------------------------------------------- learned proposal parts

def _mlp_params(rng, k=5, hdim=7):
    return (rng.standard_normal((k, hdim)) * 0.5, rng.standard_normal(hdim) * 0.1,
            rng.standard_normal(hdim) * 0.5, 0.3)


def test_mlp_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((9, 5))
    y = (rng.random(9) < 0.4).astype(float)
    W1, b1, w2, b2 = _mlp_params(rng)
    loss, dW1, db1, dw2, db2 = orc.mlp_loss_grad(X, y, W1, b1, w2, b2, pos_weight=3.0)
    f = lambda W1_, b1_, w2_, b2_: orc.mlp_loss_grad(X, y, W1_, b1_, w2_, b2_, pos_weight=3.0)[0]
    h = 1e-6
    for (i, j) in [(0, 0), (2, 5), (4, 6)]:
        E = np.zeros_like(W1); E[i, j] = h
        assert (f(W1 + E, b1, w2, b2) - f(W1 - E, b1, w2, b2)) / (2 * h) == pytest.approx(dW1[i, j], rel=1e-5, abs=1e-9)
    for j in (0, 3):
        e = np.zeros_like(b1); e[j] = h
        assert (f(W1, b1 + e, w2, b2) - f(W1, b1 - e, w2, b2)) / (2 * h) == pytest.approx(db1[j], rel=1e-5, abs=1e-9)
        e = np.zeros_like(w2); e[j] = h
        assert (f(W1, b1, w2 + e, b2) - f(W1, b1, w2 - e, b2)) / (2 * h) == pytest.approx(dw2[j], rel=1e-5, abs=1e-9)
    assert (f(W1, b1, w2, b2 + h) - f(W1, b1, w2, b2 - h)) / (2 * h) == pytest.approx(db2, rel=1e-5)


def test_mlp_loss_closed_form_and_sketch_of_rank_one():
    # zero weights: every score is b2, the loss is log(1 + e^-b2) on positives, log(1 + e^b2) else
    X = np.ones((4, 3))
    y = np.array([1.0, 0.0, 0.0, 1.0])
    z = np.zeros((3, 2))
    loss = orc.mlp_loss_grad(X, y, z, np.zeros(2), np.zeros(2), 0.7)[0]
    assert loss == pytest.approx((2 * math.log1p(math.exp(-0.7)) + 2 * math.log1p(math.exp(0.7))) / 4)
    rng = np.random.default_rng(1)
    u, v = rng.standard_normal(6), rng.standard_normal(5)
    S, T = rng.standard_normal((5, 3)), rng.standard_normal((6, 3))
    Y, Z = orc.sketch(np.outer(u, v), S, T)
    np.testing.assert_allclose(Y, np.outer(u, v @ S), rtol=1e-12)
    np.testing.assert_allclose(Z, np.outer(v, u @ T), rtol=1e-12)


def test_propose_and_cross_from():
    assert orc.propose([0.5, 2.0, 2.0, -1.0, 3.0], 3) == [4, 1, 2]
    a = wl.gaussian_kernel(300, 120, 0.25, seed=3, dtype=np.float64)
    I, J, info = orc.cross(a, 6, 2, 1)
    I2, J2, info2 = orc.cross_from(a, 6, I, J)       # a converged cross stays put
    assert sorted(I2) == sorted(I) and sorted(J2) == sorted(J) and info2["sweep_swaps"] == [0]
    _, _, bad = orc.cross_from(a, 6, [0] * 6, list(range(6)))
    assert bad["status"] == orc.ERR_SINGULAR


def test_adam_first_step_moves_by_lr_and_follows_its_recurrence():
    # step 1 from zero moments: m1/c1 = g and sqrt(m2/c2) = |g|, so each parameter moves
    # by lr * g / (|g| + eps), i.e. by about lr against the sign of its gradient
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    p1, m1, m2 = orc.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    np.testing.assert_allclose(p1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    # a constant gradient keeps m1/c1 = g and m2/c2 = g^2 at every step
    p, a, b = np.zeros(4), np.zeros(4), np.zeros(4)
    for t in range(1, 6):
        p, a, b = orc.adam_step(p, g, a, b, t, lr=0.01)
    np.testing.assert_allclose(p, -5 * 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-10)


# ---------------------------------------------------------------- padding, features, merge chain

def test_pad_indices_takes_the_lowest_unused_by_enumeration():
    """Every short selection of range(6) (every subset, every order, up to length 3) is
    filled up to r with the smallest indices not in it, in increasing order; the given
    prefix is kept as it is and nothing repeats (rank-deficient start, reading 6)."""
    size = 6
    for k in range(0, 4):
        for sel in itertools.permutations(range(size), k):
            for r in range(k, size + 1):
                out = orc.pad_indices(list(sel), size, r)
                unused = [x for x in range(size) if x not in sel]
                assert out == list(sel) + unused[:r - k]
                assert len(set(out)) == len(out) == r


def test_pad_indices_hand_cases():
    assert orc.pad_indices([3, 0, 5], 8, 6) == [3, 0, 5, 1, 2, 4]
    assert orc.pad_indices([0, 1, 2], 8, 5) == [0, 1, 2, 3, 4]      # low indices already held
    assert orc.pad_indices([], 4, 2) == [0, 1]
    assert orc.pad_indices([7, 2], 8, 2) == [7, 2]                    # nothing to add
    assert orc.pad_indices([1], 2, 3) == [1, 0]                       # only `size` indices exist


def test_proposal_features_divide_by_the_largest_row_norm():
    """Closed form: rows (3,4), (0,1), (1,0), (0,0) have norms 5, 1, 1, 0, so every row is
    divided by 5 (one global divisor: a per-row normalisation would give norms 1, 1, 1)."""
    Y = np.array([[0.0, 1.0], [3.0, 4.0], [1.0, 0.0], [0.0, 0.0]])
    F = orc.proposal_features(Y)
    assert np.array_equal(F, Y / 5.0)
    assert np.allclose(np.sqrt((F * F).sum(axis=1)), [0.2, 1.0, 0.2, 0.0], rtol=0, atol=1e-15)
    # invariant to a positive scale of the sketch and equivariant to a row permutation
    rng = np.random.default_rng(5)
    Z = rng.standard_normal((50, 32))
    perm = rng.permutation(50)
    assert np.allclose(orc.proposal_features(7.5 * Z), orc.proposal_features(Z), rtol=1e-14, atol=0)
    assert np.array_equal(orc.proposal_features(Z[perm]), orc.proposal_features(Z)[perm])
    assert np.array_equal(orc.proposal_features(np.zeros((3, 2))), np.zeros((3, 2)))


def _dominant(Cb, S, delta):
    """No single swap of row i (outside S) into position j raises |det Cb(S,:)| by more
    than 1 + delta: enumerated with numpy determinants."""
    base = abs(np.linalg.det(Cb[S, :]))
    for j in range(len(S)):
        for i in range(Cb.shape[0]):
            if i in S:
                continue
            T = list(S)
            T[j] = i
            if abs(np.linalg.det(Cb[T, :])) > (1 + delta) * base * (1 + 1e-12):
                return False
    return True


def test_merge_singular_left_start_goes_to_the_right_set():
    """Left set {(1,0), (1,0)} is singular. The right set {(0.995,0), (0,1)} is dominant in
    the union (|det| 0.995; replacing (0.995,0) by (1,0) gains 1.005 < 1 + delta), so a
    maxvol started there makes no swap and returns it. Algorithm 3 on the union would start
    at {(1,0), (0,1)} instead (first maximum of the norms), so a chain that skipped the
    right start returns a different set."""
    C = np.array([[1.0, 0.0], [1.0, 0.0], [0.995, 0.0], [0.0, 1.0]])
    left, right = [0, 1], [2, 3]
    assert abs(np.linalg.det(C[left])) == 0.0
    assert _dominant(C, right, 1e-2)
    out, swaps = orc.merge(C, [left, right])
    assert out == right and swaps == 0
    aca, _ = orc.aca_select(C, 0, 2, 1)
    assert sorted(aca) == [0, 3]


def test_merge_both_starts_singular_uses_algorithm3_on_the_union():
    """Left {(1,0), (2,0)} and right {(0,1), (0,3)} each have rank 1; their union has rank
    2 and its unique maximal-volume pair is {(2,0), (0,3)} (|det| 6, by enumeration), which
    Algorithm 3 on the union picks (norms 1, 4, 1, 9: first (0,3), then (2,0))."""
    C = np.array([[1.0, 0.0], [2.0, 0.0], [0.0, 1.0], [0.0, 3.0]])
    out, swaps = orc.merge(C, [[0, 1], [2, 3]])
    best, vol = orc.bruteforce_rows(C, 2)
    assert best == [1, 3] and vol == pytest.approx(6.0)
    assert out == [3, 1] and swaps == 0


def test_merge_singular_left_then_right_converges_to_bruteforce_maximum():
    """Singular left start; the right start is not dominant and the swaps lead to the
    union's maximal-volume set (tiny p, enumerated)."""
    rng = np.random.default_rng(11)
    for _ in range(20):
        C = rng.standard_normal((6, 3))
        C[1] = 2.0 * C[0]                      # left set rows 0, 1, 2 is singular
        out, _sw = orc.merge(C, [[0, 1, 2], [3, 4, 5]])
        U = C[[0, 1, 2, 3, 4, 5]]
        assert _dominant(U, out, 1e-2)
        best, vol = orc.bruteforce_rows(U, 3)
        # Hadamard bound for a (1+delta)-dominant set of a 3-column basis
        assert abs(np.linalg.det(U[out])) >= vol / ((1.01 * math.sqrt(3)) ** 3)


def test_merge_union_of_rank_below_r_keeps_the_padded_start():
    """Every row of the union lies on one line: Algorithm 3 stops after one pick, the pad
    adds the lowest unused position, the start stays singular and is returned as is."""
    C = np.array([[1.0, 0.0], [2.0, 0.0], [3.0, 0.0], [4.0, 0.0]])
    out, swaps = orc.merge(C, [[0, 1], [2, 3]])
    assert out == [3, 0] and swaps == 0
