"""FP64 CPU oracle for the scalable binary CUR cross (test infrastructure only).

This module is test infrastructure. Only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the CUDA library never
does, and it never calls the CUDA library. It is written for reading, not speed:
plain NumPy in float64, one step of the method after another, in the paper's
order and notation, with a library matmul as the only borrowed primitive.

What it computes (the paper: "Scalable Binary CUR Low-Rank Approximation
Algorithm", arXiv 2502.11017):

* ``aca_select``: Algorithm 3 (Blockwise Adaptive Cross Approximation), Section
  2.2: r rounds of {squared norm of every row/column of the residual, blockwise
  local maximum, cross-block maximum, pivot vector, blockwise orthogonal rank-1
  projection}.
* ``maxvol``: the maximal-volume swap iteration on a tall basis (Section 1.2,
  Definition 1 and the argmax-volume problem): B = C M^-1, swap while
  max|B_ij| > 1 + delta, Sherman-Morrison updates, refresh every r swaps.
* ``merge``: the binary (pairwise) merge of candidate index sets: a tournament
  tree in which each node runs maxvol on the union of its two children.
* ``maxvol_rows`` / ``maxvol_cols`` / ``cross``: Algorithm 2 with the blockwise
  maxvol refinement: J0 from Algorithm 3 on the columns, then row selection on
  C = A(:,J) and column selection on A(I,:)^T, then global sweeps.
* ``assemble``: C = A(:,J), U = A(I,J)^dagger, R = A(I,:) (Section 1.1).
* ``residual``: Chebyshev norm max|A - CUR| (Theorem 1) and the relative
  Frobenius error ||A - CUR||_F / ||A||_F (Section 3.1).
* ``aca_full``: Algorithm 1 (adaptive cross approximation with full pivoting),
  Section 1.3: r steps of {global argmax |R_k(i,j)|, rank-1 elimination of the
  pivot's row and column}; the paper's sequential baseline.
* ``sketch`` / ``mlp_*`` / ``propose`` / ``cross_from``: the learned proposal's parts
  (sketch features, a 2-layer scoring network with its cross-entropy gradients, top-r
  proposal, maxvol refinement of a proposed cross).
* ``bruteforce_*``: exhaustive maximal-volume search for tiny inputs.

Readings where the paper is silent or ambiguous (Algorithm 3 uses squared norms;
ties go to the lowest index; selected indices are masked; a residual at rounding
level stops the selection early; contiguous balanced blocks; the merge is a
left-first tournament; delta = 1e-2; refresh every r swaps; at most 100 r swaps;
at most 8 sweeps) are listed with the design notes of the repository.

Status codes mirror the C library's ``cur_status`` values.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

OK, ERR_ARG, ERR_SINGULAR, ERR_NONFINITE, ERR_NOCONV = 0, 1, 2, 3, 4
ERR_TIMEOUT, ERR_NOMEM, ERR_CUDA, WARN_RANK = 5, 6, 7, 8

EPS = np.finfo(np.float64).eps


# --------------------------------------------------------------------------
# Blocks
# --------------------------------------------------------------------------

def balanced_blocks(size: int, nblocks: int) -> list[tuple[int, int]]:
    """Contiguous blocks [start, stop); the first ``size mod nblocks`` blocks get
    one extra element (Algorithm 3 divides A into b blocks along one axis)."""
    base, extra = divmod(size, nblocks)
    out, s = [], 0
    for k in range(nblocks):
        e = s + base + (1 if k < extra else 0)
        out.append((s, e))
        s = e
    return out


# --------------------------------------------------------------------------
# Algorithm 3: Blockwise Adaptive Cross Approximation
# --------------------------------------------------------------------------

def aca_select(A, axis: int, r: int, nblocks: int = 1):
    """Algorithm 3 of the paper. Returns (indices in selection order, status).

    axis = 0 selects rows, axis = 1 selects columns. Each round computes the
    squared norm of every unselected row (column) of the residual block by
    block, takes the per-block maximum (strict '>' in ascending index, so the
    lowest index wins a tie), combines the block maxima the same way, takes the
    winning residual vector v, and applies the orthogonal projection
    R_blk <- R_blk - (R_blk v^T / ||v||^2) v   (rows), or
    R_blk <- R_blk - v (v^T R_blk / ||v||^2)   (columns)
    to every block. A round whose best squared norm is at rounding level,
    (max(m,n) eps ||A||_F)^2, ends the selection early with WARN_RANK.
    """
    R = np.array(A, dtype=np.float64, copy=True)
    m, n = R.shape
    size = m if axis == 0 else n
    if not (1 <= r <= size):
        return [], ERR_ARG
    blocks = balanced_blocks(size, nblocks)
    tol = (max(m, n) * EPS * np.linalg.norm(R)) ** 2
    selected: list[int] = []
    mask = np.zeros(size, dtype=bool)
    for _t in range(r):
        max_norm, max_idx = -1.0, -1
        for (s, e) in blocks:
            if e == s:
                continue
            blk = R[s:e, :] if axis == 0 else R[:, s:e]
            nu = (blk * blk).sum(axis=1 if axis == 0 else 0)
            nu = np.where(mask[s:e], -1.0, nu)
            loc = int(np.argmax(nu))          # first maximum: lowest index
            if nu[loc] > max_norm:             # strict: earlier block wins ties
                max_norm, max_idx = float(nu[loc]), s + loc
        if max_idx < 0 or max_norm <= tol:
            return selected, WARN_RANK
        if axis == 0:
            v = R[max_idx, :].copy()
            for (s, e) in blocks:
                coef = (R[s:e, :] @ v) / max_norm
                R[s:e, :] -= np.outer(coef, v)
        else:
            v = R[:, max_idx].copy()
            for (s, e) in blocks:
                coef = (v @ R[:, s:e]) / max_norm
                R[:, s:e] -= np.outer(v, coef)
        selected.append(max_idx)
        mask[max_idx] = True
    return selected, OK


def aca_full(A, r: int):
    """Algorithm 1 (ACA with full pivoting). Returns (I, J, pivots, R, status).

    R_0 = A; step k takes (i, j) = argmax |R_k(i,j)| (first maximum in row-major
    order, i.e. the smallest row, then the smallest column), appends i to I and j to
    J, and eliminates: R_{k+1} = R_k - R_k(:,j) R_k(i,:) / R_k(i,j). Row i and
    column j of R_{k+1} are zero in exact arithmetic and are set to zero. The loop
    runs r steps (the pseudocode's bound m - 1 read as r); a pivot at rounding level,
    |R_k(i,j)| <= max(m,n) eps max|A|, stops it early with WARN_RANK. R is returned
    as the residual after the last step.
    """
    R = np.array(A, dtype=np.float64, copy=True)
    m, n = R.shape
    if not (1 <= r <= min(m, n)):
        return [], [], [], R, ERR_ARG
    tol = max(m, n) * EPS * (np.abs(R).max() if R.size else 0.0)
    I, J, piv = [], [], []
    for _k in range(r):
        flat = int(np.argmax(np.abs(R)))
        i, j = divmod(flat, n)
        p = R[i, j]
        if not abs(p) > tol:
            return I, J, piv, R, WARN_RANK
        R -= np.outer(R[:, j], R[i, :]) / p
        R[i, :] = 0.0
        R[:, j] = 0.0
        I.append(i)
        J.append(j)
        piv.append(float(p))
    return I, J, piv, R, OK


def aca_full_replay(A, I, J):
    """Algorithm 1's elimination along a given pivot sequence (for checking a run whose
    near-tied choices were decided by rounding). Returns (pivot values, max |R_k| before
    each step, R after the last step)."""
    R = np.array(A, dtype=np.float64, copy=True)
    piv, mx = [], []
    for i, j in zip(I, J):
        mx.append(float(np.abs(R).max()))
        p = R[i, j]
        piv.append(float(p))
        R -= np.outer(R[:, j], R[i, :]) / p
        R[i, :] = 0.0
        R[:, j] = 0.0
    return piv, mx, R


def pad_indices(idx, size: int, r: int) -> list[int]:
    """Fill a short selection up to r with the lowest unselected indices."""
    out = list(idx)
    have = set(out)
    k = 0
    while len(out) < r and k < size:
        if k not in have:
            out.append(k)
            have.add(k)
        k += 1
    return out


# --------------------------------------------------------------------------
# Dense r x r kernels written out: LU with partial pivoting, inverse, log|det|
# --------------------------------------------------------------------------

def lu_factor(M):
    """Doolittle LU with partial pivoting, PM = LU. Returns (LU, perm, singular).

    A pivot with |u_kk| <= r eps max|M| marks M as numerically singular.
    """
    a = np.array(M, dtype=np.float64, copy=True)
    r = a.shape[0]
    perm = np.arange(r)
    thresh = r * EPS * (np.abs(a).max() if a.size else 0.0)
    singular = False
    for k in range(r):
        p = k + int(np.argmax(np.abs(a[k:, k])))
        if p != k:
            a[[k, p], :] = a[[p, k], :]
            perm[[k, p]] = perm[[p, k]]
        piv = a[k, k]
        if abs(piv) <= thresh or not np.isfinite(piv):
            singular = True
            if piv == 0.0:
                continue
        a[k + 1:, k] /= piv
        a[k + 1:, k + 1:] -= np.outer(a[k + 1:, k], a[k, k + 1:])
    return a, perm, singular


def lu_logabsdet(lu) -> float:
    d = np.abs(np.diag(lu))
    if np.any(d == 0):
        return -math.inf
    return float(np.log(d).sum())


def lu_inverse(lu, perm):
    """Inverse from PM = LU: solve L Y = P I, then U X = Y, column by column."""
    r = lu.shape[0]
    inv = np.zeros((r, r))
    for c in range(r):
        b = (perm == c).astype(np.float64)      # column c of P (P I)
        y = np.zeros(r)
        for i in range(r):
            y[i] = b[i] - lu[i, :i] @ y[:i]
        x = np.zeros(r)
        for i in range(r - 1, -1, -1):
            x[i] = (y[i] - lu[i, i + 1:] @ x[i + 1:]) / lu[i, i]
        inv[:, c] = x
    return inv


def logvol(M) -> float:
    """log vol(M) = log |det M| (Definition 1), through the LU above."""
    lu, _perm, _sing = lu_factor(M)
    return lu_logabsdet(lu)


# --------------------------------------------------------------------------
# Maximal-volume swap iteration
# --------------------------------------------------------------------------

def coefficients(Cb, S):
    """B = Cb M^-1 with M = Cb(S,:). Returns (B, Minv, logvol, singular)."""
    M = Cb[list(S), :]
    lu, perm, singular = lu_factor(M)
    if singular:
        return None, None, -math.inf, True
    Minv = lu_inverse(lu, perm)
    return Cb @ Minv, Minv, lu_logabsdet(lu), False


def argmax_abs(B):
    """(i, j) of max |B_ij|; ties go to the smallest i, then the smallest j."""
    flat = int(np.argmax(np.abs(B)))            # first maximum in row-major order
    return divmod(flat, B.shape[1])


def sm_swap(B, Minv, i: int, j: int):
    """Row i of the basis replaces position j of the submatrix.

    With b = B_ij and w = B(i,:) - e_j^T (Sherman-Morrison, 1 + w M^-1 e_j = b):
    B <- B - B(:,j) w / b and M^-1 <- M^-1 - M^-1(:,j) w / b. The volume grows by
    the factor |b|.
    """
    b = B[i, j]
    w = B[i, :].copy()
    w[j] -= 1.0
    B -= np.outer(B[:, j], w) / b
    if Minv is not None:
        Minv -= np.outer(Minv[:, j], w) / b
    return b


def maxvol(Cb, S0, delta: float = 1e-2, max_swaps: int | None = None):
    """Maxvol on the tall basis Cb (p x r) from the start rows S0 (length r).

    Returns (S, logvol, swaps, status); S is in submatrix-position order.
    Each cycle refreshes M = Cb(S,:), its inverse and B = Cb M^-1 from scratch,
    then makes at most r swaps: pick (i,j) = argmax|B_ij|, stop if
    |B_ij| <= 1 + delta, else swap with the Sherman-Morrison updates. A cycle
    that starts converged ends the iteration, so the exit B is always fresh.
    """
    Cb = np.asarray(Cb, dtype=np.float64)
    p, r = Cb.shape
    S = [int(s) for s in S0]
    if len(S) != r or len(set(S)) != r or min(S) < 0 or max(S) >= p:
        return S, -math.inf, 0, ERR_ARG
    if max_swaps is None:
        max_swaps = 100 * r
    swaps = 0
    while True:
        B, Minv, lv, singular = coefficients(Cb, S)
        if singular:
            return S, -math.inf, swaps, ERR_SINGULAR
        made = 0
        while made < r:
            i, j = argmax_abs(B)
            if abs(B[i, j]) <= 1.0 + delta:
                break
            if swaps >= max_swaps:
                return S, lv, swaps, ERR_NOCONV
            b = sm_swap(B, Minv, i, j)
            S[j] = i
            lv += math.log(abs(b))
            made += 1
            swaps += 1
        if made == 0:
            return S, lv, swaps, OK


# --------------------------------------------------------------------------
# Binary merge and the row / column selections
# --------------------------------------------------------------------------



def merge(C, sets, delta: float = 1e-2):
    """Binary tournament merge of candidate row sets of the basis C (m x r).

    Level by level, node t merges L[2t] and L[2t+1]: maxvol on the 2r rows
    L[2t] ++ L[2t+1] (left child first) started at the left child. If the left
    start is singular the right child is the start; if both are, Algorithm 3 on
    the union gives the start (and if that is singular too, that start is kept).
    An odd set at the end of a level passes through. Returns (set, swaps).
    """
    C = np.asarray(C, dtype=np.float64)
    level = [list(s) for s in sets]
    swaps = 0
    while len(level) > 1:
        nxt = []
        for t in range(0, len(level) - 1, 2):
            left, right = level[t], level[t + 1]
            r = len(left)
            U = left + right
            Cb = C[U, :]
            S, _lv, sw, st = maxvol(Cb, list(range(r)), delta)
            if st == ERR_SINGULAR:
                S, _lv, sw, st = maxvol(Cb, list(range(r, 2 * r)), delta)
                if st == ERR_SINGULAR:
                    S0, _ = aca_select(Cb, 0, r, 1)
                    S0 = pad_indices(S0, 2 * r, r)
                    S, _lv, sw, st = maxvol(Cb, S0, delta)
                    if st == ERR_SINGULAR:
                        S = S0
            swaps += sw
            nxt.append([U[x] for x in S])
        if len(level) % 2 == 1:
            nxt.append(level[-1])
        level = nxt
    return level[0], swaps


def maxvol_basis_rows(C, nblocks: int, delta: float = 1e-2, polish: bool = True):
    """Row selection on a tall basis C (p x r): blockwise start and maxvol,
    binary merge, then (polish) maxvol over all p rows from the merged set.

    Returns (rows, logvol, swaps, status, info) with rows in position order.
    """
    C = np.asarray(C, dtype=np.float64)
    p, r = C.shape
    blocks = balanced_blocks(p, nblocks)
    if any(e - s < r for (s, e) in blocks):
        return [], -math.inf, 0, ERR_ARG, {}
    sets, swaps, block_swaps = [], 0, []
    for (s, e) in blocks:
        Ck = C[s:e, :]
        S0, _st = aca_select(Ck, 0, r, 1)
        S0 = pad_indices(S0, e - s, r)
        S, _lv, sw, st = maxvol(Ck, S0, delta)
        if st == ERR_SINGULAR:
            S = S0
        swaps += sw
        block_swaps.append(sw)
        sets.append([s + x for x in S])
    merged, msw = merge(C, sets, delta)
    swaps += msw
    info = dict(block_sets=sets, merged=list(merged), block_swaps=block_swaps,
                merge_swaps=msw)
    if not polish:
        lv = logvol(C[merged, :])
        return merged, lv, swaps, OK, info
    S, lv, sw, st = maxvol(C, merged, delta)
    swaps += sw
    info["polish_swaps"] = sw
    if st == ERR_SINGULAR:
        return merged, -math.inf, swaps, st, info
    return S, lv, swaps, st, info


def maxvol_rows(A, J, nblocks: int, delta: float = 1e-2, polish: bool = True):
    """Rows I for the columns J: maxvol_basis_rows on C = A(:,J)."""
    A = np.asarray(A)
    C = np.asarray(A[:, list(J)], dtype=np.float64)
    return maxvol_basis_rows(C, nblocks, delta, polish)


def maxvol_cols(A, I, nblocks: int, delta: float = 1e-2, polish: bool = True):
    """Columns J for the rows I: maxvol_basis_rows on A(I,:)^T."""
    A = np.asarray(A)
    Rt = np.asarray(A[list(I), :], dtype=np.float64).T
    return maxvol_basis_rows(Rt, nblocks, delta, polish)


def cross(A, r: int, b_r: int, b_c: int, delta: float = 1e-2,
          max_sweeps: int = 8, polish: bool = True):
    """The whole cross (Algorithm 2 with blockwise maxvol refinement).

    J0 = Algorithm 3 on the columns of A (padded to r if the residual runs out);
    sweep 1 = {I = maxvol_rows(A, J0), J = maxvol_cols(A, I)}; sweeps 2..8 =
    {global maxvol on A(:,J) from I, global maxvol on A(I,:)^T from J}, ending
    after the first sweep that makes no swap. Returns (I, J, info).
    """
    A = np.asarray(A)
    m, n = A.shape
    if not np.isfinite(np.asarray(A, dtype=np.float64)).all():
        return [], [], dict(status=ERR_NONFINITE)
    if not (1 <= r < min(m, n)):
        return [], [], dict(status=ERR_ARG)
    J0, st0 = aca_select(A, 1, r, b_c)
    J0 = pad_indices(J0, n, r)
    I, _lv, sw_r, st_r, _ = maxvol_rows(A, J0, b_r, delta, polish)
    if st_r == ERR_ARG:
        return [], [], dict(status=ERR_ARG)
    J, _lv, sw_c, st_c, _ = maxvol_cols(A, I, b_c, delta, polish)
    if st_c == ERR_ARG:
        return [], [], dict(status=ERR_ARG)
    sweeps, sweep_swaps = 1, [sw_r + sw_c]
    status = OK if st0 == OK else st0
    for st in (st_r, st_c):
        if st not in (OK,):
            status = st
    while sweeps < max_sweeps:
        sweeps += 1
        I, _lv, s1, st1 = maxvol(np.asarray(A[:, J], dtype=np.float64), I, delta)
        J, lv, s2, st2 = maxvol(np.asarray(A[I, :], dtype=np.float64).T, J, delta)
        sweep_swaps.append(s1 + s2)
        if st1 != OK or st2 != OK:
            status = st1 if st1 != OK else st2
            break
        if s1 + s2 == 0:
            break
    info = dict(status=status, J0=list(J0), sweeps=sweeps, sweep_swaps=sweep_swaps,
                logvol=logvol(np.asarray(A, dtype=np.float64)[np.ix_(I, J)]))
    return list(I), list(J), info


def cross_batched(mats, ranks, blocks, delta: float = 1e-2):
    """The cross of every matrix of a batch, one after another: mats[t] with rank
    ranks[t] and (b_r, b_c) = blocks[t]. Returns a list of (I, J, info)."""
    return [cross(A, r, br, bc, delta) for A, r, (br, bc) in zip(mats, ranks, blocks)]


# --------------------------------------------------------------------------
# Learned proposal: sketch features and a 2-layer scoring network
# --------------------------------------------------------------------------

def sketch(A, S, T):
    """Row features A S (m x k) and column features (T^T A)^T (n x k) for Gaussian test
    matrices S (n x k) and T (m x k)."""
    A = np.asarray(A, dtype=np.float64)
    return A @ np.asarray(S, np.float64), (np.asarray(T, np.float64).T @ A).T


def proposal_features(Y):
    """Features of the rows of a sketch: each row divided by the largest row norm."""
    Y = np.asarray(Y, dtype=np.float64)
    mx = np.sqrt((Y * Y).sum(axis=1)).max()
    return Y / mx if mx > 0 else Y


def mlp_forward(X, W1, b1, w2, b2):
    """Scores s = relu(X W1 + b1) w2 + b2 and the hidden layer H."""
    H = np.maximum(np.asarray(X, np.float64) @ W1 + b1, 0.0)
    return H @ w2 + b2, H


def mlp_loss_grad(X, y, W1, b1, w2, b2, pos_weight: float = 1.0):
    """Mean binary cross-entropy of the scores against labels y (0/1), positives weighted
    by pos_weight, and its gradients (loss, dW1, db1, dw2, db2)."""
    X = np.asarray(X, np.float64)
    y = np.asarray(y, np.float64)
    s, H = mlp_forward(X, W1, b1, w2, b2)
    wt = np.where(y > 0.5, pos_weight, 1.0)
    N = X.shape[0]
    # log(1 + e^-s) for y = 1, log(1 + e^s) for y = 0, in a stable form
    loss = float((wt * (np.logaddexp(0.0, -s) * y + np.logaddexp(0.0, s) * (1.0 - y))).sum() / N)
    ds = wt * (1.0 / (1.0 + np.exp(-s)) - y) / N
    dw2 = H.T @ ds
    db2 = float(ds.sum())
    dH = np.outer(ds, w2) * (H > 0.0)
    dW1 = X.T @ dH
    db1 = dH.sum(axis=0)
    return loss, dW1, db1, dw2, db2


def adam_step(p, g, m1, m2, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam step (Kingma and Ba, 2015): returns the new (p, m1, m2)."""
    m1 = beta1 * np.asarray(m1, np.float64) + (1 - beta1) * np.asarray(g, np.float64)
    m2 = beta2 * np.asarray(m2, np.float64) + (1 - beta2) * np.asarray(g, np.float64) ** 2
    mh = m1 / (1 - beta1 ** t)
    vh = m2 / (1 - beta2 ** t)
    return np.asarray(p, np.float64) - lr * mh / (np.sqrt(vh) + eps), m1, m2


def propose(scores, r: int):
    """The r highest scores (ties: the lowest index), in decreasing score."""
    order = np.lexsort((np.arange(len(scores)), -np.asarray(scores, np.float64)))
    return [int(i) for i in order[:r]]


def cross_from(A, r: int, I0, J0, delta: float = 1e-2, max_sweeps: int = 8):
    """Maxvol refinement of a proposed cross (I0, J0): sweeps of global maxvol on the rows
    of A(:,J), then on the columns of A(I,:), until a sweep makes no swap. Returns
    (I, J, info); status SINGULAR when A(I0,J0) is singular (the caller falls back)."""
    A64 = np.asarray(A, dtype=np.float64)
    I, J = list(I0), list(J0)
    lu, _p, sing = lu_factor(A64[np.ix_(I, J)])
    if sing:
        return I, J, dict(status=ERR_SINGULAR, sweeps=0, sweep_swaps=[], logvol=-math.inf)
    sweeps, sweep_swaps, status = 0, [], OK
    while sweeps < max_sweeps:
        sweeps += 1
        I, _lv, s1, st1 = maxvol(A64[:, J], I, delta)
        J, lv, s2, st2 = maxvol(A64[I, :].T, J, delta)
        sweep_swaps.append(s1 + s2)
        if st1 != OK or st2 != OK:
            status = st1 if st1 != OK else st2
            break
        if s1 + s2 == 0:
            break
    info = dict(status=status, sweeps=sweeps, sweep_swaps=sweep_swaps,
                logvol=logvol(A64[np.ix_(I, J)]))
    return I, J, info


# --------------------------------------------------------------------------
# Assembly and residual
# --------------------------------------------------------------------------

def jacobi_svd(M, tol: float = 1e-15, max_sweeps: int = 80):
    """One-sided (Hestenes) Jacobi SVD, M = U diag(s) V^T, s descending."""
    a = np.array(M, dtype=np.float64, copy=True)
    n = a.shape[1]
    v = np.eye(n)
    for _ in range(max_sweeps):
        rotated = False
        for p in range(n - 1):
            for q in range(p + 1, n):
                alpha = a[:, p] @ a[:, p]
                beta = a[:, q] @ a[:, q]
                gamma = a[:, p] @ a[:, q]
                if gamma == 0.0 or abs(gamma) <= tol * math.sqrt(alpha * beta):
                    continue
                rotated = True
                zeta = (beta - alpha) / (2.0 * gamma)
                t = math.copysign(1.0, zeta) / (abs(zeta) + math.sqrt(1.0 + zeta * zeta))
                c = 1.0 / math.sqrt(1.0 + t * t)
                s = c * t
                ap, aq = a[:, p].copy(), a[:, q].copy()
                a[:, p], a[:, q] = c * ap - s * aq, s * ap + c * aq
                vp, vq = v[:, p].copy(), v[:, q].copy()
                v[:, p], v[:, q] = c * vp - s * vq, s * vp + c * vq
        if not rotated:
            break
    s = np.sqrt((a * a).sum(axis=0))
    order = np.argsort(-s, kind="stable")
    s = s[order]
    a = a[:, order]
    v = v[:, order]
    u = np.zeros_like(a)
    nz = s > 0
    u[:, nz] = a[:, nz] / s[nz]
    return u, s, v


def pinv(M):
    """Moore-Penrose pseudo-inverse through the Jacobi SVD, cutoff r eps s_max."""
    u, s, v = jacobi_svd(M)
    r = M.shape[0]
    cut = r * EPS * (s[0] if s.size else 0.0)
    inv_s = np.where(s > cut, 1.0 / np.where(s > cut, s, 1.0), 0.0)
    return (v * inv_s[None, :]) @ u.T


def assemble(A, I, J, rcond_min: float = 1e-13):
    """C = A(:,J), U = A(I,J)^dagger, R = A(I,:) (Section 1.1).

    U is the LU inverse when rcond = 1/(||M||_1 ||M^-1||_1) >= rcond_min, else
    the Jacobi-SVD pseudo-inverse. Returns (C, U, R, rcond, used_pinv).
    """
    A64 = np.asarray(A, dtype=np.float64)
    I, J = list(I), list(J)
    C = A64[:, J]
    R = A64[I, :]
    M = A64[np.ix_(I, J)]
    lu, perm, singular = lu_factor(M)
    rcond = 0.0
    if not singular:
        Minv = lu_inverse(lu, perm)
        rcond = 1.0 / (np.abs(M).sum(axis=0).max() * np.abs(Minv).sum(axis=0).max())
        if rcond >= rcond_min:
            return C, Minv, R, rcond, False
    return C, pinv(M), R, rcond, True


def residual(A, C, U, R, chunk_rows: int = 4096):
    """(max_ij |A - C (U R)|, ||A - CUR||_F / ||A||_F), in float64, by row chunks."""
    W = np.asarray(U, dtype=np.float64) @ np.asarray(R, dtype=np.float64)
    cheb, num, den = 0.0, 0.0, 0.0
    m = A.shape[0]
    for s in range(0, m, chunk_rows):
        a = np.asarray(A[s:s + chunk_rows], dtype=np.float64)
        e = a - np.asarray(C[s:s + chunk_rows], dtype=np.float64) @ W
        if e.size:
            cheb = max(cheb, float(np.abs(e).max()))
        num += float((e * e).sum())
        den += float((a * a).sum())
    return cheb, (math.sqrt(num / den) if den > 0 else 0.0)


def dominance(A, I, J):
    """(max|A(:,J) A(I,J)^-1|, max|A(I,J)^-1 A(I,:)|): both are <= 1 + delta for a
    cross that maxvol leaves unchanged on both sides."""
    A = np.asarray(A)
    CJ = np.asarray(A[:, list(J)], dtype=np.float64)
    RI = np.asarray(A[list(I), :], dtype=np.float64)
    return dominance_parts(CJ, RI, CJ[list(I), :])


def dominance_parts(CJ, RI, M):
    """dominance() from the parts C = A(:,J), R = A(I,:) and M = A(I,J), for matrices too
    large to convert whole."""
    lu, perm, _ = lu_factor(np.asarray(M, dtype=np.float64))
    Minv = lu_inverse(lu, perm)
    rows = np.abs(np.asarray(CJ, dtype=np.float64) @ Minv).max()
    cols = np.abs(Minv @ np.asarray(RI, dtype=np.float64)).max()
    return float(rows), float(cols)


# --------------------------------------------------------------------------
# Exhaustive search (tiny inputs only)
# --------------------------------------------------------------------------

def bruteforce_rows(Cb, r: int):
    """Row set S (sorted) of maximal |det Cb(S,:)| over all r-subsets."""
    Cb = np.asarray(Cb, dtype=np.float64)
    best, best_s = -math.inf, None
    for S in itertools.combinations(range(Cb.shape[0]), r):
        v = abs(np.linalg.det(Cb[list(S), :]))
        if v > best:
            best, best_s = v, list(S)
    return best_s, best


def bruteforce_cross(A, r: int):
    """(I, J) sorted, of maximal |det A(I,J)| over all r x r submatrices."""
    A = np.asarray(A, dtype=np.float64)
    best, best_ij = -math.inf, None
    for I in itertools.combinations(range(A.shape[0]), r):
        sub = A[list(I), :]
        for J in itertools.combinations(range(A.shape[1]), r):
            v = abs(np.linalg.det(sub[:, list(J)]))
            if v > best:
                best, best_ij = v, (list(I), list(J))
    return best_ij[0], best_ij[1], best


def theorem1_bound(sigma, r: int) -> float:
    """(r+1) sigma_{r+1} (Theorem 1)."""
    return (r + 1) * float(sigma[r])


def theorem2_bound(sigma, r: int) -> float:
    """(r+1) sigma_{r+1} / sqrt(1 + sum_k sigma_{r+1}^2 / sigma_k^2) (Theorem 2)."""
    s = np.asarray(sigma, dtype=np.float64)
    return (r + 1) * float(s[r]) / math.sqrt(1.0 + float(((s[r] / s[:r]) ** 2).sum()))
