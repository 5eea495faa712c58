"""A CPU stand-in for the per-rank kernels of the sharded cross (test infrastructure).

``NumpyRankOps`` has the interface of ``paper_2502_11017_gb300.shard.CudaRankOps`` and does
each step in FP64 NumPy on the rank's slab, so that the sharded driver (the partition, the
merge tree across ranks, the MAXLOC agreement of each swap, the collectives) runs on CPU
ranks under gloo and can be compared with the single-process oracle. The block stage and
the merge node are the oracle's own steps; the slab-local Algorithm 3 and maxvol steps
follow the kernels' contract (include/cur.h) written out plainly.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from oracle import cur_oracle as orc

OK, SINGULAR, WARN_RANK = 0, 2, 8
I64_MAX = np.iinfo(np.int64).max


def _t(x, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dtype)


class NumpyRankOps:
    def __init__(self, A_k: np.ndarray, r: int):
        self.A = _t(A_k)
        self.a = np.asarray(A_k, dtype=np.float64)
        self.r = r
        self.status = OK

    # -- plumbing
    def zeros(self, shape, dtype=None):
        return torch.zeros(shape, dtype=dtype or torch.float64)

    def empty(self, shape, dtype=None):
        return torch.zeros(shape, dtype=dtype or torch.float64)

    def cat(self, xs):
        return torch.cat(xs)

    def item(self, t):
        return t.item()

    def sync_status(self):
        s, self.status = self.status, OK
        return s

    def _warn(self, code):
        if self.status == OK or (self.status == WARN_RANK and code != WARN_RANK):
            self.status = code

    # -- Algorithm 3 on the columns of the slab (implicit residual)
    def aca_begin(self, m_global):
        m, n = self.a.shape
        self.mg = m_global
        self.nu = np.zeros(n)
        self.mask = np.zeros(n, dtype=bool)
        self.Q = []
        self.W = []
        self.stop = False
        self.idx = [-1] * self.r
        self.count = 0
        return _t((self.a * self.a).sum(axis=0))

    def aca_pick(self, t, red):
        red = red.numpy()
        if self.stop:
            return _t(np.zeros(self.r))
        if t == 0:
            self.nu = red.copy()
            self.frob2 = float(red.sum())
        else:
            self.W.append(red.copy())
            self.nu = self.nu - red * red
        cand = np.where(self.mask, -np.inf, self.nu)
        self.p = int(np.argmax(cand))
        Wp = np.array([w[self.p] for w in self.W])
        self.v = self.a[:, self.p] - (np.array(self.Q).T @ Wp if t else 0.0)
        out = np.zeros(self.r)
        if t:
            out[:t] = np.array(self.Q) @ self.v
        out[t] = self.v @ self.v
        return _t(out)

    def aca_commit(self, t, red2):
        n = self.a.shape[1]
        if self.stop:
            return _t(np.zeros(n))
        red2 = red2.numpy()
        c = red2[:t]
        s = float(red2[t] - c @ c)   # ||v - Q^T c||^2 = ||v||^2 - ||c||^2
        mx = max(self.mg, n) * orc.EPS
        if not s > mx * mx * self.frob2:
            self.stop = True
            self._warn(WARN_RANK)
            return _t(np.zeros(n))
        if t:
            self.v = self.v - np.array(self.Q).T @ c
        self.idx[t] = self.p
        self.mask[self.p] = True
        self.count = t + 1
        q = self.v / math.sqrt(s)
        self.Q.append(q)
        return _t(self.a.T @ q)

    def aca_finish(self):
        return _t(orc.pad_indices(self.idx[:self.count], self.a.shape[1], self.r), torch.int32)

    # -- bases, gathers
    def gather_cols(self, J):
        return _t(self.a[:, J.numpy()])

    def rows_at(self, X, offset, ids):
        x = X.numpy()
        out = np.zeros((len(ids), x.shape[1]))
        for j, g in enumerate(ids.tolist()):
            i = g - offset
            if 0 <= i < x.shape[0]:
                out[j] = x[i]
        return _t(out, X.dtype)

    def transpose(self, X):
        return _t(X.numpy().T.copy(), X.dtype)

    def offset_ids(self, ids, offset):
        return _t(ids.numpy().astype(np.int64) + offset, torch.int32)

    def local_select(self, basis, nblocks, delta):
        S, _lv, sw, _st, _info = orc.maxvol_basis_rows(basis.numpy(), nblocks, delta, polish=False)
        return _t(np.array(S), torch.int32), sw

    def merge_pair(self, rows, ids, delta):
        r = self.r
        pos, sw = orc.merge(rows.numpy(), [list(range(r)), list(range(r, 2 * r))], delta)
        return _t(ids.numpy()[pos], torch.int32), _t(rows.numpy()[pos], rows.dtype), sw

    # -- maxvol over a distributed basis
    def _factor(self, basis, offset):
        lu, perm, sing = orc.lu_factor(self.M)
        if sing:
            self.st = SINGULAR
            self.logvol = -math.inf
            self.keyv, self.keyi = -1.0, I64_MAX
            return _t(np.array([-1.0]))
        self.Minv = orc.lu_inverse(lu, perm)
        self.logvol = orc.lu_logabsdet(lu)
        self.B = basis.numpy() @ self.Minv
        return self._key(offset)

    def _key(self, offset):
        flat = int(np.argmax(np.abs(self.B)))
        i, j = divmod(flat, self.r)
        self.keyv = float(abs(self.B[i, j]))
        self.keyi = (offset + i) * self.r + j
        return _t(np.array([self.keyv]))

    def dmv_begin(self, basis, offset, S, M_rows):
        self.S = [int(x) for x in S.tolist()]
        self.M = M_rows.numpy().astype(np.float64).copy()
        self.swaps, self.st = 0, OK
        return self._factor(basis, offset)

    def dmv_refresh(self, basis, offset):
        return self._factor(basis, offset)

    def dmv_holder(self, basis, keyv_glob):
        return _t(np.array([self.keyi if self.keyv == keyv_glob.item() else I64_MAX]), torch.int64)

    def dmv_fill(self, basis, offset, keyi_glob):
        i = int(keyi_glob.item()) // self.r - offset
        x = basis.numpy()
        return _t(x[i] if 0 <= i < x.shape[0] else np.zeros(self.r), basis.dtype)

    def dmv_swap(self, basis, offset, keyi_glob, row):
        i, j = divmod(int(keyi_glob.item()), self.r)
        c = row.numpy().astype(np.float64)
        b = c @ self.Minv
        w = b.copy()
        w[j] -= 1.0
        self.Minv -= np.outer(self.Minv[:, j], w) / b[j]
        self.B -= np.outer(self.B[:, j], w) / b[j]
        self.M[j] = c
        self.S[j] = i
        self.logvol += math.log(abs(b[j]))
        self.swaps += 1
        return self._key(offset)

    def dmv_result(self, basis):
        return _t(np.array(self.S), torch.int32), self.logvol, self.swaps, self.st

    # -- assembly and residual
    def inverse(self, M):
        r = self.r
        _C, U, _R, _rc, _p = orc.assemble(M.numpy(), list(range(r)), list(range(r)))
        return _t(U)

    def residual_parts(self, C, U, R):
        E = self.a - C.numpy() @ (U.numpy() @ R.numpy())
        return _t(np.array([np.abs(E).max(), (E * E).sum(), (self.a * self.a).sum()]))
