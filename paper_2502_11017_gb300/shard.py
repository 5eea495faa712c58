"""The cross with A partitioned by rows over P processes (one per GPU).

The paper divides A into blocks handled by separate processes (Section 2.2): Algorithm 3
reduces each round's (norm, index) over the blocks and broadcasts the pivot vector, and
Section 3.2 attributes the flattening of its speed-up beyond 16 processes to that
communication. Here rank k of P holds a contiguous slab of the rows of A: the row blocks
k b_r/P .. (k+1) b_r/P - 1 of the single-process cross (b_r/P a power of two, so that a
rank's blocks are one subtree of the binary merge), and for the column selection the
column blocks k b_c/P .. (k+1) b_c/P - 1 of R^T = A(I,:)^T. The steps:

* J0 (Algorithm 3 on the columns): per round two allreduce-sums, the slab partials of
  A^T q, and those of Q^T v (the second Gram-Schmidt pass) together with ||v||^2 (the norm
  of the re-orthogonalised vector is ||v||^2 - ||Q^T v||^2, so it needs no third).
* Row selection: every rank runs its blocks and its part of the merge tree alone
  (cur_maxvol_rows without the polish); the top log2 P levels of the tree cross ranks: the
  right child's owner sends its r ids and r x r rows of C to the left child's owner, which
  merges (cur_merge_pair); the root's set is broadcast.
* Polish and later sweeps: maxvol over all rows with the ranks agreeing on each swap by an
  allreduce-MAX of |B_ij|, an allreduce-MIN of the flat index among the holders of that
  value (the lowest index wins a tie, as on one GPU), and an allreduce-sum that carries
  the winner's row from its owner (cur_dmv_*).
* Column selection: R = A(I,:) is summed from the slabs' rows, each rank takes its column
  slab of R^T, then as for the rows.
* Assembly and residual: A(I,J) and R by allreduce-sum, the residual's parts by
  allreduce-max and -sum.

The transport is an interface (``Transport``): ``TorchTransport`` over torch.distributed
(NCCL between GPUs, gloo between CPU processes) and ``ThreadGroup`` for ranks that are
threads of one process. The per-rank arithmetic is an interface too (``CudaRankOps``:
every step in libcur's kernels); nothing here computes a step of the method itself.
"""
from __future__ import annotations

import math
import threading

import numpy as np

from . import (CUR_ERR_ARG, CUR_ERR_NOCONV, CUR_ERR_SINGULAR, CUR_ERR_TIMEOUT, CUR_F32, CUR_F64, CUR_OK,
               CUR_WARN_RANK)


class PeerLost(RuntimeError):
    """A collective could not complete: a rank left or did not answer in time."""


def balanced_blocks(size: int, nblocks: int):
    """Contiguous blocks [start, stop); the first size mod nblocks blocks get one more."""
    base, extra = divmod(size, nblocks)
    out, s = [], 0
    for k in range(nblocks):
        e = s + base + (1 if k < extra else 0)
        out.append((s, e))
        s = e
    return out


def slab(size: int, nblocks: int, world: int, rank: int):
    """(start, stop) of rank's contiguous share: blocks rank*nblocks/world ..
    (rank+1)*nblocks/world - 1 of balanced_blocks(size, nblocks)."""
    check_partition(nblocks, world)
    per = nblocks // world
    bl = balanced_blocks(size, nblocks)
    return bl[rank * per][0], bl[(rank + 1) * per - 1][1]


def check_partition(nblocks: int, world: int) -> None:
    per = nblocks // world if world else 0
    if world < 1 or nblocks % world or per & (per - 1):
        raise ValueError(f"{nblocks} blocks over {world} ranks: each rank needs the same power-of-two count")


# ------------------------------------------------------------------ transports

class Transport:
    """Collectives among the ranks on small tensors (in place)."""
    rank = 0
    world = 1

    def allreduce(self, t, op: str):
        raise NotImplementedError

    def send(self, t, dst: int):
        raise NotImplementedError

    def recv(self, t, src: int):
        raise NotImplementedError

    def broadcast(self, t, src: int):
        raise NotImplementedError


class TorchTransport(Transport):
    """torch.distributed: NCCL on device tensors, or gloo (device tensors pass through the
    host). A failed collective (a peer that left, a timeout) raises PeerLost."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.host = dist.get_backend(group) == "gloo"

    def _run(self, fn, t):
        host = self.host and t.is_cuda
        x = t.cpu() if host else t
        try:
            fn(x)
        except Exception as e:          # a collective that cannot complete
            raise PeerLost(str(e)) from e
        if host:
            t.copy_(x)
        return t

    def allreduce(self, t, op: str):
        ops = {"sum": self.dist.ReduceOp.SUM, "max": self.dist.ReduceOp.MAX, "min": self.dist.ReduceOp.MIN}
        return self._run(lambda x: self.dist.all_reduce(x, ops[op], group=self.group), t)

    def send(self, t, dst: int):
        return self._run(lambda x: self.dist.send(x, dst, group=self.group), t)

    def recv(self, t, src: int):
        return self._run(lambda x: self.dist.recv(x, src, group=self.group), t)

    def broadcast(self, t, src: int):
        return self._run(lambda x: self.dist.broadcast(x, src, group=self.group), t)


class ThreadGroup:
    """Ranks that are threads of one process: a barrier-based rendezvous, reductions done on
    the host in rank order (identical results on every rank). ``transport(k)`` is rank k's."""

    def __init__(self, world: int, timeout: float = 60.0):
        self.world = world
        self.timeout = timeout
        self._bar = threading.Barrier(world)
        self._slots = [None] * world
        self._result = None
        self._mail = {}
        self._cv = threading.Condition()

    def transport(self, rank: int) -> "ThreadTransport":
        return ThreadTransport(self, rank)

    def _wait(self):
        try:
            self._bar.wait(self.timeout)
        except threading.BrokenBarrierError as e:
            raise PeerLost("a rank did not reach the collective in time") from e


class ThreadTransport(Transport):
    def __init__(self, group: ThreadGroup, rank: int):
        self.g = group
        self.rank = rank
        self.world = group.world

    def allreduce(self, t, op: str):
        g = self.g
        g._slots[self.rank] = t.detach().cpu().numpy().copy()
        g._wait()
        if self.rank == 0:
            acc = g._slots[0].copy()
            for x in g._slots[1:]:
                if op == "sum":
                    acc = acc + x
                elif op == "max":
                    acc = np.maximum(acc, x)
                else:
                    acc = np.minimum(acc, x)
            g._result = acc
        g._wait()
        import torch
        t.copy_(torch.from_numpy(g._result.copy()))
        g._wait()
        return t

    def send(self, t, dst: int):
        with self.g._cv:
            self.g._mail.setdefault((self.rank, dst), []).append(t.detach().cpu().numpy().copy())
            self.g._cv.notify_all()
        return t

    def recv(self, t, src: int):
        import torch
        with self.g._cv:
            ok = self.g._cv.wait_for(lambda: self.g._mail.get((src, self.rank)), self.g.timeout)
            if not ok:
                raise PeerLost(f"nothing from rank {src} in time")
            x = self.g._mail[(src, self.rank)].pop(0)
        t.copy_(torch.from_numpy(x))
        return t

    def broadcast(self, t, src: int):
        g = self.g
        if self.rank == src:
            g._result = t.detach().cpu().numpy().copy()
        g._wait()
        import torch
        t.copy_(torch.from_numpy(g._result.copy()))
        g._wait()
        return t


# ------------------------------------------------------------------ per-rank steps on the GPU

class CudaRankOps:
    """The per-rank steps in libcur's kernels, on this rank's slab A_k (a CUDA tensor, FP32
    or FP64, rows row0 .. row0 + A_k.shape[0] - 1 of A)."""

    def __init__(self, A_k, r: int, workspace_rows: int | None = None, stream=None):
        import torch
        from . import Handle, _dtype_code
        self.torch = torch
        self.A = A_k
        self.dev = A_k.device
        self.dtype = A_k.dtype
        self.code = _dtype_code(A_k)
        if self.code not in (CUR_F32, CUR_F64):
            raise ValueError("the sharded cross takes FP32 or FP64 slabs")
        self.r = r
        m_k, n = A_k.shape
        rows = workspace_rows or max(m_k, n)
        self.hd = Handle(rows, n, r, self.code)
        self.h = self.hd.h
        self.stream = stream
        self.aca_state = None

    # -- plumbing
    def zeros(self, shape, dtype=None):
        return self.torch.zeros(shape, dtype=dtype or self.dtype, device=self.dev)

    def empty(self, shape, dtype=None):
        return self.torch.empty(shape, dtype=dtype or self.dtype, device=self.dev)

    def cat(self, xs):
        return self.torch.cat(xs)

    def item(self, t):
        return t.item()

    def sync_status(self) -> int:
        from . import cur_sync_status
        return cur_sync_status(self.h, self.stream)

    def close(self):
        self.hd.close()

    # -- Algorithm 3 on the columns
    def aca_begin(self, m_global: int):
        from . import cur_shard_aca_begin, cur_shard_aca_state_bytes
        n = self.A.shape[1]
        self.aca_state = self.empty(cur_shard_aca_state_bytes(self.h, self.A, self.r), self.torch.uint8)
        self.idx = self.empty(self.r, self.torch.int32)
        red = self.empty(n, self.torch.float64)
        cur_shard_aca_begin(self.h, self.A, m_global, self.r, self.aca_state, self.idx, red, self.stream)
        return red

    def aca_pick(self, t: int, red):
        from . import cur_shard_aca_pick
        red2 = self.empty(self.r, self.torch.float64)
        cur_shard_aca_pick(self.h, self.A, self.r, t, self.aca_state, red, red2, self.stream)
        return red2

    def aca_commit(self, t: int, red2):
        from . import cur_shard_aca_commit
        red = self.empty(self.A.shape[1], self.torch.float64)
        cur_shard_aca_commit(self.h, self.A, self.r, t, self.aca_state, red2, self.idx, red, self.stream)
        return red

    def aca_finish(self):
        from . import cur_shard_aca_finish
        cur_shard_aca_finish(self.h, self.A, self.r, self.aca_state, self.idx, self.stream)
        return self.idx

    # -- bases, gathers
    def gather_cols(self, J):
        from . import cur_gather_cols
        C = self.empty((self.A.shape[0], self.r))
        cur_gather_cols(self.h, self.A, J, self.r, C, self.stream)
        return C

    def rows_at(self, X, offset: int, ids):
        from . import cur_rows_at
        out = self.empty((ids.shape[0], X.shape[1]), X.dtype)
        cur_rows_at(self.h, X, offset, ids, ids.shape[0], out, self.stream)
        return out

    def transpose(self, X):
        from . import cur_transpose
        out = self.empty((X.shape[1], X.shape[0]), X.dtype)
        cur_transpose(self.h, X, out, self.stream)
        return out

    def offset_ids(self, ids, offset: int):
        from . import cur_offset_ids
        out = self.empty(ids.shape[0], self.torch.int32)
        cur_offset_ids(self.h, ids, ids.shape[0], offset, out, self.stream)
        return out

    def local_select(self, basis, nblocks: int, delta: float):
        """Blocks and their merge tree on this rank's basis (no polish): local ids, swaps."""
        from . import cur_maxvol_rows, opts
        iota = self.torch.arange(self.r, dtype=self.torch.int32, device=self.dev)
        I = self.empty(self.r, self.torch.int32)
        sw = self.empty(1, self.torch.int32)
        cur_maxvol_rows(self.h, basis, iota, self.r, opts(delta, nblocks=nblocks, polish=False), I, None, sw,
                        self.stream)
        return I, int(sw.item())

    def merge_pair(self, rows, ids, delta: float):
        from . import cur_merge_pair, opts
        ids_out = self.empty(self.r, self.torch.int32)
        rows_out = self.empty((self.r, self.r), rows.dtype)
        sw = self.empty(1, self.torch.int32)
        cur_merge_pair(self.h, rows, ids, opts(delta), ids_out, rows_out, sw, self.stream)
        return ids_out, rows_out, int(sw.item())

    # -- maxvol over a distributed basis
    def dmv_begin(self, basis, offset: int, S, M_rows):
        from . import cur_dmv_begin, cur_dmv_state_bytes
        self.dmv_state = self.empty(cur_dmv_state_bytes(basis.shape[0], self.r, self.code), self.torch.uint8)
        keyv = self.empty(1, self.torch.float64)
        cur_dmv_begin(self.h, basis, offset, S, M_rows, self.dmv_state, keyv, self.stream)
        return keyv

    def dmv_refresh(self, basis, offset: int):
        from . import cur_dmv_refresh
        keyv = self.empty(1, self.torch.float64)
        cur_dmv_refresh(self.h, basis, offset, self.dmv_state, keyv, self.stream)
        return keyv

    def dmv_holder(self, basis, keyv_glob):
        from . import cur_dmv_holder
        keyi = self.empty(1, self.torch.int64)
        cur_dmv_holder(self.h, basis, self.dmv_state, keyv_glob, keyi, self.stream)
        return keyi

    def dmv_fill(self, basis, offset: int, keyi_glob):
        from . import cur_dmv_fill
        row = self.empty(self.r, basis.dtype)
        cur_dmv_fill(self.h, basis, offset, keyi_glob, row, self.stream)
        return row

    def dmv_swap(self, basis, offset: int, keyi_glob, row):
        from . import cur_dmv_swap
        keyv = self.empty(1, self.torch.float64)
        cur_dmv_swap(self.h, basis, offset, self.dmv_state, keyi_glob, row, keyv, self.stream)
        return keyv

    def dmv_result(self, basis):
        from . import cur_dmv_result
        S = self.empty(self.r, self.torch.int32)
        lv = self.empty(1, self.torch.float64)
        cnt = self.empty(2, self.torch.int32)
        cur_dmv_result(self.h, basis, self.dmv_state, S, lv, cnt, self.stream)
        c = cnt.tolist()
        return S, float(lv.item()), int(c[0]), int(c[1])

    # -- assembly and residual
    def inverse(self, M):
        """U = M^dagger for the r x r M (cur_assemble on M itself: LU inverse, pinv fallback)."""
        from . import cur_assemble
        iota = self.torch.arange(self.r, dtype=self.torch.int32, device=self.dev)
        U = self.empty((self.r, self.r), self.torch.float64)
        rc = self.empty(1, self.torch.float64)
        cur_assemble(self.h, M, iota, iota, self.r, None, U, None, rc, self.stream)
        return U

    def residual_parts(self, C, U, R):
        from . import cur_residual_parts
        parts = self.empty(3, self.torch.float64)
        cur_residual_parts(self.h, self.A, C, U, R, self.r, parts, self.stream)
        return parts


# ------------------------------------------------------------------ the driver

def aca_columns(T: Transport, ops, m: int, r: int):
    """J0 = Algorithm 3 on the columns of A over the row slabs (padded after an early stop)."""
    red = T.allreduce(ops.aca_begin(m), "sum")
    for t in range(r):
        red2 = T.allreduce(ops.aca_pick(t, red), "sum")
        red = ops.aca_commit(t, red2)
        if t + 1 < r:
            T.allreduce(red, "sum")
    return ops.aca_finish()


def dmaxvol(T: Transport, ops, basis, offset: int, S, M_rows, r: int, delta: float, max_swaps: int | None = None):
    """Maxvol over all rows of the distributed basis from S (replicated). Returns
    (S, logvol, swaps, status) as the single-process iteration does."""
    if max_swaps is None:
        max_swaps = 100 * r
    keyv = ops.dmv_begin(basis, offset, S, M_rows)
    swaps, status = 0, CUR_OK
    while True:
        made = 0
        while made < r:
            T.allreduce(keyv, "max")
            v = ops.item(keyv)
            if v < 0:                       # M numerically singular (identical on every rank)
                status = CUR_ERR_SINGULAR
                break
            if v <= 1.0 + delta:
                break
            if swaps >= max_swaps:
                status = CUR_ERR_NOCONV
                break
            keyi = T.allreduce(ops.dmv_holder(basis, keyv), "min")
            row = T.allreduce(ops.dmv_fill(basis, offset, keyi), "sum")
            keyv = ops.dmv_swap(basis, offset, keyi, row)
            made += 1
            swaps += 1
        if made == 0 or status != CUR_OK:
            break
        keyv = ops.dmv_refresh(basis, offset)
    S_out, lv, _sw, st = ops.dmv_result(basis)
    if st == CUR_ERR_SINGULAR:
        status = CUR_ERR_SINGULAR
    return S_out, lv, swaps, status


def select(T: Transport, ops, basis, offset: int, nblocks_local: int, r: int, delta: float, polish: bool = True):
    """Row selection on a basis distributed by slabs (the blocks of this rank, the merge tree,
    the polish). Returns (ids, logvol, swaps, status) with ids replicated on every rank."""
    loc, sw_local = ops.local_select(basis, nblocks_local, delta)
    ids = ops.offset_ids(loc, offset)
    rows = ops.rows_at(basis, offset, ids)
    swaps_here = sw_local
    owners = list(range(T.world))
    while len(owners) > 1:
        nxt = []
        for t in range(0, len(owners) - 1, 2):
            a, b = owners[t], owners[t + 1]
            if T.rank == b:
                T.send(ids, a)
                T.send(rows, a)
            elif T.rank == a:
                ids_b, rows_b = ops.empty(r, ids.dtype), ops.empty((r, r), rows.dtype)
                T.recv(ids_b, b)
                T.recv(rows_b, b)
                ids, rows, sw = ops.merge_pair(ops.cat([rows, rows_b]), ops.cat([ids, ids_b]), delta)
                swaps_here += sw
            nxt.append(a)
        if len(owners) % 2:
            nxt.append(owners[-1])
        owners = nxt
    T.broadcast(ids, owners[0])
    T.broadcast(rows, owners[0])
    import torch
    tot = ops.zeros(1, torch.int64)
    tot += swaps_here
    swaps = int(ops.item(T.allreduce(tot, "sum")))
    if not polish:
        return ids, None, swaps, CUR_OK
    S, lv, sw, st = dmaxvol(T, ops, basis, offset, ids, rows, r, delta)
    swaps += sw
    if st == CUR_ERR_SINGULAR:
        return ids, -math.inf, swaps, st
    return S, lv, swaps, st


def cross(T: Transport, ops, m: int, n: int, r: int, b_r: int, b_c: int, delta: float = 1e-2,
          max_sweeps: int = 8, residual: bool = True):
    """The cross of A (m x n) whose row slab ops holds (rows of ``slab(m, b_r, P, rank)``).

    Returns a dict with I, J (host lists, position order), logvol, status, sweeps,
    sweep_swaps, J0 and, with ``residual``, cheb = max|A - CUR| and fro_rel. A rank that
    leaves makes the others' next collective fail: they return status CUR_ERR_TIMEOUT."""
    P, k = T.world, T.rank
    check_partition(b_r, P)
    check_partition(b_c, P)
    if not (1 <= r < min(m, n)) or m // b_r < r or n // b_c < r:
        return dict(status=CUR_ERR_ARG)
    row0, row1 = slab(m, b_r, P, k)
    col0, col1 = slab(n, b_c, P, k)
    try:
        J0 = aca_columns(T, ops, m, r)
        J0_host = [int(x) for x in J0.tolist()]
        # sweep 1: blockwise rows, then blockwise columns
        C = ops.gather_cols(J0)
        I, _lv, sw_r, st_r = select(T, ops, C, row0, b_r // P, r, delta)

        def col_basis(I):
            R = T.allreduce(ops.rows_at(ops.A, row0, I), "sum")          # A(I,:), r x n
            return R, ops.transpose(R[:, col0:col1])

        R, Rt = col_basis(I)
        J, lv, sw_c, st_c = select(T, ops, Rt, col0, b_c // P, r, delta)
        sweeps, sweep_swaps = 1, [sw_r + sw_c]
        status = CUR_OK
        for st in (st_r, st_c):
            if st != CUR_OK:
                status = st
        while sweeps < max_sweeps:
            sweeps += 1
            C = ops.gather_cols(J)
            M = T.allreduce(ops.rows_at(C, row0, I), "sum")
            I, _lv, s1, st1 = dmaxvol(T, ops, C, row0, I, M, r, delta)
            R, Rt = col_basis(I)
            Mt = T.allreduce(ops.rows_at(Rt, col0, J), "sum")
            J, lv, s2, st2 = dmaxvol(T, ops, Rt, col0, J, Mt, r, delta)
            sweep_swaps.append(s1 + s2)
            if st1 != CUR_OK or st2 != CUR_OK:
                status = st1 if st1 != CUR_OK else st2
                break
            if s1 + s2 == 0:
                break
        out = dict(I=[int(x) for x in I.tolist()], J=[int(x) for x in J.tolist()], logvol=lv, sweeps=sweeps,
                   sweep_swaps=sweep_swaps, J0=J0_host)
        if residual:
            C = ops.gather_cols(J)
            M = T.allreduce(ops.rows_at(C, row0, I), "sum")                # A(I,J)
            U = ops.inverse(M)
            R = T.allreduce(ops.rows_at(ops.A, row0, I), "sum")
            parts = ops.residual_parts(C, U, R)
            mx = T.allreduce(parts[0:1].clone(), "max")
            sums = T.allreduce(parts[1:3].clone(), "sum")
            s = sums.tolist()
            out["cheb"] = float(mx.item())
            out["fro_rel"] = math.sqrt(s[0] / s[1]) if s[1] > 0 else 0.0
        # the device status word: an error found there wins; Algorithm 3's early stop
        # (CUR_WARN_RANK) is kept unless a stage ended with an error
        dev_status = ops.sync_status()
        if dev_status not in (CUR_OK, CUR_WARN_RANK) or status == CUR_OK:
            status = dev_status if dev_status != CUR_OK else status
        out["status"] = status
        return out
    except PeerLost as e:
        return dict(status=CUR_ERR_TIMEOUT, error=str(e))
