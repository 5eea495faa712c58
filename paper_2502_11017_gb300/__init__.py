"""GB300 (sm_103a) scalable binary CUR cross: Python binding of libcur.

The functions below carry the names of the C ABI in include/cur.h and only
marshal arguments: PyTorch tensors supply device memory and the stream, every
step runs in libcur's CUDA kernels. If the library is missing the calls raise
instead of falling back to anything else; build it with ``build()``.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libcur.so")

CUR_OK, CUR_ERR_ARG, CUR_ERR_SINGULAR, CUR_ERR_NONFINITE, CUR_ERR_NOCONV = 0, 1, 2, 3, 4
CUR_ERR_TIMEOUT, CUR_ERR_NOMEM, CUR_ERR_CUDA, CUR_WARN_RANK = 5, 6, 7, 8
CUR_F64, CUR_F32, CUR_BF16 = 0, 1, 2
CUR_FLAG_POLISH = 1
CUR_FLAG_PREC_BF16 = 2
CUR_FLAG_PREC_FP8 = 4
CUR_FLAG_REFACTOR_ALWAYS = 8

# Every symbol include/cur.h declares.
EXPORTS = ["cur_create", "cur_destroy", "cur_workspace_size", "cur_aca_select", "cur_aca_full",
           "cur_batch_workspace_size", "cur_cross_batched",
           "cur_maxvol_rows", "cur_maxvol_cols", "cur_merge", "cur_assemble",
           "cur_residual_cheb", "cur_cross", "cur_sync_status", "cur_default_opts",
           "cur_status_string", "cur_prof_enable", "cur_prof_read", "cur_prof_refactors",
           "cur_residual_cheb_noalloc", "cur_selftest_wait_timeout",
           "cur_sketch", "cur_mlp_forward", "cur_mlp_grad", "cur_adam_step", "cur_propose",
           "cur_cross_from", "cur_maxvol_global",
           "cur_shard_aca_state_bytes", "cur_shard_aca_begin", "cur_shard_aca_pick",
           "cur_shard_aca_commit", "cur_shard_aca_finish",
           "cur_dmv_state_bytes", "cur_dmv_begin", "cur_dmv_refresh", "cur_dmv_holder", "cur_dmv_fill",
           "cur_dmv_swap", "cur_dmv_result", "cur_merge_pair", "cur_rows_at", "cur_transpose",
           "cur_offset_ids", "cur_gather_cols", "cur_residual_parts", "cur_coef_tf32"]


class CurMat(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("rows", ctypes.c_int64), ("cols", ctypes.c_int64),
                ("ld", ctypes.c_int64), ("dtype", ctypes.c_int)]


class CurOpts(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("max_swaps", ctypes.c_int32),
                ("nblocks", ctypes.c_int32), ("flags", ctypes.c_uint32)]


class CurCrossInfo(ctypes.Structure):
    _fields_ = [("logvol", ctypes.c_double), ("sweeps", ctypes.c_int32),
                ("swaps_total", ctypes.c_int32), ("sweep_swaps", ctypes.c_int32 * 8),
                ("aca_selected", ctypes.c_int32), ("status", ctypes.c_int32)]


class CurBatchItem(ctypes.Structure):
    _fields_ = [("offset", ctypes.c_int64), ("rows", ctypes.c_int64), ("cols", ctypes.c_int64),
                ("ld", ctypes.c_int64), ("r", ctypes.c_int32), ("b_r", ctypes.c_int32), ("b_c", ctypes.c_int32)]


_lib = None


def build(verbose: bool = False) -> str:
    from . import buildlib
    return buildlib.build(verbose=verbose)


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libcur.so and declare its signatures. Raises if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libcur.so not found at {path}: run "
                           "paper_2502_11017_gb300.build() first (no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    pmat, popts = ctypes.POINTER(CurMat), ctypes.POINTER(CurOpts)
    sig = {
        "cur_create": ([ctypes.POINTER(P), ctypes.c_size_t], ctypes.c_int),
        "cur_destroy": ([P], ctypes.c_int),
        "cur_workspace_size": ([I64, I64, I32, ctypes.c_int], ctypes.c_size_t),
        "cur_aca_select": ([P, pmat, ctypes.c_int, I32, I32, P, P], ctypes.c_int),
        "cur_aca_full": ([P, pmat, I32, P, P, P, P, P], ctypes.c_int),
        "cur_batch_workspace_size": ([ctypes.POINTER(CurBatchItem), I32], ctypes.c_size_t),
        "cur_cross_batched": ([P, P, ctypes.c_int, ctypes.POINTER(CurBatchItem), I32, popts, P, P, P],
                              ctypes.c_int),
        "cur_maxvol_rows": ([P, pmat, P, I32, popts, P, P, P, P], ctypes.c_int),
        "cur_maxvol_cols": ([P, pmat, P, I32, popts, P, P, P, P], ctypes.c_int),
        "cur_merge": ([P, pmat, P, I32, I32, popts, P, P], ctypes.c_int),
        "cur_assemble": ([P, pmat, P, P, I32, P, P, P, P, P], ctypes.c_int),
        "cur_residual_cheb": ([P, pmat, P, P, P, I32, P, P, P], ctypes.c_int),
        "cur_cross": ([P, pmat, I32, I32, I32, popts, P, P, P, P], ctypes.c_int),
        "cur_sync_status": ([P, P], ctypes.c_int),
        "cur_default_opts": ([], CurOpts),
        "cur_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "cur_prof_enable": ([P, ctypes.c_int], ctypes.c_int),
        "cur_residual_cheb_noalloc": ([pmat, P, P, P, I32, P, P, P], ctypes.c_int),
        "cur_selftest_wait_timeout": ([P, P], ctypes.c_int),
        "cur_prof_read": ([P, P, ctypes.POINTER(D), ctypes.POINTER(I32),
                           ctypes.POINTER(I64)], ctypes.c_int),
        "cur_prof_refactors": ([P, P, ctypes.POINTER(I64)], ctypes.c_int),
        "cur_sketch": ([P, pmat, P, P, I32, P, P, I32, P], ctypes.c_int),
        "cur_mlp_forward": ([P, P, I64, I32, I32, P, P, P], ctypes.c_int),
        "cur_mlp_grad": ([P, P, P, I64, P, I64, I32, I32, P, ctypes.c_float, P, P, P], ctypes.c_int),
        "cur_adam_step": ([P, P, P, P, P, I64, I32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                           ctypes.c_float, P], ctypes.c_int),
        "cur_propose": ([P, P, I64, I32, P, P], ctypes.c_int),
        "cur_cross_from": ([P, pmat, I32, P, P, popts, P, P, P, P], ctypes.c_int),
        "cur_maxvol_global": ([P, pmat, P, I32, popts, P, P, P, P], ctypes.c_int),
        "cur_shard_aca_state_bytes": ([P, pmat, I32], ctypes.c_size_t),
        "cur_shard_aca_begin": ([P, pmat, I64, I32, P, P, P, P], ctypes.c_int),
        "cur_shard_aca_pick": ([P, pmat, I32, I32, P, P, P, P], ctypes.c_int),
        "cur_shard_aca_commit": ([P, pmat, I32, I32, P, P, P, P, P], ctypes.c_int),
        "cur_shard_aca_finish": ([P, pmat, I32, P, P, P], ctypes.c_int),
        "cur_dmv_state_bytes": ([I64, I32, ctypes.c_int], ctypes.c_size_t),
        "cur_dmv_begin": ([P, pmat, I64, P, P, P, P, P], ctypes.c_int),
        "cur_dmv_refresh": ([P, pmat, I64, P, P, P], ctypes.c_int),
        "cur_dmv_holder": ([P, pmat, P, P, P, P], ctypes.c_int),
        "cur_dmv_fill": ([P, pmat, I64, P, P, P], ctypes.c_int),
        "cur_dmv_swap": ([P, pmat, I64, P, P, P, P, P], ctypes.c_int),
        "cur_dmv_result": ([P, pmat, P, P, P, P, P], ctypes.c_int),
        "cur_merge_pair": ([P, pmat, P, popts, P, P, P, P], ctypes.c_int),
        "cur_rows_at": ([P, pmat, I64, P, I32, P, P], ctypes.c_int),
        "cur_transpose": ([P, pmat, P, P], ctypes.c_int),
        "cur_offset_ids": ([P, P, I32, I64, P, P], ctypes.c_int),
        "cur_gather_cols": ([P, pmat, P, I32, P, P], ctypes.c_int),
        "cur_residual_parts": ([P, pmat, P, P, P, I32, P, P], ctypes.c_int),
        "cur_coef_tf32": ([P, pmat, P, P, P], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


class CurError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = load().cur_status_string(status).decode()
        super().__init__(f"{what}: {msg} (status {status})")


def _check(st: int, what: str) -> int:
    if st not in (CUR_OK, CUR_WARN_RANK):
        raise CurError(st, what)
    return st


def cur_status_string(status: int) -> str:
    return load().cur_status_string(status).decode()


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float64:
        return CUR_F64
    if t.dtype == torch.float32:
        return CUR_F32
    if t.dtype == torch.bfloat16:
        return CUR_BF16
    raise TypeError(f"unsupported dtype {t.dtype}")


def mat(t) -> CurMat:
    """cur_mat view of a 2-D row-major CUDA tensor (unit stride in columns)."""
    if t.dim() != 2 or t.stride(1) != 1 or not t.is_cuda:
        raise ValueError("expected a 2-D CUDA tensor with unit column stride")
    return CurMat(t.data_ptr(), t.shape[0], t.shape[1], t.stride(0), _dtype_code(t))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def opts(delta: float = 1e-2, max_swaps: int = 0, nblocks: int = 1, polish: bool = True,
         bf16: bool = False, fp8: bool = False, refactor_always: bool = False) -> CurOpts:
    return CurOpts(delta, max_swaps, nblocks, (CUR_FLAG_POLISH if polish else 0) | (CUR_FLAG_PREC_BF16 if bf16 else 0)
                   | (CUR_FLAG_PREC_FP8 if fp8 else 0) | (CUR_FLAG_REFACTOR_ALWAYS if refactor_always else 0))


# ------------------------------------------------------------------ C ABI names

def cur_workspace_size(m: int, n: int, r: int, dtype: int) -> int:
    return load().cur_workspace_size(m, n, r, dtype)


def cur_create(workspace_bytes: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().cur_create(ctypes.byref(h), workspace_bytes), "cur_create")
    return h


def cur_destroy(h) -> None:
    _check(load().cur_destroy(h), "cur_destroy")


def cur_sync_status(h, stream=None) -> int:
    return load().cur_sync_status(h, _stream(stream))


def cur_aca_select(h, A, axis: int, r: int, nblocks: int, idx_out, stream=None) -> int:
    return _check(load().cur_aca_select(h, ctypes.byref(mat(A)), axis, r, nblocks,
                                        _ptr(idx_out), _stream(stream)), "cur_aca_select")


def cur_aca_full(h, A, r: int, R_work, I_out, J_out, piv_out=None, stream=None) -> int:
    return _check(load().cur_aca_full(h, ctypes.byref(mat(A)), r, _ptr(R_work), _ptr(I_out),
                                      _ptr(J_out), _ptr(piv_out), _stream(stream)), "cur_aca_full")


def batch_items(shapes, offsets):
    """ctypes array of cur_batch_item from (rows, cols, r, b_r, b_c) tuples and element offsets
    (contiguous rows: ld = cols)."""
    arr = (CurBatchItem * len(shapes))()
    for t, ((m, n, r, br, bc), off) in enumerate(zip(shapes, offsets)):
        arr[t] = CurBatchItem(int(off), int(m), int(n), int(n), int(r), int(br), int(bc))
    return arr


def cur_batch_workspace_size(items) -> int:
    return load().cur_batch_workspace_size(items, len(items))


def cur_cross_batched(h, data, items, opts_, IJ_out, info_out=None, stream=None) -> int:
    """data: packed device tensor; items: a batch_items() array."""
    return _check(load().cur_cross_batched(h, _ptr(data), _dtype_code(data), items, len(items),
                                           ctypes.byref(opts_), _ptr(IJ_out), _ptr(info_out),
                                           _stream(stream)), "cur_cross_batched")


def cur_maxvol_rows(h, A, J, r: int, o: CurOpts, I_out, logvol_out=None, swaps_out=None,
                    stream=None) -> int:
    return _check(load().cur_maxvol_rows(h, ctypes.byref(mat(A)), _ptr(J), r, ctypes.byref(o),
                                         _ptr(I_out), _ptr(logvol_out), _ptr(swaps_out),
                                         _stream(stream)), "cur_maxvol_rows")


def cur_maxvol_cols(h, A, I, r: int, o: CurOpts, J_out, logvol_out=None, swaps_out=None,
                    stream=None) -> int:
    return _check(load().cur_maxvol_cols(h, ctypes.byref(mat(A)), _ptr(I), r, ctypes.byref(o),
                                         _ptr(J_out), _ptr(logvol_out), _ptr(swaps_out),
                                         _stream(stream)), "cur_maxvol_cols")


def cur_merge(h, basis, cand, nsets: int, r: int, o: CurOpts, out, stream=None) -> int:
    return _check(load().cur_merge(h, ctypes.byref(mat(basis)), _ptr(cand), nsets, r,
                                   ctypes.byref(o), _ptr(out), _stream(stream)), "cur_merge")


def cur_assemble(h, A, I, J, r: int, C_out, U_out, R_out, rcond_out, stream=None) -> int:
    return _check(load().cur_assemble(h, ctypes.byref(mat(A)), _ptr(I), _ptr(J), r, _ptr(C_out),
                                      _ptr(U_out), _ptr(R_out), _ptr(rcond_out), _stream(stream)),
                  "cur_assemble")


def cur_residual_cheb(h, A, C, U, R, r: int, cheb_out, fro_out=None, stream=None) -> int:
    return _check(load().cur_residual_cheb(h, ctypes.byref(mat(A)), _ptr(C), _ptr(U), _ptr(R), r,
                                           _ptr(cheb_out), _ptr(fro_out), _stream(stream)),
                  "cur_residual_cheb")


def cur_residual_cheb_noalloc(A, C, U, R, r: int, cheb_out, fro_out=None, stream=None) -> int:
    """The residual without a handle or any allocation (scratch compiled into libcur)."""
    return _check(load().cur_residual_cheb_noalloc(ctypes.byref(mat(A)), _ptr(C), _ptr(U), _ptr(R),
                                                   r, _ptr(cheb_out), _ptr(fro_out),
                                                   _stream(stream)), "cur_residual_cheb_noalloc")


def cur_cross(h, A, r: int, b_r: int, b_c: int, o: CurOpts, I_out, J_out, info_out=None,
              stream=None) -> int:
    return _check(load().cur_cross(h, ctypes.byref(mat(A)), r, b_r, b_c, ctypes.byref(o),
                                   _ptr(I_out), _ptr(J_out), _ptr(info_out), _stream(stream)),
                  "cur_cross")


def cur_prof_enable(h, on: bool = True) -> None:
    _check(load().cur_prof_enable(h, 1 if on else 0), "cur_prof_enable")


def cur_prof_read(h, stream=None):
    """(pass_ms, pass_launches, kernel_launches) since the last read."""
    ms, n, k = ctypes.c_double(), ctypes.c_int32(), ctypes.c_int64()
    _check(load().cur_prof_read(h, _stream(stream), ctypes.byref(ms), ctypes.byref(n),
                                ctypes.byref(k)), "cur_prof_read")
    return ms.value, n.value, k.value


def cur_prof_refactors(h, stream=None) -> int:
    """Cycle refactorisations of C(S,:) made by the handle's calls since the last read."""
    n = ctypes.c_int64()
    _check(load().cur_prof_refactors(h, _stream(stream), ctypes.byref(n)), "cur_prof_refactors")
    return n.value


def cur_selftest_wait_timeout(h, stream=None) -> None:
    """Launch a device wait that must run out; its timeout lands in the status word."""
    _check(load().cur_selftest_wait_timeout(h, _stream(stream)), "cur_selftest_wait_timeout")


# ------------------------------------------------------------------ sharded cross (per-rank steps)

def cur_shard_aca_state_bytes(h, A_k, r: int) -> int:
    return load().cur_shard_aca_state_bytes(h, ctypes.byref(mat(A_k)), r)


def cur_shard_aca_begin(h, A_k, m_global: int, r: int, state, idx_out, red, stream=None) -> int:
    return _check(load().cur_shard_aca_begin(h, ctypes.byref(mat(A_k)), m_global, r, _ptr(state), _ptr(idx_out),
                                             _ptr(red), _stream(stream)), "cur_shard_aca_begin")


def cur_shard_aca_pick(h, A_k, r: int, t: int, state, red, red2, stream=None) -> int:
    return _check(load().cur_shard_aca_pick(h, ctypes.byref(mat(A_k)), r, t, _ptr(state), _ptr(red), _ptr(red2),
                                            _stream(stream)), "cur_shard_aca_pick")


def cur_shard_aca_commit(h, A_k, r: int, t: int, state, red2, idx_out, red, stream=None) -> int:
    return _check(load().cur_shard_aca_commit(h, ctypes.byref(mat(A_k)), r, t, _ptr(state), _ptr(red2),
                                              _ptr(idx_out), _ptr(red), _stream(stream)), "cur_shard_aca_commit")


def cur_shard_aca_finish(h, A_k, r: int, state, idx_out, stream=None) -> int:
    return _check(load().cur_shard_aca_finish(h, ctypes.byref(mat(A_k)), r, _ptr(state), _ptr(idx_out),
                                              _stream(stream)), "cur_shard_aca_finish")


def cur_dmv_state_bytes(p_local: int, r: int, dtype: int) -> int:
    return load().cur_dmv_state_bytes(p_local, r, dtype)


def cur_dmv_begin(h, C_k, offset: int, S, M_rows, state, keyv_out, stream=None) -> int:
    return _check(load().cur_dmv_begin(h, ctypes.byref(mat(C_k)), offset, _ptr(S), _ptr(M_rows), _ptr(state),
                                       _ptr(keyv_out), _stream(stream)), "cur_dmv_begin")


def cur_dmv_refresh(h, C_k, offset: int, state, keyv_out, stream=None) -> int:
    return _check(load().cur_dmv_refresh(h, ctypes.byref(mat(C_k)), offset, _ptr(state), _ptr(keyv_out),
                                         _stream(stream)), "cur_dmv_refresh")


def cur_dmv_holder(h, C_k, state, keyv_glob, keyi_out, stream=None) -> int:
    return _check(load().cur_dmv_holder(h, ctypes.byref(mat(C_k)), _ptr(state), _ptr(keyv_glob), _ptr(keyi_out),
                                        _stream(stream)), "cur_dmv_holder")


def cur_dmv_fill(h, C_k, offset: int, keyi_glob, row_out, stream=None) -> int:
    return _check(load().cur_dmv_fill(h, ctypes.byref(mat(C_k)), offset, _ptr(keyi_glob), _ptr(row_out),
                                      _stream(stream)), "cur_dmv_fill")


def cur_dmv_swap(h, C_k, offset: int, state, keyi_glob, row, keyv_out, stream=None) -> int:
    return _check(load().cur_dmv_swap(h, ctypes.byref(mat(C_k)), offset, _ptr(state), _ptr(keyi_glob), _ptr(row),
                                      _ptr(keyv_out), _stream(stream)), "cur_dmv_swap")


def cur_dmv_result(h, C_k, state, S_out=None, logvol_out=None, counts_out=None, stream=None) -> int:
    return _check(load().cur_dmv_result(h, ctypes.byref(mat(C_k)), _ptr(state), _ptr(S_out), _ptr(logvol_out),
                                        _ptr(counts_out), _stream(stream)), "cur_dmv_result")


def cur_merge_pair(h, rows, ids, o: CurOpts, ids_out, rows_out, swaps_out=None, stream=None) -> int:
    return _check(load().cur_merge_pair(h, ctypes.byref(mat(rows)), _ptr(ids), ctypes.byref(o), _ptr(ids_out),
                                        _ptr(rows_out), _ptr(swaps_out), _stream(stream)), "cur_merge_pair")


def cur_rows_at(h, X, offset: int, ids, count: int, out, stream=None) -> int:
    return _check(load().cur_rows_at(h, ctypes.byref(mat(X)), offset, _ptr(ids), count, _ptr(out),
                                     _stream(stream)), "cur_rows_at")


def cur_transpose(h, X, Xt_out, stream=None) -> int:
    return _check(load().cur_transpose(h, ctypes.byref(mat(X)), _ptr(Xt_out), _stream(stream)), "cur_transpose")


def cur_offset_ids(h, ids, count: int, offset: int, out, stream=None) -> int:
    return _check(load().cur_offset_ids(h, _ptr(ids), count, offset, _ptr(out), _stream(stream)), "cur_offset_ids")


def cur_gather_cols(h, A, J, r: int, C_out, stream=None) -> int:
    return _check(load().cur_gather_cols(h, ctypes.byref(mat(A)), _ptr(J), r, _ptr(C_out), _stream(stream)),
                  "cur_gather_cols")


def cur_residual_parts(h, A, C, U, R, r: int, parts_out, stream=None) -> int:
    return _check(load().cur_residual_parts(h, ctypes.byref(mat(A)), _ptr(C), _ptr(U), _ptr(R), r,
                                            _ptr(parts_out), _stream(stream)), "cur_residual_parts")


def cur_coef_tf32(h, basis, minv, B_out, stream=None) -> int:
    """B_out = basis minv on the tensor cores (3xTF32); basis p x r FP32, minv r x r FP64."""
    return _check(load().cur_coef_tf32(h, ctypes.byref(mat(basis)), _ptr(minv), _ptr(B_out), _stream(stream)),
                  "cur_coef_tf32")


def info_from_tensor(t) -> CurCrossInfo:
    """Decode a cur_cross_info written into a uint8 tensor (copied to the host)."""
    raw = bytes(t.cpu().numpy().tobytes())
    return CurCrossInfo.from_buffer_copy(raw[:ctypes.sizeof(CurCrossInfo)])


# ------------------------------------------------------------------ convenience

class Handle:
    """Owns a cur_handle and its workspace."""

    def __init__(self, m: int, n: int, r: int, dtype: int = CUR_F32, workspace_bytes: int = 0):
        size = workspace_bytes or cur_workspace_size(m, n, r, dtype)
        self.h = cur_create(size)

    def close(self):
        if self.h is not None:
            cur_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cross(A, r: int, b_r: int, b_c: int, delta: float = 1e-2, handle: Handle | None = None,
          stream=None):
    """Run cur_cross on a CUDA tensor; returns (I, J, info) with I, J int32 CUDA tensors."""
    import torch
    own = handle is None
    hd = handle or Handle(A.shape[0], A.shape[1], r, _dtype_code(A))
    try:
        I = torch.empty(r, dtype=torch.int32, device=A.device)
        J = torch.empty(r, dtype=torch.int32, device=A.device)
        info = torch.zeros(ctypes.sizeof(CurCrossInfo), dtype=torch.uint8, device=A.device)
        cur_cross(hd.h, A, r, b_r, b_c, opts(delta), I, J, info, stream)
        st = cur_sync_status(hd.h, stream)
        _check(st, "cur_cross (device)")
        return I, J, info_from_tensor(info)
    finally:
        if own:
            hd.close()


# ------------------------------------------------------------------ learned proposal

def mlp_param_count(k: int = 32, H: int = 256) -> int:
    """Length of the scoring network's parameter array: W1 (k x H), b1, w2, b2."""
    return k * H + 2 * H + 1


def cur_sketch(h, A, S, T, Y_out, Zt_out, normalize: bool = True, stream=None) -> int:
    """Y = A S (m x k) and Zt = A^T T (n x k); S: n x k, T: m x k, FP32 CUDA tensors."""
    return _check(load().cur_sketch(h, ctypes.byref(mat(A)), _ptr(S), _ptr(T), S.shape[1], _ptr(Y_out),
                                    _ptr(Zt_out), 1 if normalize else 0, _stream(stream)), "cur_sketch")


def cur_mlp_forward(h, X, params, scores_out, H: int = 256, stream=None) -> int:
    return _check(load().cur_mlp_forward(h, _ptr(X), X.shape[0], X.shape[1], H, _ptr(params),
                                         _ptr(scores_out), _stream(stream)), "cur_mlp_forward")


def cur_mlp_grad(h, X, y, params, grads_out, loss_out=None, idx=None, N=None, pos_weight: float = 1.0,
                 H: int = 256, stream=None) -> int:
    """Gradient over the samples idx[0..N) (all rows of X when idx is None)."""
    n = (X.shape[0] if idx is None else idx.shape[0]) if N is None else N
    return _check(load().cur_mlp_grad(h, _ptr(X), _ptr(y), X.shape[0], _ptr(idx), n, X.shape[1], H, _ptr(params),
                                      pos_weight, _ptr(grads_out), _ptr(loss_out), _stream(stream)),
                  "cur_mlp_grad")


def cur_adam_step(h, params, grads, m1, m2, t: int, lr: float = 1e-3, beta1: float = 0.9,
                  beta2: float = 0.999, eps: float = 1e-8, stream=None) -> int:
    return _check(load().cur_adam_step(h, _ptr(params), _ptr(grads), _ptr(m1), _ptr(m2), params.numel(), t,
                                       lr, beta1, beta2, eps, _stream(stream)), "cur_adam_step")


def cur_propose(h, scores, r: int, idx_out, stream=None) -> int:
    return _check(load().cur_propose(h, _ptr(scores), scores.numel(), r, _ptr(idx_out), _stream(stream)),
                  "cur_propose")


def cur_cross_from(h, A, r: int, I0, J0, o: CurOpts, I_out, J_out, info_out=None, stream=None) -> int:
    return _check(load().cur_cross_from(h, ctypes.byref(mat(A)), r, _ptr(I0), _ptr(J0), ctypes.byref(o),
                                        _ptr(I_out), _ptr(J_out), _ptr(info_out), _stream(stream)),
                  "cur_cross_from")


def cur_maxvol_global(h, basis, S0, r: int, o: CurOpts, S_out, logvol_out=None, swaps_out=None, stream=None) -> int:
    """Maxvol over all rows of basis (p x r CUDA tensor) from S0; swaps_out: 2 int32."""
    return _check(load().cur_maxvol_global(h, ctypes.byref(mat(basis)), _ptr(S0), r, ctypes.byref(o), _ptr(S_out),
                                           _ptr(logvol_out), _ptr(swaps_out), _stream(stream)), "cur_maxvol_global")
