"""The C ABI library builds, loads and exports what include/cur.h declares (CPU only:
no call here touches a GPU)."""
import os
import re
import subprocess

import pytest

import paper_2502_11017_gb300 as cur

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(cur.LIB_PATH):
        cur.build()
    return cur.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "cur.h")).read()
    return sorted(set(re.findall(r"^\s*(?:cur_status|size_t|cur_opts|const char\*)\s+(cur_\w+)\s*\(",
                                 text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("cur_maxvol_rows", "cur_maxvol_cols", "cur_merge", "cur_assemble",
                 "cur_residual_cheb", "cur_aca_select", "cur_cross", "cur_create",
                 "cur_destroy", "cur_sync_status", "cur_status_string"):
        assert must in names
    assert sorted(cur.EXPORTS) == names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", cur.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(cur_\w+)$", out, flags=re.M))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)


def test_host_only_calls(lib):
    o = lib.cur_default_opts()
    assert o.delta == pytest.approx(1e-2)
    assert o.flags & cur.CUR_FLAG_POLISH
    assert o.nblocks == 1
    assert lib.cur_status_string(cur.CUR_ERR_SINGULAR) == b"singular submatrix"
    assert lib.cur_status_string(cur.CUR_OK) == b"ok"
    small = lib.cur_workspace_size(100, 80, 8, cur.CUR_F32)
    big = lib.cur_workspace_size(65536, 8192, 64, cur.CUR_F32)
    assert 0 < small < big
    assert lib.cur_workspace_size(0, 10, 4, cur.CUR_F32) == 0


def test_null_arguments_are_rejected_without_a_device(lib):
    import ctypes
    assert lib.cur_create(None, 0) == cur.CUR_ERR_ARG
    assert lib.cur_destroy(None) == cur.CUR_ERR_ARG
    assert lib.cur_aca_select(None, None, 1, 4, 1, None, None) == cur.CUR_ERR_ARG
    assert lib.cur_cross(None, None, 4, 1, 1, None, None, None, None, None) == cur.CUR_ERR_ARG
    assert lib.cur_sync_status(None, None) == cur.CUR_ERR_ARG
    m = cur.CurMat(ctypes.c_void_p(16), 10, 10, 5, cur.CUR_F32)   # ld < cols
    assert lib.cur_maxvol_rows(ctypes.c_void_p(1), ctypes.byref(m), ctypes.c_void_p(16), 2,
                               None, ctypes.c_void_p(16), None, None, None) == cur.CUR_ERR_ARG


def test_binding_fails_loudly_without_library(tmp_path):
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        saved = cur._lib
        cur._lib = None
        try:
            cur.load(str(tmp_path / "missing.so"))
        finally:
            cur._lib = saved
