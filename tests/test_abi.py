"""The C ABI library loads and exports every entry point include/minjoin.h
declares (no GPU needed: nothing is computed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "minjoin.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mj_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1810_08833_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("mj_create", "mj_join", "mj_partition", "mj_candidates", "mj_verify", "mj_join_host"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib_path):
    import paper_1810_08833_gb300 as mj
    assert set(declared_functions()) <= set(mj.exported_symbols())
    mj.library()


def test_binding_fails_loudly_without_library(tmp_path):
    import paper_1810_08833_gb300 as mj
    with pytest.raises(RuntimeError):
        mj._lib_backup = mj._lib
        try:
            mj._lib = None
            mj.library(str(tmp_path / "missing.so"))
        finally:
            mj._lib = mj._lib_backup


def test_strerror_without_device(lib_path):
    import paper_1810_08833_gb300 as mj
    lib = mj.library()
    assert lib.mj_strerror(0) == b"ok"
    assert lib.mj_strerror(-1) == b"invalid argument"
    h = ctypes.c_void_p()
    # no device here: creation fails with a status, never aborts
    st = lib.mj_create(ctypes.byref(h), 0)
    import torch
    if not torch.cuda.is_available():
        assert st != 0
    else:
        lib.mj_destroy(h)
