"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every function include/catfhe.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "catfhe.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(catfhe_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2503_22227_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_exports_every_declared_symbol(lib):
    names = header_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_2503_22227_gb300 import api
    assert sorted(api.EXPORTS) == header_functions()


def test_strerror_and_null_arguments(lib):
    lib.catfhe_strerror.restype = ctypes.c_char_p
    assert lib.catfhe_strerror(0) == b"ok"
    assert lib.catfhe_strerror(-3) == b"key-switching key missing"
    # argument checks happen before any CUDA call
    lib.catfhe_ctx_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.catfhe_ctx_create(None, None) == -1
    lib.catfhe_workspace_bytes.restype = ctypes.c_size_t
    lib.catfhe_workspace_bytes.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32,
                                           ctypes.c_uint32]
    assert lib.catfhe_workspace_bytes(None, 1, 3, 1) == 0
