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
    assert lib.catfhe_strerror(-8) == b"a kernel's bounded wait timed out"
    lib.catfhe_sync.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.catfhe_sync(None, None) == -1
    # argument checks happen before any CUDA call
    lib.catfhe_ctx_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.catfhe_ctx_create(None, None) == -1
    lib.catfhe_workspace_bytes.restype = ctypes.c_size_t
    lib.catfhe_workspace_bytes.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32,
                                           ctypes.c_uint32]
    assert lib.catfhe_workspace_bytes(None, 1, 3, 1) == 0


def _params(**kw):
    from paper_2503_22227_gb300 import api, workloads as W
    p = api.params_from_preset(W.PRESETS["ckks_n12"])
    for k, v in kw.items():
        if k == "q_bits0":
            p.q_bits[0] = v
        elif k == "p_bits0":
            p.p_bits[0] = v
        else:
            setattr(p, k, v)
    return p


@pytest.mark.parametrize("bad", [
    dict(scheme=3), dict(scheme=-1), dict(log_n=11), dict(log_n=17), dict(log_n_max=11),
    dict(log_n_max=21), dict(L=0), dict(L=33), dict(K=0), dict(K=16), dict(dnum=0), dict(dnum=4),
    dict(q_bits0=19), dict(q_bits0=62), dict(p_bits0=19), dict(p_bits0=62),
    dict(scheme=1, t=2), dict(scheme=2, t=65536), dict(scheme=1, t=1 << 61),
])
def test_context_parameters_rejected_before_any_device_call(lib, bad):
    """Invalid parameter sets return CATFHE_EINVAL from the host checks, so
    this runs without a GPU."""
    import ctypes as C
    p = _params(**bad)
    h = C.c_void_p()
    lib.catfhe_ctx_create.argtypes = [C.c_void_p, C.c_void_p]
    assert lib.catfhe_ctx_create(C.byref(p), C.byref(h)) == -1
    assert not h.value


def test_null_handles_rejected(lib):
    import ctypes as C
    vp = C.c_void_p
    lib.catfhe_add.argtypes = [vp, vp, vp, vp, C.c_uint32, C.c_uint32, vp]
    assert lib.catfhe_add(None, None, None, None, 1, 1, None) == -1
    lib.catfhe_rotate_hoisted.argtypes = [vp, vp, vp, vp, C.c_uint32, vp, C.c_uint32, C.c_uint32,
                                          vp, C.c_size_t, vp]
    assert lib.catfhe_rotate_hoisted(None, None, None, None, 0, None, 1, 1, None, 0, None) == -1
    lib.catfhe_run_batch.argtypes = [vp, C.c_uint32, C.c_uint32, vp, C.c_size_t, vp]
    assert lib.catfhe_run_batch(None, 0, 1, None, 0, None) == -1
    lib.catfhe_batch_workspace_bytes.restype = C.c_size_t
    lib.catfhe_batch_workspace_bytes.argtypes = [vp, C.c_uint32, C.c_uint32]
    assert lib.catfhe_batch_workspace_bytes(None, 0, 1) == 0
