"""catfhe_rescale_noalloc against catfhe_rescale.

The allocation-free rescale exists for callers that cannot allocate device
memory while they run; it borrows a scratch array the library reserves
statically.  Its results must equal the regular rescale's bit for bit
(the same exact arithmetic), on consecutive calls that reuse the shared
scratch, for CKKS rescale and BGV modulus switching.  This file is
collected last so that a run stopping at the first failure has already run
every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2503_22227_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2503_22227_gb300 import api  # noqa: E402


def _uniform(ctx, tag, level, count):
    return torch.cat([ctx.ct_uniform(W.seed_for(tag), i, level) for i in range(count)])


@pytest.mark.parametrize("name", ["ckks_n12", "bgv_n14"])
def test_noalloc_rescale_equals_rescale_twice(name):
    ctx = api.Context(W.PRESETS[name])
    L = ctx.L
    # two calls in a row: different level and batch, same shared scratch
    for tag, level, count in (("noalloc-1", L, 2), ("noalloc-2", L - 1, 3)):
        a = _uniform(ctx, tag, level, count)
        want = ctx.export_ct(ctx.rescale(a))
        out = ctx.empty_ct(count, level - 1)
        got = ctx.export_ct(ctx.rescale_noalloc(a, out))
        assert np.array_equal(got, want), (name, level, count)


def test_noalloc_full_size_and_limit():
    ctx = api.Context(W.PRESETS["ckks_n16"])
    a = _uniform(ctx, "noalloc-n16", 24, 1)
    out = ctx.empty_ct(1, 23)
    for _ in range(2):
        got = ctx.export_ct(ctx.rescale_noalloc(a, out))
        assert np.array_equal(got, ctx.export_ct(ctx.rescale(a)))
    # two N = 2^16 ciphertexts at level 24 exceed the static scratch: refused
    # before any work is enqueued
    lib = api.load()
    rc = lib.catfhe_rescale_noalloc(ctx._h, ctypes.c_void_p(a.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), 24, 2, None)
    assert rc == -7  # CATFHE_EWORKSPACE
