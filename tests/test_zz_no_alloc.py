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
    """N = 2^16: the scratch holds 16 KiB + 16 count level N bytes of at most
    32 MiB, so count * level <= 31.  Calls at the limit run and equal
    catfhe_rescale; calls one step past it are refused before any launch."""
    ctx = api.Context(W.PRESETS["ckks_n16"])
    lib = api.load()
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    for count, level in ((1, 24), (2, 15)):
        a = _uniform(ctx, f"noalloc-n16-{count}", level, count)
        out = ctx.empty_ct(count, level - 1)
        for _ in range(2):
            got = ctx.export_ct(ctx.rescale_noalloc(a, out))
            assert np.array_equal(got, ctx.export_ct(ctx.rescale(a))), (count, level)
    a = _uniform(ctx, "noalloc-n16-big", 24, 2)
    out = ctx.empty_ct(2, 23)
    keep = out.clone()
    for count, level in ((2, 16), (3, 11), (2, 24)):
        rc = lib.catfhe_rescale_noalloc(ctx._h, P(a), P(out), level, count, None)
        assert rc == -7, (count, level)  # CATFHE_EWORKSPACE
    torch.cuda.synchronize()
    assert torch.equal(out, keep)        # nothing was written


def test_noalloc_refuses_overlap():
    """The output may not overlap the input: in place, or shifted by a limb."""
    ctx = api.Context(W.PRESETS["ckks_n12"])
    lib = api.load()
    a = _uniform(ctx, "noalloc-overlap", 3, 2)
    P = lambda p: ctypes.c_void_p(p)
    base = a.data_ptr()
    assert lib.catfhe_rescale_noalloc(ctx._h, P(base), P(base), 3, 2, None) == -1
    assert lib.catfhe_rescale_noalloc(ctx._h, P(base), P(base + 8 * ctx.n), 3, 2, None) == -1
