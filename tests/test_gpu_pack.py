"""The bit-packed transfer form on the device: catfhe_ct_import_packed of the
host codec's words equals the native (at-rest) import, catfhe_ct_export_packed
decodes to the native export, bit for bit; at the end-to-end workload's size
(8 ciphertexts, N = 2^16, level 24) and at N = 2^12 with mixed prime sizes."""
import numpy as np
import pytest

from paper_2503_22227_gb300 import api, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

MIXED = W.Preset("pack_mixed", W.CKKS, 12, (40, 50, 61, 33), (60,), 2, log_n_max=12)


@pytest.mark.parametrize("preset,count,level", [(MIXED, 3, 4), (MIXED, 2, 2),
                                                (W.PRESETS["ckks_n16"], 8, 24)],
                         ids=["mixed-l4", "mixed-l2", "n16-l24"])
def test_packed_transfers_equal_native(preset, count, level):
    ctx = api.Context(preset)
    seed = W.seed_for(f"pack-{preset.name}")
    ct = torch.cat([ctx.ct_uniform(seed, i, level) for i in range(count)])
    native = ctx.export_ct(ct, api.FORM_NATIVE)
    packed = ctx.pack(native)
    words = ctx.packed_words(level, count)
    assert packed.size == words == 2 * count * sum(preset.n * int(b) // 64
                                                   for b in ctx.bits(level))
    # host -> device
    ws = torch.empty(words, dtype=torch.int64, device="cuda")
    got = ctx.import_packed(packed, level, count, ws=ws)
    assert torch.equal(got, ct)
    # pinned host buffer and the asynchronous flag
    hp = torch.from_numpy(packed.view(np.int64)).pin_memory()
    got2 = ctx.import_packed(hp, level, count, ws=ws, flags=api.FORM_ASYNC)
    torch.cuda.synchronize()
    assert torch.equal(got2, ct)
    # device -> host
    back = ctx.export_packed(ct, ws=ws)
    assert np.array_equal(back, packed)
    assert np.array_equal(ctx.unpack(back, count, level), native)
    # too small a workspace is refused
    with pytest.raises(api.CatfheError):
        ctx.import_packed(packed, level, count, ws=ws[: words - 1])


def test_unpack_reduces_out_of_range_fields():
    ctx = api.Context(MIXED)
    level, count = 4, 1
    bits = ctx.bits(level)
    ones = np.full((count, 2, level, MIXED.n), 2 ** 64 - 1, dtype=np.uint64)
    packed = ctx.pack(ones)                      # every field all ones
    got = ctx.export_ct(ctx.import_packed(packed, level, count), api.FORM_NATIVE)
    for i, (b, q) in enumerate(zip(bits, ctx.q)):
        want = (1 << int(b)) - 1 - int(q)
        assert 0 <= want < int(q)
        assert (got[:, :, i] == np.uint64(want)).all(), i


def test_zero_count_is_a_noop():
    ctx = api.Context(MIXED)
    out = torch.full((1, 2, 4, MIXED.n), 7, dtype=torch.int64, device="cuda")
    packed = np.zeros(16, dtype=np.uint64)
    ctx.import_packed(packed, 4, 0, out=out)
    torch.cuda.synchronize()
    assert bool((out == 7).all())


def test_misaligned_workspace_is_refused_before_any_launch():
    """A workspace pointer that is not 16-byte aligned is refused on the host
    (EINVAL) by the packed transfers, the key-switching calls and batches;
    nothing is enqueued and the output is untouched."""
    ctx = api.Context(MIXED)
    keys = ctx.keygen(W.seed_for("pack-ws"))
    a = ctx.ct_uniform(W.seed_for("pack-ws"), 0, 4)
    out = torch.full_like(a, 7)
    raw = torch.empty(1 << 24, dtype=torch.uint8, device="cuda")
    bad = raw[8:]
    packed = ctx.pack(ctx.export_ct(a, api.FORM_NATIVE))
    with pytest.raises(api.CatfheError) as e:
        ctx.import_packed(packed, 4, 1, out=out, ws=bad)
    assert e.value.code == -1
    import ctypes
    L = api.load()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.catfhe_mul_relin(ctx._h, keys._h, ctypes.c_void_p(a.data_ptr()),
                            ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(out.data_ptr()), 4, 1,
                            ctypes.c_void_p(bad.data_ptr()), bad.numel(), s)
    assert rc == -1
    with pytest.raises(api.CatfheError) as e:
        api.run_batch([api.make_op(api.OP_ADD, ctx, a, out, b=a)], lanes=1, ws=bad)
    assert e.value.code == -1
    torch.cuda.synchronize()
    assert bool((out == 7).all())


def test_misaligned_ciphertext_buffers_are_refused():
    """Ciphertext buffers must be 16-byte aligned (kernels move 16-byte words):
    a view that starts one word into an allocation is refused with EINVAL by
    single calls and by batch entries, before anything is enqueued."""
    ctx = api.Context(MIXED)
    keys = ctx.keygen(W.seed_for("pack-align"))
    a = ctx.ct_uniform(W.seed_for("pack-align"), 0, 4)
    flat = torch.empty(a.numel() + 2, dtype=torch.int64, device="cuda")
    shifted = flat[1:1 + a.numel()].view(a.shape)
    shifted.copy_(a)
    out = torch.full_like(a, 7)
    for call in (lambda: ctx.mul_relin(keys, shifted, a, out),
                 lambda: ctx.add(shifted, a, out),
                 lambda: ctx.rescale(shifted, out[:, :, :3].contiguous())):
        with pytest.raises(api.CatfheError) as e:
            call()
        assert e.value.code == -1
    with pytest.raises(api.CatfheError) as e:
        api.run_batch([api.make_op(api.OP_ADD, ctx, shifted, out, b=a)], lanes=1)
    assert e.value.code == -1
    torch.cuda.synchronize()
    assert bool((out == 7).all())
