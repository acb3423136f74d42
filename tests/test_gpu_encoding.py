"""CKKS encoding and decoding on the device against the oracle's canonical
embedding (`oracle.encode_ckks` / `oracle.decode_ckks`, evaluated directly
at the slot roots, O(N^2)): the device plaintext's coefficients equal the
oracle's up to a rounding tie (float64 operation order differs: |diff| <= 1,
almost all equal), every limb holds the same integers, and decoded slots
match the oracle's decode of the oracle's decryption within 2^-30 and the
message within 2^-20.  At N = 2^16 (too large for the O(N^2) oracle) the
device is compared with the host FFT encoder, itself tied to the oracle
at N = 2^11 on the CPU."""
import numpy as np
import pytest

import oracle
from paper_2503_22227_gb300 import encoding, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2503_22227_gb300 import api  # noqa: E402


def _centred(r, q):
    r = r.astype(object)
    return np.array([int(x) - q if 2 * int(x) > q else int(x) for x in r], dtype=object)


def _device_coeffs(ctx, pt):
    coeff = pt.clone().reshape(1, ctx.L, ctx.n)
    ctx.ntt(coeff, inverse=True)
    limbs = coeff[0].cpu().numpy().view(np.uint64)
    first = _centred(limbs[0], ctx.q[0])
    for i in range(1, ctx.L):
        assert np.array_equal(_centred(limbs[i], ctx.q[i]), first), i
    return first


def test_encode_decode_match_oracle():
    p = W.PRESETS["ckks_n12"]
    ctx = api.Context(p)
    octx = oracle.Context(p.scheme, p.log_n, p.q_bits, p.p_bits, p.dnum, log_n_max=p.log_n)
    seed_k = W.seed_for("enc-keys-oracle")
    keys, okeys = ctx.keygen(seed_k), octx.keygen(seed_k)
    n, scale = p.n, 2.0 ** 40
    z = W.complex_slots(W.rng_for("enc-oracle"), n)
    got = _device_coeffs(ctx, ctx.encode_ckks(z, scale))
    want = oracle.encode_ckks(z, n, scale).astype(object)
    diff = np.abs((got - want).astype(np.int64))
    assert diff.max() <= 1 and np.mean(diff == 0) > 0.98
    # decode: the device decrypts and decodes; the oracle decrypts the same
    # ciphertext and evaluates the embedding directly
    m = oracle.encode_ckks(z, n, scale)
    ct = ctx.encrypt(keys, m, W.seed_for("enc-oracle-ct"))
    dec = ctx.decode_ckks(keys, ct, scale)
    ref = oracle.decode_ckks(octx.decrypt(okeys, ctx.export_ct(ct)[0]), n, scale)
    assert np.max(np.abs(dec - ref)) < 2.0 ** -30
    assert np.max(np.abs(dec - z)) < 2.0 ** -20
    # special inputs: all-zero slots encode to zero; a constant to a constant
    # (|0.375 scale| < q_i / 2 for these 40-bit primes, so every limb centres
    # to the same integer)
    assert not _device_coeffs(ctx, ctx.encode_ckks(np.zeros(n // 2, complex), scale)).any()
    c = _device_coeffs(ctx, ctx.encode_ckks(np.full(n // 2, -0.375 + 0j), scale))
    assert c[0] == oracle.encode_ckks(np.full(n // 2, -0.375 + 0j), n, scale)[0]
    assert not c[1:].any()


def test_encode_full_size_matches_host_and_round_trips():
    p = W.PRESETS["ckks_n16_k8"]
    ctx = api.Context(p)
    keys = ctx.keygen(W.seed_for("enc-keys-" + p.name))
    n, scale = p.n, 2.0 ** 50
    z = W.complex_slots(W.rng_for("enc-" + p.name), n)
    got = _device_coeffs(ctx, ctx.encode_ckks(z, scale))
    want = encoding.encode(z, n, scale).astype(object)
    diff = np.abs((got - want).astype(np.int64))
    assert diff.max() <= 1 and np.mean(diff == 0) > 0.99
    ct = ctx.encrypt(keys, encoding.encode(z, n, scale), W.seed_for("enc-ct-" + p.name))
    dec = ctx.decode_ckks(keys, ct, scale)
    assert np.max(np.abs(dec - z)) < 2.0 ** -20


def test_device_plaintext_product():
    p = W.PRESETS["ckks_n12"]
    ctx = api.Context(p)
    keys = ctx.keygen(W.seed_for("enc-mul"))
    n, scale = p.n, 2.0 ** 40
    rng = W.rng_for("enc-mul")
    z1, z2 = W.complex_slots(rng, n), W.complex_slots(rng, n)
    ct = ctx.encrypt(keys, encoding.encode(z1, n, scale), W.seed_for("enc-mul-ct"))
    prod = ctx.rescale(ctx.mul_plain(ct, ctx.encode_ckks(z2, scale)))
    dec = ctx.decode_ckks(keys, prod, scale * scale / ctx.q[-1])
    assert np.max(np.abs(dec - z1 * z2)) < 2.0 ** -20


def test_encode_decode_errors():
    bfv = api.Context(W.PRESETS["bfv_n14"])
    with pytest.raises(api.CatfheError) as e:
        bfv.encode_ckks(np.zeros(bfv.n // 2), 2.0 ** 20)
    assert e.value.code == -6
    ctx = api.Context(W.PRESETS["ckks_n12"])
    with pytest.raises(api.CatfheError) as e:
        ctx.encode_ckks(np.zeros(ctx.n // 2), 0.0)
    assert e.value.code == -1
