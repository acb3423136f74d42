"""CKKS encoding and decoding on the device against the host encoder
(`encoding.py`, itself pinned against the O(N^2) definition): the device
plaintext's coefficients equal the host's up to a rounding tie (float64
operation order differs), decoded slots match within 2^-20, and a
device-encoded plaintext multiplies into a ciphertext as expected."""
import numpy as np
import pytest

from paper_2503_22227_gb300 import encoding, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2503_22227_gb300 import api  # noqa: E402


def _centred(r, q):
    r = r.astype(object)
    return np.array([int(x) - q if 2 * int(x) > q else int(x) for x in r], dtype=object)


@pytest.mark.parametrize("name,log_scale", [("ckks_n12", 40), ("ckks_n16_k8", 50)])
def test_encode_matches_host_and_decode_round_trips(name, log_scale):
    p = W.PRESETS[name]
    ctx = api.Context(p)
    keys = ctx.keygen(W.seed_for("enc-keys-" + name))
    n, scale = p.n, 2.0 ** log_scale
    rng = W.rng_for("enc-" + name)
    z = W.complex_slots(rng, n)
    pt = ctx.encode_ckks(z, scale)
    coeff = pt.clone().reshape(1, ctx.L, n)
    ctx.ntt(coeff, inverse=True)
    got = _centred(coeff[0, 0].cpu().numpy().view(np.uint64), ctx.q[0])
    want = encoding.encode(z, n, scale).astype(object)
    diff = np.abs((got - want).astype(np.int64))
    assert diff.max() <= 1 and np.mean(diff == 0) > 0.99
    # every limb holds the same integers
    for i in range(1, ctx.L):
        assert np.array_equal(_centred(coeff[0, i].cpu().numpy().view(np.uint64), ctx.q[i]), got)
    # decode of a real encryption
    ct = ctx.encrypt(keys, encoding.encode(z, n, scale), W.seed_for("enc-ct-" + name))
    dec = ctx.decode_ckks(keys, ct, scale)
    assert np.max(np.abs(dec - z)) < 2.0 ** -20
    host = encoding.decode(ctx.decrypt(keys, ct), n, scale)
    assert np.max(np.abs(dec - host)) < 2.0 ** -30


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
