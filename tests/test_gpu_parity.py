"""Bit-exact parity of the CUDA path (through the C ABI) with the CPU oracle.

Every ciphertext limb, key limb and decrypted coefficient must be equal;
the arithmetic is exact modular integer arithmetic on both sides.  Inputs
are seeded: uniform ciphertexts and keys come from the ChaCha20 stream that
each side implements on its own, messages from workloads.py.
"""
import numpy as np
import pytest

import oracle
from paper_2503_22227_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2503_22227_gb300 import api  # noqa: E402

SEED = W.seed_for("parity-keys")


def octx_for(p: W.Preset):
    return oracle.Context(p.scheme, p.log_n, p.q_bits, p.p_bits, p.dnum, t=p.t,
                          log_n_max=p.log_n_max or p.log_n, b_bits=p.b_bits)


class Pair:
    """GPU context + keys and oracle context + keys for one preset."""

    def __init__(self, p: W.Preset, galois=()):
        self.p = p
        self.g = api.Context(p)
        self.o = octx_for(p)
        self.gk = self.g.keygen(SEED)
        self.ok = self.o.keygen(SEED)
        for e in galois:
            self.gk.gen_galois(e)
            self.ok.gen_galois(e)


SMALL_BGV = W.Preset("bgv_small", W.BGV, 12, (55,) * 4, (60,), 4, t=65537, log_n_max=12)
SMALL_BFV = W.Preset("bfv_small", W.BFV, 12, (55,) * 4, (60,), 4, t=65537, log_n_max=12)
CKKS_DIGITS = W.Preset("ckks_digits", W.CKKS, 12, (45,) * 5, (50, 50), 2, log_n_max=12)


@pytest.fixture(scope="module")
def ckks12():
    p = W.PRESETS["ckks_n12"]
    pr = Pair(p)
    for r in (1, -3):
        e = pr.g.galois_elt(r)
        pr.gk.gen_galois(e)
        pr.ok.gen_galois(e)
    conj = 2 * p.n - 1
    pr.gk.gen_galois(conj)
    pr.ok.gen_galois(conj)
    return pr


# ---------------------------------------------------------------- set-up

@pytest.mark.parametrize("name", list(W.PRESETS))
def test_prime_chains_match(name):
    p = W.PRESETS[name]
    g, o = api.Context(p), octx_for(p)
    assert (g.q, g.p, g.b) == (o.q, o.p, o.b)
    assert (g.alpha, g.beta) == (o.alpha, o.beta)


@pytest.mark.parametrize("log_n", [12, 13, 14, 15, 16])
def test_ntt_matches_oracle(log_n):
    p = W.Preset("ntt", W.CKKS, log_n, (50, 61, 40), (60,), 1, log_n_max=16)
    ctx = api.Context(p)
    rng = np.random.default_rng(log_n)
    count = 2
    host = W.uniform_residues(rng, ctx.q, (count,), ctx.n)     # [count][L][N]
    dev = torch.from_numpy(host.view(np.int64)).cuda()
    ctx.ntt(dev)
    got = dev.cpu().numpy().view(np.uint64)
    for c in range(count):
        for i, q in enumerate(ctx.q):
            psi = oracle.min_psi(q, log_n)
            assert np.array_equal(got[c, i], oracle.ntt(host[c, i], log_n, q, psi)), (c, i)
    ctx.ntt(dev, inverse=True)
    assert np.array_equal(dev.cpu().numpy().view(np.uint64), host)
    # edge values: all q-1, all zero, a single one
    edge = np.zeros((1, ctx.L, ctx.n), dtype=np.uint64)
    for i, q in enumerate(ctx.q):
        edge[0, i, :] = q - 1
    edge[0, 0, 5] = 0
    d = torch.from_numpy(edge.view(np.int64).copy()).cuda()
    ctx.ntt(d)
    got = d.cpu().numpy().view(np.uint64)
    for i, q in enumerate(ctx.q):
        assert np.array_equal(got[0, i], oracle.ntt(edge[0, i], log_n, q, oracle.min_psi(q, log_n)))


# ---------------------------------------------------------------- keys, encryption

@pytest.mark.parametrize("preset", [W.PRESETS["ckks_n12"], SMALL_BGV, SMALL_BFV, CKKS_DIGITS],
                         ids=lambda p: p.name)
def test_keys_match_oracle(preset):
    pr = Pair(preset)
    s, pk, ksk = pr.gk.export(0)
    assert np.array_equal(s, pr.ok.secret())
    assert np.array_equal(pk, pr.ok.public())
    assert np.array_equal(ksk, pr.ok.ksk(0))
    g = pr.g.galois_elt(2)
    pr.gk.gen_galois(g)
    pr.ok.gen_galois(g)
    assert np.array_equal(pr.gk.export(g, s=False, pk=False)[2], pr.ok.ksk(g))


@pytest.mark.parametrize("preset", [W.PRESETS["ckks_n12"], SMALL_BGV, SMALL_BFV],
                         ids=lambda p: p.name)
def test_encrypt_decrypt_match_oracle(preset):
    pr = Pair(preset)
    rng = W.rng_for("enc-" + preset.name)
    if preset.scheme == W.CKKS:
        msg = rng.integers(-2 ** 45, 2 ** 45, preset.n, dtype=np.int64)
    else:
        msg = W.int_messages(rng, preset.n, preset.t)
    es = W.seed_for("enc-seed-" + preset.name)
    ct = pr.g.encrypt(pr.gk, msg, es)
    want = pr.o.encrypt(pr.ok, msg, es)
    assert np.array_equal(pr.g.export_ct(ct)[0], want)
    dec = pr.g.decrypt(pr.gk, ct)
    assert np.array_equal(dec, pr.o.decrypt(pr.ok, want))
    if preset.scheme != W.CKKS:
        assert np.array_equal(dec, msg)


# ---------------------------------------------------------------- hot path, CKKS

def _uniform_pair(pr: Pair, level: int, count: int, tag: str):
    a = np.stack([pr.o.ct_uniform(W.seed_for(tag), 2 * i, level) for i in range(count)])
    b = np.stack([pr.o.ct_uniform(W.seed_for(tag), 2 * i + 1, level) for i in range(count)])
    return a, b


@pytest.mark.parametrize("level", [3, 2, 1])
def test_ckks_ops_match_oracle(ckks12, level):
    pr = ckks12
    a, b = _uniform_pair(pr, level, 3, f"ckks-ops-{level}")
    da, db = pr.g.import_ct(a), pr.g.import_ct(b)
    got = pr.g.export_ct(pr.g.mul_relin(pr.gk, da, db))
    for c in range(3):
        assert np.array_equal(got[c], pr.o.mul_relin(pr.ok, a[c], b[c])), c
    got = pr.g.export_ct(pr.g.add(da, db))
    for c in range(3):
        assert np.array_equal(got[c], pr.o.add(a[c], b[c]))
    for r in (1, -3):
        g = pr.g.galois_elt(r)
        got = pr.g.export_ct(pr.g.rotate(pr.gk, da, g))
        for c in range(3):
            assert np.array_equal(got[c], pr.o.rotate(pr.ok, a[c], g)), (r, c)
    conj = 2 * pr.p.n - 1
    got = pr.g.export_ct(pr.g.rotate(pr.gk, da, conj))
    assert np.array_equal(got[0], pr.o.rotate(pr.ok, a[0], conj))
    if level >= 2:
        got = pr.g.export_ct(pr.g.rescale(da))
        for c in range(3):
            assert np.array_equal(got[c], pr.o.rescale(a[c]))
        got = pr.g.export_ct(pr.g.mul_relin_rescale(pr.gk, da, db))
        for c in range(3):
            assert np.array_equal(got[c], pr.o.rescale(pr.o.mul_relin(pr.ok, a[c], b[c]))), c


@pytest.mark.parametrize("level", [5, 4, 3])
def test_ckks_multi_prime_digits_match_oracle(level):
    """alpha = 3 primes per digit and 2 special primes: partial last digits."""
    pr = Pair(CKKS_DIGITS, galois=(5,))
    a, b = _uniform_pair(pr, level, 2, f"digits-{level}")
    da, db = pr.g.import_ct(a), pr.g.import_ct(b)
    got = pr.g.export_ct(pr.g.mul_relin_rescale(pr.gk, da, db))
    for c in range(2):
        assert np.array_equal(got[c], pr.o.rescale(pr.o.mul_relin(pr.ok, a[c], b[c])))
    got = pr.g.export_ct(pr.g.rotate(pr.gk, da, 5))
    for c in range(2):
        assert np.array_equal(got[c], pr.o.rotate(pr.ok, a[c], 5))


def test_batched_equals_single(ckks12):
    pr = ckks12
    a, b = _uniform_pair(pr, 3, 5, "batch")
    da, db = pr.g.import_ct(a), pr.g.import_ct(b)
    batched = pr.g.export_ct(pr.g.mul_relin_rescale(pr.gk, da, db))
    for c in range(5):
        single = pr.g.export_ct(pr.g.mul_relin_rescale(pr.gk, da[c:c + 1], db[c:c + 1]))
        assert np.array_equal(batched[c], single[0])


def test_ckks_accuracy(ckks12):
    """Decrypted slots within 2^-20 of the product at scale 2^40."""
    pr = ckks12
    n, scale = pr.p.n, 2.0 ** 40
    rng = W.rng_for("gpu-ckks-accuracy")
    za, zb = W.complex_slots(rng, n), W.complex_slots(rng, n)
    ma, mb = oracle.encode_ckks(za, n, scale), oracle.encode_ckks(zb, n, scale)
    ca = pr.g.encrypt(pr.gk, ma, W.seed_for("acc-a"))
    cb = pr.g.encrypt(pr.gk, mb, W.seed_for("acc-b"))
    prod = pr.g.mul_relin_rescale(pr.gk, ca, cb)
    dec = pr.g.decrypt(pr.gk, prod)
    assert np.array_equal(dec, pr.o.decrypt(pr.ok, pr.g.export_ct(prod)[0]))
    z = oracle.decode_ckks(dec, n, scale * scale / pr.g.q[-1])
    assert np.max(np.abs(z - za * zb)) < 2.0 ** -20
    g = pr.g.galois_elt(1)
    z = oracle.decode_ckks(pr.g.decrypt(pr.gk, pr.g.rotate(pr.gk, ca, g)), n, scale)
    assert np.max(np.abs(z - np.roll(za, -1))) < 2.0 ** -20


@pytest.mark.parametrize("preset", [W.PRESETS["ckks_n12"], SMALL_BGV, SMALL_BFV],
                         ids=lambda p: p.name)
def test_elementwise_ops_match_oracle(preset):
    """sub, integer multiply, constant add (not BFV), level drop: direct
    calls and the same entries through an uneven batch, at a full and a
    lower level, with positive, negative and zero constants."""
    pr = Pair(preset)
    L = preset.L
    for level in (L, max(1, L - 1)):
        a, b = _uniform_pair(pr, level, 2, f"ew-{preset.name}-{level}")
        da, db = pr.g.import_ct(a), pr.g.import_ct(b)
        got = pr.g.export_ct(pr.g.sub(da, db))
        for c in range(2):
            assert np.array_equal(got[c], pr.o.sub(a[c], b[c]))
        for k in (0, 3, -(2 ** 40) - 7, 2 ** 62 + 11):
            got = pr.g.export_ct(pr.g.mul_int(da, k))
            for c in range(2):
                assert np.array_equal(got[c], pr.o.mul_int(a[c], k)), k
            if preset.scheme != W.BFV:
                got = pr.g.export_ct(pr.g.add_const(da, k))
                for c in range(2):
                    assert np.array_equal(got[c], pr.o.add_const(a[c], k)), k
        for nl in range(1, level + 1):
            got = pr.g.export_ct(pr.g.drop_level(da, nl))
            for c in range(2):
                assert np.array_equal(got[c], pr.o.drop(a[c], nl)), nl
        # the same through one batch
        entries, outs, wants = [], [], []
        kinds = [(api.OP_SUB, 0, level), (api.OP_MUL_INT, -12345, level),
                 (api.OP_DROP, 0, max(1, level - 1))]
        if preset.scheme != W.BFV:
            kinds.append((api.OP_ADD_CONST, 987654321, level))
        for kind, k, lo in kinds:
            out = pr.g.empty_ct(2, lo)
            entries.append(api.make_op(kind, pr.g, da, out, b=db if kind == api.OP_SUB else None,
                                       const=k))
            outs.append(out)
            if kind == api.OP_SUB:
                wants.append([pr.o.sub(a[c], b[c]) for c in range(2)])
            elif kind == api.OP_MUL_INT:
                wants.append([pr.o.mul_int(a[c], k) for c in range(2)])
            elif kind == api.OP_DROP:
                wants.append([pr.o.drop(a[c], lo) for c in range(2)])
            else:
                wants.append([pr.o.add_const(a[c], k) for c in range(2)])
        api.run_batch(entries, lanes=2)
        for out, want in zip(outs, wants):
            got = pr.g.export_ct(out)
            for c in range(2):
                assert np.array_equal(got[c], want[c])
    if preset.scheme == W.BFV:
        with pytest.raises(api.CatfheError) as e:
            pr.g.add_const(pr.g.import_ct(_uniform_pair(pr, L, 1, "ew-bfv")[0]), 1)
        assert e.value.code == -6     # ESCHEME


# ---------------------------------------------------------------- hot path, BGV / BFV

@pytest.mark.parametrize("preset", [SMALL_BGV, SMALL_BFV], ids=lambda p: p.name)
def test_integer_schemes_match_oracle(preset):
    g5 = None
    pr = Pair(preset)
    g5 = pr.g.galois_elt(1)
    pr.gk.gen_galois(g5)
    pr.ok.gen_galois(g5)
    level = preset.L
    a, b = _uniform_pair(pr, level, 2, "int-" + preset.name)
    da, db = pr.g.import_ct(a), pr.g.import_ct(b)
    got = pr.g.export_ct(pr.g.mul_relin(pr.gk, da, db))
    for c in range(2):
        assert np.array_equal(got[c], pr.o.mul_relin(pr.ok, a[c], b[c])), c
    got = pr.g.export_ct(pr.g.rotate(pr.gk, da, g5))
    for c in range(2):
        assert np.array_equal(got[c], pr.o.rotate(pr.ok, a[c], g5))
    if preset.scheme == W.BGV:
        got = pr.g.export_ct(pr.g.rescale(da))
        assert np.array_equal(got[0], pr.o.rescale(a[0]))
        # lower level: partial digit set
        a2, b2 = a[:, :, :level - 1].copy(), b[:, :, :level - 1].copy()
        got = pr.g.export_ct(pr.g.mul_relin(pr.gk, pr.g.import_ct(a2), pr.g.import_ct(b2)))
        assert np.array_equal(got[0], pr.o.mul_relin(pr.ok, a2[0], b2[0]))
    # decryption invariant on real encryptions
    rng = W.rng_for("inv-" + preset.name)
    ma, mb = W.int_messages(rng, preset.n, preset.t), W.int_messages(rng, preset.n, preset.t)
    ca = pr.g.encrypt(pr.gk, ma, W.seed_for("inv-a"))
    cb = pr.g.encrypt(pr.gk, mb, W.seed_for("inv-b"))
    prod = pr.g.decrypt(pr.gk, pr.g.mul_relin(pr.gk, ca, cb))
    n, t = preset.n, preset.t
    # negacyclic product mod t via the oracle-independent numpy route
    full = np.zeros(2 * n, dtype=object)
    A, B = [int(x) for x in ma], [int(x) for x in mb]
    conv = np.convolve(np.array(A, dtype=object), np.array(B, dtype=object))
    full[:len(conv)] = conv
    want = [(int(full[i]) - int(full[i + n])) % t for i in range(n)]
    assert [int(x) for x in prod] == want


@pytest.mark.parametrize("name", ["bfv_n14", "bgv_n14"])
def test_integer_schemes_full_size(name):
    """The N = 2^14, 8 x 55-bit chain, t = 65537 in the benchmark's launch
    configuration: one HMult+relin launch over the batch of 16 pairs (the
    benchmark's seeds and keys); the first and last outputs checked limb for
    limb against the oracle."""
    p = W.PRESETS[name]
    g_ctx, o_ctx = api.Context(p), octx_for(p)
    gk = g_ctx.keygen(W.seed_for("bench-keys-" + name))
    ok = o_ctx.keygen(W.seed_for("bench-keys-" + name))
    seed = W.seed_for("bench-inputs-" + name)
    x = torch.cat([g_ctx.ct_uniform(seed, 2 * i, p.L) for i in range(p.batch)])
    y = torch.cat([g_ctx.ct_uniform(seed, 2 * i + 1, p.L) for i in range(p.batch)])
    got = g_ctx.export_ct(g_ctx.mul_relin(gk, x, y))
    for i in (0, p.batch - 1):
        oa, ob = o_ctx.ct_uniform(seed, 2 * i, p.L), o_ctx.ct_uniform(seed, 2 * i + 1, p.L)
        assert np.array_equal(got[i], o_ctx.mul_relin(ok, oa, ob)), i


@pytest.mark.slow
def test_ckks_n16_full_size():
    """N = 2^16, L = 24, K = 4, dnum = 3 in the benchmark's launch
    configuration: the batch of 8 uniform pairs (the benchmark's seeds and
    keys) through one fused HMult+relin+rescale launch, and HRotate(1) on the
    batch; the first and last ciphertexts checked limb for limb against the
    oracle."""
    p = W.PRESETS["ckks_n16"]
    g_ctx, o_ctx = api.Context(p), octx_for(p)
    gk, ok = g_ctx.keygen(W.seed_for("bench-keys")), o_ctx.keygen(W.seed_for("bench-keys"))
    g = g_ctx.galois_elt(1)
    gk.gen_galois(g)
    ok.gen_galois(g)
    seed = W.seed_for("bench-inputs")
    a = torch.cat([g_ctx.ct_uniform(seed, 2 * i, p.L) for i in range(8)])
    b = torch.cat([g_ctx.ct_uniform(seed, 2 * i + 1, p.L) for i in range(8)])
    out = g_ctx.empty_ct(8, p.L - 1)
    g_ctx.mul_relin_rescale(gk, a, b, out)
    got = g_ctx.export_ct(out)
    rot = g_ctx.export_ct(g_ctx.rotate(gk, a, g))
    for i in (0, 7):
        oa, ob = o_ctx.ct_uniform(seed, 2 * i, p.L), o_ctx.ct_uniform(seed, 2 * i + 1, p.L)
        assert np.array_equal(got[i], o_ctx.rescale(o_ctx.mul_relin(ok, oa, ob))), i
        assert np.array_equal(rot[i], o_ctx.rotate(ok, oa, g)), i


def test_ckks_n16_noise_valid_accuracy():
    """K = 8 special primes: decrypted slots of the batched HMult+relin+rescale
    and of HRotate(1) within 2^-20 of the exact results, slots uniform in the
    complex unit square at scale 2^50."""
    from paper_2503_22227_gb300 import encoding
    p = W.PRESETS["ckks_n16_k8"]
    ctx = api.Context(p)
    keys = ctx.keygen(W.seed_for("k8-accuracy"))
    g = ctx.galois_elt(1)
    keys.gen_galois(g)
    n, scale = p.n, 2.0 ** 50
    rng = W.rng_for("k8-accuracy")
    zs = [(W.complex_slots(rng, n), W.complex_slots(rng, n)) for _ in range(4)]
    a = torch.cat([ctx.encrypt(keys, encoding.encode(za, n, scale), W.seed_for(f"k8a{i}"))
                   for i, (za, _) in enumerate(zs)])
    b = torch.cat([ctx.encrypt(keys, encoding.encode(zb, n, scale), W.seed_for(f"k8b{i}"))
                   for i, (_, zb) in enumerate(zs)])
    prod = ctx.mul_relin_rescale(keys, a, b)
    rot = ctx.rotate(keys, a, g)
    s2 = scale * scale / ctx.q[-1]
    for i, (za, zb) in enumerate(zs):
        z = encoding.decode(ctx.decrypt(keys, prod[i:i + 1]), n, s2)
        assert np.max(np.abs(z - za * zb)) < 2.0 ** -20, i
        z = encoding.decode(ctx.decrypt(keys, rot[i:i + 1]), n, scale)
        assert np.max(np.abs(z - np.roll(za, -1))) < 2.0 ** -20, i


# ---------------------------------------------------------------- errors and edges

def test_error_codes(ckks12):
    pr = ckks12
    a, b = _uniform_pair(pr, 1, 1, "errors")
    da = pr.g.import_ct(a)
    with pytest.raises(api.CatfheError) as e:
        pr.g.rescale(da)
    assert e.value.code == -2  # ELEVEL
    with pytest.raises(api.CatfheError) as e:
        pr.g.rotate(pr.gk, da, pr.g.galois_elt(7))
    assert e.value.code == -3  # ENOKEY
    lib = api.load()
    import ctypes
    out = pr.g.empty_ct(1, 1)
    rc = lib.catfhe_mul_relin(pr.g._h, pr.gk._h, ctypes.c_void_p(da.data_ptr()),
                              ctypes.c_void_p(da.data_ptr()), ctypes.c_void_p(out.data_ptr()), 1, 1,
                              ctypes.c_void_p(out.data_ptr()), 16, None)
    assert rc == -7  # EWORKSPACE
    # count = 0 is a no-op
    assert lib.catfhe_mul_relin(pr.g._h, pr.gk._h, ctypes.c_void_p(da.data_ptr()),
                                ctypes.c_void_p(da.data_ptr()), ctypes.c_void_p(out.data_ptr()), 1, 0,
                                None, 0, None) == 0
    bfv = api.Context(SMALL_BFV)
    x = bfv.empty_ct(1, 2)
    with pytest.raises(api.CatfheError) as e:
        bfv.rescale(x)
    assert e.value.code == -6  # ESCHEME


def test_async_import_export_round_trip(ckks12):
    pr = ckks12
    a, _ = _uniform_pair(pr, 3, 2, "async-io")
    host = torch.from_numpy(a.view(np.int64).copy()).pin_memory()
    dev = pr.g.import_ct(host, api.FORM_COEFF | api.FORM_ASYNC)
    back = torch.empty_like(host).pin_memory()
    pr.g.export_into(dev, back, api.FORM_NATIVE | api.FORM_ASYNC)
    native = torch.empty_like(host).pin_memory()
    pr.g.export_into(dev, native, api.FORM_NATIVE)
    torch.cuda.synchronize()
    assert torch.equal(back, native)
    dev2 = pr.g.import_ct(back, api.FORM_NATIVE | api.FORM_ASYNC)
    assert np.array_equal(pr.g.export_ct(dev2, api.FORM_COEFF), a)
    with pytest.raises(api.CatfheError) as e:
        pr.g.import_ct(host, api.FORM_NATIVE | 0x200)
    assert e.value.code == -1


@pytest.mark.parametrize("preset", [W.PRESETS["ckks_n12"], CKKS_DIGITS, SMALL_BGV],
                         ids=lambda p: p.name)
def test_hoisted_rotations_equal_single_rotations(preset):
    """One shared ModUp for several Galois elements (rotations by 1, -3, 5
    and the conjugation 2N-1): every output equals catfhe_rotate, and the
    first equals the oracle's rotation."""
    pr = Pair(preset)
    gs = [pr.g.galois_elt(r) for r in (1, -3, 5)] + [2 * preset.n - 1]
    for g in gs:
        pr.gk.gen_galois(g)
        pr.ok.gen_galois(g)
    for level in sorted({preset.L, max(1, preset.L - 2)}):
        a, _ = _uniform_pair(pr, level, 3, f"hoist-{preset.name}-{level}")
        da = pr.g.import_ct(a)
        out = pr.g.rotate_hoisted(pr.gk, da, gs)
        assert tuple(out.shape) == (len(gs), 3, 2, level, preset.n)
        for r, g in enumerate(gs):
            assert torch.equal(out[r], pr.g.rotate(pr.gk, da, g)), (level, g)
        got = pr.g.export_ct(out[0])
        assert np.array_equal(got[1], pr.o.rotate(pr.ok, a[1], gs[0]))


def test_hoisted_rotation_errors(ckks12):
    pr = ckks12
    a, _ = _uniform_pair(pr, 3, 1, "hoist-err")
    da = pr.g.import_ct(a)
    with pytest.raises(api.CatfheError) as e:      # no key for 7 steps, nothing enqueued
        pr.g.rotate_hoisted(pr.gk, da, [pr.g.galois_elt(1), pr.g.galois_elt(7)])
    assert e.value.code == -3
    with pytest.raises(api.CatfheError) as e:
        pr.g.rotate_hoisted(pr.gk, da, [4])
    assert e.value.code == -1
    empty = pr.g.rotate_hoisted(pr.gk, da, [])
    assert empty.shape[0] == 0
    bfv = Pair(SMALL_BFV)
    b, _ = _uniform_pair(bfv, SMALL_BFV.L, 1, "hoist-bfv")
    with pytest.raises(api.CatfheError) as e:
        bfv.g.rotate_hoisted(bfv.gk, bfv.g.import_ct(b), [bfv.g.galois_elt(1)])
    assert e.value.code == -6


@pytest.mark.parametrize("preset", [W.PRESETS["ckks_n12"], SMALL_BGV, SMALL_BFV],
                         ids=lambda p: p.name)
def test_mul_plain_matches_oracle(preset):
    pr = Pair(preset)
    rng = np.random.default_rng(41)
    pt = rng.integers(-2 ** 40, 2 ** 40, preset.n)
    for level in sorted({preset.L, max(1, preset.L - 1)}):
        a, _ = _uniform_pair(pr, level, 2, f"mulplain-{preset.name}-{level}")
        da = pr.g.import_ct(a)
        dpt = pr.g.plain_import(pt, level)
        got = pr.g.export_ct(pr.g.mul_plain(da, dpt))
        for c in range(2):
            assert np.array_equal(got[c], pr.o.mul_plain(a[c], pt)), (level, c)
        out = pr.g.empty_ct(2, level)
        api.run_batch([api.make_op(api.OP_MUL_PLAIN, pr.g, da, out, b=dpt)], lanes=1)
        assert np.array_equal(pr.g.export_ct(out), got)
        # out aliasing a
        pr.g.mul_plain(da, dpt, da)
        assert np.array_equal(pr.g.export_ct(da), got)


def test_zero_count_is_a_noop(ckks12):
    """count = 0 with valid buffers enqueues nothing and leaves out untouched."""
    import ctypes
    pr = ckks12
    L = api.load()
    a = pr.g.ct_uniform(W.seed_for("zero"), 0, 3)
    out = torch.full_like(a, 7)
    ws = pr.g.workspace(api.OP_MUL_RELIN_RESCALE, 3, 1)
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    h, kh = pr.g._h, pr.gk._h
    g = pr.g.galois_elt(1)
    rcs = [
        L.catfhe_mul_relin(h, kh, P(a), P(a), P(out), 3, 0, P(ws), ws.numel(), s),
        L.catfhe_mul_relin_rescale(h, kh, P(a), P(a), P(out), 3, 0, P(ws), ws.numel(), s),
        L.catfhe_rotate(h, kh, P(a), g, P(out), 3, 0, P(ws), ws.numel(), s),
        L.catfhe_rescale(h, P(a), P(out), 3, 0, P(ws), ws.numel(), s),
        L.catfhe_add(h, P(a), P(a), P(out), 3, 0, s),
        L.catfhe_sub(h, P(a), P(a), P(out), 3, 0, s),
        L.catfhe_mul_int(h, P(a), 5, P(out), 3, 0, s),
        L.catfhe_add_const(h, P(a), 5, P(out), 3, 0, s),
        L.catfhe_drop_level(h, P(a), 3, 2, P(out), 0, s),
        L.catfhe_mul_plain(h, P(a), P(a), P(out), 3, 0, s),
    ]
    assert rcs == [0] * len(rcs)
    torch.cuda.synchronize()
    assert bool((out == 7).all())


def test_split_and_alternating_paths_equal_single_calls():
    """N = 2^14: key switching on 5 ciphertexts runs as halves of 3 and 2 on
    two streams, and hoisted rotations alternate over two streams; every
    output must equal the single-ciphertext (unsplit) call."""
    p = W.Preset("ckks_n14_small", W.CKKS, 14, (50,) * 6, (60, 60), 3, log_n_max=14)
    ctx = api.Context(p)
    keys = ctx.keygen(W.seed_for("split-keys"))
    gs = [ctx.galois_elt(r) for r in (1, 2, -5)] + [2 * p.n - 1]
    for g in gs:
        keys.gen_galois(g)
    seed = W.seed_for("split-in")
    a = torch.cat([ctx.ct_uniform(seed, 2 * i, p.L) for i in range(5)])
    b = torch.cat([ctx.ct_uniform(seed, 2 * i + 1, p.L) for i in range(5)])
    for fused in (False, True):
        whole = ctx.mul_relin_rescale(keys, a, b) if fused else ctx.mul_relin(keys, a, b)
        for i in range(5):
            one = (ctx.mul_relin_rescale(keys, a[i:i + 1], b[i:i + 1]) if fused
                   else ctx.mul_relin(keys, a[i:i + 1], b[i:i + 1]))
            assert torch.equal(whole[i:i + 1], one), (fused, i)
    rot = ctx.rotate(keys, a, gs[0])
    for i in range(5):
        assert torch.equal(rot[i:i + 1], ctx.rotate(keys, a[i:i + 1], gs[0])), i
    hoisted = ctx.rotate_hoisted(keys, a[:2], gs)
    for r, g in enumerate(gs):
        assert torch.equal(hoisted[r], ctx.rotate(keys, a[:2], g)), g


# ---------------------------------------------------------------- conversion layouts at the edges
# The key-switching presets above keep digits of at most 8 primes below 2^60,
# so their exact conversions run in the split-weight Montgomery layout.  These
# reach the other layouts and the largest sizes:
#  - 12 primes per digit: Montgomery constants without split weights;
#  - 32 primes in one digit (the most a context holds);
#  - 61-bit primes: ModUp's constants no longer sum below 2^64, so the
#    exact layout (128-bit sums reduced by Shoup products) runs; ModDown's
#    three 61-bit sources stay in the Montgomery layout.
EDGE_PRESETS = [
    W.Preset("ckks_wide_digit", W.CKKS, 12, (50,) * 12, (60, 60), 1, log_n_max=12),
    W.Preset("ckks_max_l", W.CKKS, 12, (40,) * 32, (50, 50), 1, log_n_max=12),
    W.Preset("ckks_61bit", W.CKKS, 12, (61,) * 10, (61, 61), 1, log_n_max=12),
]


@pytest.mark.parametrize("preset", EDGE_PRESETS, ids=lambda p: p.name)
def test_conversion_layouts_at_the_edges_match_oracle(preset):
    pr = Pair(preset, galois=(5,))
    L = preset.L
    for level in (L, L - 1, 2):
        a, b = _uniform_pair(pr, level, 2, f"edge-{preset.name}-{level}")
        da, db = pr.g.import_ct(a), pr.g.import_ct(b)
        got = pr.g.export_ct(pr.g.mul_relin(pr.gk, da, db))
        want = [pr.o.mul_relin(pr.ok, a[c], b[c]) for c in range(2)]
        for c in range(2):
            assert np.array_equal(got[c], want[c]), (level, c)
        got = pr.g.export_ct(pr.g.mul_relin_rescale(pr.gk, da, db))
        for c in range(2):
            assert np.array_equal(got[c], pr.o.rescale(want[c])), (level, c)
        got = pr.g.export_ct(pr.g.rotate(pr.gk, da, 5))
        for c in range(2):
            assert np.array_equal(got[c], pr.o.rotate(pr.ok, a[c], 5)), (level, c)
