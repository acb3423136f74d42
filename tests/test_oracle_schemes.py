"""Pins of the oracle's schemes by their defining invariants:
keys decrypt to small errors, Dec(Enc(m)) = m, Dec(HMult(Enc a, Enc b)) =
a b mod t (BFV, BGV, exact) and ~ a b for CKKS, rotations permute slots,
rescale / modulus switch keep the message, key switching leaves a small
error (checked with Python big integers)."""
import numpy as np
import pytest

import oracle
from paper_2503_22227_gb300 import workloads as W


def crt(res, mods):
    x, step = 0, 1
    for r, m in zip(res, mods):
        k = ((int(r) - x) * pow(step, -1, m)) % m
        x += k * step
        step *= m
    return x, step


def centred(x, M):
    x %= M
    return x - M if 2 * x > M else x


def negamul_int(a, b, mod=None):
    n = len(a)
    out = [0] * n
    for i in range(n):
        if a[i] == 0:
            continue
        for j in range(n):
            s = a[i] * b[j]
            if i + j < n:
                out[i + j] += s
            else:
                out[i + j - n] -= s
    return [x % mod for x in out] if mod else out


def poly_big(ct_poly, mods):
    n = ct_poly.shape[-1]
    M = 1
    for m in mods:
        M *= m
    return [centred(crt([ct_poly[i][j] for i in range(len(mods))], mods)[0], M) for j in range(n)], M


SEED = W.seed_for("oracle-tests")


@pytest.fixture(scope="module")
def bfv_small():
    ctx = oracle.Context(oracle.BFV, 6, [55] * 3, [60], 3, t=257)
    return ctx, ctx.keygen(SEED)


@pytest.fixture(scope="module")
def bgv_small():
    ctx = oracle.Context(oracle.BGV, 6, [55] * 3, [60], 3, t=257)
    return ctx, ctx.keygen(SEED)


@pytest.fixture(scope="module")
def ckks_n12():
    p = W.PRESETS["ckks_n12"]
    ctx = oracle.Context(oracle.CKKS, p.log_n, p.q_bits, p.p_bits, p.dnum, log_n_max=p.log_n_max)
    return ctx, ctx.keygen(SEED)


@pytest.mark.parametrize("which", ["bfv_small", "bgv_small"])
def test_keys_decrypt_to_small_error(which, request):
    ctx, keys = request.getfixturevalue(which)
    n = ctx.n
    s = [int(x) for x in keys.secret()]
    assert set(s) <= {-1, 0, 1}
    te = ctx.t if ctx.scheme == oracle.BGV else 1
    pk = keys.public()
    for i, q in enumerate(ctx.q):
        e = [(int(x) + int(y)) % q for x, y in zip(pk[0, i], negamul_int([int(v) for v in pk[1, i]], s, q))]
        e = [centred(v, q) for v in e]
        assert max(abs(v) for v in e) <= 19 * te and all(v % te == 0 for v in e)
    ksk = keys.ksk(0)
    s2 = negamul_int(s, s)
    mods = ctx.q + ctx.p
    P = 1
    for p in ctx.p:
        P *= p
    for j in range(ctx.beta):
        for i, m in enumerate(mods):
            a = [int(v) for v in ksk[j, 1, i]]
            as_ = negamul_int(a, s, m)
            gadget = (P % m) if (i < ctx.L and i // ctx.alpha == j) else 0
            e = [centred(int(ksk[j, 0, i, x]) + as_[x] - gadget * s2[x], m) for x in range(n)]
            assert max(abs(v) for v in e) <= 19 * te and all(v % te == 0 for v in e)


@pytest.mark.parametrize("which", ["bfv_small", "bgv_small"])
def test_integer_schemes_encrypt_multiply_rotate(which, request):
    ctx, keys = request.getfixturevalue(which)
    n, t = ctx.n, ctx.t
    rng = np.random.default_rng(12)
    a = W.int_messages(rng, n, t)
    b = W.int_messages(rng, n, t)
    ca = ctx.encrypt(keys, a, W.seed_for("enc-a"))
    cb = ctx.encrypt(keys, b, W.seed_for("enc-b"))
    assert np.array_equal(ctx.decrypt(keys, ca), a)
    assert np.array_equal(ctx.decrypt(keys, ctx.add(ca, cb)), (a + b) % t)
    prod = ctx.mul_relin(keys, ca, cb)
    expect = negamul_int([int(x) for x in a], [int(x) for x in b], t)
    assert [int(x) for x in ctx.decrypt(keys, prod)] == expect
    # rotation of rows: the plaintext polynomial goes through X -> X^g
    g = ctx.galois_elt(1)
    keys.gen_galois(g)
    rot = ctx.rotate(keys, ca, g)
    sig = [0] * n
    for i in range(n):
        k = i * g % (2 * n)
        if k < n:
            sig[k] = int(a[i]) % t
        else:
            sig[k - n] = (-int(a[i])) % t
    assert [int(x) for x in ctx.decrypt(keys, rot)] == sig
    # modulus switch / rescale keeps the message
    if ctx.scheme == oracle.BGV:
        ms = ctx.rescale(prod)
        f = ctx.bgv_factor_after_rescale(1, ctx.L)
        assert [int(x) for x in ctx.decrypt(keys, ms, factor=f)] == expect
        # without the factor the plaintext is multiplied by q_{l-1}^{-1} mod t
        qinv = pow(ctx.q[-1], -1, t)
        assert [int(x) for x in ctx.decrypt(keys, ms)] == [e * qinv % t for e in expect]


def test_keyswitch_error_is_small(bgv_small, bfv_small):
    for ctx, keys in (bfv_small, bgv_small):
        n = ctx.n
        rng = np.random.default_rng(13)
        c = np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in ctx.q])
        k = ctx.keyswitch(keys, c, 0)
        s = [int(x) for x in keys.secret()]
        s2 = negamul_int(s, s)
        Q = 1
        for q in ctx.q:
            Q *= q
        cbig = [crt(c[:, j], ctx.q)[0] for j in range(n)]
        k0 = [crt(k[0, :, j], ctx.q)[0] for j in range(n)]
        k1 = [crt(k[1, :, j], ctx.q)[0] for j in range(n)]
        lhs = [x + y for x, y in zip(k0, negamul_int(k1, s))]
        rhs = negamul_int(cbig, s2)
        err = [centred(x - y, Q) for x, y in zip(lhs, rhs)]
        bound = ctx.beta * n * max(ctx.q) * 19 * (ctx.t if ctx.scheme == oracle.BGV else 1)
        bound = bound // min(ctx.p) + n * ctx.t * 2
        assert max(abs(e) for e in err) < bound
        if ctx.scheme == oracle.BGV:
            assert all(e % ctx.t == 0 for e in err)


def test_ckks_hmult_relin_rescale_and_rotate(ckks_n12):
    ctx, keys = ckks_n12
    n = ctx.n
    scale = 2.0 ** 40
    rng = W.rng_for("ckks-accuracy")
    za, zb = W.complex_slots(rng, n), W.complex_slots(rng, n)
    ma, mb = oracle.encode_ckks(za, n, scale), oracle.encode_ckks(zb, n, scale)
    ca = ctx.encrypt(keys, ma, W.seed_for("ckks-a"))
    cb = ctx.encrypt(keys, mb, W.seed_for("ckks-b"))
    dec = oracle.decode_ckks(ctx.decrypt(keys, ca), n, scale)
    assert np.max(np.abs(dec - za)) < 2.0 ** -20
    prod = ctx.rescale(ctx.mul_relin(keys, ca, cb))
    scale2 = scale * scale / ctx.q[-1]
    got = oracle.decode_ckks(ctx.decrypt(keys, prod), n, scale2)
    assert np.max(np.abs(got - za * zb)) < 2.0 ** -20
    g = ctx.galois_elt(1)
    keys.gen_galois(g)
    rot = oracle.decode_ckks(ctx.decrypt(keys, ctx.rotate(keys, ca, g)), n, scale)
    assert np.max(np.abs(rot - np.roll(za, -1))) < 2.0 ** -20


def test_ckks_encoder_closed_forms():
    n, scale = 64, 2.0 ** 30
    c = 0.375
    m = oracle.encode_ckks(np.full(n // 2, c, dtype=complex), n, scale)
    assert m[0] == round(c * scale) and not m[1:].any()
    rng = np.random.default_rng(1)
    z1, z2 = W.complex_slots(rng, n), W.complex_slots(rng, n)
    m1, m2 = oracle.encode_ckks(z1, n, scale), oracle.encode_ckks(z2, n, scale)
    prod = negamul_int([int(x) for x in m1], [int(x) for x in m2])
    got = oracle.decode_ckks(np.array(prod, dtype=np.float64), n, scale * scale)
    assert np.max(np.abs(got - z1 * z2)) < 1e-6
    # X -> X^5 rotates the slots left by one
    rot = [0] * n
    for i in range(n):
        k = 5 * i % (2 * n)
        if k < n:
            rot[k] = int(m1[i])
        else:
            rot[k - n] = -int(m1[i])
    assert np.max(np.abs(oracle.decode_ckks(rot, n, scale) - np.roll(z1, -1))) < 1e-6


def test_ckks_keyswitch_output_matches_definition_small():
    """Tiny CKKS ring: KS(c) checked against the big-integer definition."""
    ctx = oracle.Context(oracle.CKKS, 3, [40] * 4, [40, 40], 2)
    keys = ctx.keygen(SEED)
    n = ctx.n
    rng = np.random.default_rng(2)
    for level in (4, 3):
        c = np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in ctx.q[:level]])
        got = ctx.keyswitch(keys, c, 0)
        ksk = keys.ksk(0)
        mods = ctx.q[:level] + ctx.p
        P = ctx.p[0] * ctx.p[1]
        QP = 1
        for m in mods:
            QP *= m
        beta = -(-level // ctx.alpha)
        acc = [[0] * n for _ in range(2)]
        for j in range(beta):
            dq = ctx.q[j * ctx.alpha: min((j + 1) * ctx.alpha, level)]
            dig = c[j * ctx.alpha: min((j + 1) * ctx.alpha, level)]
            D = 1
            for m in dq:
                D *= m
            lifted = [centred(crt(dig[:, x], dq)[0], D) for x in range(n)]
            for poly in range(2):
                key_rows = list(range(level)) + [ctx.L + k for k in range(ctx.K)]
                kb = [crt([ksk[j, poly, r, x] for r in key_rows], mods)[0] for x in range(n)]
                prod = negamul_int(lifted, kb)
                acc[poly] = [u + v for u, v in zip(acc[poly], prod)]
        for poly in range(2):
            for x in range(n):
                y = round(__import__("fractions").Fraction(acc[poly][x] % QP, P))
                assert [int(got[poly, i, x]) for i in range(level)] == [y % q for q in ctx.q[:level]]


def test_elementwise_ops_by_decryption(bgv_small, ckks_n12):
    """sub / integer multiply / constant add / level drop, pinned by what
    decryption must give (exact for BGV mod t; exact integers for CKKS,
    whose decryption is the centred plaintext polynomial)."""
    ctx, keys = bgv_small
    n, t = ctx.n, ctx.t
    rng = np.random.default_rng(21)
    a, b = W.int_messages(rng, n, t), W.int_messages(rng, n, t)
    ca = ctx.encrypt(keys, a, W.seed_for("ew-a"))
    cb = ctx.encrypt(keys, b, W.seed_for("ew-b"))
    assert np.array_equal(ctx.decrypt(keys, ctx.sub(ca, cb)), (a - b) % t)
    assert np.array_equal(ctx.add(ctx.sub(ca, cb), cb), ca)
    for k in (0, 1, 7, -3, t - 1):
        assert np.array_equal(ctx.decrypt(keys, ctx.mul_int(ca, k)), (a * k) % t)
    # BGV in coefficient form: the constant k lands on plaintext coefficient 0
    want = a.copy()
    want[0] = (want[0] + 5) % t
    assert np.array_equal(ctx.decrypt(keys, ctx.add_const(ca, 5)), want)
    d = ctx.drop(ca, ctx.L - 1)
    assert d.shape == (2, ctx.L - 1, n)
    assert np.array_equal(d, ca[:, : ctx.L - 1])
    # dropping a prime is a modulus switch without the division: the
    # plaintext survives when the noise is far below the smaller modulus
    assert np.array_equal(ctx.decrypt(keys, d), a)

    ctx, keys = ckks_n12
    n = ctx.n
    rng = np.random.default_rng(22)
    ma = rng.integers(-2 ** 30, 2 ** 30, n)
    mb = rng.integers(-2 ** 30, 2 ** 30, n)
    ca = ctx.encrypt(keys, ma, W.seed_for("ew-ckks-a"))
    cb = ctx.encrypt(keys, mb, W.seed_for("ew-ckks-b"))
    da, db = ctx.decrypt(keys, ca), ctx.decrypt(keys, cb)
    assert np.max(np.abs(da - ma)) < 2 ** 12            # fresh-encryption noise
    assert np.array_equal(ctx.decrypt(keys, ctx.sub(ca, cb)), da - db)
    assert np.array_equal(ctx.decrypt(keys, ctx.mul_int(ca, -1234)), da * -1234)
    want = da.copy()
    want[0] += -(2 ** 35)
    assert np.array_equal(ctx.decrypt(keys, ctx.add_const(ca, -(2 ** 35))), want)
    assert np.array_equal(ctx.decrypt(keys, ctx.drop(ca, 1)), da)


def test_mul_plain_by_decryption(bgv_small, bfv_small, ckks_n12):
    """Multiplication by a plaintext polynomial: decryption is linear, so
    Dec(c pt) = Dec(c) pt in Z[X]/(X^N + 1) (mod t for BGV and BFV, where
    c0 + c1 s = Delta m + e becomes Delta m pt + e pt; exactly, as integers,
    for small CKKS messages)."""
    for (ctx, keys), tag in ((bgv_small, "bgv"), (bfv_small, "bfv")):
        n, t = ctx.n, ctx.t
        rng = np.random.default_rng(31)
        m = W.int_messages(rng, n, t)
        pt = rng.integers(-3, 4, n)
        c = ctx.encrypt(keys, m, W.seed_for(f"mp-{tag}"))
        want = negamul_int([int(x) for x in m], [int(x) for x in pt], t)
        assert [int(x) for x in ctx.decrypt(keys, ctx.mul_plain(c, pt))] == want, tag

    ctx, keys = ckks_n12
    n = ctx.n
    rng = np.random.default_rng(32)
    m = rng.integers(-2 ** 20, 2 ** 20, n)
    pt = rng.integers(-2 ** 10, 2 ** 10, n)
    c = ctx.encrypt(keys, m, W.seed_for("mp-ckks"))
    d = ctx.decrypt(keys, c)
    want = negamul_int([int(x) for x in d], [int(x) for x in pt])
    assert [int(x) for x in ctx.decrypt(keys, ctx.mul_plain(c, pt))] == want
