"""Pins of the oracle's randomness: ChaCha20 (RFC 8439) and the samplers."""
import numpy as np
import pytest

import oracle


def test_chacha20_rfc8439_block_vector():
    # RFC 8439 Sec. 2.3.2: key 00..1f, nonce 000000090000004a00000000, counter 1
    key = bytes(range(32))
    nonce = bytes.fromhex("000000090000004a00000000")
    blk = oracle.chacha20_block(key, 1, nonce)
    assert blk[:16].hex() == "10f1e7e4d13b5915500fdd1fa32071c4"
    assert blk[-4:].hex() == "a2503c4e"


def test_chacha20_matches_library_keystream():
    crypto = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    rng = np.random.default_rng(9)
    for trial in range(8):
        key = rng.bytes(32)
        tag, i0, i1 = (int(x) for x in rng.integers(0, 2 ** 32, 3))
        nonce = b"".join(int(v).to_bytes(4, "little") for v in (tag, i0, i1))
        counter = int(rng.integers(0, 1000))
        enc = crypto.Cipher(crypto.algorithms.ChaCha20(key, counter.to_bytes(4, "little") + nonce),
                            mode=None).encryptor()
        ks = enc.update(bytes(64 * 3))
        for w in range(24):
            expect = int.from_bytes(ks[8 * w: 8 * w + 8], "little")
            assert oracle.stream_word(key, tag, i0, i1, counter * 8 + w) == expect


def test_cdt_table_matches_high_precision():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    sigma = mpmath.mpf("3.2")
    p = [mpmath.e ** (-(k * k) / (2 * sigma ** 2)) for k in range(20)]
    total = p[0] + 2 * sum(p[1:])
    cum, expect = p[0], []
    for k in range(19):
        v = cum / total * 2 ** 40
        # the double-precision table is only well defined away from half-integers
        assert abs(v - mpmath.floor(v) - mpmath.mpf("0.5")) > mpmath.mpf("1e-3")
        expect.append(int(mpmath.floor(v + mpmath.mpf("0.5"))))
        cum += 2 * p[k + 1]
    assert oracle.cdt_table() == expect


def test_sampler_statistics():
    key = bytes(range(32))
    g = np.concatenate([oracle.sample_gaussian(key, 3, i, 0, 16) for i in range(16)])  # 2^20
    assert abs(g.mean()) < 0.02
    assert abs(g.std() - 3.2) / 3.2 < 0.01
    assert np.abs(g).max() <= 19
    assert abs((g > 0).mean() - (g < 0).mean()) < 0.01
    t = oracle.sample_ternary(key, 1, 0, 0, 16)
    for v in (-1, 0, 1):
        assert abs((t == v).mean() - 1 / 3) < 0.01
    q = oracle.gen_primes(50, 2, 2 ** 17)
    u = oracle.sample_uniform(key, 9, 0, 0, q, 14)
    for i, m in enumerate(q):
        assert u[i].max() < m
        assert abs(u[i].astype(np.float64).mean() / m - 0.5) < 0.01


def test_sampler_word_layout():
    """Uniform limb i coefficient j uses words 2k, 2k+1 with k = i N + j."""
    key = bytes(range(1, 33))
    q = oracle.gen_primes(40, 2, 2 ** 5)
    log_n = 4
    u = oracle.sample_uniform(key, 9, 1, 2, q, log_n)
    for i in range(2):
        for j in range(16):
            k = i * 16 + j
            hi = oracle.stream_word(key, 9, 1, 2, 2 * k)
            lo = oracle.stream_word(key, 9, 1, 2, 2 * k + 1)
            assert int(u[i, j]) == ((hi << 64) | lo) % q[i]
    t = oracle.sample_ternary(key, 6, 0, 0, log_n)
    assert [int(x) for x in t] == [oracle.stream_word(key, 6, 0, 0, j) % 3 - 1 for j in range(16)]
