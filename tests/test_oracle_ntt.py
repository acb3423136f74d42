"""Pins of the oracle's NTT (paper Sec. 3.1.3, butterfly NTT):
the O(N^2) definition out[bitrev(i)] = sum_j a_j psi^((2i+1) j), the
inverse, and the negacyclic convolution it implements (schoolbook)."""
import random

import numpy as np
import pytest

import oracle


def bitrev(x, bits):
    return int(format(x, f"0{bits}b")[::-1], 2) if bits else 0


def ntt_definition(a, log_n, q, psi):
    n = 1 << log_n
    out = [0] * n
    for i in range(n):
        out[bitrev(i, log_n)] = sum(int(a[j]) * pow(psi, (2 * i + 1) * j, q) for j in range(n)) % q
    return out


def schoolbook_negacyclic(a, b, q):
    n = len(a)
    out = [0] * n
    for i in range(n):
        for j in range(n):
            k = i + j
            if k < n:
                out[k] += int(a[i]) * int(b[j])
            else:
                out[k - n] -= int(a[i]) * int(b[j])
    return [x % q for x in out]


@pytest.mark.parametrize("log_n", [1, 3, 4, 6, 8])
@pytest.mark.parametrize("bits", [40, 60])
def test_ntt_matches_definition(log_n, bits):
    n = 1 << log_n
    q = oracle.gen_primes(bits, 1, 2 * n)[0]
    psi = oracle.min_psi(q, log_n)
    rng = random.Random(log_n * 100 + bits)
    a = [rng.randrange(q) for _ in range(n)]
    assert list(map(int, oracle.ntt(a, log_n, q, psi))) == ntt_definition(a, log_n, q, psi)


def test_ntt_special_inputs():
    log_n, n = 5, 32
    q = oracle.gen_primes(50, 1, 2 * n)[0]
    psi = oracle.min_psi(q, log_n)
    # NTT(1) = all ones; NTT(X)[bitrev(i)] = psi^(2i+1)
    delta = np.zeros(n, dtype=np.uint64)
    delta[0] = 1
    assert list(map(int, oracle.ntt(delta, log_n, q, psi))) == [1] * n
    x = np.zeros(n, dtype=np.uint64)
    x[1] = 1
    out = oracle.ntt(x, log_n, q, psi)
    for i in range(n):
        assert int(out[bitrev(i, log_n)]) == pow(psi, 2 * i + 1, q)


@pytest.mark.parametrize("log_n", [4, 12])
def test_inverse_roundtrip(log_n):
    n = 1 << log_n
    q = oracle.gen_primes(55, 1, 2 * n)[0]
    psi = oracle.min_psi(q, log_n)
    a = np.random.default_rng(3).integers(0, q, n, dtype=np.uint64)
    assert np.array_equal(oracle.intt(oracle.ntt(a, log_n, q, psi), log_n, q, psi), a)


@pytest.mark.parametrize("log_n", [2, 4, 6])
def test_negacyclic_mul_matches_schoolbook(log_n):
    n = 1 << log_n
    q = oracle.gen_primes(60, 1, 2 * n)[0]
    psi = oracle.min_psi(q, log_n)
    rng = random.Random(log_n)
    a = [rng.randrange(q) for _ in range(n)]
    b = [rng.randrange(q) for _ in range(n)]
    got = oracle.negacyclic_mul(np.array(a, dtype=np.uint64), np.array(b, dtype=np.uint64),
                                log_n, q, psi)
    assert list(map(int, got)) == schoolbook_negacyclic(a, b, q)


def test_automorphism_composition_and_definition():
    log_n, n = 5, 32
    q = oracle.gen_primes(50, 1, 2 * n)[0]
    rng = np.random.default_rng(5)
    a = rng.integers(0, q, n, dtype=np.uint64)
    for g, h in [(5, 25), (3, 2 * n - 1), (5, 2 * n - 1)]:
        lhs = oracle.automorphism(oracle.automorphism(a, h, q), g, q)
        rhs = oracle.automorphism(a, g * h % (2 * n), q)
        assert np.array_equal(lhs, rhs)
    # definition: sigma_g(X^i) = X^(ig) with X^N = -1
    for i in range(n):
        e = np.zeros(n, dtype=np.uint64)
        e[i] = 7
        out = oracle.automorphism(e, 5, q)
        k = i * 5 % (2 * n)
        expect = np.zeros(n, dtype=np.uint64)
        expect[k % n] = 7 if k < n else q - 7
        assert np.array_equal(out, expect)
