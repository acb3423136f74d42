"""Pins of the oracle's number theory: primality, prime chains, NTT roots.

Each check uses an independent route (sympy, Python integers, brute force).
"""
import random

import pytest

import oracle

sympy = pytest.importorskip("sympy")


def test_is_prime_matches_sympy():
    rng = random.Random(1)
    cands = [rng.getrandbits(64) | 1 for _ in range(300)]
    # strong pseudoprimes to small bases and Carmichael numbers
    cands += [561, 1105, 2047, 3215031751, 3825123056546413051, 318665857834031151167461,
              2 ** 61 - 1, 2 ** 61 + 1, (1 << 64) - 59]
    for c in cands:
        if c >= 1 << 64:
            continue
        assert oracle.is_prime(c) == sympy.isprime(c), c


@pytest.mark.parametrize("bits,two_n,count", [(40, 2 ** 13, 4), (50, 2 ** 17, 5), (55, 2 ** 15, 4),
                                              (60, 2 ** 17, 3)])
def test_prime_chain_definition(bits, two_n, count):
    """Largest primes below 2^bits with q = 1 mod 2N, descending (sympy scan)."""
    expect = []
    c = ((2 ** bits - 2) // two_n) * two_n + 1
    while len(expect) < count:
        if sympy.isprime(c):
            expect.append(c)
        c -= two_n
    assert oracle.gen_primes(bits, count, two_n) == expect
    # skipping already used primes gives the next ones
    assert oracle.gen_primes(bits, 1, two_n, exclude=expect[:2]) == [expect[2]]


@pytest.mark.parametrize("log_n", [1, 3, 6, 10])
def test_min_psi_is_smallest_primitive_root(log_n):
    n = 1 << log_n
    for q in oracle.gen_primes(40, 2, 2 * n) + oracle.gen_primes(20, 1, 2 * n):
        psi = oracle.min_psi(q, log_n)
        g = sympy.primitive_root(q)
        w = pow(g, (q - 1) // (2 * n), q)           # a primitive 2N-th root
        roots = {pow(w, 2 * k + 1, q) for k in range(n)}  # all of them
        assert psi == min(roots)
        assert pow(psi, n, q) == q - 1 and pow(psi, 2 * n, q) == 1


def test_modular_helpers():
    L = oracle.lib()
    rng = random.Random(2)
    for _ in range(200):
        m = rng.getrandbits(62) | 1
        a, b = rng.getrandbits(64), rng.getrandbits(64)
        assert L.oc_mulmod(a, b, m) == a * b % m
        e = rng.getrandbits(64)
        assert L.oc_powmod(a, e, m) == pow(a, e, m)
    q = oracle.gen_primes(60, 1, 2)[0]
    for a in (1, 2, 3, q - 1, 123456789):
        assert L.oc_invmod(a, q) * a % q == 1
