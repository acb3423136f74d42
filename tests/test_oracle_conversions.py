"""Pins of the oracle's exact base conversions against Python integers.

ModUp lift, ModDown round(x/P), CKKS rescale round(c/q), the t-preserving
division of BGV, the BFV tensor round(t x / Q) and the ModDown+rescale
fusion identity, each checked by an independent characterisation
(Fraction rounding, divisibility and size properties), not by retyping the
oracle's formula."""
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle


def crt(res, mods):
    M = 1
    for m in mods:
        M *= m
    # brute-force-free but independent route: successive substitution (Garner)
    x, step = 0, 1
    for r, m in zip(res, mods):
        k = ((r - x) * pow(step, -1, m)) % m
        x += k * step
        step *= m
    return x % M, M


def centred(x, M):
    x %= M
    return x - M if 2 * x > M else x


def residues(x, mods):
    return [x % m for m in mods]


PR = oracle.gen_primes(50, 10, 2 ** 17)
PP = oracle.gen_primes(60, 6, 2 ** 17)


@pytest.mark.parametrize("k,T", [(1, 3), (2, 5), (3, 4), (8, 12)])
def test_lift_centred(k, T):
    src, dst = PR[:k], PR[k:k + min(T, 10 - k)] + PP[:max(0, T - (10 - k))]
    M = 1
    for m in src:
        M *= m
    rng = random.Random(k * 10 + T)
    xs = [rng.randrange(M) for _ in range(60)] + [0, 1, M - 1, (M - 1) // 2, (M + 1) // 2]
    arr = np.array([residues(x, src) for x in xs], dtype=np.uint64).T.copy()
    got = oracle.lift_centred(arr, src, dst)
    for j, x in enumerate(xs):
        xc = centred(x, M)
        assert -M < 2 * xc <= M
        assert [int(v) for v in got[:, j]] == [xc % m for m in dst]


@pytest.mark.parametrize("kq,kd", [(3, 1), (4, 2), (6, 4), (2, 5)])
def test_div_round_is_nearest_integer(kq, kd):
    qs, ds = PR[:kq], PP[:kd]
    Q = D = 1
    for m in qs:
        Q *= m
    for m in ds:
        D *= m
    rng = random.Random(kq * 7 + kd)
    xs = [rng.randrange(Q * D) for _ in range(60)] + [0, D // 2, D // 2 + 1, Q * D - 1,
                                                      Q * D - D // 2, Q * D - D // 2 - 1]
    arr = np.array([residues(x, qs + ds) for x in xs], dtype=np.uint64).T.copy()
    got = oracle.div_round(arr, qs, ds)
    for j, x in enumerate(xs):
        y = round(Fraction(x, D))       # nearest integer (D odd: never a tie)
        assert [int(v) for v in got[:, j]] == [y % m for m in qs]
        assert abs(x - D * y) * 2 < D


@pytest.mark.parametrize("kq,kd,t", [(3, 1, 65537), (4, 2, 257), (5, 3, 65537)])
def test_div_t_exact_properties(kq, kd, t):
    qs, ds = PR[:kq], PP[:kd]
    Q = D = 1
    for m in qs:
        Q *= m
    for m in ds:
        D *= m
    rng = random.Random(kq + kd + t)
    xs = [rng.randrange(Q * D) for _ in range(60)]
    arr = np.array([residues(x, qs + ds) for x in xs], dtype=np.uint64).T.copy()
    got = oracle.div_t_exact(arr, qs, ds, t)
    for j, x in enumerate(xs):
        y, _ = crt([int(v) for v in got[:, j]], qs)
        d = centred(x - D * y, Q * D)    # the correction actually applied
        assert d % D == x % D            # removes x mod D
        assert d % t == 0                # keeps the plaintext mod t
        assert 2 * abs(d) <= t * D       # and is the small one
        # y D = x - d (mod QD), and the plaintext maps to x D^{-1} mod t
        assert (y * D - (x - d)) % (Q * D) == 0


def test_moddown_then_rescale_equals_one_division():
    """round(round(x/P)/q) == round(x/(P q)): the identity that lets the
    key switch's ModDown and the CKKS rescale run as one exact division."""
    qs, ds = PR[:5], PP[:4]
    rng = np.random.default_rng(11)
    n = 256
    x = np.stack([rng.integers(0, m, n, dtype=np.uint64) for m in qs + ds])
    step1 = oracle.div_round(x, qs, ds)                    # over q_0..q_4
    seq = oracle.div_round(step1, qs[:4], qs[4:])          # then / q_4
    reorder = np.concatenate([x[:4], x[5:], x[4:5]])       # divisor P u {q_4}
    fused = oracle.div_round(reorder, qs[:4], ds + qs[4:5])
    assert np.array_equal(seq, fused)


def test_tensor_and_bfv_scale_round_small():
    """BFV tensor on a tiny ring: centred lifts, exact integer negacyclic
    products (Python schoolbook), round(t x / Q) by Fraction."""
    ctx = oracle.Context(oracle.BFV, 3, [30, 30], [31], 2, t=257)
    n, Q = ctx.n, ctx.q[0] * ctx.q[1]
    rng = np.random.default_rng(4)
    a = np.stack([np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in ctx.q])
                  for _ in range(2)])
    b = np.stack([np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in ctx.q])
                  for _ in range(2)])

    def big(poly):
        return [centred(crt([int(poly[i][j]) for i in range(2)], ctx.q)[0], Q) for j in range(n)]

    def negamul(u, v):
        out = [0] * n
        for i in range(n):
            for j in range(n):
                if i + j < n:
                    out[i + j] += u[i] * v[j]
                else:
                    out[i + j - n] -= u[i] * v[j]
        return out

    A0, A1, B0, B1 = big(a[0]), big(a[1]), big(b[0]), big(b[1])
    d0 = negamul(A0, B0)
    d1 = [x + y for x, y in zip(negamul(A0, B1), negamul(A1, B0))]
    d2 = negamul(A1, B1)
    got = ctx.tensor(a, b)
    for k, d in enumerate((d0, d1, d2)):
        for j in range(n):
            y = round(Fraction(257 * d[j], Q))
            assert [int(got[k, i, j]) for i in range(2)] == [y % q for q in ctx.q]


def test_tensor_ckks_small():
    ctx = oracle.Context(oracle.CKKS, 3, [40, 40], [40], 2)
    n = ctx.n
    rng = np.random.default_rng(6)
    a = np.stack([np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in ctx.q]) for _ in range(2)])
    b = np.stack([np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in ctx.q]) for _ in range(2)])
    got = ctx.tensor(a, b)
    for i, q in enumerate(ctx.q):
        def nm(u, v):
            out = [0] * n
            for x in range(n):
                for y in range(n):
                    s = 1 if x + y < n else -1
                    out[(x + y) % n] += s * int(u[x]) * int(v[y])
            return [o % q for o in out]
        assert list(map(int, got[0, i])) == nm(a[0, i], b[0, i])
        assert list(map(int, got[1, i])) == [(x + y) % q for x, y in zip(nm(a[0, i], b[1, i]),
                                                                         nm(a[1, i], b[0, i]))]
        assert list(map(int, got[2, i])) == nm(a[1, i], b[1, i])
