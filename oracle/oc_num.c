/*
 * Oracle: modular arithmetic, primality, prime chains and roots of unity.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper (Sec. 2.2, RNS representation) writes q as a product of
 * word-sized pairwise coprime moduli and never lists them.  Reading taken
 * here: for each requested bit size b, the largest primes below 2^b with
 * q = 1 mod 2N_max, scanned downwards, skipping primes already taken;
 * ciphertext primes first, then the special primes, then the auxiliary
 * primes of BFV.  The NTT root is the smallest primitive 2N-th root of
 * unity mod q.
 */
#include "oracle.h"

uint64_t oc_mulmod(uint64_t a, uint64_t b, uint64_t m) {
    return (uint64_t)(((oc_u128)a * b) % m);
}

uint64_t oc_addmod(uint64_t a, uint64_t b, uint64_t m) {
    return (uint64_t)(((oc_u128)a + b) % m);
}

uint64_t oc_submod(uint64_t a, uint64_t b, uint64_t m) {
    return (uint64_t)(((oc_u128)a + m - (b % m)) % m);
}

uint64_t oc_powmod(uint64_t a, uint64_t e, uint64_t m) {
    uint64_t r = 1 % m, x = a % m;
    while (e) {
        if (e & 1) r = oc_mulmod(r, x, m);
        x = oc_mulmod(x, x, m);
        e >>= 1;
    }
    return r;
}

/* Inverse by the extended Euclidean algorithm; returns 0 if gcd != 1. */
uint64_t oc_invmod(uint64_t a, uint64_t m) {
    __int128 t = 0, newt = 1;
    __int128 r = m, newr = a % m;
    while (newr != 0) {
        __int128 quo = r / newr, tmp;
        tmp = t - quo * newt; t = newt; newt = tmp;
        tmp = r - quo * newr; r = newr; newr = tmp;
    }
    if (r != 1) return 0;
    if (t < 0) t += m;
    return (uint64_t)t;
}

/* Least non-negative residue of a signed integer. */
uint64_t oc_reduce_i64(int64_t x, uint64_t m) {
    __int128 r = (__int128)x % (__int128)m;
    if (r < 0) r += m;
    return (uint64_t)r;
}

/* Miller-Rabin with the first twelve primes as bases: deterministic for
 * every n < 3.3e24, so for every 64-bit n. */
int oc_is_prime(uint64_t n) {
    static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        uint64_t x = oc_powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int composite = 1;
        for (int r = 1; r < s; r++) {
            x = oc_mulmod(x, x, n);
            if (x == n - 1) { composite = 0; break; }
        }
        if (composite) return 0;
    }
    return 1;
}

/* The `count` largest primes below 2^bits that are 1 mod two_n and are not
 * in `exclude`, in descending order.  Returns the number found. */
int oc_gen_primes(int bits, int count, uint64_t two_n, const uint64_t *exclude,
                  int n_exclude, uint64_t *out) {
    uint64_t top = (bits >= 64) ? UINT64_MAX : ((uint64_t)1 << bits) - 1;
    uint64_t c = ((top - 1) / two_n) * two_n + 1; /* largest c <= top, c = 1 mod 2N */
    int found = 0;
    while (found < count && c > two_n) {
        int used = 0;
        for (int i = 0; i < n_exclude; i++) used |= (exclude[i] == c);
        for (int i = 0; i < found; i++) used |= (out[i] == c);
        if (!used && oc_is_prime(c)) out[found++] = c;
        c -= two_n;
    }
    return found;
}

/* Smallest primitive 2N-th root of unity mod q (q prime, q = 1 mod 2N).
 * First any primitive root psi0 = g^((q-1)/2N) with psi0^N = -1, then the
 * minimum over all N primitive 2N-th roots psi0^(2k+1). */
uint64_t oc_min_psi(uint64_t q, int log_n) {
    uint64_t n = (uint64_t)1 << log_n;
    uint64_t psi0 = 0;
    for (uint64_t g = 2; g < q; g++) {
        uint64_t c = oc_powmod(g, (q - 1) / (2 * n), q);
        if (oc_powmod(c, n, q) == q - 1) { psi0 = c; break; }
    }
    uint64_t best = psi0, sq = oc_mulmod(psi0, psi0, q), cur = psi0;
    for (uint64_t k = 1; k < n; k++) {
        cur = oc_mulmod(cur, sq, q);
        if (cur < best) best = cur;
    }
    return best;
}
