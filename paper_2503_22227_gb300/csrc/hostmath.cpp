// Host-side number theory of the library: primality, roots of unity,
// Shoup constants, the discrete Gaussian table.  Written independently of
// the CPU oracle; both follow the same published definitions.
#include <math.h>

#include "internal.h"

namespace catfhe {

typedef unsigned __int128 u128;

uint64_t h_mulmod(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((u128)a * b % m); }

uint64_t h_powmod(uint64_t a, uint64_t e, uint64_t m) {
    uint64_t r = 1 % m;
    a %= m;
    for (; e; e >>= 1) {
        if (e & 1) r = h_mulmod(r, a, m);
        a = h_mulmod(a, a, m);
    }
    return r;
}

// Inverse modulo m by the extended Euclidean algorithm (0 if none).
uint64_t h_invmod(uint64_t a, uint64_t m) {
    uint64_t r0 = a % m, r1 = m;
    // the Bezout coefficient of a, tracked in signed 128 bits (no overflow)
    __int128 x0 = 1, x1 = 0;
    while (r1) {
        uint64_t qt = r0 / r1;
        uint64_t r2 = r0 - qt * r1;
        __int128 x2 = x0 - (__int128)qt * x1;
        r0 = r1;
        r1 = r2;
        x0 = x1;
        x1 = x2;
    }
    if (r0 != 1) return 0;
    __int128 v = x0 % (__int128)m;
    if (v < 0) v += m;
    return (uint64_t)v;
}

// Deterministic Miller-Rabin for 64-bit n (bases: the primes up to 37).
bool h_is_prime(uint64_t n) {
    if (n < 2) return false;
    const uint64_t small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (uint64_t p : small) {
        if (n % p == 0) return n == p;
    }
    uint64_t d = n - 1;
    int r = 0;
    while (!(d & 1)) {
        d >>= 1;
        r++;
    }
    for (uint64_t a : small) {
        uint64_t x = h_powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool witness = true;
        for (int i = 1; i < r && witness; i++) {
            x = h_mulmod(x, x, n);
            if (x == n - 1) witness = false;
        }
        if (witness) return false;
    }
    return true;
}

uint64_t h_shoup(uint64_t w, uint64_t q) { return (uint64_t)(((u128)w << 64) / q); }

// Smallest primitive 2N-th root of unity mod q: take any one, w, then the
// minimum of w^(2k+1) over k < N (these are all of them).
uint64_t h_min_psi(uint64_t q, int log_n) {
    const uint64_t n = uint64_t(1) << log_n;
    uint64_t w = 0;
    for (uint64_t g = 2; g < q && !w; g++) {
        uint64_t c = h_powmod(g, (q - 1) >> (log_n + 1), q);
        if (h_powmod(c, n, q) == q - 1) w = c;
    }
    uint64_t w2 = h_mulmod(w, w, q), cur = w, best = w;
    for (uint64_t k = 1; k < n; k++) {
        cur = h_mulmod(cur, w2, q);
        if (cur < best) best = cur;
    }
    return best;
}

// CDT thresholds of |X|, X discrete Gaussian with sigma = 3.2 on
// [-19, 19]: T_k = round(2^40 P(|X| <= k)), k = 0 .. 18.
void h_cdt(uint64_t out[19]) {
    const double s2 = 2.0 * 3.2 * 3.2;
    double rho[20];
    for (int k = 0; k < 20; k++) rho[k] = exp(-(double)(k * k) / s2);
    double total = rho[0];
    for (int k = 1; k < 20; k++) total += 2.0 * rho[k];
    double acc = rho[0];
    for (int k = 0; k < 19; k++) {
        out[k] = (uint64_t)floor(acc / total * 1099511627776.0 + 0.5);
        acc += 2.0 * rho[k + 1];
    }
}

DevMod h_devmod(uint64_t q, uint64_t n, uint64_t psi) {
    DevMod m{};
    m.q = q;
    m.r64 = (uint64_t)(((u128)1 << 64) % q);
    m.r64_s = h_shoup(m.r64, q);
    m.one_s = h_shoup(1, q);
    uint64_t x = q;  // -q^-1 mod 2^64 by Newton's iteration (q odd)
    for (int i = 0; i < 6; i++) x *= 2 - q * x;
    m.qinv = 0 - x;
    m.m64 = q > (uint64_t(1) << 33) ? (uint64_t)(((u128)1 << 64) / q) : 0;
    if (n) {
        m.ninv = h_invmod(n % q, q);
        m.ninv_s = h_shoup(m.ninv, q);
        // psi^-bitrev(1) = psi^-(N/2)
        uint64_t wi = h_powmod(h_invmod(psi, q), n / 2, q);
        m.ninvw = h_mulmod(m.ninv, wi, q);
        m.ninvw_s = h_shoup(m.ninvw, q);
    }
    return m;
}

}  // namespace catfhe
