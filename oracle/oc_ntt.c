/*
 * Oracle: negacyclic number-theoretic transform.  TEST INFRASTRUCTURE ONLY.
 *
 * Definition (the butterfly NTT of Sec. 3.1.3 of the paper, "NTT_BM"):
 *   out[bitrev(i)] = sum_j a_j psi^((2i+1) j) mod q,   i, j in [0, N)
 * with psi a primitive 2N-th root of unity.  Computed by the textbook
 * iterative Cooley-Tukey recursion with bit-reversed powers of psi
 * (forward) and Gentleman-Sande with inverse powers (inverse), each
 * product reduced with '%' and every value kept in [0, q).
 */
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static uint64_t bitrev(uint64_t x, int bits) {
    uint64_t r = 0;
    for (int i = 0; i < bits; i++) r |= ((x >> i) & 1) << (bits - 1 - i);
    return r;
}

/* tab[i] = root^bitrev(i) for i in [0, N). */
static uint64_t *bitrev_powers(uint64_t root, int log_n, uint64_t q) {
    uint64_t n = (uint64_t)1 << log_n;
    uint64_t *pw = malloc(sizeof(uint64_t) * n), *tab = malloc(sizeof(uint64_t) * n);
    pw[0] = 1;
    for (uint64_t i = 1; i < n; i++) pw[i] = oc_mulmod(pw[i - 1], root, q);
    for (uint64_t i = 0; i < n; i++) tab[i] = pw[bitrev(i, log_n)];
    free(pw);
    return tab;
}

void oc_ntt_fwd(uint64_t *a, int log_n, uint64_t q, uint64_t psi) {
    uint64_t n = (uint64_t)1 << log_n;
    uint64_t *w = bitrev_powers(psi, log_n, q);
    for (uint64_t m = 1, t = n / 2; m < n; m *= 2, t /= 2) {
        for (uint64_t i = 0; i < m; i++) {
            uint64_t wi = w[m + i];
            for (uint64_t j = 2 * i * t; j < 2 * i * t + t; j++) {
                uint64_t u = a[j], v = oc_mulmod(a[j + t], wi, q);
                a[j] = oc_addmod(u, v, q);
                a[j + t] = oc_submod(u, v, q);
            }
        }
    }
    free(w);
}

void oc_ntt_inv(uint64_t *a, int log_n, uint64_t q, uint64_t psi) {
    uint64_t n = (uint64_t)1 << log_n;
    uint64_t *w = bitrev_powers(oc_invmod(psi, q), log_n, q);
    for (uint64_t m = n / 2, t = 1; m >= 1; m /= 2, t *= 2) {
        for (uint64_t i = 0; i < m; i++) {
            uint64_t wi = w[m + i];
            for (uint64_t j = 2 * i * t; j < 2 * i * t + t; j++) {
                uint64_t u = a[j], v = a[j + t];
                a[j] = oc_addmod(u, v, q);
                a[j + t] = oc_mulmod(oc_submod(u, v, q), wi, q);
            }
        }
    }
    uint64_t ninv = oc_invmod(n % q, q);
    for (uint64_t j = 0; j < n; j++) a[j] = oc_mulmod(a[j], ninv, q);
    free(w);
}

/* out = a * b in Z_q[X]/(X^N + 1), by NTT, pointwise product, inverse NTT. */
void oc_negacyclic_mul(uint64_t *out, const uint64_t *a, const uint64_t *b,
                       int log_n, uint64_t q, uint64_t psi) {
    uint64_t n = (uint64_t)1 << log_n;
    uint64_t *x = malloc(sizeof(uint64_t) * n), *y = malloc(sizeof(uint64_t) * n);
    memcpy(x, a, sizeof(uint64_t) * n);
    memcpy(y, b, sizeof(uint64_t) * n);
    oc_ntt_fwd(x, log_n, q, psi);
    oc_ntt_fwd(y, log_n, q, psi);
    for (uint64_t j = 0; j < n; j++) x[j] = oc_mulmod(x[j], y[j], q);
    oc_ntt_inv(x, log_n, q, psi);
    memcpy(out, x, sizeof(uint64_t) * n);
    free(x);
    free(y);
}
