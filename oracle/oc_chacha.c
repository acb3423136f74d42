/*
 * Oracle: ChaCha20 keystream (RFC 8439, Sec. 2.3) and the samplers of
 * secrets, errors and uniform polynomials.  TEST INFRASTRUCTURE ONLY.
 *
 * The paper does not say how randomness is drawn (its key generation and
 * encryption are named in Sec. 3 and Tables 1-3 only).  Reading taken:
 *  - keystream: ChaCha20 with key = 32-byte seed, counter = block index,
 *    nonce = three little-endian 32-bit words (tag, i0, i1);
 *    word w = keystream bytes 8w..8w+7, little endian;
 *  - uniform mod q_i, limb i, coefficient j: with k = i*N + j,
 *    (word(2k) * 2^64 + word(2k+1)) mod q_i;
 *  - ternary coefficient j: (word(j) mod 3) - 1;
 *  - discrete Gaussian, sigma = 3.2, coefficient j: u = low 40 bits of
 *    word(j), |x| = number of thresholds T_k (k = 0..18) with u >= T_k,
 *    T_k = round(2^40 F(k)), F the distribution function of |X| with
 *    P(|X| = 0) proportional to 1 and P(|X| = k) to 2 exp(-k^2 / 2 sigma^2);
 *    bit 63 of word(j) is the sign of a non-zero |x|.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static uint32_t rotl32(uint32_t x, int r) { return (x << r) | (x >> (32 - r)); }

static void quarter_round(uint32_t *s, int a, int b, int c, int d) {
    s[a] += s[b]; s[d] ^= s[a]; s[d] = rotl32(s[d], 16);
    s[c] += s[d]; s[b] ^= s[c]; s[b] = rotl32(s[b], 12);
    s[a] += s[b]; s[d] ^= s[a]; s[d] = rotl32(s[d], 8);
    s[c] += s[d]; s[b] ^= s[c]; s[b] = rotl32(s[b], 7);
}

static uint32_t load_le32(const uint8_t *p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) |
           ((uint32_t)p[3] << 24);
}

void oc_chacha20_block(const uint8_t key[32], uint32_t counter,
                       const uint8_t nonce[12], uint8_t out[64]) {
    uint32_t init[16], s[16];
    init[0] = 0x61707865u; init[1] = 0x3320646eu; /* "expand 32-byte k" */
    init[2] = 0x79622d32u; init[3] = 0x6b206574u;
    for (int i = 0; i < 8; i++) init[4 + i] = load_le32(key + 4 * i);
    init[12] = counter;
    for (int i = 0; i < 3; i++) init[13 + i] = load_le32(nonce + 4 * i);
    memcpy(s, init, sizeof(s));
    for (int r = 0; r < 10; r++) {
        quarter_round(s, 0, 4, 8, 12);
        quarter_round(s, 1, 5, 9, 13);
        quarter_round(s, 2, 6, 10, 14);
        quarter_round(s, 3, 7, 11, 15);
        quarter_round(s, 0, 5, 10, 15);
        quarter_round(s, 1, 6, 11, 12);
        quarter_round(s, 2, 7, 8, 13);
        quarter_round(s, 3, 4, 9, 14);
    }
    for (int i = 0; i < 16; i++) {
        uint32_t v = s[i] + init[i];
        out[4 * i + 0] = (uint8_t)v;
        out[4 * i + 1] = (uint8_t)(v >> 8);
        out[4 * i + 2] = (uint8_t)(v >> 16);
        out[4 * i + 3] = (uint8_t)(v >> 24);
    }
}

static void make_nonce(uint8_t nonce[12], uint32_t tag, uint32_t i0, uint32_t i1) {
    uint32_t w[3] = {tag, i0, i1};
    for (int i = 0; i < 3; i++)
        for (int b = 0; b < 4; b++) nonce[4 * i + b] = (uint8_t)(w[i] >> (8 * b));
}

uint64_t oc_stream_word(const uint8_t key[32], uint32_t tag, uint32_t i0,
                        uint32_t i1, uint64_t w) {
    uint8_t nonce[12], blk[64];
    make_nonce(nonce, tag, i0, i1);
    oc_chacha20_block(key, (uint32_t)(w / 8), nonce, blk);
    uint64_t v = 0;
    for (int b = 7; b >= 0; b--) v = (v << 8) | blk[8 * (w % 8) + (uint64_t)b];
    return v;
}

/* Reads `count` consecutive keystream words starting at word 0. */
static void stream_words(const uint8_t key[32], uint32_t tag, uint32_t i0,
                         uint32_t i1, uint64_t count, uint64_t *out) {
    uint8_t nonce[12], blk[64];
    make_nonce(nonce, tag, i0, i1);
    for (uint64_t blkno = 0; blkno * 8 < count; blkno++) {
        oc_chacha20_block(key, (uint32_t)blkno, nonce, blk);
        for (uint64_t k = 0; k < 8 && blkno * 8 + k < count; k++) {
            uint64_t v = 0;
            for (int b = 7; b >= 0; b--) v = (v << 8) | blk[8 * k + (uint64_t)b];
            out[blkno * 8 + k] = v;
        }
    }
}

void oc_cdt_table(uint64_t out[19]) {
    const double two_sigma_sq = 2.0 * 3.2 * 3.2;
    double p[20], total;
    for (int k = 0; k < 20; k++) p[k] = exp(-(double)(k * k) / two_sigma_sq);
    total = p[0];
    for (int k = 1; k < 20; k++) total += 2.0 * p[k];
    double cum = p[0];
    for (int k = 0; k < 19; k++) {
        out[k] = (uint64_t)floor(cum / total * 1099511627776.0 + 0.5); /* 2^40 */
        cum += 2.0 * p[k + 1];
    }
}

void oc_sample_uniform(const uint8_t key[32], uint32_t tag, uint32_t i0,
                       uint32_t i1, const uint64_t *mods, int n_limbs,
                       int log_n, uint64_t *out) {
    uint64_t n = (uint64_t)1 << log_n, total = 2 * n * (uint64_t)n_limbs;
    uint64_t *w = malloc(sizeof(uint64_t) * total);
    stream_words(key, tag, i0, i1, total, w);
    for (int i = 0; i < n_limbs; i++)
        for (uint64_t j = 0; j < n; j++) {
            uint64_t k = (uint64_t)i * n + j;
            oc_u128 v = ((oc_u128)w[2 * k] << 64) | w[2 * k + 1];
            out[k] = (uint64_t)(v % mods[i]);
        }
    free(w);
}

void oc_sample_ternary(const uint8_t key[32], uint32_t tag, uint32_t i0,
                       uint32_t i1, int log_n, int64_t *out) {
    uint64_t n = (uint64_t)1 << log_n;
    uint64_t *w = malloc(sizeof(uint64_t) * n);
    stream_words(key, tag, i0, i1, n, w);
    for (uint64_t j = 0; j < n; j++) out[j] = (int64_t)(w[j] % 3) - 1;
    free(w);
}

void oc_sample_gaussian(const uint8_t key[32], uint32_t tag, uint32_t i0,
                        uint32_t i1, int log_n, int64_t *out) {
    uint64_t n = (uint64_t)1 << log_n, cdt[19];
    uint64_t *w = malloc(sizeof(uint64_t) * n);
    oc_cdt_table(cdt);
    stream_words(key, tag, i0, i1, n, w);
    for (uint64_t j = 0; j < n; j++) {
        uint64_t u = w[j] & (((uint64_t)1 << 40) - 1);
        int64_t mag = 0;
        for (int k = 0; k < 19; k++) mag += (u >= cdt[k]);
        out[j] = (w[j] >> 63) ? -mag : mag;
    }
    free(w);
}
