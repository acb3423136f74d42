/*
 * Oracle: CKKS, BFV and BGV on RNS limbs in coefficient form.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper implements these three schemes (Sec. 1 and 3; operator lists
 * in Tables 1-3: encrypt, decrypt, add, multiply, relinearize, rescale,
 * rotate) but states them only by citation (CKKS: Cheon et al. 2017,
 * BFV: Fan-Vercauteren 2012, BGV: Brakerski-Gentry-Vaikuntanathan 2014;
 * BFV multiplication with an auxiliary basis after Al Badawi et al.).
 * Every function below is the textbook definition, with these readings:
 *
 *  - ciphertexts are pairs (c0, c1) over Q_l = q_0 ... q_{l-1}; decryption
 *    is [c0 + c1 s]_{Q_l} (centred);
 *  - key switching is the hybrid method: beta = ceil(l / alpha) digits
 *    D_j = {q_{j alpha} .. q_{min((j+1) alpha, l) - 1}}, alpha = ceil(L / dnum);
 *    each digit is lifted exactly (centred CRT) to Q_l and the special
 *    primes P = p_0 ... p_{K-1}; the key for s' holds, per digit j and
 *    prime m, b_j = -a_j s + e_j + [m in D_j] (P mod m) s'  (BGV: t e_j);
 *  - ModDown is round(x / P) mod Q_l (CKKS, BFV) and (x - d) / P with
 *    d = t [x t^{-1}]_P (BGV), computed on the big integer x;
 *  - CKKS rescale is round(c / q_{l-1}); BGV modulus switching is
 *    (c - d) / q_{l-1} with d = t [c t^{-1}]_{q_{l-1}}, after which the
 *    plaintext carries the factor q_{l-1}^{-1} mod t;
 *  - BFV multiplication: centred lifts of both ciphertexts to Q u B, their
 *    exact integer tensor product (held exactly in Q u B because
 *    |B| is chosen with prod(B) > 2 t N Q), then round(t x / Q) mod Q;
 *  - rotation applies X -> X^g to both components (g = 5^r mod 2N rotates
 *    CKKS slots left by r) and key switches sigma_g(c1) with the key for
 *    sigma_g(s).
 */
#include <assert.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

typedef struct {
    int scheme, log_n;
    uint64_t n;
    int L, K, nb, alpha, beta;
    uint64_t t;
    uint64_t q[64], p[16], b[64];
    uint64_t psi_q[64], psi_p[16], psi_b[64];
} oc_ctx;

typedef struct {
    uint8_t seed[32];
    int64_t *s;   /* [N] ternary secret                       */
    uint64_t *pk; /* [2][L][N]                                */
    int n_ksk;
    uint64_t ksk_id[256];
    uint64_t *ksk[256]; /* [beta][2][L+K][N]; id 0 relin, g Galois */
} oc_keys;

/* ---------------------------------------------------------------- */

static uint64_t ext_mod(const oc_ctx *c, int level, int i) {
    return i < level ? c->q[i] : c->p[i - level];
}
static uint64_t ext_psi(const oc_ctx *c, int level, int i) {
    return i < level ? c->psi_q[i] : c->psi_p[i - level];
}
/* Key limb of extended position i at level `level`. */
static int key_limb(const oc_ctx *c, int level, int i) {
    return i < level ? i : c->L + (i - level);
}

void *oc_ctx_new(int scheme, int log_n, int log_n_max, int L, const int *q_bits,
                 int K, const int *p_bits, int dnum, uint64_t t, int nb_override,
                 int b_bits) {
    oc_ctx *c = calloc(1, sizeof(oc_ctx));
    uint64_t used[160];
    int n_used = 0;
    uint64_t two_n = (uint64_t)2 << log_n_max;
    c->scheme = scheme;
    c->log_n = log_n;
    c->n = (uint64_t)1 << log_n;
    c->L = L;
    c->K = K;
    c->t = t;
    c->alpha = (L + dnum - 1) / dnum;
    c->beta = (L + c->alpha - 1) / c->alpha;
    for (int i = 0; i < L; i++) {
        if (oc_gen_primes(q_bits[i], 1, two_n, used, n_used, &c->q[i]) != 1) goto fail;
        used[n_used++] = c->q[i];
    }
    for (int i = 0; i < K; i++) {
        if (oc_gen_primes(p_bits[i], 1, two_n, used, n_used, &c->p[i]) != 1) goto fail;
        used[n_used++] = c->p[i];
    }
    if (scheme == OC_BFV) {
        /* Smallest auxiliary basis with prod(B) > 2 t N Q. */
        oc_bn bound, tmp, prodb;
        oc_bn_from_u64(&bound, 2 * t);
        oc_bn_from_u64(&tmp, c->n);
        oc_bn_mul(&bound, &bound, &tmp);
        for (int i = 0; i < L; i++) {
            oc_bn_from_u64(&tmp, c->q[i]);
            oc_bn_mul(&bound, &bound, &tmp);
        }
        oc_bn_from_u64(&prodb, 1);
        int nb = 0;
        while (nb_override > 0 ? nb < nb_override : oc_bn_cmp(&prodb, &bound) <= 0) {
            if (oc_gen_primes(b_bits, 1, two_n, used, n_used, &c->b[nb]) != 1) goto fail;
            used[n_used++] = c->b[nb];
            oc_bn_from_u64(&tmp, c->b[nb]);
            oc_bn_mul(&prodb, &prodb, &tmp);
            nb++;
        }
        c->nb = nb;
    }
    for (int i = 0; i < L; i++) c->psi_q[i] = oc_min_psi(c->q[i], log_n);
    for (int i = 0; i < K; i++) c->psi_p[i] = oc_min_psi(c->p[i], log_n);
    for (int i = 0; i < c->nb; i++) c->psi_b[i] = oc_min_psi(c->b[i], log_n);
    return c;
fail:
    free(c);
    return NULL;
}

void oc_ctx_free(void *ctx) { free(ctx); }

void oc_ctx_moduli(const void *ctx, uint64_t *q, uint64_t *p, uint64_t *b,
                   int *counts /* L, K, nb, alpha, beta */) {
    const oc_ctx *c = ctx;
    if (q) memcpy(q, c->q, sizeof(uint64_t) * (size_t)c->L);
    if (p) memcpy(p, c->p, sizeof(uint64_t) * (size_t)c->K);
    if (b) memcpy(b, c->b, sizeof(uint64_t) * (size_t)c->nb);
    if (counts) {
        counts[0] = c->L; counts[1] = c->K; counts[2] = c->nb;
        counts[3] = c->alpha; counts[4] = c->beta;
    }
}

/* ---------------------------------------------------------------- */
/* Base conversions on big integers (per coefficient).              */

/* dst[t][x] = (centred CRT of src[.][x] over src_mod) mod dst_mod[t]. */
void oc_lift_centred(const uint64_t *src, const uint64_t *src_mod, int k,
                     const uint64_t *dst_mod, int T, uint64_t *dst, uint64_t n) {
    oc_basis *bs = malloc(sizeof(oc_basis));
    oc_basis_init(bs, src_mod, k);
    uint64_t r[64];
    oc_bn x;
    for (uint64_t j = 0; j < n; j++) {
        for (int i = 0; i < k; i++) r[i] = src[(uint64_t)i * n + j];
        oc_crt_centred(&x, bs, r);
        for (int t = 0; t < T; t++) dst[(uint64_t)t * n + j] = oc_bn_mod_u64(&x, dst_mod[t]);
    }
    free(bs);
}

/* Residues src[0..kq+kd) of x over (q_0..q_{kq-1}, d_0..d_{kd-1}); writes
 * round(x / D) mod q_i, D = prod d, for x the representative in [0, QD). */
void oc_div_round(const uint64_t *src, const uint64_t *mods, int kq, int kd,
                  uint64_t *dst, uint64_t n) {
    oc_basis *bs = malloc(sizeof(oc_basis));
    oc_basis_init(bs, mods, kq + kd);
    oc_bn D, tmp, twoD, num, y;
    oc_bn_from_u64(&D, 1);
    for (int i = 0; i < kd; i++) {
        oc_bn_from_u64(&tmp, mods[kq + i]);
        oc_bn_mul(&D, &D, &tmp);
    }
    oc_bn_add(&twoD, &D, &D);
    uint64_t r[64];
    oc_bn x;
    for (uint64_t j = 0; j < n; j++) {
        for (int i = 0; i < kq + kd; i++) r[i] = src[(uint64_t)i * n + j];
        oc_crt(&x, bs, r);
        /* round(x/D) = floor((2x + D) / 2D); D is odd so there is no tie. */
        oc_bn_add(&num, &x, &x);
        oc_bn_add(&num, &num, &D);
        oc_bn_divmod_floor(&y, NULL, &num, &twoD);
        for (int i = 0; i < kq; i++) dst[(uint64_t)i * n + j] = oc_bn_mod_u64(&y, mods[i]);
    }
    free(bs);
}

/* Same inputs; writes (x - d) / D mod q_i with d = t [x t^{-1}]_D (centred):
 * the division that keeps the plaintext modulo t (BGV). */
void oc_div_t_exact(const uint64_t *src, const uint64_t *mods, int kq, int kd,
                    uint64_t t, uint64_t *dst, uint64_t n) {
    oc_basis *bs = malloc(sizeof(oc_basis)), *bd = malloc(sizeof(oc_basis));
    oc_basis_init(bs, mods, kq + kd);
    oc_basis_init(bd, mods + kq, kd);
    uint64_t tinv_res[64];
    for (int i = 0; i < kd; i++) tinv_res[i] = oc_invmod(t % mods[kq + i], mods[kq + i]);
    oc_bn tinv, tb, x, xd, u, twice, d, diff, y, rem;
    oc_crt(&tinv, bd, tinv_res); /* t^{-1} mod D */
    oc_bn_from_u64(&tb, t);
    uint64_t r[64];
    for (uint64_t j = 0; j < n; j++) {
        for (int i = 0; i < kq + kd; i++) r[i] = src[(uint64_t)i * n + j];
        oc_crt(&x, bs, r);
        oc_bn_divmod_floor(NULL, &xd, &x, &bd->M);   /* x mod D          */
        oc_bn_mul(&u, &xd, &tinv);
        oc_bn_divmod_floor(NULL, &u, &u, &bd->M);    /* x t^{-1} mod D   */
        oc_bn_add(&twice, &u, &u);
        if (oc_bn_cmp(&twice, &bd->M) > 0) oc_bn_sub(&u, &u, &bd->M); /* centred */
        oc_bn_mul(&d, &u, &tb);
        oc_bn_sub(&diff, &x, &d);
        oc_bn_divmod_floor(&y, &rem, &diff, &bd->M);
        assert(rem.n == 0);
        for (int i = 0; i < kq; i++) dst[(uint64_t)i * n + j] = oc_bn_mod_u64(&y, mods[i]);
    }
    free(bs);
    free(bd);
}

/* ---------------------------------------------------------------- */
/* Polynomial helpers.                                              */

static void poly_from_small(uint64_t *out, const int64_t *s, uint64_t n, uint64_t m) {
    for (uint64_t j = 0; j < n; j++) out[j] = oc_reduce_i64(s[j], m);
}

/* sigma_g(a)(X) = a(X^g) in Z_m[X]/(X^N + 1): coefficient i moves to i*g
 * mod 2N, negated when that index is >= N. */
void oc_automorphism(uint64_t *out, const uint64_t *a, uint64_t n, uint64_t g, uint64_t m) {
    for (uint64_t i = 0; i < n; i++) {
        uint64_t k = (i * g) % (2 * n);
        if (k < n) out[k] = a[i];
        else out[k - n] = a[i] ? m - a[i] : 0;
    }
}

static void automorphism_small(int64_t *out, const int64_t *a, uint64_t n, uint64_t g) {
    for (uint64_t i = 0; i < n; i++) {
        uint64_t k = (i * g) % (2 * n);
        if (k < n) out[k] = a[i];
        else out[k - n] = -a[i];
    }
}

/* ---------------------------------------------------------------- */
/* Keys.                                                            */

static void gen_ksk(const oc_ctx *c, oc_keys *k, uint64_t id, const uint64_t *sp /* [L+K][N] */) {
    uint64_t n = c->n;
    int M = c->L + c->K;
    uint64_t mods[80];
    for (int i = 0; i < M; i++) mods[i] = ext_mod(c, c->L, i);
    uint64_t *key = malloc(sizeof(uint64_t) * (size_t)c->beta * 2 * (size_t)M * n);
    uint64_t *a = malloc(sizeof(uint64_t) * (size_t)M * n);
    int64_t *e = malloc(sizeof(int64_t) * n);
    uint64_t *s_i = malloc(sizeof(uint64_t) * n), *as = malloc(sizeof(uint64_t) * n);
    uint64_t te = (c->scheme == OC_BGV) ? c->t : 1;
    for (int j = 0; j < c->beta; j++) {
        oc_sample_uniform(k->seed, OC_TAG_KSK_A, (uint32_t)j, (uint32_t)id, mods, M, c->log_n, a);
        oc_sample_gaussian(k->seed, OC_TAG_KSK_E, (uint32_t)j, (uint32_t)id, c->log_n, e);
        for (int i = 0; i < M; i++) {
            uint64_t m = mods[i];
            uint64_t *bj = key + (((size_t)j * 2 + 0) * (size_t)M + (size_t)i) * n;
            uint64_t *aj = key + (((size_t)j * 2 + 1) * (size_t)M + (size_t)i) * n;
            poly_from_small(s_i, k->s, n, m);
            oc_negacyclic_mul(as, a + (size_t)i * n, s_i, c->log_n, m, ext_psi(c, c->L, i));
            /* P mod m for a digit prime of D_j, else 0 (P = 0 mod p_k). */
            uint64_t pfac = 0;
            if (i < c->L && i / c->alpha == j) {
                pfac = 1;
                for (int kk = 0; kk < c->K; kk++) pfac = oc_mulmod(pfac, c->p[kk] % m, m);
            }
            for (uint64_t x = 0; x < n; x++) {
                uint64_t v = oc_submod(oc_mulmod(te % m, oc_reduce_i64(e[x], m), m), as[x], m);
                v = oc_addmod(v, oc_mulmod(pfac, sp[(size_t)i * n + x], m), m);
                bj[x] = v;
                aj[x] = a[(size_t)i * n + x];
            }
        }
    }
    k->ksk_id[k->n_ksk] = id;
    k->ksk[k->n_ksk] = key;
    k->n_ksk++;
    free(a); free(e); free(s_i); free(as);
}

static const uint64_t *find_ksk(const oc_keys *k, uint64_t id) {
    for (int i = 0; i < k->n_ksk; i++)
        if (k->ksk_id[i] == id) return k->ksk[i];
    return NULL;
}

void *oc_keygen(const void *ctx, const uint8_t seed[32]) {
    const oc_ctx *c = ctx;
    uint64_t n = c->n;
    int L = c->L, M = c->L + c->K;
    oc_keys *k = calloc(1, sizeof(oc_keys));
    memcpy(k->seed, seed, 32);
    k->s = malloc(sizeof(int64_t) * n);
    oc_sample_ternary(seed, OC_TAG_SK, 0, 0, c->log_n, k->s);

    /* Public key (-a s + e, a) over Q_L (BGV: t e). */
    k->pk = malloc(sizeof(uint64_t) * 2 * (size_t)L * n);
    uint64_t *a = malloc(sizeof(uint64_t) * (size_t)L * n);
    int64_t *e = malloc(sizeof(int64_t) * n);
    uint64_t *s_i = malloc(sizeof(uint64_t) * n), *as = malloc(sizeof(uint64_t) * n);
    oc_sample_uniform(seed, OC_TAG_PK_A, 0, 0, c->q, L, c->log_n, a);
    oc_sample_gaussian(seed, OC_TAG_PK_E, 0, 0, c->log_n, e);
    uint64_t te = (c->scheme == OC_BGV) ? c->t : 1;
    for (int i = 0; i < L; i++) {
        uint64_t m = c->q[i];
        poly_from_small(s_i, k->s, n, m);
        oc_negacyclic_mul(as, a + (size_t)i * n, s_i, c->log_n, m, c->psi_q[i]);
        for (uint64_t x = 0; x < n; x++) {
            k->pk[(size_t)i * n + x] =
                oc_submod(oc_mulmod(te % m, oc_reduce_i64(e[x], m), m), as[x], m);
            k->pk[((size_t)L + (size_t)i) * n + x] = a[(size_t)i * n + x];
        }
    }
    /* Relinearisation key: s' = s^2. */
    uint64_t *sp = malloc(sizeof(uint64_t) * (size_t)M * n);
    for (int i = 0; i < M; i++) {
        uint64_t m = ext_mod(c, L, i);
        poly_from_small(s_i, k->s, n, m);
        oc_negacyclic_mul(sp + (size_t)i * n, s_i, s_i, c->log_n, m, ext_psi(c, L, i));
    }
    gen_ksk(c, k, 0, sp);
    free(a); free(e); free(s_i); free(as); free(sp);
    return k;
}

/* Galois key for X -> X^g: s' = sigma_g(s). */
int oc_gen_galois(const void *ctx, void *keys, uint64_t g) {
    const oc_ctx *c = ctx;
    oc_keys *k = keys;
    if (find_ksk(k, g)) return 0;
    if (k->n_ksk >= 256 || (g & 1) == 0) return -1;
    uint64_t n = c->n;
    int M = c->L + c->K;
    int64_t *sg = malloc(sizeof(int64_t) * n);
    uint64_t *sp = malloc(sizeof(uint64_t) * (size_t)M * n);
    automorphism_small(sg, k->s, n, g % (2 * n));
    for (int i = 0; i < M; i++) poly_from_small(sp + (size_t)i * n, sg, n, ext_mod(c, c->L, i));
    gen_ksk(c, k, g % (2 * n), sp);
    free(sg);
    free(sp);
    return 0;
}

void oc_keys_free(void *keys) {
    oc_keys *k = keys;
    if (!k) return;
    free(k->s);
    free(k->pk);
    for (int i = 0; i < k->n_ksk; i++) free(k->ksk[i]);
    free(k);
}

void oc_keys_export(const void *ctx, const void *keys, int64_t *s, uint64_t *pk) {
    const oc_ctx *c = ctx;
    const oc_keys *k = keys;
    if (s) memcpy(s, k->s, sizeof(int64_t) * c->n);
    if (pk) memcpy(pk, k->pk, sizeof(uint64_t) * 2 * (size_t)c->L * c->n);
}

int oc_ksk_export(const void *ctx, const void *keys, uint64_t id, uint64_t *out) {
    const oc_ctx *c = ctx;
    const uint64_t *key = find_ksk(keys, id);
    if (!key) return -1;
    memcpy(out, key, sizeof(uint64_t) * (size_t)c->beta * 2 * (size_t)(c->L + c->K) * c->n);
    return 0;
}

/* ---------------------------------------------------------------- */
/* Encryption, decryption, uniform ciphertexts.                     */

void oc_encrypt(const void *ctx, const void *keys, const int64_t *msg,
                const uint8_t seed[32], uint64_t *out /* [2][L][N] */) {
    const oc_ctx *c = ctx;
    const oc_keys *k = keys;
    uint64_t n = c->n;
    int L = c->L;
    int64_t *v = malloc(sizeof(int64_t) * n), *e0 = malloc(sizeof(int64_t) * n),
            *e1 = malloc(sizeof(int64_t) * n);
    uint64_t *v_i = malloc(sizeof(uint64_t) * n), *t0 = malloc(sizeof(uint64_t) * n),
             *t1 = malloc(sizeof(uint64_t) * n);
    oc_sample_ternary(seed, OC_TAG_ENC_V, 0, 0, c->log_n, v);
    oc_sample_gaussian(seed, OC_TAG_ENC_E0, 0, 0, c->log_n, e0);
    oc_sample_gaussian(seed, OC_TAG_ENC_E1, 0, 0, c->log_n, e1);
    uint64_t te = (c->scheme == OC_BGV) ? c->t : 1;
    /* BFV: Delta = floor(Q / t). */
    oc_bn Q, tmp, delta;
    oc_bn_from_u64(&Q, 1);
    for (int i = 0; i < L; i++) {
        oc_bn_from_u64(&tmp, c->q[i]);
        oc_bn_mul(&Q, &Q, &tmp);
    }
    oc_bn_from_u64(&tmp, c->t ? c->t : 1);
    oc_bn_divmod_floor(&delta, NULL, &Q, &tmp);
    for (int i = 0; i < L; i++) {
        uint64_t m = c->q[i];
        poly_from_small(v_i, v, n, m);
        oc_negacyclic_mul(t0, v_i, k->pk + (size_t)i * n, c->log_n, m, c->psi_q[i]);
        oc_negacyclic_mul(t1, v_i, k->pk + ((size_t)L + (size_t)i) * n, c->log_n, m, c->psi_q[i]);
        uint64_t dm = oc_bn_mod_u64(&delta, m);
        for (uint64_t x = 0; x < n; x++) {
            uint64_t mm = oc_reduce_i64(msg[x], m);
            if (c->scheme == OC_BFV) mm = oc_mulmod(dm, mm, m);
            uint64_t c0 = oc_addmod(t0[x], oc_mulmod(te % m, oc_reduce_i64(e0[x], m), m), m);
            out[(size_t)i * n + x] = oc_addmod(c0, mm, m);
            out[((size_t)L + (size_t)i) * n + x] =
                oc_addmod(t1[x], oc_mulmod(te % m, oc_reduce_i64(e1[x], m), m), m);
        }
    }
    free(v); free(e0); free(e1); free(v_i); free(t0); free(t1);
}

void oc_ct_uniform(const void *ctx, const uint8_t seed[32], uint32_t ct_index, int level,
                   uint64_t *out /* [2][level][N] */) {
    const oc_ctx *c = ctx;
    for (uint32_t poly = 0; poly < 2; poly++)
        oc_sample_uniform(seed, OC_TAG_CT_UNIFORM, poly, ct_index, c->q, level, c->log_n,
                          out + (size_t)poly * (size_t)level * c->n);
}

/* x = [c0 + c1 s]_{Q_l} centred; CKKS: x (two's complement mod 2^64);
 * BFV: round(t x / Q_l) mod t; BGV: x factor^{-1} mod t. */
void oc_decrypt(const void *ctx, const void *keys, const uint64_t *ct, int level,
                uint64_t factor, int64_t *out) {
    const oc_ctx *c = ctx;
    const oc_keys *k = keys;
    uint64_t n = c->n;
    uint64_t *x = malloc(sizeof(uint64_t) * (size_t)level * n);
    uint64_t *s_i = malloc(sizeof(uint64_t) * n), *cs = malloc(sizeof(uint64_t) * n);
    for (int i = 0; i < level; i++) {
        uint64_t m = c->q[i];
        poly_from_small(s_i, k->s, n, m);
        oc_negacyclic_mul(cs, ct + ((size_t)level + (size_t)i) * n, s_i, c->log_n, m, c->psi_q[i]);
        for (uint64_t j = 0; j < n; j++) x[(size_t)i * n + j] = oc_addmod(ct[(size_t)i * n + j], cs[j], m);
    }
    oc_basis *bs = malloc(sizeof(oc_basis));
    oc_basis_init(bs, c->q, level);
    oc_bn X, tb, num, twoQ, y;
    oc_bn_from_u64(&tb, c->t ? c->t : 1);
    oc_bn_add(&twoQ, &bs->M, &bs->M);
    uint64_t finv = (c->scheme == OC_BGV) ? oc_invmod(factor % c->t, c->t) : 1;
    uint64_t r[64];
    for (uint64_t j = 0; j < n; j++) {
        for (int i = 0; i < level; i++) r[i] = x[(size_t)i * n + j];
        oc_crt_centred(&X, bs, r);
        if (c->scheme == OC_CKKS) {
            out[j] = oc_bn_to_i64_wrap(&X);
        } else if (c->scheme == OC_BFV) {
            /* round(t X / Q) = floor((2 t X + Q) / 2Q) */
            oc_bn_mul(&num, &X, &tb);
            oc_bn_add(&num, &num, &num);
            oc_bn_add(&num, &num, &bs->M);
            oc_bn_divmod_floor(&y, NULL, &num, &twoQ);
            out[j] = (int64_t)oc_bn_mod_u64(&y, c->t);
        } else {
            out[j] = (int64_t)oc_mulmod(oc_bn_mod_u64(&X, c->t), finv, c->t);
        }
    }
    free(bs); free(x); free(s_i); free(cs);
}

/* ---------------------------------------------------------------- */
/* Homomorphic operations.                                          */

void oc_add(const void *ctx, const uint64_t *a, const uint64_t *b, uint64_t *out, int level) {
    const oc_ctx *c = ctx;
    uint64_t n = c->n;
    for (int p = 0; p < 2; p++)
        for (int i = 0; i < level; i++)
            for (uint64_t j = 0; j < n; j++) {
                size_t o = ((size_t)p * (size_t)level + (size_t)i) * n + j;
                out[o] = oc_addmod(a[o], b[o], c->q[i]);
            }
}

/* Ciphertext subtraction (Table 1 "sub"): out = a - b limb by limb. */
void oc_sub(const void *ctx, const uint64_t *a, const uint64_t *b, uint64_t *out, int level) {
    const oc_ctx *c = ctx;
    uint64_t n = c->n;
    for (int p = 0; p < 2; p++)
        for (int i = 0; i < level; i++)
            for (uint64_t j = 0; j < n; j++) {
                size_t o = ((size_t)p * (size_t)level + (size_t)i) * n + j;
                out[o] = oc_submod(a[o], b[o], c->q[i]);
            }
}

/* Multiplication by the integer k (a constant plaintext, Table 1
 * "multiply_plain"): both polynomials times k mod q_i. */
void oc_mul_int(const void *ctx, const uint64_t *a, int64_t k, uint64_t *out, int level) {
    const oc_ctx *c = ctx;
    uint64_t n = c->n;
    for (int p = 0; p < 2; p++)
        for (int i = 0; i < level; i++) {
            uint64_t kq = oc_reduce_i64(k, c->q[i]);
            for (uint64_t j = 0; j < n; j++) {
                size_t o = ((size_t)p * (size_t)level + (size_t)i) * n + j;
                out[o] = oc_mulmod(a[o], kq, c->q[i]);
            }
        }
}

/* Adds the constant polynomial k to the plaintext: coefficient 0 of c0
 * plus k mod q_i (coefficient form); everything else copied. */
void oc_add_const(const void *ctx, const uint64_t *a, int64_t k, uint64_t *out, int level) {
    const oc_ctx *c = ctx;
    uint64_t n = c->n;
    memcpy(out, a, sizeof(uint64_t) * 2 * (size_t)level * n);
    for (int i = 0; i < level; i++)
        out[(size_t)i * n] = oc_addmod(a[(size_t)i * n], oc_reduce_i64(k, c->q[i]), c->q[i]);
}

/* Multiplication by a plaintext polynomial (Table 1 "multiply_plain"): each
 * polynomial of the ciphertext times pt (signed coefficients reduced mod
 * q_i), a negacyclic product per limb. */
void oc_mul_plain(const void *ctx, const uint64_t *a, const int64_t *pt, uint64_t *out, int level) {
    const oc_ctx *c = ctx;
    uint64_t n = c->n;
    uint64_t *pi = malloc(sizeof(uint64_t) * n);
    for (int i = 0; i < level; i++) {
        uint64_t m = c->q[i];
        for (uint64_t j = 0; j < n; j++) pi[j] = oc_reduce_i64(pt[j], m);
        for (int p = 0; p < 2; p++) {
            size_t o = ((size_t)p * (size_t)level + (size_t)i) * n;
            oc_negacyclic_mul(out + o, a + o, pi, c->log_n, m, c->psi_q[i]);
        }
    }
    free(pi);
}

/* Level drop: keeps the limbs of q_0 .. q_{new_level-1} of each polynomial. */
void oc_drop(const void *ctx, const uint64_t *a, int level, int new_level, uint64_t *out) {
    const oc_ctx *c = ctx;
    uint64_t n = c->n;
    for (int p = 0; p < 2; p++)
        memcpy(out + (size_t)p * (size_t)new_level * n, a + (size_t)p * (size_t)level * n,
               sizeof(uint64_t) * (size_t)new_level * n);
}

/* Key switch of one polynomial cin (over Q_l) with key `id`:
 * (k0, k1) with k0 + k1 s = cin s' + small (CKKS, BFV) or + t small (BGV). */
int oc_keyswitch(const void *ctx, const void *keys, const uint64_t *cin, int level,
                 uint64_t id, uint64_t *out /* [2][level][N] */) {
    const oc_ctx *c = ctx;
    const uint64_t *key = find_ksk(keys, id);
    if (!key) return -1;
    uint64_t n = c->n;
    int M = level + c->K, Mk = c->L + c->K;
    int beta = (level + c->alpha - 1) / c->alpha;
    uint64_t mods[80];
    for (int i = 0; i < M; i++) mods[i] = ext_mod(c, level, i);
    uint64_t *acc = calloc((size_t)2 * (size_t)M * n, sizeof(uint64_t));
    uint64_t *hat = malloc(sizeof(uint64_t) * (size_t)M * n);
    uint64_t *prod = malloc(sizeof(uint64_t) * n);
    for (int j = 0; j < beta; j++) {
        int lo = j * c->alpha, hi = (j + 1) * c->alpha < level ? (j + 1) * c->alpha : level;
        /* Exact centred lift of the digit c mod D_j to every prime of Q_l u P. */
        oc_lift_centred(cin + (size_t)lo * n, c->q + lo, hi - lo, mods, M, hat, n);
        for (int i = 0; i < M; i++) {
            int kl = key_limb(c, level, i);
            for (int poly = 0; poly < 2; poly++) {
                const uint64_t *kp = key + (((size_t)j * 2 + (size_t)poly) * (size_t)Mk + (size_t)kl) * n;
                oc_negacyclic_mul(prod, hat + (size_t)i * n, kp, c->log_n, mods[i], ext_psi(c, level, i));
                uint64_t *ap = acc + ((size_t)poly * (size_t)M + (size_t)i) * n;
                for (uint64_t x = 0; x < n; x++) ap[x] = oc_addmod(ap[x], prod[x], mods[i]);
            }
        }
    }
    for (int poly = 0; poly < 2; poly++) {
        const uint64_t *ap = acc + (size_t)poly * (size_t)M * n;
        uint64_t *op = out + (size_t)poly * (size_t)level * n;
        if (c->scheme == OC_BGV) oc_div_t_exact(ap, mods, level, c->K, c->t, op, n);
        else oc_div_round(ap, mods, level, c->K, op, n);
    }
    free(acc); free(hat); free(prod);
    return 0;
}

/* CKKS rescale / BGV modulus switch of one ciphertext from level l to l-1. */
void oc_rescale(const void *ctx, const uint64_t *a, uint64_t *out, int level) {
    const oc_ctx *c = ctx;
    uint64_t n = c->n;
    for (int poly = 0; poly < 2; poly++) {
        const uint64_t *ap = a + (size_t)poly * (size_t)level * n;
        uint64_t *op = out + (size_t)poly * (size_t)(level - 1) * n;
        if (c->scheme == OC_BGV) oc_div_t_exact(ap, c->q, level - 1, 1, c->t, op, n);
        else oc_div_round(ap, c->q, level - 1, 1, op, n);
    }
}

static void tensor(const oc_ctx *c, const uint64_t *a, const uint64_t *b, int limbs,
                   const uint64_t *mods, const uint64_t *psis, uint64_t *d /* [3][limbs][N] */) {
    uint64_t n = c->n;
    uint64_t *t = malloc(sizeof(uint64_t) * n);
    for (int i = 0; i < limbs; i++) {
        const uint64_t *a0 = a + (size_t)i * n, *a1 = a + ((size_t)limbs + (size_t)i) * n;
        const uint64_t *b0 = b + (size_t)i * n, *b1 = b + ((size_t)limbs + (size_t)i) * n;
        uint64_t *d0 = d + (size_t)i * n, *d1 = d + ((size_t)limbs + (size_t)i) * n,
                 *d2 = d + (2 * (size_t)limbs + (size_t)i) * n;
        oc_negacyclic_mul(d0, a0, b0, c->log_n, mods[i], psis[i]);
        oc_negacyclic_mul(d1, a0, b1, c->log_n, mods[i], psis[i]);
        oc_negacyclic_mul(t, a1, b0, c->log_n, mods[i], psis[i]);
        for (uint64_t x = 0; x < n; x++) d1[x] = oc_addmod(d1[x], t[x], mods[i]);
        oc_negacyclic_mul(d2, a1, b1, c->log_n, mods[i], psis[i]);
    }
    free(t);
}

/* BFV tensor: lift to Q u B, exact product, round(t x / Q) mod Q_l. */
static void bfv_tensor(const oc_ctx *c, const uint64_t *a, const uint64_t *b, int level,
                       uint64_t *d /* [3][level][N] */) {
    uint64_t n = c->n;
    int kb = level + c->nb;
    uint64_t mods[128], psis[128];
    for (int i = 0; i < level; i++) { mods[i] = c->q[i]; psis[i] = c->psi_q[i]; }
    for (int i = 0; i < c->nb; i++) { mods[level + i] = c->b[i]; psis[level + i] = c->psi_b[i]; }
    uint64_t *A = malloc(sizeof(uint64_t) * 2 * (size_t)kb * n);
    uint64_t *Bx = malloc(sizeof(uint64_t) * 2 * (size_t)kb * n);
    uint64_t *D = malloc(sizeof(uint64_t) * 3 * (size_t)kb * n);
    for (int poly = 0; poly < 2; poly++) {
        oc_lift_centred(a + (size_t)poly * (size_t)level * n, c->q, level, mods, kb,
                        A + (size_t)poly * (size_t)kb * n, n);
        oc_lift_centred(b + (size_t)poly * (size_t)level * n, c->q, level, mods, kb,
                        Bx + (size_t)poly * (size_t)kb * n, n);
    }
    tensor(c, A, Bx, kb, mods, psis, D);
    oc_basis *bs = malloc(sizeof(oc_basis)), *bq = malloc(sizeof(oc_basis));
    oc_basis_init(bs, mods, kb);
    oc_basis_init(bq, c->q, level);
    oc_bn X, tb, num, twoQ, y;
    oc_bn_from_u64(&tb, c->t);
    oc_bn_add(&twoQ, &bq->M, &bq->M);
    uint64_t r[128];
    for (int poly = 0; poly < 3; poly++)
        for (uint64_t j = 0; j < n; j++) {
            for (int i = 0; i < kb; i++) r[i] = D[((size_t)poly * (size_t)kb + (size_t)i) * n + j];
            oc_crt_centred(&X, bs, r); /* the exact integer coefficient */
            oc_bn_mul(&num, &X, &tb);
            oc_bn_add(&num, &num, &num);
            oc_bn_add(&num, &num, &bq->M);
            oc_bn_divmod_floor(&y, NULL, &num, &twoQ);
            for (int i = 0; i < level; i++)
                d[((size_t)poly * (size_t)level + (size_t)i) * n + j] = oc_bn_mod_u64(&y, c->q[i]);
        }
    free(A); free(Bx); free(D); free(bs); free(bq);
}

int oc_mul_relin(const void *ctx, const void *keys, const uint64_t *a, const uint64_t *b,
                 uint64_t *out, int level) {
    const oc_ctx *c = ctx;
    uint64_t n = c->n;
    size_t lim = (size_t)level * n;
    uint64_t *d = malloc(sizeof(uint64_t) * 3 * lim);
    uint64_t *ks = malloc(sizeof(uint64_t) * 2 * lim);
    if (c->scheme == OC_BFV) bfv_tensor(c, a, b, level, d);
    else tensor(c, a, b, level, c->q, c->psi_q, d);
    int rc = oc_keyswitch(ctx, keys, d + 2 * lim, level, 0, ks);
    if (rc == 0)
        for (int poly = 0; poly < 2; poly++)
            for (int i = 0; i < level; i++)
                for (uint64_t x = 0; x < n; x++) {
                    size_t o = (size_t)poly * lim + (size_t)i * n + x;
                    out[o] = oc_addmod(d[o], ks[o], c->q[i]);
                }
    free(d);
    free(ks);
    return rc;
}

/* The three tensor components before relinearisation (for step checks). */
void oc_tensor(const void *ctx, const uint64_t *a, const uint64_t *b, uint64_t *d, int level) {
    const oc_ctx *c = ctx;
    if (c->scheme == OC_BFV) bfv_tensor(c, a, b, level, d);
    else tensor(c, a, b, level, c->q, c->psi_q, d);
}

int oc_rotate(const void *ctx, const void *keys, const uint64_t *a, uint64_t *out,
              int level, uint64_t g) {
    const oc_ctx *c = ctx;
    uint64_t n = c->n;
    size_t lim = (size_t)level * n;
    g %= 2 * n;
    uint64_t *s0 = malloc(sizeof(uint64_t) * lim), *s1 = malloc(sizeof(uint64_t) * lim);
    uint64_t *ks = malloc(sizeof(uint64_t) * 2 * lim);
    for (int i = 0; i < level; i++) {
        oc_automorphism(s0 + (size_t)i * n, a + (size_t)i * n, n, g, c->q[i]);
        oc_automorphism(s1 + (size_t)i * n, a + lim + (size_t)i * n, n, g, c->q[i]);
    }
    int rc = oc_keyswitch(ctx, keys, s1, level, g, ks);
    if (rc == 0) {
        for (int i = 0; i < level; i++)
            for (uint64_t x = 0; x < n; x++) {
                size_t o = (size_t)i * n + x;
                out[o] = oc_addmod(s0[o], ks[o], c->q[i]);
                out[lim + o] = ks[lim + o];
            }
    }
    free(s0); free(s1); free(ks);
    return rc;
}

/* Galois element for a left rotation of CKKS slots (BFV/BGV rows) by r. */
uint64_t oc_galois_elt(int log_n, int64_t r) {
    uint64_t two_n = (uint64_t)2 << log_n, slots = (uint64_t)1 << (log_n - 1);
    uint64_t e = (uint64_t)(((r % (int64_t)slots) + (int64_t)slots) % (int64_t)slots);
    return oc_powmod(5, e, two_n);
}
