/*
 * Oracle: sign-magnitude arbitrary precision integers (32-bit words) and
 * the Chinese remainder reconstruction.  TEST INFRASTRUCTURE ONLY.
 *
 * Division is the schoolbook long division of Knuth (TAOCP vol. 2,
 * Sec. 4.3.1, Algorithm D).  The CRT reconstruction is the textbook
 * formula x = sum_i r_i (M/m_i) [(M/m_i)^{-1}]_{m_i} mod M, which is what
 * the paper's RNS representation (Sec. 2.2) relies on.
 */
#include <assert.h>
#include <string.h>
#include "oracle.h"

#define B32 ((uint64_t)1 << 32)

static int mag_norm(const uint32_t *w, int n) {
    while (n > 0 && w[n - 1] == 0) n--;
    return n;
}

static int mag_cmp(const uint32_t *a, int an, const uint32_t *b, int bn) {
    if (an != bn) return an < bn ? -1 : 1;
    for (int i = an - 1; i >= 0; i--)
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    return 0;
}

static int mag_add(uint32_t *r, const uint32_t *a, int an, const uint32_t *b, int bn) {
    int n = an > bn ? an : bn;
    uint64_t carry = 0;
    for (int i = 0; i < n; i++) {
        uint64_t s = carry;
        if (i < an) s += a[i];
        if (i < bn) s += b[i];
        r[i] = (uint32_t)s;
        carry = s >> 32;
    }
    assert(n < OC_BN_WORDS);
    r[n] = (uint32_t)carry;
    return mag_norm(r, n + 1);
}

/* r = a - b for |a| >= |b|. */
static int mag_sub(uint32_t *r, const uint32_t *a, int an, const uint32_t *b, int bn) {
    uint64_t borrow = 0;
    for (int i = 0; i < an; i++) {
        uint64_t sub = borrow + (i < bn ? b[i] : 0);
        uint64_t cur = a[i];
        if (cur >= sub) { r[i] = (uint32_t)(cur - sub); borrow = 0; }
        else { r[i] = (uint32_t)(cur + B32 - sub); borrow = 1; }
    }
    assert(borrow == 0);
    return mag_norm(r, an);
}

static int mag_mul(uint32_t *r, const uint32_t *a, int an, const uint32_t *b, int bn) {
    uint32_t tmp[OC_BN_WORDS];
    assert(an + bn <= OC_BN_WORDS);
    memset(tmp, 0, sizeof(uint32_t) * (size_t)(an + bn));
    for (int i = 0; i < an; i++) {
        uint64_t carry = 0;
        for (int j = 0; j < bn; j++) {
            uint64_t t = (uint64_t)a[i] * b[j] + tmp[i + j] + carry;
            tmp[i + j] = (uint32_t)t;
            carry = t >> 32;
        }
        tmp[i + bn] = (uint32_t)carry;
    }
    memcpy(r, tmp, sizeof(uint32_t) * (size_t)(an + bn));
    return mag_norm(r, an + bn);
}

static int clz32(uint32_t x) {
    int n = 0;
    while (!(x & 0x80000000u)) { x <<= 1; n++; }
    return n;
}

/* Long division of magnitudes: u = q v + r, 0 <= r < v (v != 0). */
static void mag_divmod(uint32_t *q, int *qn, uint32_t *r, int *rn,
                       const uint32_t *u, int un, const uint32_t *v, int vn) {
    assert(vn > 0 && v[vn - 1] != 0);
    if (mag_cmp(u, un, v, vn) < 0) {
        memcpy(r, u, sizeof(uint32_t) * (size_t)un);
        *rn = un;
        *qn = 0;
        return;
    }
    if (vn == 1) {
        uint64_t rem = 0;
        for (int i = un - 1; i >= 0; i--) {
            uint64_t cur = (rem << 32) | u[i];
            q[i] = (uint32_t)(cur / v[0]);
            rem = cur % v[0];
        }
        *qn = mag_norm(q, un);
        r[0] = (uint32_t)rem;
        *rn = rem ? 1 : 0;
        return;
    }
    /* Normalise so that the top word of the divisor has its high bit set. */
    int s = clz32(v[vn - 1]);
    uint32_t vs[OC_BN_WORDS], us[OC_BN_WORDS + 1];
    for (int i = vn - 1; i > 0; i--)
        vs[i] = (v[i] << s) | (s ? (uint32_t)((uint64_t)v[i - 1] >> (32 - s)) : 0);
    vs[0] = v[0] << s;
    us[un] = s ? (uint32_t)((uint64_t)u[un - 1] >> (32 - s)) : 0;
    for (int i = un - 1; i > 0; i--)
        us[i] = (u[i] << s) | (s ? (uint32_t)((uint64_t)u[i - 1] >> (32 - s)) : 0);
    us[0] = u[0] << s;

    for (int j = un - vn; j >= 0; j--) {
        /* Estimate the quotient word from the top two words of the window. */
        uint64_t num = ((uint64_t)us[j + vn] << 32) | us[j + vn - 1];
        uint64_t qhat = num / vs[vn - 1];
        uint64_t rhat = num % vs[vn - 1];
        while (qhat >= B32 || qhat * vs[vn - 2] > ((rhat << 32) | us[j + vn - 2])) {
            qhat--;
            rhat += vs[vn - 1];
            if (rhat >= B32) break;
        }
        /* Subtract qhat * v from the window us[j .. j+vn]. */
        uint64_t carry = 0, borrow = 0;
        for (int i = 0; i < vn; i++) {
            uint64_t p = qhat * vs[i] + carry;
            carry = p >> 32;
            uint64_t sub = (p & 0xffffffffu) + borrow;
            uint64_t cur = us[i + j];
            if (cur >= sub) { us[i + j] = (uint32_t)(cur - sub); borrow = 0; }
            else { us[i + j] = (uint32_t)(cur + B32 - sub); borrow = 1; }
        }
        uint64_t sub = carry + borrow;
        uint64_t cur = us[j + vn];
        int negative = cur < sub;
        us[j + vn] = (uint32_t)(cur + (negative ? B32 : 0) - sub);
        if (negative) {
            /* qhat was one too large: add v back. */
            qhat--;
            uint64_t c = 0;
            for (int i = 0; i < vn; i++) {
                uint64_t t = (uint64_t)us[i + j] + vs[i] + c;
                us[i + j] = (uint32_t)t;
                c = t >> 32;
            }
            us[j + vn] = (uint32_t)((uint64_t)us[j + vn] + c);
        }
        q[j] = (uint32_t)qhat;
    }
    *qn = mag_norm(q, un - vn + 1);
    for (int i = 0; i < vn; i++)
        r[i] = (us[i] >> s) | (s ? (uint32_t)((uint64_t)us[i + 1] << (32 - s)) : 0);
    *rn = mag_norm(r, vn);
}

void oc_bn_from_u64(oc_bn *r, uint64_t v) {
    r->neg = 0;
    r->w[0] = (uint32_t)v;
    r->w[1] = (uint32_t)(v >> 32);
    r->n = mag_norm(r->w, 2);
}

void oc_bn_from_i64(oc_bn *r, int64_t v) {
    uint64_t mag = v < 0 ? (uint64_t)0 - (uint64_t)v : (uint64_t)v;
    oc_bn_from_u64(r, mag);
    r->neg = (v < 0);
}

int oc_bn_cmp(const oc_bn *a, const oc_bn *b) {
    int an = a->n ? a->neg : 0, bneg = b->n ? b->neg : 0;
    if (an != bneg) return an ? -1 : 1;
    int c = mag_cmp(a->w, a->n, b->w, b->n);
    return an ? -c : c;
}

static void bn_signed_add(oc_bn *r, const oc_bn *a, int aneg, const oc_bn *b, int bneg) {
    oc_bn t;
    if (aneg == bneg) {
        t.n = mag_add(t.w, a->w, a->n, b->w, b->n);
        t.neg = aneg;
    } else if (mag_cmp(a->w, a->n, b->w, b->n) >= 0) {
        t.n = mag_sub(t.w, a->w, a->n, b->w, b->n);
        t.neg = aneg;
    } else {
        t.n = mag_sub(t.w, b->w, b->n, a->w, a->n);
        t.neg = bneg;
    }
    if (t.n == 0) t.neg = 0;
    *r = t;
}

void oc_bn_add(oc_bn *r, const oc_bn *a, const oc_bn *b) {
    bn_signed_add(r, a, a->neg, b, b->neg);
}

void oc_bn_sub(oc_bn *r, const oc_bn *a, const oc_bn *b) {
    bn_signed_add(r, a, a->neg, b, b->n ? !b->neg : 0);
}

void oc_bn_mul(oc_bn *r, const oc_bn *a, const oc_bn *b) {
    oc_bn t;
    t.n = mag_mul(t.w, a->w, a->n, b->w, b->n);
    t.neg = t.n ? (a->neg ^ b->neg) : 0;
    *r = t;
}

/* q = floor(a / b), r = a - q b, for b > 0 (so 0 <= r < b). */
void oc_bn_divmod_floor(oc_bn *q, oc_bn *r, const oc_bn *a, const oc_bn *b) {
    assert(b->n > 0 && !b->neg);
    oc_bn qq, rr;
    mag_divmod(qq.w, &qq.n, rr.w, &rr.n, a->w, a->n, b->w, b->n);
    qq.neg = 0;
    rr.neg = 0;
    if (a->neg && a->n) {
        /* -|a| = -(q0 b + r0): floor quotient is -q0 (r0 == 0) or -q0-1. */
        if (rr.n) {
            oc_bn one;
            oc_bn_from_u64(&one, 1);
            qq.n = mag_add(qq.w, qq.w, qq.n, one.w, one.n);
            rr.n = mag_sub(rr.w, b->w, b->n, rr.w, rr.n);
        }
        qq.neg = qq.n ? 1 : 0;
    }
    if (q) *q = qq;
    if (r) *r = rr;
}

/* Least non-negative residue of a mod m. */
uint64_t oc_bn_mod_u64(const oc_bn *a, uint64_t m) {
    oc_u128 rem = 0;
    for (int i = a->n - 1; i >= 0; i--) rem = ((rem << 32) | a->w[i]) % m;
    uint64_t r = (uint64_t)rem;
    if (a->neg && r) r = m - r;
    return r;
}

/* The value modulo 2^64, as a two's complement signed integer. */
int64_t oc_bn_to_i64_wrap(const oc_bn *a) {
    uint64_t lo = 0;
    if (a->n > 0) lo |= a->w[0];
    if (a->n > 1) lo |= (uint64_t)a->w[1] << 32;
    if (a->neg) lo = (uint64_t)0 - lo;
    return (int64_t)lo;
}

int oc_bn_bits(const oc_bn *a) {
    if (a->n == 0) return 0;
    return 32 * (a->n - 1) + (32 - clz32(a->w[a->n - 1]));
}

int oc_bn_to_words(const oc_bn *a, uint32_t *out, int max_words) {
    int n = a->n < max_words ? a->n : max_words;
    for (int i = 0; i < n; i++) out[i] = a->w[i];
    return a->neg ? -n : n;
}

void oc_basis_init(oc_basis *b, const uint64_t *m, int k) {
    assert(k > 0 && k <= 64);
    b->k = k;
    oc_bn_from_u64(&b->M, 1);
    for (int i = 0; i < k; i++) {
        oc_bn mi;
        b->m[i] = m[i];
        oc_bn_from_u64(&mi, m[i]);
        oc_bn_mul(&b->M, &b->M, &mi);
    }
    for (int i = 0; i < k; i++) {
        oc_bn mi, rem;
        oc_bn_from_u64(&mi, m[i]);
        oc_bn_divmod_floor(&b->Mi[i], &rem, &b->M, &mi);
        assert(rem.n == 0);
        b->inv[i] = oc_invmod(oc_bn_mod_u64(&b->Mi[i], m[i]), m[i]);
        assert(b->inv[i] != 0);
    }
}

void oc_crt(oc_bn *x, const oc_basis *b, const uint64_t *r) {
    oc_bn acc, term, c;
    oc_bn_from_u64(&acc, 0);
    for (int i = 0; i < b->k; i++) {
        oc_bn_from_u64(&c, oc_mulmod(r[i] % b->m[i], b->inv[i], b->m[i]));
        oc_bn_mul(&term, &b->Mi[i], &c);
        oc_bn_add(&acc, &acc, &term);
    }
    oc_bn_divmod_floor(NULL, x, &acc, &b->M);
}

void oc_crt_centred(oc_bn *x, const oc_basis *b, const uint64_t *r) {
    oc_bn twice;
    oc_crt(x, b, r);
    oc_bn_add(&twice, x, x);
    if (oc_bn_cmp(&twice, &b->M) > 0) oc_bn_sub(x, x, &b->M);
}
