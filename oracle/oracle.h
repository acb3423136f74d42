/*
 * CPU oracle for the RNS hot path of CKKS / BFV / BGV homomorphic
 * multiplication, relinearisation, rotation and rescale.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links,
 * includes or calls this code; only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark load it.  It shares no source
 * with the CUDA path.
 *
 * Every function is the plain definition of what it computes: 128-bit
 * products reduced with '%', a textbook iterative NTT, and arbitrary
 * precision integers for every base conversion (the CRT reconstruction
 * written out, then a real big-integer division for each rounding).
 * There is no blocking, fusion or lazy reduction anywhere.
 *
 * Paper: "CAT: A GPU-Accelerated FHE Framework ..." (arXiv 2503.22227).
 * The paper states the schemes only by citation; the readings taken
 * where it is silent are listed next to each function.
 */
#ifndef CATFHE_ORACLE_H
#define CATFHE_ORACLE_H

#include <stdint.h>
#include <stddef.h>

typedef unsigned __int128 oc_u128;

/* ---------------- number theory (oc_num.c) ---------------- */
uint64_t oc_mulmod(uint64_t a, uint64_t b, uint64_t m);
uint64_t oc_addmod(uint64_t a, uint64_t b, uint64_t m);
uint64_t oc_submod(uint64_t a, uint64_t b, uint64_t m);
uint64_t oc_powmod(uint64_t a, uint64_t e, uint64_t m);
uint64_t oc_invmod(uint64_t a, uint64_t m);
uint64_t oc_reduce_i64(int64_t x, uint64_t m);
int oc_is_prime(uint64_t n);
int oc_gen_primes(int bits, int count, uint64_t two_n, const uint64_t *exclude,
                  int n_exclude, uint64_t *out);
uint64_t oc_min_psi(uint64_t q, int log_n);

/* ---------------- arbitrary precision integers (oc_bigint.c) ---------------- */
#define OC_BN_WORDS 160 /* 5120 bits, far above the largest modulus used */
typedef struct {
    int neg;                 /* sign of the value (0 for zero)            */
    int n;                   /* number of significant 32-bit words        */
    uint32_t w[OC_BN_WORDS]; /* magnitude, least significant word first   */
} oc_bn;

void oc_bn_from_u64(oc_bn *r, uint64_t v);
void oc_bn_from_i64(oc_bn *r, int64_t v);
int oc_bn_cmp(const oc_bn *a, const oc_bn *b);
void oc_bn_add(oc_bn *r, const oc_bn *a, const oc_bn *b);
void oc_bn_sub(oc_bn *r, const oc_bn *a, const oc_bn *b);
void oc_bn_mul(oc_bn *r, const oc_bn *a, const oc_bn *b);
void oc_bn_divmod_floor(oc_bn *q, oc_bn *r, const oc_bn *a, const oc_bn *b);
uint64_t oc_bn_mod_u64(const oc_bn *a, uint64_t m);
int64_t oc_bn_to_i64_wrap(const oc_bn *a);
int oc_bn_bits(const oc_bn *a);
int oc_bn_to_words(const oc_bn *a, uint32_t *out, int max_words);

/* A residue basis {m_0..m_{k-1}} with the constants of the CRT formula. */
typedef struct {
    int k;
    uint64_t m[64];
    oc_bn M;           /* product of all m_i                    */
    oc_bn Mi[64];      /* M / m_i                               */
    uint64_t inv[64];  /* (M / m_i)^{-1} mod m_i                */
} oc_basis;

void oc_basis_init(oc_basis *b, const uint64_t *m, int k);
/* x in [0, M) with x = r_i mod m_i (Chinese remainder theorem). */
void oc_crt(oc_bn *x, const oc_basis *b, const uint64_t *r);
/* Centred representative in (-M/2, M/2]. */
void oc_crt_centred(oc_bn *x, const oc_basis *b, const uint64_t *r);

/* ---------------- NTT (oc_ntt.c) ---------------- */
void oc_ntt_fwd(uint64_t *a, int log_n, uint64_t q, uint64_t psi);
void oc_ntt_inv(uint64_t *a, int log_n, uint64_t q, uint64_t psi);
void oc_negacyclic_mul(uint64_t *out, const uint64_t *a, const uint64_t *b,
                       int log_n, uint64_t q, uint64_t psi);

/* ---------------- ChaCha20 and samplers (oc_chacha.c) ---------------- */
void oc_chacha20_block(const uint8_t key[32], uint32_t counter,
                       const uint8_t nonce[12], uint8_t out[64]);
uint64_t oc_stream_word(const uint8_t key[32], uint32_t tag, uint32_t i0,
                        uint32_t i1, uint64_t w);
void oc_cdt_table(uint64_t out[19]);
void oc_sample_uniform(const uint8_t key[32], uint32_t tag, uint32_t i0,
                       uint32_t i1, const uint64_t *mods, int n_limbs,
                       int log_n, uint64_t *out);
void oc_sample_ternary(const uint8_t key[32], uint32_t tag, uint32_t i0,
                       uint32_t i1, int log_n, int64_t *out);
void oc_sample_gaussian(const uint8_t key[32], uint32_t tag, uint32_t i0,
                        uint32_t i1, int log_n, int64_t *out);

/* Domain tags of the keystream (nonce word 0). */
enum {
    OC_TAG_SK = 1,
    OC_TAG_PK_A = 2,
    OC_TAG_PK_E = 3,
    OC_TAG_KSK_A = 4,
    OC_TAG_KSK_E = 5,
    OC_TAG_ENC_V = 6,
    OC_TAG_ENC_E0 = 7,
    OC_TAG_ENC_E1 = 8,
    OC_TAG_CT_UNIFORM = 9
};

/* ---------------- schemes (oc_fhe.c) ---------------- */
enum { OC_CKKS = 0, OC_BFV = 1, OC_BGV = 2 };

#endif
