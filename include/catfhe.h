/*
 * catfhe: the RNS hot path of CKKS / BFV / BGV homomorphic multiplication
 * with relinearisation, rotation and rescale / modulus switching, as
 * hand-written CUDA for GB300 (sm_103a), behind a plain C ABI.
 *
 * Paper: Q. Li, R. Zong, "CAT: A GPU-Accelerated FHE Framework with Its
 * Application to High-Precision Private Dataset Query" (arXiv 2503.22227).
 * The operations are the upper-layer operators of its Sec. 3 (key
 * generation, encrypt / decrypt, add, multiply, relinearize, rescale,
 * rotate; Tables 1-3), over the RNS representation of its Sec. 2.2.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Return value: CATFHE_OK (0) on success, else a negative CATFHE_E* code;
 *   catfhe_strerror() names it.  On error nothing is written to outputs.
 * Handles: catfhe_ctx and catfhe_keys are created and owned by the library
 *   and freed by their _destroy call.  They hold device memory (prime and
 *   NTT tables, keys) allocated once with cudaMalloc on the current device.
 * Ciphertexts: plain device pointers to uint64 residues, "limb-major"
 *   (Sec. 3.1.5 of the paper: the residues of one modulus are contiguous,
 *   one modulus after another).  A batch of `count` ciphertexts at level l
 *   (primes q_0 .. q_{l-1}) is  u64[count][2][l][N],  every residue in
 *   [0, q_i).  At rest, CKKS and BGV ciphertexts are in NTT (evaluation)
 *   form and BFV ciphertexts in coefficient form; the NTT order is
 *   internal.  catfhe_ct_export gives the coefficient form.
 *   Device buffers are caller-owned and 16-byte aligned (a pointer that is
 *   not is refused with EINVAL before any work is enqueued); the library only
 *   reads inputs and writes outputs during the stream-ordered work it
 *   enqueues.  `out` may
 *   alias an input of the same shape.
 * Workspace: operations that need scratch take (ws, ws_bytes): a device
 *   buffer of at least catfhe_workspace_bytes(...) bytes, 256-byte aligned
 *   (a pointer that is not even 16-byte aligned is refused with EINVAL),
 *   caller-owned, not touched after the enqueued work completes.  ws = NULL
 *   makes the library use a scratch buffer owned by the context (grown
 *   with cudaMalloc on demand; calls that share it must be ordered on one
 *   stream).
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  All
 *   device work is enqueued on it and is asynchronous, except where a
 *   function says it synchronises (those that write host memory).
 * Seeds: 32 bytes.  All randomness is ChaCha20 (RFC 8439) keyed by the
 *   seed, so keys and encryptions are reproducible bit for bit.
 */
#ifndef CATFHE_H
#define CATFHE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    CATFHE_OK = 0,
    CATFHE_EINVAL = -1,     /* bad argument, shape or parameter set          */
    CATFHE_ELEVEL = -2,     /* level out of range, or rescale at level 1     */
    CATFHE_ENOKEY = -3,     /* the key-switching key is missing              */
    CATFHE_ENOMEM = -4,     /* device allocation failed                      */
    CATFHE_ECUDA = -5,      /* a CUDA call or kernel launch failed           */
    CATFHE_ESCHEME = -6,    /* operation not defined for this scheme         */
    CATFHE_EWORKSPACE = -7, /* workspace smaller than required               */
    CATFHE_ETIMEOUT = -8    /* a kernel's bounded wait gave up (catfhe_sync)  */
};

enum { CATFHE_CKKS = 0, CATFHE_BFV = 1, CATFHE_BGV = 2 };

/* Operation codes for catfhe_workspace_bytes. */
enum {
    CATFHE_OP_MUL_RELIN = 1,
    CATFHE_OP_MUL_RELIN_RESCALE = 2,
    CATFHE_OP_ROTATE = 3,
    CATFHE_OP_RESCALE = 4,
    CATFHE_OP_DECRYPT = 5,
    CATFHE_OP_EXPORT = 6,
    CATFHE_OP_NTT = 7,
    /* element-wise operations (batch entries; no workspace) */
    CATFHE_OP_ADD = 8,
    CATFHE_OP_SUB = 9,
    CATFHE_OP_MUL_INT = 10,
    CATFHE_OP_ADD_CONST = 11,
    CATFHE_OP_DROP = 12,
    /* workspace of catfhe_rotate_hoisted (any number of rotations) */
    CATFHE_OP_ROTATE_HOISTED = 13,
    /* batch entry: out = a * plaintext b (catfhe_mul_plain; no workspace) */
    CATFHE_OP_MUL_PLAIN = 14,
    /* workspaces of catfhe_encode_ckks / catfhe_decode_ckks */
    CATFHE_OP_ENCODE = 15,
    CATFHE_OP_DECODE = 16
};

/* Forms for catfhe_ct_import / catfhe_ct_export. */
enum { CATFHE_FORM_COEFF = 0, CATFHE_FORM_NATIVE = 1 };
/* OR-ed into the form of catfhe_ct_import / catfhe_ct_export: return
 * without synchronising; the copy completes in the order of `stream`. */
enum { CATFHE_FORM_ASYNC = 0x100 };

/*
 * Parameter set (paper Sec. 2.2: q = prod q_i of word-sized coprime
 * moduli; Sec. 5.1 fixes N, L and log Q per experiment).
 *   scheme     CATFHE_CKKS / _BFV / _BGV
 *   log_n      ring degree N = 2^log_n, 12 <= log_n <= 16
 *   log_n_max  every prime is 1 mod 2^(log_n_max+1) (>= log_n; lets one
 *              chain serve several ring degrees)
 *   L, q_bits  L <= 32 ciphertext primes; prime i is the largest unused prime
 *              below 2^q_bits[i] that is 1 mod 2^(log_n_max+1)
 *   K, p_bits  K special primes for hybrid key switching (chosen after Q)
 *   dnum       number of key-switching digits: alpha = ceil(L/dnum)
 *              primes per digit
 *   t          plaintext modulus (BFV, BGV; ignored for CKKS), odd,
 *              coprime to every prime, t < 2^61
 *   aux_count  BFV auxiliary basis size; 0 = the smallest count with
 *              prod(B) > 2 t N Q
 *   aux_bits   BFV auxiliary prime size (0 = 60)
 * Prime sizes: 20 <= bits <= 61.
 */
typedef struct {
    int32_t scheme;
    int32_t log_n;
    int32_t log_n_max;
    int32_t L;
    int32_t K;
    int32_t dnum;
    int32_t q_bits[64];
    int32_t p_bits[16];
    uint64_t t;
    int32_t aux_count;
    int32_t aux_bits;
} catfhe_params;

typedef struct {
    int32_t n;       /* ring degree                         */
    int32_t L, K;    /* ciphertext and special prime counts */
    int32_t nb;      /* BFV auxiliary primes (0 otherwise)  */
    int32_t alpha;   /* primes per key-switching digit      */
    int32_t beta;    /* digits at the top level             */
} catfhe_info;

typedef struct catfhe_ctx catfhe_ctx;
typedef struct catfhe_keys catfhe_keys;

const char *catfhe_strerror(int code);

/* Creates a context on the current CUDA device: generates the primes,
 * the NTT tables (smallest primitive 2N-th root of each prime, powers in
 * bit-reversed order) and the base-conversion constants.  Synchronises. */
int catfhe_ctx_create(const catfhe_params *params, catfhe_ctx **out);
void catfhe_ctx_destroy(catfhe_ctx *ctx);
int catfhe_ctx_info(const catfhe_ctx *ctx, catfhe_info *out);
/* Copies the primes to host arrays of L, K and nb entries (any may be NULL). */
int catfhe_ctx_moduli(const catfhe_ctx *ctx, uint64_t *q, uint64_t *p, uint64_t *b);

/* Galois element 5^steps mod 2N (left rotation of CKKS slots / BFV and
 * BGV rows by `steps`); steps may be negative.  Returns 0 on bad ctx. */
uint64_t catfhe_galois_elt(const catfhe_ctx *ctx, int64_t steps);

/* Key generation from a seed (paper Sec. 3: "key generation periods of
 * various types"): ternary secret s, public key (-a s + e, a) (BGV: t e),
 * and the relinearisation key switching s^2 -> s.  Synchronises. */
int catfhe_keygen(catfhe_ctx *ctx, const uint8_t seed[32], catfhe_keys **out);
/* Adds the key switching sigma_g(s) -> s, g odd (rotation / conjugation). */
int catfhe_gen_galois_key(catfhe_ctx *ctx, catfhe_keys *keys, uint64_t galois_elt);
void catfhe_keys_destroy(catfhe_keys *keys);
/* Exports keys in coefficient form to host memory (for checking):
 * s: int64[N]; pk: u64[2][L][N]; ksk (key_id 0 = relinearisation, else a
 * Galois element): u64[beta][2][L+K][N].  Any pointer may be NULL.
 * Synchronises. */
int catfhe_keys_export(catfhe_ctx *ctx, const catfhe_keys *keys, uint64_t key_id,
                       int64_t *s, uint64_t *pk, uint64_t *ksk);

/* Public-key encryption of the integer polynomial msg (host, int64[N]) at
 * the top level L into ct (device, u64[2][L][N]).  CKKS: msg is the
 * encoded, scaled plaintext; BFV / BGV: msg in [0, t).  Synchronises on
 * the upload of msg. */
int catfhe_encrypt(catfhe_ctx *ctx, const catfhe_keys *keys, const int64_t *msg,
                   const uint8_t seed[32], uint64_t *ct, void *stream);

/* A ciphertext with residues uniform mod q_i (coefficient form, ChaCha20
 * domain "ct_uniform", indexes poly and `index`), stored at rest. */
int catfhe_ct_uniform(catfhe_ctx *ctx, const uint8_t seed[32], uint32_t index,
                      uint32_t level, uint64_t *ct, void *stream);

/* Host <-> device transfer of `count` ciphertexts u64[count][2][level][N].
 * FORM_COEFF: host data in coefficient form (converted to / from the at-
 * rest form on the device).  FORM_NATIVE: host data in the at-rest form
 * (plain copies).  export needs workspace only for FORM_COEFF; it
 * synchronises `stream`.  import synchronises on the host copy.  With
 * CATFHE_FORM_ASYNC neither synchronises: the host buffer must then stay
 * allocated and unchanged (import) or unread (export) until the work
 * enqueued on `stream` so far has completed; page-locked host memory lets
 * the copy overlap with other work. */
int catfhe_ct_import(catfhe_ctx *ctx, const uint64_t *host, uint32_t level, uint32_t count,
                     int form, uint64_t *ct, void *stream);
int catfhe_ct_export(catfhe_ctx *ctx, const uint64_t *ct, uint32_t level, uint32_t count,
                     int form, uint64_t *host, void *ws, size_t ws_bytes, void *stream);

/* Bit-packed transfer form (an addition of this library; the paper moves
 * whole words).  Each limb's N residues of prime q_i, in the at-rest form
 * and order [count][2][level], as a little-endian bit stream of
 * b_i = bitlen(q_i) bits per residue: residue k occupies bits
 * [k b_i, (k+1) b_i) of the limb's N b_i / 64 words, limbs one after
 * another.  catfhe_packed_words gives the words of `count` ciphertexts at
 * `level` (0 on bad arguments).  import copies the packed words from host
 * memory into `ws` (at least that many words, 16-byte aligned; NULL = the
 * context's scratch) and unpacks them into ct; an unpacked value >= q_i is
 * reduced by one subtraction of q_i.  export packs ct into `ws` and copies
 * the words to host memory.  flags = 0 synchronises (as catfhe_ct_import /
 * _export), CATFHE_FORM_ASYNC does not (the host buffer must stay valid and
 * unchanged, or unread, until the stream's work completes).
 * catfhe_pack_host / catfhe_unpack_host convert `polys` polynomials of
 * `level` limbs of N = 2^log_n words between the two forms on the host,
 * with bits[i] = b_i (1..64); pack keeps the low b_i bits of each word. */
size_t catfhe_packed_words(const catfhe_ctx *ctx, uint32_t level, uint32_t count);
int catfhe_ct_import_packed(catfhe_ctx *ctx, const uint64_t *packed, uint32_t level,
                            uint32_t count, uint64_t *ct, void *ws, size_t ws_bytes, int flags,
                            void *stream);
int catfhe_ct_export_packed(catfhe_ctx *ctx, const uint64_t *ct, uint32_t level, uint32_t count,
                            uint64_t *packed, void *ws, size_t ws_bytes, int flags, void *stream);
int catfhe_pack_host(const uint8_t *bits, uint32_t level, uint32_t polys, uint32_t log_n,
                     const uint64_t *limbs, uint64_t *packed);
int catfhe_unpack_host(const uint8_t *bits, uint32_t level, uint32_t polys, uint32_t log_n,
                       const uint64_t *packed, uint64_t *limbs);

/* out = a + b (Table 1-3 "add"), count ciphertexts at `level`. */
int catfhe_add(catfhe_ctx *ctx, const uint64_t *a, const uint64_t *b, uint64_t *out,
               uint32_t level, uint32_t count, void *stream);

/* Homomorphic multiplication with relinearisation (Tables 1-3 "multiply"
 * then "relinearize"): tensor (d0, d1, d2) = (a0 b0, a0 b1 + a1 b0, a1 b1)
 * (BFV: exact round(t x / Q) of the tensor over Q u B), then hybrid key
 * switching of d2 with the relinearisation key: exact ModUp of each digit
 * to Q_l u P, inner product with the key, exact ModDown round(x / P)
 * (BGV: (x - d) / P with d = t [x t^-1]_P).  Output at `level`.
 * With count >= 4 and N >= 2^14 the ciphertexts run as two halves on two
 * library streams forked from `stream` and joined back (results identical;
 * this and catfhe_rotate enqueue under a process-wide lock). */
int catfhe_mul_relin(catfhe_ctx *ctx, const catfhe_keys *keys, const uint64_t *a,
                     const uint64_t *b, uint64_t *out, uint32_t level, uint32_t count,
                     void *ws, size_t ws_bytes, void *stream);

/* CKKS only: multiply, relinearise and rescale in one fused pass; the
 * ModDown and the rescale are one exact division by P q_{l-1}, equal bit
 * for bit to catfhe_mul_relin followed by catfhe_rescale.  Output at
 * level-1, u64[count][2][level-1][N]. */
int catfhe_mul_relin_rescale(catfhe_ctx *ctx, const catfhe_keys *keys, const uint64_t *a,
                             const uint64_t *b, uint64_t *out, uint32_t level,
                             uint32_t count, void *ws, size_t ws_bytes, void *stream);

/* out = a - b (ciphertext subtraction), count ciphertexts at `level`. */
int catfhe_sub(catfhe_ctx *ctx, const uint64_t *a, const uint64_t *b, uint64_t *out,
               uint32_t level, uint32_t count, void *stream);

/* Multiplication by a plaintext integer constant k (Table 1
 * "multiply_plain" for a constant plaintext): both polynomials times k mod
 * q_i, no rescale.  For CKKS multiply by round(c q_{l-1}) and then rescale
 * to scale by a real c while keeping the scale.  Any scheme. */
int catfhe_mul_int(catfhe_ctx *ctx, const uint64_t *a, int64_t k, uint64_t *out, uint32_t level,
                   uint32_t count, void *stream);

/* Addition of the plaintext constant k to every slot (CKKS: k is the
 * scaled value, round(c * scale); BGV: k mod t): c0 += k, which in NTT form
 * is the constant polynomial k.  ESCHEME for BFV. */
int catfhe_add_const(catfhe_ctx *ctx, const uint64_t *a, int64_t k, uint64_t *out,
                     uint32_t level, uint32_t count, void *stream);

/* A plaintext polynomial for catfhe_mul_plain (Table 1 "multiply_plain"):
 * host int64[N] signed coefficients (CKKS: the encoded, scaled message;
 * BFV / BGV: a polynomial mod t) reduced mod q_0 .. q_{level-1} into the
 * device buffer pt u64[level][N], in NTT form.  Synchronises on the host
 * copy. */
int catfhe_plain_import(catfhe_ctx *ctx, const int64_t *coeffs, uint32_t level, uint64_t *pt,
                        void *stream);

/* CKKS encoding on the device (Table 1 "encode"): host slots z, N/2
 * complex numbers as interleaved (re, im) doubles, become the plaintext
 * m with m(zeta^(5^k)) ~ scale z_k (zeta = exp(i pi / N), conjugate slots
 * implied): one length-N DFT of float64, coefficients rounded half away
 * from zero (|m_i| must stay below 2^62), reduced mod q_0 .. q_{level-1}
 * and NTT'd into pt u64[level][N] (a plaintext for catfhe_mul_plain).
 * ESCHEME unless CKKS.  Workspace: catfhe_workspace_bytes(CATFHE_OP_ENCODE,
 * level, 1) or NULL.  Synchronises. */
int catfhe_encode_ckks(catfhe_ctx *ctx, const double *slots, double scale, uint32_t level,
                       uint64_t *pt, void *ws, size_t ws_bytes, void *stream);

/* CKKS decryption and decoding on the device (Table 1 "decrypt",
 * "decode"): the centred plaintext of ct (as catfhe_decrypt, exact while
 * below 2^63 in magnitude), evaluated at the slot roots by one float64 DFT
 * and divided by scale, into host slots (N/2 interleaved complex doubles).
 * ESCHEME unless CKKS.  Workspace: CATFHE_OP_DECODE.  Synchronises. */
int catfhe_decode_ckks(catfhe_ctx *ctx, const catfhe_keys *keys, const uint64_t *ct,
                       uint32_t level, double scale, double *slots, void *ws, size_t ws_bytes,
                       void *stream);

/* Multiplication by a plaintext (Table 1 "multiply_plain"): both
 * polynomials times pt, limb by limb in NTT form; pt u64[>= level][N] from
 * catfhe_plain_import (its first `level` limbs are used).  No relinearisation;
 * a CKKS product carries the scale of a times the plaintext's scale.  BFV
 * ciphertexts (coefficient form) are transformed, multiplied and transformed
 * back inside out; out may alias a. */
int catfhe_mul_plain(catfhe_ctx *ctx, const uint64_t *a, const uint64_t *pt, uint64_t *out,
                     uint32_t level, uint32_t count, void *stream);

/* Keeps primes q_0 .. q_{new_level-1}: out is u64[count][2][new_level][N]
 * (CKKS scale and plaintext unchanged); out must not alias a. */
int catfhe_drop_level(catfhe_ctx *ctx, const uint64_t *a, uint32_t level, uint32_t new_level,
                      uint64_t *out, uint32_t count, void *stream);

/* Rotation (Table 1 "rotate_vector_one_step", Tables 2-3 rotate rows /
 * columns): out = (sigma_g(a0), 0) + KS(sigma_g(a1)) with the Galois key of
 * g; g = catfhe_galois_elt(steps), or 2N-1 for conjugation / columns. */
int catfhe_rotate(catfhe_ctx *ctx, const catfhe_keys *keys, const uint64_t *a,
                  uint64_t galois_elt, uint64_t *out, uint32_t level, uint32_t count,
                  void *ws, size_t ws_bytes, void *stream);

/* Several rotations of the same ciphertexts with one shared ModUp (Table 1
 * "rotate_vector_random" over many steps; hoisting): the exact lift of each
 * digit of a1 commutes with sigma_g (a signed permutation of coefficients;
 * the centred lift is odd), so ModUp(sigma_g(a1)) = sigma_g(ModUp(a1)) and
 * each rotation only permutes the lifted digits, then runs the inner product
 * and ModDown.  out[r] = catfhe_rotate(a, galois_elts[r]) bit for bit, for
 * r < n_rot; out is u64[n_rot][count][2][level][N].  CKKS and BGV (ESCHEME
 * for BFV); every key is checked (ENOKEY) before anything is enqueued.
 * Workspace: catfhe_workspace_bytes(CATFHE_OP_ROTATE_HOISTED, level, count),
 * independent of n_rot.  galois_elts is host memory; with n_rot = 0 nothing
 * is read or written (out may be NULL). */
int catfhe_rotate_hoisted(catfhe_ctx *ctx, const catfhe_keys *keys, const uint64_t *a,
                          const uint64_t *galois_elts, uint32_t n_rot, uint64_t *out,
                          uint32_t level, uint32_t count, void *ws, size_t ws_bytes,
                          void *stream);

/* CKKS rescale round(c / q_{l-1}) (Table 1 "rescale"), or BGV modulus
 * switch (c - d) / q_{l-1}, d = t [c t^-1]_{q_{l-1}} (the plaintext then
 * carries the factor q_{l-1}^-1 mod t, see catfhe_decrypt).  Output at
 * level-1.  ESCHEME for BFV, ELEVEL at level 1. */
int catfhe_rescale(catfhe_ctx *ctx, const uint64_t *a, uint64_t *out, uint32_t level,
                   uint32_t count, void *ws, size_t ws_bytes, void *stream);

/* catfhe_rescale without any device allocation, for callers that may not
 * allocate device memory while they run (a host callback, a loop whose
 * memory budget is fixed at start-up, a plugin whose host process owns all
 * device allocations).  The paper has no counterpart; the result is the
 * same as catfhe_rescale's, bit for bit.
 * Scratch: a 32 MiB array that the library reserves statically on every
 * GPU that loads it (held until the process exits); enough for count
 * ciphertexts when 16 KiB + 16 * count * level * N bytes fit in 32 MiB
 * (one N = 2^16 ciphertext at level 24), else CATFHE_EWORKSPACE and nothing
 * is enqueued.  No call allocates or frees memory.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress), so
 * make that first call before any stream capture.  All calls share the
 * array and it keeps the last call's contents (nothing in it needs to start
 * at zero); calls whose device work overlaps race on it, so order them on
 * one stream.  Inputs and outputs are caller-owned device buffers as for
 * catfhe_rescale; `out` must not overlap `a` (EINVAL, nothing enqueued).
 * The context's device must be the caller's current device (EINVAL
 * otherwise): the array has a different address on every GPU. */
int catfhe_rescale_noalloc(catfhe_ctx *ctx, const uint64_t *a, uint64_t *out, uint32_t level,
                           uint32_t count, void *stream);

/* Decryption of one ciphertext at `level` into host msg (int64[N]):
 * x = [c0 + c1 s]_{Q_l} centred; CKKS: x as two's complement (exact when
 * |x| < 2^63); BFV: round(t x / Q_l) mod t; BGV: x factor^-1 mod t where
 * `factor` is the plaintext factor accumulated by modulus switches (1 for
 * a fresh or multiplied ciphertext).  Synchronises. */
int catfhe_decrypt(catfhe_ctx *ctx, const catfhe_keys *keys, const uint64_t *ct,
                   uint32_t level, uint64_t factor, int64_t *msg, void *ws, size_t ws_bytes,
                   void *stream);

/* Batched negacyclic NTT (paper Sec. 3.1.3) in place over count*level
 * limbs u64[count][level][N], limb i of each group mod q_i.  inverse != 0
 * runs the inverse transform (N^-1 folded in).  No workspace. */
int catfhe_ntt(catfhe_ctx *ctx, uint64_t *limbs, uint32_t level, uint32_t count, int inverse,
               void *stream);

/* Kernel watchdog.  Kernels that wait on an mbarrier for bulk copies bound
 * every wait (about one second of global time); on timeout they set a bit in
 * the context's device status word and return instead of waiting on (bit 1:
 * the inner product's copies; bit 2: catfhe_wait_selftest; bit 4: the
 * ModDown / rescale combine's copy in the NTT row pass).  The paper has
 * no counterpart.  catfhe_device_status synchronises `stream`, stores the
 * word in *flags and clears it if `clear`.  catfhe_wait_selftest launches
 * one CTA whose barrier expects data that never comes: its wait gives up
 * after limit_ns nanoseconds (1e3 .. 1e10) and sets bit 2, so a caller can
 * check that a timed-out wait ends and is reported. */
int catfhe_device_status(catfhe_ctx *ctx, int32_t *flags, int clear, void *stream);
int catfhe_wait_selftest(catfhe_ctx *ctx, uint64_t limit_ns, void *stream);

/* Waits until everything enqueued on `stream` has finished (operations are
 * stream-ordered and asynchronous; import/export without CATFHE_FORM_ASYNC,
 * decrypt and decode synchronise by themselves).  Returns CATFHE_ECUDA if
 * the stream reports an error, CATFHE_ETIMEOUT if any bounded wait of this
 * context's kernels has given up since the status word was last cleared
 * (any bit of catfhe_device_status, the self-test's included; the word is
 * left as it is), else CATFHE_OK. */
int catfhe_sync(catfhe_ctx *ctx, void *stream);

/* Diagnostics.  catfhe_measure_int_peak times register-resident loops of
 * independent 64-bit Shoup products by a constant (fully reduced) and of
 * the forward NTT's butterflies exactly as the transform runs them: for
 * primes of 57 bits or more (`butterfly_per_s`: lazy product, one
 * conditional subtraction, add, subtract) and for smaller primes
 * (`butterfly_wide_per_s`: no conditional subtraction).  The loops fill the
 * whole GPU; each result is the best of five launches in operations per
 * second (any pointer may be NULL); `stream` is synchronised.  These are
 * the integer-pipe ceilings the hot path is measured against.
 * catfhe_kernel_launches returns how many kernels the library has launched
 * since it was loaded. */
int catfhe_measure_int_peak(double *modmul_per_s, double *butterfly_per_s,
                            double *butterfly_wide_per_s, void *stream);
/* The device's rates, over the whole GPU, of the three 32-bit multiply
 * instructions the 64-bit modular arithmetic is made of: low product
 * (mad.lo.u32), high product (mad.hi.u32) and widening product
 * (mad.wide.u32), each in register-resident loops of independent chains,
 * best of five launches, in instructions (thread operations) per second
 * (any pointer may be NULL); `stream` is synchronised.  With how many of
 * each a butterfly issues (a profiler's count), they bound the transform
 * from the hardware side. */
int catfhe_measure_imad_rates(double *lo_per_s, double *hi_per_s, double *wide_per_s,
                              void *stream);
uint64_t catfhe_kernel_launches(void);

/* ---- Uneven batches (many independent operations in one submission) ----
 * Each entry is one operation of any context (ring degree), level and kind;
 * the entries must not depend on one another.  catfhe_run_batch spreads
 * them over `lanes` (1..32) concurrent streams forked from `stream`, each
 * lane with its own slice of `ws` (at least catfhe_batch_workspace_bytes),
 * assigning operations longest-first by modular-product count, and joins
 * the lanes back into `stream` (paper Sec. 3.1.6 spreads per-modulus work
 * over a stream pool; here whole operations are spread).
 * catfhe_batch_capture runs the batch once, then captures it into a CUDA
 * graph (buffers and workspace are baked in: replaying it recomputes the
 * same operations on whatever the buffers then hold); catfhe_graph_launch
 * replays it on a stream.  The lane streams are shared by all calls on a
 * device: call from one host thread at a time.  op codes and the fields
 * they use: CATFHE_OP_MUL_RELIN, _MUL_RELIN_RESCALE (keys, a, b, out);
 * _ROTATE (keys, a, out, arg = Galois element); _RESCALE (a, out);
 * _ADD, _SUB (a, b, out); _MUL_INT, _ADD_CONST (a, out, arg = the int64
 * constant as two's complement); _DROP (a, out, level_out); _MUL_PLAIN
 * (a, b = plaintext from catfhe_plain_import, out). */
typedef struct {
    int32_t op;
    uint32_t level;
    uint32_t count;
    uint32_t level_out;
    catfhe_ctx *ctx;
    const catfhe_keys *keys;
    const uint64_t *a;
    const uint64_t *b;
    uint64_t *out;
    uint64_t arg;
} catfhe_op;

typedef struct catfhe_graph catfhe_graph;

size_t catfhe_batch_workspace_bytes(const catfhe_op *ops, uint32_t n, uint32_t lanes);
int catfhe_run_batch(const catfhe_op *ops, uint32_t n, uint32_t lanes, void *ws, size_t ws_bytes,
                     void *stream);
int catfhe_batch_capture(const catfhe_op *ops, uint32_t n, uint32_t lanes, void *ws,
                         size_t ws_bytes, catfhe_graph **out);
int catfhe_graph_launch(catfhe_graph *graph, void *stream);
size_t catfhe_graph_nodes(const catfhe_graph *graph);
void catfhe_graph_destroy(catfhe_graph *graph);

/* ---- NTT schedules (paper Sec. 3.1.3) ----
 * Each ring degree has a few two-pass schedules (how many of the log N
 * stages the column pass takes, how many words each thread holds, and each
 * pass's threads per CTA and CTAs per SM).  The
 * context keeps one choice per launch size class: launches of up to 64
 * limbs, up to 256, and more.  catfhe_tune_ntt times every schedule of
 * ctx's ring degree on `limbs` limbs (rounded up to whole groups of L;
 * forward + inverse, best of five, synchronises `stream`), keeps the
 * fastest for later launches of that size class and writes its index to
 * *chosen and each schedule's time in microseconds to us[] (either may be
 * NULL).  catfhe_ntt_schedule reports the schedule used for launches of
 * `limbs` limbs, how many exist and its shape {column log size, column log
 * words/thread, row log size, row log words/thread};
 * catfhe_set_ntt_schedule picks one by index for every class. */
int catfhe_tune_ntt(catfhe_ctx *ctx, uint32_t limbs, void *stream, int32_t *chosen, float *us);
int catfhe_ntt_schedule(const catfhe_ctx *ctx, uint32_t limbs, int32_t *index, int32_t *count,
                        int32_t shape[4]);
int catfhe_set_ntt_schedule(catfhe_ctx *ctx, int32_t index);

/* Workspace bytes that `op` needs for `count` ciphertexts at `level`. */
size_t catfhe_workspace_bytes(const catfhe_ctx *ctx, int op, uint32_t level, uint32_t count);

#ifdef __cplusplus
}
#endif

#endif /* CATFHE_H */
