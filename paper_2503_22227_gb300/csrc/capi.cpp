// The C ABI (include/catfhe.h): argument checks and dispatch.
#include <string.h>

#include <new>

#include "internal.h"


namespace catfhe {
int ctx_init(Context &c, const catfhe_params &p);
void ctx_free(Context &c);
size_t ws_bytes(const Context &c, int op, uint32_t level, uint32_t count);
int op_mul_relin(Context &c, const Keys &keys, const uint64_t *a, const uint64_t *b,
                 uint64_t *out, uint32_t level, uint32_t count, bool fused, void *ws,
                 size_t ws_bytes_in, cudaStream_t s,
                 const Gather *gth = nullptr, bool split = false);
int op_rotate(Context &c, const Keys &keys, const uint64_t *a, uint64_t g, uint64_t *out,
              uint32_t level, uint32_t count, void *ws, size_t ws_bytes_in, cudaStream_t s,
              const Gather *gth = nullptr, bool split = false);
int op_plain_import(Context &c, const int64_t *coeffs, uint32_t level, uint64_t *pt,
                    cudaStream_t s);
int op_encode_ckks(Context &c, const double *slots, double scale, uint32_t level, uint64_t *pt,
                   void *ws, size_t ws_bytes_in, cudaStream_t s);
int op_decode_ckks(Context &c, const Keys &k, const uint64_t *ct, uint32_t level, double scale,
                   double *slots, void *ws, size_t ws_bytes_in, cudaStream_t s);
int op_mul_plain(Context &c, const uint64_t *a, const uint64_t *pt, uint64_t *out, uint32_t level,
                 uint32_t count, cudaStream_t s);
int op_rotate_hoisted(Context &c, const Keys &keys, const uint64_t *a, const uint64_t *gs,
                      uint32_t n_rot, uint64_t *out, uint32_t level, uint32_t count, void *ws,
                      size_t ws_bytes_in, cudaStream_t s);
int op_rescale(Context &c, const uint64_t *a, uint64_t *out, uint32_t level, uint32_t count,
               void *ws, size_t ws_bytes_in, cudaStream_t s);
int op_add(Context &c, const uint64_t *a, const uint64_t *b, uint64_t *out, uint32_t level,
           uint32_t count, cudaStream_t s);
int op_ntt(Context &c, uint64_t *limbs, uint32_t level, uint32_t count, int inverse,
           cudaStream_t s);
int op_sub(Context &c, const uint64_t *a, const uint64_t *b, uint64_t *out, uint32_t level,
           uint32_t count, cudaStream_t s);
int op_mul_int(Context &c, const uint64_t *a, int64_t k, uint64_t *out, uint32_t level,
               uint32_t count, cudaStream_t s);
int op_add_const(Context &c, const uint64_t *a, int64_t k, uint64_t *out, uint32_t level,
                 uint32_t count, cudaStream_t s);
int op_drop_level(Context &c, const uint64_t *a, uint32_t level, uint32_t new_level,
                  uint64_t *out, uint32_t count, cudaStream_t s);
int op_keygen(Context &c, const uint8_t seed[32], Keys **out);
int op_gen_galois(Context &c, Keys &k, uint64_t g);
void keys_free(Keys *k);
int op_keys_export(Context &c, const Keys &k, uint64_t id, int64_t *s_out, uint64_t *pk_out,
                   uint64_t *ksk_out);
int op_encrypt(Context &c, const Keys &k, const int64_t *msg, const uint8_t seed[32],
               uint64_t *ct, cudaStream_t s);
int op_ct_uniform(Context &c, const uint8_t seed[32], uint32_t index, uint32_t level, uint64_t *ct,
                  cudaStream_t s);
int op_import(Context &c, const uint64_t *host, uint32_t level, uint32_t count, int form,
              bool sync, uint64_t *ct, cudaStream_t s);
int op_export(Context &c, const uint64_t *ct, uint32_t level, uint32_t count, int form,
              bool sync, uint64_t *host, void *ws, size_t ws_bytes_in, cudaStream_t s);
int op_import_packed(Context &c, const uint64_t *host, uint32_t level, uint32_t count, bool sync,
                     uint64_t *ct, void *ws, size_t ws_bytes, cudaStream_t s);
int op_export_packed(Context &c, const uint64_t *ct, uint32_t level, uint32_t count, bool sync,
                     uint64_t *host, void *ws, size_t ws_bytes, cudaStream_t s);
size_t packed_words(const Context &c, uint32_t level);
int op_decrypt(Context &c, const Keys &k, const uint64_t *ct, uint32_t level, uint64_t factor,
               int64_t *msg, void *ws, size_t ws_bytes_in, cudaStream_t s);
int measure_imad_rates(double *lo_per_s, double *hi_per_s, double *wide_per_s, cudaStream_t s);
int measure_int_peak(double *modmul_per_s, double *bfly_per_s, double *bfly_wide_per_s,
                     cudaStream_t s);
int op_rescale_noalloc_impl(Context &c, const uint64_t *a, uint64_t *out, uint32_t level,
                            uint32_t count, cudaStream_t s);
}  // namespace catfhe

using namespace catfhe;

static cudaStream_t S(void *s) { return static_cast<cudaStream_t>(s); }

static bool keys_ok(const catfhe_ctx *ctx, const catfhe_keys *k) {
    return ctx && k && k->k && k->owner == ctx;
}

// Device buffers of the caller: kernels read and write them in 8- and 16-byte
// words, so a pointer that is not 16-byte aligned is refused (EINVAL) before
// anything is enqueued, as is a null one.
static bool dev(const void *p) { return p && !(reinterpret_cast<uintptr_t>(p) & 15); }

extern "C" {

const char *catfhe_strerror(int code) {
    switch (code) {
        case CATFHE_OK: return "ok";
        case CATFHE_EINVAL: return "invalid argument";
        case CATFHE_ELEVEL: return "level out of range";
        case CATFHE_ENOKEY: return "key-switching key missing";
        case CATFHE_ENOMEM: return "device allocation failed";
        case CATFHE_ECUDA: return "CUDA error";
        case CATFHE_ESCHEME: return "operation not defined for this scheme";
        case CATFHE_EWORKSPACE: return "workspace too small";
        case CATFHE_ETIMEOUT: return "a kernel's bounded wait timed out";
        default: return "unknown error";
    }
}

int catfhe_ctx_create(const catfhe_params *params, catfhe_ctx **out) {
    if (!params || !out) return CATFHE_EINVAL;
    catfhe_ctx *ctx = new (std::nothrow) catfhe_ctx();
    if (!ctx) return CATFHE_ENOMEM;
    int rc = ctx_init(ctx->c, *params);
    if (rc != CATFHE_OK) {
        ctx_free(ctx->c);
        delete ctx;
        return rc;
    }
    *out = ctx;
    return CATFHE_OK;
}

void catfhe_ctx_destroy(catfhe_ctx *ctx) {
    if (!ctx) return;
    ctx_free(ctx->c);
    delete ctx;
}

int catfhe_ctx_info(const catfhe_ctx *ctx, catfhe_info *out) {
    if (!ctx || !out) return CATFHE_EINVAL;
    const Context &c = ctx->c;
    out->n = int32_t(c.n);
    out->L = c.L;
    out->K = c.K;
    out->nb = c.nb;
    out->alpha = c.alpha;
    out->beta = c.beta;
    return CATFHE_OK;
}

int catfhe_ctx_moduli(const catfhe_ctx *ctx, uint64_t *q, uint64_t *p, uint64_t *b) {
    if (!ctx) return CATFHE_EINVAL;
    const Context &c = ctx->c;
    for (int i = 0; i < c.L && q; i++) q[i] = c.mod(i);
    for (int i = 0; i < c.K && p; i++) p[i] = c.mod(c.pp(i));
    for (int i = 0; i < c.nb && b; i++) b[i] = c.mod(c.pb(i));
    return CATFHE_OK;
}

uint64_t catfhe_galois_elt(const catfhe_ctx *ctx, int64_t steps) {
    if (!ctx) return 0;
    const uint64_t two_n = 2 * ctx->c.n, slots = ctx->c.n / 2;
    int64_t r = steps % int64_t(slots);
    if (r < 0) r += int64_t(slots);
    return h_powmod(5, uint64_t(r), two_n);
}

int catfhe_keygen(catfhe_ctx *ctx, const uint8_t seed[32], catfhe_keys **out) {
    if (!ctx || !seed || !out) return CATFHE_EINVAL;
    Keys *k = nullptr;
    int rc = op_keygen(ctx->c, seed, &k);
    if (rc != CATFHE_OK) return rc;
    catfhe_keys *h = new (std::nothrow) catfhe_keys{k, ctx};
    if (!h) {
        keys_free(k);
        return CATFHE_ENOMEM;
    }
    *out = h;
    return CATFHE_OK;
}

int catfhe_gen_galois_key(catfhe_ctx *ctx, catfhe_keys *keys, uint64_t galois_elt) {
    if (!keys_ok(ctx, keys)) return CATFHE_EINVAL;
    return op_gen_galois(ctx->c, *keys->k, galois_elt);
}

void catfhe_keys_destroy(catfhe_keys *keys) {
    if (!keys) return;
    keys_free(keys->k);
    delete keys;
}

int catfhe_keys_export(catfhe_ctx *ctx, const catfhe_keys *keys, uint64_t key_id, int64_t *s,
                       uint64_t *pk, uint64_t *ksk) {
    if (!keys_ok(ctx, keys)) return CATFHE_EINVAL;
    return op_keys_export(ctx->c, *keys->k, key_id, s, pk, ksk);
}

int catfhe_encrypt(catfhe_ctx *ctx, const catfhe_keys *keys, const int64_t *msg,
                   const uint8_t seed[32], uint64_t *ct, void *stream) {
    if (!keys_ok(ctx, keys) || !msg || !seed || !dev(ct)) return CATFHE_EINVAL;
    return op_encrypt(ctx->c, *keys->k, msg, seed, ct, S(stream));
}

int catfhe_ct_uniform(catfhe_ctx *ctx, const uint8_t seed[32], uint32_t index, uint32_t level,
                      uint64_t *ct, void *stream) {
    if (!ctx || !seed || !dev(ct)) return CATFHE_EINVAL;
    return op_ct_uniform(ctx->c, seed, index, level, ct, S(stream));
}

static bool split_form(int form, int *base, bool *sync) {
    if (form & ~(0xff | CATFHE_FORM_ASYNC)) return false;
    *base = form & 0xff;
    *sync = !(form & CATFHE_FORM_ASYNC);
    return *base == CATFHE_FORM_COEFF || *base == CATFHE_FORM_NATIVE;
}

int catfhe_ct_import(catfhe_ctx *ctx, const uint64_t *host, uint32_t level, uint32_t count,
                     int form, uint64_t *ct, void *stream) {
    int base;
    bool sync;
    if (!ctx || !host || !dev(ct) || !split_form(form, &base, &sync)) return CATFHE_EINVAL;
    return op_import(ctx->c, host, level, count, base, sync, ct, S(stream));
}

int catfhe_ct_export(catfhe_ctx *ctx, const uint64_t *ct, uint32_t level, uint32_t count,
                     int form, uint64_t *host, void *ws, size_t ws_bytes, void *stream) {
    int base;
    bool sync;
    if (!ctx || !host || !dev(ct) || !split_form(form, &base, &sync)) return CATFHE_EINVAL;
    return op_export(ctx->c, ct, level, count, base, sync, host, ws, ws_bytes, S(stream));
}

size_t catfhe_packed_words(const catfhe_ctx *ctx, uint32_t level, uint32_t count) {
    if (!ctx || level < 1 || int(level) > ctx->c.L) return 0;
    return size_t(2) * count * packed_words(ctx->c, level);
}

int catfhe_ct_import_packed(catfhe_ctx *ctx, const uint64_t *packed, uint32_t level,
                            uint32_t count, uint64_t *ct, void *ws, size_t ws_bytes, int flags,
                            void *stream) {
    if (!ctx || !packed || !dev(ct) || (flags & ~CATFHE_FORM_ASYNC)) return CATFHE_EINVAL;
    return op_import_packed(ctx->c, packed, level, count, !(flags & CATFHE_FORM_ASYNC), ct, ws,
                            ws_bytes, S(stream));
}

int catfhe_ct_export_packed(catfhe_ctx *ctx, const uint64_t *ct, uint32_t level, uint32_t count,
                            uint64_t *packed, void *ws, size_t ws_bytes, int flags, void *stream) {
    if (!ctx || !packed || !dev(ct) || (flags & ~CATFHE_FORM_ASYNC)) return CATFHE_EINVAL;
    return op_export_packed(ctx->c, ct, level, count, !(flags & CATFHE_FORM_ASYNC), packed, ws,
                            ws_bytes, S(stream));
}

// Host side of the packed form (the client's encoder / decoder): plain loops
// over the same bit layout as the device kernels.
static bool pack_shape(const uint8_t *bits, uint32_t level, uint32_t log_n) {
    if (!bits || level < 1 || level > 64 || log_n < 6 || log_n > 20) return false;
    for (uint32_t i = 0; i < level; i++)
        if (bits[i] < 1 || bits[i] > 64) return false;
    return true;
}

int catfhe_pack_host(const uint8_t *bits, uint32_t level, uint32_t polys, uint32_t log_n,
                     const uint64_t *limbs, uint64_t *packed) {
    if (!pack_shape(bits, level, log_n) || (polys && (!limbs || !packed))) return CATFHE_EINVAL;
    const uint64_t n = uint64_t(1) << log_n;
    for (uint32_t p = 0; p < polys; p++)
        for (uint32_t i = 0; i < level; i++) {
            const uint32_t b = bits[i];
            const uint64_t mask = b == 64 ? ~uint64_t(0) : (uint64_t(1) << b) - 1;
            const uint64_t words = n * b / 64;
            for (uint64_t w = 0; w < words; w++) packed[w] = 0;
            for (uint64_t k = 0; k < n; k++) {
                const uint64_t v = limbs[k] & mask, o = k * b;
                const uint64_t w = o >> 6, sh = o & 63;
                packed[w] |= v << sh;
                if (sh + b > 64) packed[w + 1] |= v >> (64 - sh);
            }
            limbs += n;
            packed += words;
        }
    return CATFHE_OK;
}

int catfhe_unpack_host(const uint8_t *bits, uint32_t level, uint32_t polys, uint32_t log_n,
                       const uint64_t *packed, uint64_t *limbs) {
    if (!pack_shape(bits, level, log_n) || (polys && (!limbs || !packed))) return CATFHE_EINVAL;
    const uint64_t n = uint64_t(1) << log_n;
    for (uint32_t p = 0; p < polys; p++)
        for (uint32_t i = 0; i < level; i++) {
            const uint32_t b = bits[i];
            const uint64_t mask = b == 64 ? ~uint64_t(0) : (uint64_t(1) << b) - 1;
            for (uint64_t k = 0; k < n; k++) {
                const uint64_t o = k * b, w = o >> 6, sh = o & 63;
                uint64_t v = packed[w] >> sh;
                if (sh + b > 64) v |= packed[w + 1] << (64 - sh);
                limbs[k] = v & mask;
            }
            limbs += n;
            packed += n * b / 64;
        }
    return CATFHE_OK;
}

int catfhe_add(catfhe_ctx *ctx, const uint64_t *a, const uint64_t *b, uint64_t *out,
               uint32_t level, uint32_t count, void *stream) {
    if (!ctx || !dev(a) || !dev(b) || !dev(out)) return CATFHE_EINVAL;
    return op_add(ctx->c, a, b, out, level, count, S(stream));
}

int catfhe_sub(catfhe_ctx *ctx, const uint64_t *a, const uint64_t *b, uint64_t *out,
               uint32_t level, uint32_t count, void *stream) {
    if (!ctx || !dev(a) || !dev(b) || !dev(out)) return CATFHE_EINVAL;
    return op_sub(ctx->c, a, b, out, level, count, S(stream));
}

int catfhe_mul_int(catfhe_ctx *ctx, const uint64_t *a, int64_t k, uint64_t *out, uint32_t level,
                   uint32_t count, void *stream) {
    if (!ctx || !dev(a) || !dev(out)) return CATFHE_EINVAL;
    return op_mul_int(ctx->c, a, k, out, level, count, S(stream));
}

int catfhe_add_const(catfhe_ctx *ctx, const uint64_t *a, int64_t k, uint64_t *out,
                     uint32_t level, uint32_t count, void *stream) {
    if (!ctx || !dev(a) || !dev(out)) return CATFHE_EINVAL;
    return op_add_const(ctx->c, a, k, out, level, count, S(stream));
}

int catfhe_drop_level(catfhe_ctx *ctx, const uint64_t *a, uint32_t level, uint32_t new_level,
                      uint64_t *out, uint32_t count, void *stream) {
    if (!ctx || !dev(a) || !dev(out) || a == out) return CATFHE_EINVAL;
    return op_drop_level(ctx->c, a, level, new_level, out, count, S(stream));
}

int catfhe_mul_relin(catfhe_ctx *ctx, const catfhe_keys *keys, const uint64_t *a,
                     const uint64_t *b, uint64_t *out, uint32_t level, uint32_t count,
                     void *ws, size_t ws_bytes, void *stream) {
    if (!keys_ok(ctx, keys) || !dev(a) || !dev(b) || !dev(out)) return CATFHE_EINVAL;
    return op_mul_relin(ctx->c, *keys->k, a, b, out, level, count, false, ws, ws_bytes, S(stream),
                        nullptr, true);
}

int catfhe_mul_relin_rescale(catfhe_ctx *ctx, const catfhe_keys *keys, const uint64_t *a,
                             const uint64_t *b, uint64_t *out, uint32_t level, uint32_t count,
                             void *ws, size_t ws_bytes, void *stream) {
    if (!keys_ok(ctx, keys) || !dev(a) || !dev(b) || !dev(out)) return CATFHE_EINVAL;
    return op_mul_relin(ctx->c, *keys->k, a, b, out, level, count, true, ws, ws_bytes, S(stream),
                        nullptr, true);
}

int catfhe_rotate(catfhe_ctx *ctx, const catfhe_keys *keys, const uint64_t *a,
                  uint64_t galois_elt, uint64_t *out, uint32_t level, uint32_t count, void *ws,
                  size_t ws_bytes, void *stream) {
    if (!keys_ok(ctx, keys) || !dev(a) || !dev(out)) return CATFHE_EINVAL;
    return op_rotate(ctx->c, *keys->k, a, galois_elt, out, level, count, ws, ws_bytes, S(stream),
                     nullptr, true);
}

int catfhe_device_status(catfhe_ctx *ctx, int32_t *flags, int clear, void *stream) {
    if (!ctx || !flags) return CATFHE_EINVAL;
    cudaStream_t s = S(stream);
    int v = 0;
    if (cudaMemcpyAsync(&v, ctx->c.d_status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return CATFHE_ECUDA;
    if (clear && cudaMemsetAsync(ctx->c.d_status, 0, sizeof(int), s) != cudaSuccess)
        return CATFHE_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CATFHE_ECUDA;
    *flags = v;
    return CATFHE_OK;
}

int catfhe_sync(catfhe_ctx *ctx, void *stream) {
    int32_t flags = 0;
    const int rc = catfhe_device_status(ctx, &flags, 0, stream);
    if (rc) return rc;
    return flags ? CATFHE_ETIMEOUT : CATFHE_OK;
}

int catfhe_wait_selftest(catfhe_ctx *ctx, uint64_t limit_ns, void *stream) {
    if (!ctx || limit_ns < 1000 || limit_ns > 10000000000ull) return CATFHE_EINVAL;
    return launch_wait_selftest(ctx->c, limit_ns, S(stream));
}

int catfhe_plain_import(catfhe_ctx *ctx, const int64_t *coeffs, uint32_t level, uint64_t *pt,
                        void *stream) {
    if (!ctx || !coeffs || !dev(pt)) return CATFHE_EINVAL;
    return op_plain_import(ctx->c, coeffs, level, pt, S(stream));
}

int catfhe_encode_ckks(catfhe_ctx *ctx, const double *slots, double scale, uint32_t level,
                       uint64_t *pt, void *ws, size_t ws_bytes, void *stream) {
    if (!ctx || !slots || !dev(pt)) return CATFHE_EINVAL;
    return op_encode_ckks(ctx->c, slots, scale, level, pt, ws, ws_bytes, S(stream));
}

int catfhe_decode_ckks(catfhe_ctx *ctx, const catfhe_keys *keys, const uint64_t *ct,
                       uint32_t level, double scale, double *slots, void *ws, size_t ws_bytes,
                       void *stream) {
    if (!keys_ok(ctx, keys) || !dev(ct) || !slots) return CATFHE_EINVAL;
    return op_decode_ckks(ctx->c, *keys->k, ct, level, scale, slots, ws, ws_bytes, S(stream));
}

int catfhe_mul_plain(catfhe_ctx *ctx, const uint64_t *a, const uint64_t *pt, uint64_t *out,
                     uint32_t level, uint32_t count, void *stream) {
    if (!ctx || !dev(a) || !dev(pt) || !dev(out)) return CATFHE_EINVAL;
    return op_mul_plain(ctx->c, a, pt, out, level, count, S(stream));
}

int catfhe_rotate_hoisted(catfhe_ctx *ctx, const catfhe_keys *keys, const uint64_t *a,
                          const uint64_t *galois_elts, uint32_t n_rot, uint64_t *out,
                          uint32_t level, uint32_t count, void *ws, size_t ws_bytes,
                          void *stream) {
    if (!keys_ok(ctx, keys) || !dev(a) || (n_rot > 0 && !dev(out))) return CATFHE_EINVAL;
    return op_rotate_hoisted(ctx->c, *keys->k, a, galois_elts, n_rot, out, level, count, ws,
                             ws_bytes, S(stream));
}

int catfhe_rescale(catfhe_ctx *ctx, const uint64_t *a, uint64_t *out, uint32_t level,
                   uint32_t count, void *ws, size_t ws_bytes, void *stream) {
    if (!ctx || !dev(a)) return CATFHE_EINVAL;
    if (ctx->c.scheme == CATFHE_BFV) return CATFHE_ESCHEME;
    if (level < 2 || int(level) > ctx->c.L) return CATFHE_ELEVEL;
    if (!dev(out)) return CATFHE_EINVAL;
    return op_rescale(ctx->c, a, out, level, count, ws, ws_bytes, S(stream));
}

int catfhe_rescale_noalloc(catfhe_ctx *ctx, const uint64_t *a, uint64_t *out, uint32_t level,
                           uint32_t count, void *stream) {
    if (!ctx || !dev(a)) return CATFHE_EINVAL;
    if (ctx->c.scheme == CATFHE_BFV) return CATFHE_ESCHEME;
    if (level < 2 || int(level) > ctx->c.L) return CATFHE_ELEVEL;
    if (!dev(out) || out == a) return CATFHE_EINVAL;
    return op_rescale_noalloc_impl(ctx->c, a, out, level, count, S(stream));
}

int catfhe_decrypt(catfhe_ctx *ctx, const catfhe_keys *keys, const uint64_t *ct, uint32_t level,
                   uint64_t factor, int64_t *msg, void *ws, size_t ws_bytes, void *stream) {
    if (!keys_ok(ctx, keys) || !dev(ct) || !msg) return CATFHE_EINVAL;
    return op_decrypt(ctx->c, *keys->k, ct, level, factor, msg, ws, ws_bytes, S(stream));
}

int catfhe_ntt(catfhe_ctx *ctx, uint64_t *limbs, uint32_t level, uint32_t count, int inverse,
               void *stream) {
    if (!ctx || !dev(limbs)) return CATFHE_EINVAL;
    return op_ntt(ctx->c, limbs, level, count, inverse, S(stream));
}

int catfhe_measure_int_peak(double *modmul_per_s, double *butterfly_per_s,
                            double *butterfly_wide_per_s, void *stream) {
    return measure_int_peak(modmul_per_s, butterfly_per_s, butterfly_wide_per_s, S(stream));
}

int catfhe_measure_imad_rates(double *lo_per_s, double *hi_per_s, double *wide_per_s,
                              void *stream) {
    return measure_imad_rates(lo_per_s, hi_per_s, wide_per_s, S(stream));
}

uint64_t catfhe_kernel_launches(void) { return launches_total(); }

size_t catfhe_workspace_bytes(const catfhe_ctx *ctx, int op, uint32_t level, uint32_t count) {
    if (!ctx) return 0;
    return ws_bytes(ctx->c, op, level, count);
}

}  // extern "C"
