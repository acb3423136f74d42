// Internal structures shared by the host orchestration and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <string>
#include <vector>

#include "catfhe.h"

namespace catfhe {

constexpr int kMaxPrimes = 128;   // global prime table (q, p, b)
constexpr int kMapMax = 128;      // limbs per group in one LimbMap
// Largest number of separately addressed ciphertexts in one operation (Gather).
constexpr int kGatherMax = 8;
constexpr int kConvMaxK = 32;     // sources of one exact base conversion
constexpr int kConvMaxT = 48;     // targets of one exact base conversion
// Bound, in multiples of q, of the forward NTT's unreduced words for primes
// below 2^57 (inputs below 4q, 4q more per stage over at most 16 stages).
constexpr uint64_t kWideWordsQ = 68;

// One modulus as the kernels see it.  q < 2^62.
struct DevMod {
    uint64_t q;
    uint64_t r64, r64_s;      // 2^64 mod q and its Shoup quotient
    uint64_t one_s;           // floor(2^64 / q): Shoup quotient of 1
    uint64_t ninv, ninv_s;    // N^-1 mod q
    uint64_t ninvw, ninvw_s;  // N^-1 * psi^-1(bitrev 1) mod q (last inverse stage)
    uint64_t qinv;            // -q^-1 mod 2^64 (Montgomery reduction)
    uint64_t m64;             // floor(2^64 / q) when q > 2^33 (fits 32 bits), else 0
};

// Addressing of a batch of limbs: limb l of a launch is entry r = l % period
// of group g = l / period; it lives at base + (g * stride + off[r]) * N and
// is reduced mod prime[r] (index into the context's prime table).
struct LimbMap {
    uint32_t period;
    uint32_t src_stride, dst_stride;  // in limbs
    uint16_t src_off[kMapMax];
    uint16_t dst_off[kMapMax];
    uint8_t prime[kMapMax];
};

// Constants of one exact, centred base conversion from k source moduli to T
// target moduli (mixed-radix form of the CRT; see conv.cu), packed into a
// flat array of 64-bit words.  Word 0 is the header
//   k | T << 16 | wrap64 << 32 | lazy << 33 | mont << 34 | split << 35
// (wrap64: targets are 2^64; lazy: outputs may lie in [0, 2q) instead of
// [0, q), for an NTT to consume; mont: the Montgomery layout below; split:
// the same layout with every weight of C and Ct stored as its two 30-bit
// halves lo | hi << 32, for k <= 8 and moduli below 2^60).
// Then src_off[k], dst_off[T] (limb offsets per item) and
//  exact layout:  smod[k][4] (q, 2^64 mod q, its Shoup quotient, floor(2^64/q)),
//                 dmod[T][4], pre[k], pre_s[k], W[k][k] (prod_{l<i} m_l mod m_j),
//                 Minv[k], Minv_s[k] ((prod_{l<j} m_l)^-1 mod m_j), h[k]
//                 (mixed-radix digits of (M-1)/2), Wt[k][T] (prod_{l<i} m_l
//                 mod p_t), Mt[T] (M mod p_t), post[T], post_s[T];
//  Montgomery layout (every constant times 2^64 mod its modulus, so one
//                 Montgomery reduction per sum returns the plain value):
//                 smod[k][2] (m, -m^-1 mod 2^64), dmod[T][2],
//                 C[k][k] (row i, column j: the weight of digit a_i, or for
//                 i = j of the residue r_j, in the mixed-radix step of a_j),
//                 h[k], Ct[k][T] (weight of a_i for target t, post-multiplier
//                 folded in), Mneg[T] (-M mod p_t, post-multiplier folded in).
__host__ __device__ inline size_t plan_words(uint32_t k, uint32_t T, bool mont) {
    return mont ? 1 + 4 * size_t(k) + 4 * size_t(T) + size_t(k) * k + size_t(k) * T
                : 1 + 10 * size_t(k) + 8 * size_t(T) + size_t(k) * k + size_t(k) * T;
}
__host__ __device__ inline size_t plan_words(uint64_t header) {
    return plan_words(uint32_t(header & 0xffff), uint32_t((header >> 16) & 0xffff),
                      ((header >> 34) & 1) != 0);
}

// Source / target description of a conversion plan.  A target modulus of 0
// means 2^64 (two's complement output).  Empty pre / post mean 1.
struct PlanSpec {
    bool lazy = false;
    bool exact = false;  // force the exact layout (else Montgomery when it fits)
    bool split = false;  // Montgomery with split weights (when it fits)
    std::vector<uint64_t> src_mod;
    std::vector<uint32_t> src_off;
    std::vector<uint64_t> pre;
    std::vector<uint64_t> dst_mod;
    std::vector<uint32_t> dst_off;
    std::vector<uint64_t> post;
};
std::vector<uint64_t> build_plan(const PlanSpec &s);
// The Montgomery layout needs sum(src_mod) + 1 < 2^64 (every accumulated sum
// stays below 2^64 times its modulus).
bool plan_fits_mont(const PlanSpec &s);
// Split weights need k <= 8 and every source and target modulus in (0, 2^60)
// (then the 30-bit half products of a sum accumulate below 2^64), besides
// the Montgomery bound.
bool plan_fits_split(const PlanSpec &s);
struct PlanRef {
    const uint64_t *p = nullptr;  // device copy
    uint32_t words = 0;
    bool mont = false;
    bool split = false;
};
struct Context;
PlanRef get_plan(Context &c, const std::string &key, const PlanSpec &spec);
PlanRef get_plan_extra(Context &c, const std::string &key, const PlanSpec &spec,
                       const std::vector<uint64_t> &extra);

// Up to this many plans run in one launch (grid.z).
struct PlanList {
    const uint64_t *p[64];
    uint32_t n;      // plans in the launch
    uint32_t kmax;   // largest source count among them
    uint32_t kmin;   // smallest source count among them
    uint32_t words;  // largest packed size among them
    uint32_t mont;   // all plans use the Montgomery layout
    uint32_t split;  // ... with split weights
};

// Host-side prime record.
struct HostPrime {
    uint64_t q;
    uint64_t psi;  // smallest primitive 2N-th root of unity
};

struct Scratch {
    void *ptr = nullptr;
    size_t bytes = 0;
};

struct Context {
    catfhe_params prm{};
    int scheme = 0, log_n = 0, L = 0, K = 0, nb = 0, alpha = 0, beta = 0;
    uint64_t n = 0, t = 0;
    std::vector<HostPrime> primes;  // q_0..q_{L-1}, p_0..p_{K-1}, b_0..b_{nb-1}
    std::vector<DevMod> hmods;
    DevMod *d_mods = nullptr;
    ulonglong2 *d_twf = nullptr;  // [prime][N] (psi^bitrev(i), Shoup)
    ulonglong2 *d_twi = nullptr;  // [prime][N] (psi^-bitrev(i), Shoup)
    uint64_t cdt[19] = {};
    std::map<std::string, uint64_t *> plans;     // device copies of packed plans
    std::map<std::string, uint32_t> plan_sizes;  // words
    Scratch scratch;
    int device = 0;
    // NTT schedule index for this ring degree (see ntt.cu), per launch size
    // class (ntt_class)
    int ntt_sched[3] = {0, 0, 0};
    int *d_status = nullptr;    // device status word: bits of kernels' timed-out waits
    double2 *d_enc = nullptr;   // CKKS encoder tables (encode.cu), built on first use
    uint32_t *d_slot = nullptr;

    int pq(int i) const { return i; }                // index of q_i
    int pp(int k) const { return L + k; }            // index of p_k
    int pb(int i) const { return L + K + i; }        // index of b_i
    uint64_t mod(int idx) const { return primes[idx].q; }
};

struct Keys {
    uint8_t seed[32];
    uint64_t *s_ntt = nullptr;                 // [L+K][N] NTT form
    uint64_t *pk = nullptr;                    // [2][L][N] NTT form
    // id -> [beta][2][L+K][N], NTT form and Montgomery form (times 2^64 mod
    // the limb's prime), so the inner product needs one reduction per sum
    std::map<uint64_t, uint64_t *> ksk;
};

// Number of kernels this library has launched (all contexts, all threads).
void note_launches(uint32_t k);
// CTAs of `kernel` resident on the whole current device (SMs x CTAs per SM at
// `threads` threads and `smem` dynamic shared bytes), 0 if unknown; cached.
int resident_slots(const void *kernel, int threads, size_t smem);
uint64_t launches_total();

// ----------------------------------------------------------------- launchers
// NTT (ntt.cu)
int launch_ntt_fwd(const Context &c, const uint64_t *src, uint64_t *dst, const LimbMap &map,
                   uint32_t n_limbs, cudaStream_t s);
int launch_ntt_inv(const Context &c, const uint64_t *src, uint64_t *dst, const LimbMap &map,
                   uint32_t n_limbs, cudaStream_t s);

// Forward NTT whose last pass also finishes the ModDown: for map entry r of
// group g it writes out = (y - NTT(lift)) * dinv[r] (+ add) instead of the
// transform (the lift itself is left in its column-pass state).
struct NttEpilogue {
    const uint64_t *y, *add;
    uint64_t *out;
    uint32_t y_stride, add_stride, out_stride;  // per group, in limbs
    uint16_t y_off[kMapMax], add_off[kMapMax], out_off[kMapMax];
    uint64_t dinv[kMapMax], dinv_s[kMapMax];
    uint32_t gathered;                          // nonzero: group g writes gout[g]
    uint64_t *gout[kGatherMax];
    int *status;                                // the context's status word (bulk-copy wait)
};
// Bit-packed transfer form (pack.cu): words per polynomial at `level`, and
// the device unpack / pack of `polys` polynomials.
size_t packed_words(const Context &c, uint32_t level);
int launch_unpack(const Context &c, const uint64_t *packed, uint64_t *out, uint32_t level,
                  uint32_t polys, cudaStream_t s);
int launch_pack(const Context &c, const uint64_t *in, uint64_t *packed, uint32_t level,
                uint32_t polys, cudaStream_t s);

// Forward NTT whose outputs for primes below 2^57 are left unreduced (below
// 68q; larger primes reduced to [0, q)), for a consumer that reduces anyway.
int launch_ntt_fwd_lazy(const Context &c, const uint64_t *src, uint64_t *dst, const LimbMap &map,
                        uint32_t n_limbs, cudaStream_t s);
int launch_ntt_fwd_combine(const Context &c, uint64_t *lift, const LimbMap &map, uint32_t n_limbs,
                           const NttEpilogue &epi, cudaStream_t s);

// Launch size classes of the NTT schedule choice: up to 64 limbs in one
// launch (about one ciphertext), up to 256, more.
constexpr int kNttClasses = 3;
inline int ntt_class(uint32_t limbs) { return limbs <= 64 ? 0 : limbs <= 256 ? 1 : 2; }
int ntt_schedule_count(int log_n);
void ntt_schedule_shape(int log_n, int sched, int shape[4]);
int tune_ntt(Context &c, uint32_t limbs, cudaStream_t s, int *chosen, float *us_out);

// Exact base conversion (conv.cu): grid over (coefficient, item, plan).
// grid.z runs plan z over items item = 0..items-1 (grid.y): sources at
// src + item * src_item + src_off * N, targets at dst + item * dst_item + ...;
// plan z may add z * src_plan / dst_plan to the item bases.
int launch_conv(const Context &c, const PlanList &plans, const uint64_t *src, size_t src_item,
                size_t src_plan, uint64_t *dst, size_t dst_item, size_t dst_plan, uint32_t items,
                cudaStream_t s);
// BFV: given the tensor x over Q u B (coefficient form, Q limbs first) of
// each item, writes round(t x / Q) mod q_i: y = t x; z = (y - [y]_Q) Q^-1 over
// B (plan q_to_b lifts [y]_Q with pre = t and post = 1); then the centred
// lift of z from B back to Q (plan b_to_q).  qinv_b: Q^-1 mod b_j (Shoup).
int launch_bfv_scale_round(const Context &c, const uint64_t *q_to_b, uint32_t q_to_b_words,
                           const uint64_t *b_to_q, uint32_t b_to_q_words, const uint64_t *src,
                           size_t src_item, uint64_t *dst, size_t dst_item, uint32_t items,
                           cudaStream_t s);

// Element-wise kernels (elementwise.cu)
// Per-ciphertext base pointers of an operation whose ciphertexts are not
// contiguous: an uneven batch merges compatible single-ciphertext entries
// into one operation of count = n items; item i reads a[i] (and b[i]) and
// writes out[i], each u64[2][level][N].  Only the kernels that touch the
// caller's buffers (the tensor's loads, the automorphism's loads, ModDown's
// final stores) look at it; everything between runs on contiguous workspace.
struct Gather {
    uint32_t n = 0;
    const uint64_t *a[kGatherMax];
    const uint64_t *b[kGatherMax];
    uint64_t *out[kGatherMax];
};

struct TensorArgs {
    const uint64_t *a, *b;       // [count][2][limbs][N]
    uint64_t *d0, *d1, *d2;      // each [count][limbs][N] (item stride given)
    size_t in_item, out_item;    // item strides in elements
    uint32_t limbs;
    uint8_t prime[kMapMax];
    uint32_t gathered;           // nonzero: item i reads ga[i], gb[i]
    const uint64_t *ga[kGatherMax], *gb[kGatherMax];
};
int launch_tensor(const Context &c, const TensorArgs &a, uint32_t count, cudaStream_t s);

struct IpArgs {
    const uint64_t *ext;       // [count][beta][M][N]: lifted digits (NTT form)
    const uint64_t *own;       // [count][l][N]: d2 in NTT form (digit's own limbs), or null
    const uint64_t *key;       // [beta_L][2][L+K][N], Montgomery form
    const uint64_t *add0, *add1;  // [count][l][N] added times P (Q positions), or null
    uint64_t *y;               // [count][2][M][N]
    size_t ext_item, own_item, add_item, y_item;
    uint32_t M, level, beta, L, K;
    uint32_t alpha;
    uint8_t prime[kMapMax];    // prime of position i
    uint16_t key_limb[kMapMax];
    uint64_t pfac[kMapMax];    // P 2^64 mod prime(i) (0 for P positions)
    int *status;               // the context's status word (bulk-copy wait timeouts)
};
int launch_ip(const Context &c, const IpArgs &a, uint32_t count, cudaStream_t s);
int launch_wait_selftest(const Context &c, uint64_t limit_ns, cudaStream_t s);

struct CombineArgs {
    const uint64_t *y;         // [count][2][.][N] at y_off positions
    const uint64_t *lift;      // [count][2][lo][N]
    const uint64_t *add;       // [count][2][lo][N] or null
    uint64_t *out;             // [count][2][lo][N]
    size_t y_item, y_poly, lift_item, lift_poly, add_item, add_poly, out_item, out_poly;
    uint32_t lo;               // output limbs
    uint8_t prime[kMapMax];
    uint64_t dinv[kMapMax], dinv_s[kMapMax];
};
int launch_combine(const Context &c, const CombineArgs &a, uint32_t count, cudaStream_t s);

int launch_automorph_ntt(const Context &c, const uint64_t *in, uint64_t *out, uint32_t limbs_total,
                         uint64_t g, cudaStream_t s);
// NTT-form automorphism over the limbs a LimbMap selects (limbs_total =
// groups x period); in and out must not overlap.
int launch_automorph_ntt_map(const Context &c, const uint64_t *in, uint64_t *out,
                             const LimbMap &map, uint32_t limbs_total, uint64_t g, cudaStream_t s);
// out[ct][p][i] = a[ct][p][i] * pt[i] mod q_i (NTT form), n_limbs = count x 2 x level.
int launch_mul_plain(const Context &c, const uint64_t *a, const uint64_t *pt, uint64_t *out,
                     uint32_t level, uint32_t n_limbs, cudaStream_t s);

// CKKS canonical embedding on the device (encode.cu).  enc_tables builds
// the context's tables once; encode: N/2 device slots -> int64 m[N];
// decode: int64 m[N] -> N/2 device slots.  buf0, buf1: N complex each.
int enc_tables(Context &c);
int launch_encode_ckks(const Context &c, const double2 *slots, double scale, double2 *buf0,
                       double2 *buf1, int64_t *m, cudaStream_t s);
int launch_decode_ckks(const Context &c, const int64_t *m, double inv_scale, double2 *buf0,
                       double2 *buf1, double2 *slots, cudaStream_t s);
int launch_automorph_coeff(const Context &c, const uint64_t *in, uint64_t *out,
                           const LimbMap &map, uint32_t n_limbs, uint64_t g, cudaStream_t s);
int launch_add(const Context &c, const uint64_t *a, const uint64_t *b, uint64_t *out,
               const LimbMap &map, uint32_t n_limbs, cudaStream_t s);
int launch_copy_limbs(const Context &c, const uint64_t *src, uint64_t *dst, const LimbMap &map,
                      uint32_t n_limbs, cudaStream_t s);
int launch_sub(const Context &c, const uint64_t *a, const uint64_t *b, uint64_t *out,
               const LimbMap &map, uint32_t n_limbs, cudaStream_t s);
// per map entry r: out = a * k[r] (Shoup pair k_s[r]), or a + k[r] where add[r]
int launch_const_op(const Context &c, const uint64_t *a, uint64_t *out, const LimbMap &map,
                    uint32_t n_limbs, const uint64_t *k, const uint64_t *k_s, const uint8_t *add,
                    cudaStream_t s);

// Sampling (sample.cu)
enum SampleKind { kUniform = 0, kTernary = 1, kGaussian = 2 };
struct SampleArgs {
    uint32_t key[8];
    uint32_t tag, i0, i1;
    uint32_t kind;
    uint64_t cdt[19];
};
// Uniform: residues over the map's primes (limb index i of the stream =
// map entry r).  Ternary / Gaussian: small signed values reduced to every
// limb of the map, times mult[r] (Shoup pair) (t e for BGV).
int launch_sample(const Context &c, const SampleArgs &a, uint64_t *out, const LimbMap &map,
                  uint32_t n_limbs, const uint64_t *mult, const uint64_t *mult_s,
                  cudaStream_t s);
// int64 message -> residues (times mult, Shoup), added into out if accumulate.
int launch_small_to_rns(const Context &c, const int64_t *in, uint64_t *out, const LimbMap &map,
                        uint32_t n_limbs, const uint64_t *mult, const uint64_t *mult_s,
                        int accumulate, cudaStream_t s);
// out = c0 + c1 * s (pointwise, NTT domain), per limb.
int launch_mul_add(const Context &c, const uint64_t *c0, const uint64_t *c1, const uint64_t *sk,
                   uint64_t *out, uint32_t limbs, int negate_product, cudaStream_t s);
// out[l] = a[l] * b[l] (pointwise) over a map.
int launch_pointwise(const Context &c, const uint64_t *a, const uint64_t *b, uint64_t *out,
                     const LimbMap &map, uint32_t n_limbs, cudaStream_t s);
// Key-switching key rows: b = -a*s + e + pfac * s' (NTT domain), per limb.
int launch_ksk_row(const Context &c, const uint64_t *a, const uint64_t *sk, const uint64_t *e,
                   const uint64_t *sp, uint64_t *b, uint32_t limbs, const uint64_t *pfac,
                   const uint64_t *pfac_s, cudaStream_t s);
// x[g][i] *= w_i (Shoup constants per limb i of a group of `limbs`), groups of
// `limbs` consecutive limbs, limb i mod prime i.
int launch_scale_limbs(const Context &c, uint64_t *x, uint32_t limbs, uint32_t groups,
                       const uint64_t *w, const uint64_t *w_s, cudaStream_t s);

// host math (hostmath.cpp)
uint64_t h_mulmod(uint64_t a, uint64_t b, uint64_t m);
uint64_t h_powmod(uint64_t a, uint64_t e, uint64_t m);
uint64_t h_invmod(uint64_t a, uint64_t m);
bool h_is_prime(uint64_t n);
uint64_t h_shoup(uint64_t w, uint64_t q);
uint64_t h_min_psi(uint64_t q, int log_n);
void h_cdt(uint64_t out[19]);
DevMod h_devmod(uint64_t q, uint64_t n, uint64_t psi);

}  // namespace catfhe

// The opaque handles of the C ABI.
struct catfhe_ctx {
    catfhe::Context c;
};
struct catfhe_keys {
    catfhe::Keys *k;
    const catfhe_ctx *owner;
};
