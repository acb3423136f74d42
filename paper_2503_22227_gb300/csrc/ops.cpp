// Scheme operations: key generation, encryption, decryption, and the hot
// path (tensor -> ModUp -> inner product -> ModDown [-> rescale]), as
// sequences of batched kernel launches on one stream.
//
// Every step follows the definitions the CPU oracle computes (hybrid key
// switching with exact centred lifts; ModDown round(x / P), or
// (x - t [x t^-1]_P) / P for BGV; CKKS rescale round(c / q_{l-1}); BFV
// multiplication by exact round(t x / Q) over an auxiliary basis).
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "internal.h"

namespace catfhe {


#define TRY(x)                      \
    do {                            \
        int rc_ = (x);              \
        if (rc_ != CATFHE_OK) return rc_; \
    } while (0)

// ----------------------------------------------------------------- workspace

struct Bump {
    char *base;
    size_t off = 0;
    template <class T>
    T *take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

static int get_ws(Context &c, void *ws, size_t ws_bytes, size_t need, char **out) {
    if (ws) {
        // kernels access the workspace in 8- and 16-byte words (and bulk
        // copies need 16-byte alignment): refuse a pointer that is not
        if (reinterpret_cast<uintptr_t>(ws) & 15) return CATFHE_EINVAL;
        if (ws_bytes < need) return CATFHE_EWORKSPACE;
        *out = static_cast<char *>(ws);
        return CATFHE_OK;
    }
    if (c.scratch.bytes < need) {
        cudaFree(c.scratch.ptr);
        c.scratch.ptr = nullptr;
        c.scratch.bytes = 0;
        if (cudaMalloc(&c.scratch.ptr, need) != cudaSuccess) return CATFHE_ENOMEM;
        c.scratch.bytes = need;
    }
    *out = static_cast<char *>(c.scratch.ptr);
    return CATFHE_OK;
}

// One launch's plans, all in one layout: Montgomery when every plan fits it
// (with split weights when every plan fits those too), else exact.
static int make_list(Context &c, const std::vector<std::pair<std::string, PlanSpec>> &specs,
                     PlanList &pl) {
    bool all = true, all_split = true;
    for (const auto &s : specs) {
        all = all && plan_fits_mont(s.second);
        all_split = all_split && plan_fits_split(s.second);
    }
    pl = PlanList{};
    pl.n = uint32_t(specs.size());
    pl.mont = all ? 1 : 0;
    pl.split = all && all_split ? 1 : 0;
    for (size_t i = 0; i < specs.size(); i++) {
        PlanSpec sp = specs[i].second;
        sp.exact = !all;
        sp.split = pl.split != 0;
        const PlanRef r = get_plan(c, specs[i].first, sp);
        if (!r.p) return CATFHE_ENOMEM;
        if (r.mont != (pl.mont != 0) || r.split != (pl.split != 0)) return CATFHE_EINVAL;
        pl.p[i] = r.p;
        pl.kmax = std::max<uint32_t>(pl.kmax, uint32_t(sp.src_mod.size()));
        pl.kmin = i == 0 ? uint32_t(sp.src_mod.size())
                         : std::min<uint32_t>(pl.kmin, uint32_t(sp.src_mod.size()));
        pl.words = std::max(pl.words, r.words);
    }
    return CATFHE_OK;
}

static LimbMap map_identity(uint32_t limbs, uint32_t first_prime = 0) {
    LimbMap m{};
    m.period = limbs;
    m.src_stride = m.dst_stride = limbs;
    for (uint32_t i = 0; i < limbs; i++) {
        m.src_off[i] = m.dst_off[i] = uint16_t(i);
        m.prime[i] = uint8_t(first_prime + i);
    }
    return m;
}

static uint64_t prod_mod(const Context &c, int from, int to, uint64_t m) {
    uint64_t r = 1 % m;
    for (int i = from; i < to; i++) r = h_mulmod(r, c.mod(i) % m, m);
    return r;
}

// P = prod p_k mod m
static uint64_t pmod(const Context &c, uint64_t m) { return prod_mod(c, c.L, c.L + c.K, m); }

// ----------------------------------------------------------------- key switching pieces

// Global prime index of extended position i at level l (Q_l then P).
static int ext_prime(const Context &c, int level, int i) { return i < level ? i : c.L + (i - level); }

// ModUp: lift each digit of d2 (coefficient form, [count][level][N]) to the
// other primes of Q_l u P, written into ext ([count][beta][M][N]).
static int modup(Context &c, const uint64_t *d2c, uint64_t *ext, uint32_t count, int level,
                 bool own_too, cudaStream_t s) {
    const int M = level + c.K, beta = (level + c.alpha - 1) / c.alpha;
    std::vector<std::pair<std::string, PlanSpec>> specs;
    for (int j = 0; j < beta; j++) {
        const int lo = j * c.alpha, hi = std::min((j + 1) * c.alpha, level);
        PlanSpec sp;
        sp.lazy = true;  // the lifted limbs go straight into an NTT
        for (int i = lo; i < hi; i++) {
            sp.src_mod.push_back(c.mod(i));
            sp.src_off.push_back(uint32_t(i));
        }
        for (int i = 0; i < M; i++) {
            if (!own_too && i >= lo && i < hi) continue;
            sp.dst_mod.push_back(c.mod(ext_prime(c, level, i)));
            sp.dst_off.push_back(uint32_t(i));
        }
        specs.emplace_back("modup/" + std::to_string(level) + "/" + std::to_string(j) +
                               (own_too ? "/own" : ""),
                           sp);
    }
    PlanList pl;
    TRY(make_list(c, specs, pl));
    const size_t n = c.n;
    return launch_conv(c, pl, d2c, size_t(level) * n, 0, ext, size_t(beta) * M * n, size_t(M) * n,
                       count, s);
}

// Whether the lifted digits' forward NTT may leave its words unreduced: the
// inner product is their only reader and reduces its sums once (Montgomery,
// valid below 2^64 q); with words below 68q from an unreduced transform, its
// beta products and the folded P d term stay below (68 beta + 1) q^2.  Used
// when that bound holds for every prime below 2^57 of Q_l u P (larger
// primes are reduced anyway).
static bool ext_lazy(const Context &c, int level) {
    const int beta = (level + c.alpha - 1) / c.alpha;
    for (int i = 0; i < level + c.K; i++) {
        const uint64_t q = c.mod(ext_prime(c, level, i));
        if (q < (uint64_t(1) << 57) &&
            (unsigned __int128)(kWideWordsQ * uint64_t(beta) + 1) * q >=
                ((unsigned __int128)1 << 64))
            return false;
    }
    return true;
}

// NTT of the lifted limbs of ext (all positions if own_too).
static int ntt_ext(Context &c, uint64_t *ext, uint32_t count, int level, bool own_too,
                   cudaStream_t s) {
    const int M = level + c.K, beta = (level + c.alpha - 1) / c.alpha;
    LimbMap m{};
    uint32_t e = 0;
    for (int j = 0; j < beta; j++) {
        const int lo = j * c.alpha, hi = std::min((j + 1) * c.alpha, level);
        for (int i = 0; i < M; i++) {
            if (!own_too && i >= lo && i < hi) continue;
            if (e >= uint32_t(kMapMax)) return CATFHE_EINVAL;
            m.src_off[e] = m.dst_off[e] = uint16_t(j * M + i);
            m.prime[e] = uint8_t(ext_prime(c, level, i));
            e++;
        }
    }
    m.period = e;
    m.src_stride = m.dst_stride = uint32_t(beta * M);
    return ext_lazy(c, level) ? launch_ntt_fwd_lazy(c, ext, ext, m, e * count, s)
                              : launch_ntt_fwd(c, ext, ext, m, e * count, s);
}

static int inner_product(Context &c, const uint64_t *ext, const uint64_t *own, const uint64_t *key,
                         const uint64_t *add0, const uint64_t *add1, uint64_t *y, uint32_t count,
                         int level, cudaStream_t s) {
    const int M = level + c.K, beta = (level + c.alpha - 1) / c.alpha;
    const size_t n = c.n;
    IpArgs a{};
    a.ext = ext;
    a.own = own;
    a.key = key;
    a.add0 = add0;
    a.add1 = add1;
    a.y = y;
    a.ext_item = size_t(beta) * M * n;
    a.own_item = size_t(level) * n;
    a.add_item = size_t(level) * n;
    a.y_item = size_t(2) * M * n;
    a.M = M;
    a.level = level;
    a.beta = beta;
    a.L = c.L;
    a.K = c.K;
    a.alpha = c.alpha;
    a.status = c.d_status;
    for (int i = 0; i < M; i++) {
        const int gp = ext_prime(c, level, i);
        a.prime[i] = uint8_t(gp);
        a.key_limb[i] = uint16_t(gp);
        if (i < level) {
            const uint64_t q = c.mod(i), r = (uint64_t)(((unsigned __int128)1 << 64) % q);
            a.pfac[i] = h_mulmod(pmod(c, q), r, q);  // P in Montgomery form
        }
    }
    return launch_ip(c, a, count, s);
}

// ModDown of y ([count][2][M][N]; NTT form for CKKS/BGV, coefficient form
// for BFV) by D = P (fused: P q_{l-1}) into out ([count][2][lo][N]).
static int moddown(Context &c, uint64_t *y, uint64_t *lift, uint64_t *out, const uint64_t *add,
                   uint32_t count, int level, bool fused, cudaStream_t s,
                   const Gather *gth = nullptr) {
    const int M = level + c.K, lo = fused ? level - 1 : level;
    const size_t n = c.n;
    const bool ntt_form = c.scheme != CATFHE_BFV;
    // division basis positions in y: P, then q_{l-1} when fused
    std::vector<int> dpos;
    for (int k = 0; k < c.K; k++) dpos.push_back(level + k);
    if (fused) dpos.push_back(level - 1);
    const int Kd = int(dpos.size());
    if (ntt_form) {
        LimbMap m{};
        m.period = uint32_t(2 * Kd);
        m.src_stride = m.dst_stride = uint32_t(2 * M);
        for (int p = 0; p < 2; p++)
            for (int d = 0; d < Kd; d++) {
                m.src_off[p * Kd + d] = m.dst_off[p * Kd + d] = uint16_t(p * M + dpos[d]);
                m.prime[p * Kd + d] = uint8_t(ext_prime(c, level, dpos[d]));
            }
        TRY(launch_ntt_inv(c, y, y, m, m.period * count, s));
    }
    PlanSpec sp;
    sp.lazy = ntt_form;  // NTT schemes transform the lift before the combine
    for (int d = 0; d < Kd; d++) {
        sp.src_mod.push_back(c.mod(ext_prime(c, level, dpos[d])));
        sp.src_off.push_back(uint32_t(dpos[d]));
    }
    for (int i = 0; i < lo; i++) {
        sp.dst_mod.push_back(c.mod(i));
        sp.dst_off.push_back(uint32_t(i));
    }
    if (c.scheme == CATFHE_BGV) {
        for (int d = 0; d < Kd; d++) sp.pre.push_back(h_invmod(c.t % sp.src_mod[d], sp.src_mod[d]));
        for (int i = 0; i < lo; i++) sp.post.push_back(c.t % c.mod(i));
    }
    PlanList pl;
    TRY(make_list(c, {{"moddown/" + std::to_string(level) + (fused ? "/f" : ""), sp}}, pl));
    TRY(launch_conv(c, pl, y, size_t(M) * n, 0, lift, size_t(lo) * n, 0, 2 * count, s));
    // D^-1 mod q_i, D = P (fused: P q_{l-1})
    std::vector<uint64_t> dinv(lo), dinv_s(lo);
    for (int i = 0; i < lo; i++) {
        const uint64_t q = c.mod(i);
        uint64_t D = pmod(c, q);
        if (fused) D = h_mulmod(D, c.mod(level - 1) % q, q);
        dinv[i] = h_invmod(D, q);
        dinv_s[i] = h_shoup(dinv[i], q);
    }
    if (gth && gth->n && (!ntt_form || add || gth->n != count)) return CATFHE_EINVAL;
    if (ntt_form) {
        // NTT of the lift whose last pass writes (y - lift) D^-1 straight to out
        LimbMap m{};
        NttEpilogue e{};
        if (gth && gth->n) {
            e.gathered = 1;
            for (uint32_t i = 0; i < gth->n; i++) e.gout[i] = gth->out[i];
        }
        m.period = uint32_t(2 * lo);
        m.src_stride = m.dst_stride = uint32_t(2 * lo);
        e.y = y;
        e.add = add;
        e.out = out;
        e.status = c.d_status;
        e.y_stride = uint32_t(2 * M);
        e.add_stride = uint32_t(2 * lo);
        e.out_stride = uint32_t(2 * lo);
        for (int p = 0; p < 2; p++)
            for (int i = 0; i < lo; i++) {
                const int r = p * lo + i;
                m.src_off[r] = m.dst_off[r] = uint16_t(r);
                m.prime[r] = uint8_t(i);
                e.y_off[r] = uint16_t(p * M + i);
                e.add_off[r] = uint16_t(r);
                e.out_off[r] = uint16_t(r);
                e.dinv[r] = dinv[i];
                e.dinv_s[r] = dinv_s[i];
            }
        return launch_ntt_fwd_combine(c, lift, m, uint32_t(2 * lo) * count, e, s);
    }
    CombineArgs a{};
    a.y = y;
    a.lift = lift;
    a.add = add;
    a.out = out;
    a.y_item = size_t(2) * M * n;
    a.y_poly = size_t(M) * n;
    a.lift_item = size_t(2) * lo * n;
    a.lift_poly = size_t(lo) * n;
    a.add_item = size_t(2) * lo * n;
    a.add_poly = size_t(lo) * n;
    a.out_item = size_t(2) * lo * n;
    a.out_poly = size_t(lo) * n;
    a.lo = uint32_t(lo);
    for (int i = 0; i < lo; i++) {
        a.prime[i] = uint8_t(i);
        a.dinv[i] = dinv[i];
        a.dinv_s[i] = dinv_s[i];
    }
    return launch_combine(c, a, count, s);
}

// ----------------------------------------------------------------- op layouts

struct KsBufs {
    uint64_t *d0, *d1, *d2, *d2c, *ext, *y, *lift;
    // BFV
    uint64_t *xin, *tens, *dq, *add;
};

static void ks_layout(const Context &c, Bump &b, KsBufs &k, uint32_t count, int level,
                      bool fused) {
    const size_t n = c.n;
    const int M = level + c.K, beta = (level + c.alpha - 1) / c.alpha;
    const int lo = fused ? level - 1 : level;
    k.d0 = b.take<uint64_t>(size_t(count) * level * n);
    k.d1 = b.take<uint64_t>(size_t(count) * level * n);
    k.d2 = b.take<uint64_t>(size_t(count) * level * n);
    k.d2c = b.take<uint64_t>(size_t(count) * level * n);
    k.ext = b.take<uint64_t>(size_t(count) * beta * M * n);
    k.y = b.take<uint64_t>(size_t(count) * 2 * M * n);
    k.lift = b.take<uint64_t>(size_t(count) * 2 * lo * n);
    k.xin = k.tens = k.dq = k.add = nullptr;
    if (c.scheme == CATFHE_BFV) {
        const int kb = level + c.nb;
        k.xin = b.take<uint64_t>(size_t(count) * 4 * kb * n);
        k.tens = b.take<uint64_t>(size_t(count) * 3 * kb * n);
        k.dq = b.take<uint64_t>(size_t(count) * 3 * level * n);
        k.add = b.take<uint64_t>(size_t(count) * 2 * level * n);
    }
}

static size_t ks_bytes(const Context &c, uint32_t count, int level, bool fused) {
    Bump b{nullptr};
    KsBufs k{};
    ks_layout(c, b, k, count, level, fused);
    return (b.off + 255) & ~size_t(255);
}

// Key-switching operations on at least kSplitMin ciphertexts of N >= 2^14
// run as two halves on two streams forked from the caller's stream: one
// half's memory-bound kernels overlap the other's integer-bound ones
// (measured on the batch of 8 at N = 2^16, l = 24: 1596 -> 1526 us).  Their
// workspace holds both halves.
constexpr uint32_t kSplitMin = 4;
static bool split_ok(const Context &c, uint32_t count) { return count >= kSplitMin && c.log_n >= 14; }

static size_t ks_ws(const Context &c, uint32_t count, int level, bool fused) {
    const size_t whole = ks_bytes(c, count, level, fused);
    if (!split_ok(c, count)) return whole;
    const uint32_t c0 = (count + 1) / 2;
    return std::max(whole, ks_bytes(c, c0, level, fused) + ks_bytes(c, count - c0, level, fused));
}

size_t ws_bytes(const Context &c, int op, uint32_t level, uint32_t count) {
    Bump b{nullptr};
    const size_t n = c.n;
    switch (op) {
        case CATFHE_OP_MUL_RELIN:
        case CATFHE_OP_ROTATE:
            b.off = ks_ws(c, count, int(level), false);
            break;
        case CATFHE_OP_MUL_RELIN_RESCALE:
            b.off = ks_ws(c, count, int(level), true);
            break;
        case CATFHE_OP_ROTATE_HOISTED: {
            // two per-rotation buffer sets (rotations alternate over two
            // streams), then the shared lifted digits
            b.off = 2 * ks_bytes(c, count, int(level), false);
            const int M = int(level) + c.K, beta = (int(level) + c.alpha - 1) / c.alpha;
            b.take<uint64_t>(size_t(count) * beta * M * n);
            break;
        }
        case CATFHE_OP_RESCALE:
            b.take<uint64_t>(size_t(count) * 2 * n);
            b.take<uint64_t>(size_t(count) * 2 * (level ? level - 1 : 0) * n);
            break;
        case CATFHE_OP_DECRYPT:
            b.take<uint64_t>(size_t(level) * n);
            b.take<uint64_t>(size_t(level) * n);
            b.take<int64_t>(n);
            break;
        case CATFHE_OP_EXPORT:
            b.take<uint64_t>(size_t(count) * 2 * level * n);
            break;
        case CATFHE_OP_ENCODE:
            b.take<double2>(n / 2);
            b.take<double2>(2 * n);
            b.take<int64_t>(n);
            break;
        case CATFHE_OP_DECODE:
            b.take<uint64_t>(size_t(2) * level * n);
            b.take<int64_t>(n);
            b.take<double2>(2 * n);
            b.take<double2>(n / 2);
            break;
        default:
            return 0;
    }
    return b.off + 256;
}

// ----------------------------------------------------------------- hot path

static int key_for(const Keys &k, uint64_t id, const uint64_t **key) {
    auto it = k.ksk.find(id);
    if (it == k.ksk.end()) return CATFHE_ENOKEY;
    *key = it->second;
    return CATFHE_OK;
}

// CKKS / BGV: tensor in NTT form, INTT d2, ModUp, NTT, inner product with
// P*(d0, d1) folded in, ModDown (fused: by P q_{l-1}).
static int mul_relin_ntt(Context &c, const Keys &keys, const uint64_t *a, const uint64_t *b,
                         uint64_t *out, uint32_t count, int level, bool fused, KsBufs &k,
                         cudaStream_t s, const Gather *gth) {
    const uint64_t *rlk;
    TRY(key_for(keys, 0, &rlk));
    const size_t n = c.n;
    TensorArgs t{};
    t.a = a;
    t.b = b;
    if (gth && gth->n) {
        t.gathered = 1;
        for (uint32_t i = 0; i < gth->n; i++) {
            t.ga[i] = gth->a[i];
            t.gb[i] = gth->b[i];
        }
    }
    t.d0 = k.d0;
    t.d1 = k.d1;
    t.d2 = k.d2;
    t.in_item = size_t(2) * level * n;
    t.out_item = size_t(level) * n;
    t.limbs = uint32_t(level);
    for (int i = 0; i < level; i++) t.prime[i] = uint8_t(i);
    TRY(launch_tensor(c, t, count, s));
    LimbMap m = map_identity(uint32_t(level));
    TRY(launch_ntt_inv(c, k.d2, k.d2c, m, uint32_t(level) * count, s));
    TRY(modup(c, k.d2c, k.ext, count, level, false, s));
    TRY(ntt_ext(c, k.ext, count, level, false, s));
    TRY(inner_product(c, k.ext, k.d2, rlk, k.d0, k.d1, k.y, count, level, s));
    return moddown(c, k.y, k.lift, out, nullptr, count, level, fused, s, gth);
}

// BFV: lift to Q u B, NTT, tensor, INTT, exact round(t x / Q) back to Q,
// then relinearise d2 in coefficient form.
static int mul_relin_bfv(Context &c, const Keys &keys, const uint64_t *a, const uint64_t *b,
                         uint64_t *out, uint32_t count, int level, KsBufs &k, cudaStream_t s) {
    const uint64_t *rlk;
    TRY(key_for(keys, 0, &rlk));
    const size_t n = c.n;
    const int kb = level + c.nb;
    // 1. centred lift of the 4 input polys from Q_l to Q_l u B
    {
        PlanSpec sp;
        sp.lazy = true;  // NTT'd before the tensor
        for (int i = 0; i < level; i++) {
            sp.src_mod.push_back(c.mod(i));
            sp.src_off.push_back(uint32_t(i));
        }
        for (int i = 0; i < kb; i++) {
            sp.dst_mod.push_back(c.mod(i < level ? i : c.pb(i - level)));
            sp.dst_off.push_back(uint32_t(i));
        }
        PlanList pl;
        TRY(make_list(c, {{"bfv_lift/" + std::to_string(level), sp}}, pl));
        // items: (ct, poly) for a then for b
        TRY(launch_conv(c, pl, a, size_t(level) * n, 0, k.xin, size_t(kb) * n, 0, 2 * count, s));
        TRY(launch_conv(c, pl, b, size_t(level) * n, 0, k.xin + size_t(count) * 2 * kb * n,
                        size_t(kb) * n, 0, 2 * count, s));
    }
    LimbMap mq{};
    mq.period = uint32_t(kb);
    mq.src_stride = mq.dst_stride = uint32_t(kb);
    for (int i = 0; i < kb; i++) {
        mq.src_off[i] = mq.dst_off[i] = uint16_t(i);
        mq.prime[i] = uint8_t(i < level ? i : c.pb(i - level));
    }
    TRY(launch_ntt_fwd(c, k.xin, k.xin, mq, uint32_t(kb) * 4 * count, s));
    // 2. tensor over Q u B
    {
        TensorArgs t{};
        t.a = k.xin;
        t.b = k.xin + size_t(count) * 2 * kb * n;
        t.in_item = size_t(2) * kb * n;
        t.d0 = k.tens;
        t.d1 = k.tens + size_t(kb) * n;
        t.d2 = k.tens + size_t(2) * kb * n;
        t.out_item = size_t(3) * kb * n;
        t.limbs = uint32_t(kb);
        for (int i = 0; i < kb; i++) t.prime[i] = mq.prime[i];
        TRY(launch_tensor(c, t, count, s));
    }
    TRY(launch_ntt_inv(c, k.tens, k.tens, mq, uint32_t(kb) * 3 * count, s));
    // 3. exact round(t x / Q) back to Q_l
    {
        PlanSpec A, B;
        std::vector<uint64_t> tq;
        for (int i = 0; i < level; i++) {
            A.src_mod.push_back(c.mod(i));
            A.src_off.push_back(uint32_t(i));
            A.pre.push_back(c.t % c.mod(i));
        }
        for (int j = 0; j < c.nb; j++) {
            const uint64_t bj = c.mod(c.pb(j));
            const uint64_t qinv = h_invmod(prod_mod(c, 0, level, bj), bj);
            A.dst_mod.push_back(bj);
            A.dst_off.push_back(uint32_t(level + j));
            A.post.push_back(qinv);
            const uint64_t tqi = h_mulmod(c.t % bj, qinv, bj);
            tq.push_back(tqi);
            tq.push_back(h_shoup(tqi, bj));
            B.src_mod.push_back(bj);
            B.src_off.push_back(0);
        }
        for (int i = 0; i < level; i++) {
            B.dst_mod.push_back(c.mod(i));
            B.dst_off.push_back(uint32_t(i));
        }
        // the fused kernel needs both conversions in the Montgomery layout
        if (!plan_fits_mont(A) || !plan_fits_mont(B)) return CATFHE_EINVAL;
        const PlanRef pa = get_plan_extra(c, "bfv_sr_a/" + std::to_string(level), A, tq);
        const PlanRef pb = get_plan(c, "bfv_sr_b/" + std::to_string(level), B);
        if (!pa.p || !pb.p) return CATFHE_ENOMEM;
        TRY(launch_bfv_scale_round(c, pa.p, pa.words, pb.p, pb.words, k.tens, size_t(kb) * n, k.dq,
                                   size_t(level) * n, 3 * count, s));
    }
    // 4. relinearise d2' (coefficient form) and add (d0', d1')
    const uint64_t *d2 = k.dq + size_t(2) * level * n;
    // ModUp reads the digit limbs of d2' per ct: item stride 3*level*N
    {
        const int M = level + c.K, beta = (level + c.alpha - 1) / c.alpha;
        std::vector<std::pair<std::string, PlanSpec>> specs;
        for (int j = 0; j < beta; j++) {
            const int lo = j * c.alpha, hi = std::min((j + 1) * c.alpha, level);
            PlanSpec sp;
            sp.lazy = true;
            for (int i = lo; i < hi; i++) {
                sp.src_mod.push_back(c.mod(i));
                sp.src_off.push_back(uint32_t(i));
            }
            for (int i = 0; i < M; i++) {
                sp.dst_mod.push_back(c.mod(ext_prime(c, level, i)));
                sp.dst_off.push_back(uint32_t(i));
            }
            specs.emplace_back("modup/" + std::to_string(level) + "/" + std::to_string(j) + "/own",
                               sp);
        }
        PlanList pl;
        TRY(make_list(c, specs, pl));
        TRY(launch_conv(c, pl, d2, size_t(3) * level * n, 0, k.ext, size_t(beta) * M * n,
                        size_t(M) * n, count, s));
    }
    TRY(ntt_ext(c, k.ext, count, level, true, s));
    TRY(inner_product(c, k.ext, nullptr, rlk, nullptr, nullptr, k.y, count, level, s));
    {
        const int M = level + c.K;
        LimbMap my = map_identity(uint32_t(M));
        for (int i = 0; i < M; i++) my.prime[i] = uint8_t(ext_prime(c, level, i));
        TRY(launch_ntt_inv(c, k.y, k.y, my, uint32_t(2 * M) * count, s));
    }
    // (d0', d1') of [count][3][level] packed as [count][2][level] for the combine
    {
        LimbMap cp{};
        cp.period = uint32_t(2 * level);
        cp.src_stride = uint32_t(3 * level);
        cp.dst_stride = uint32_t(2 * level);
        for (int i = 0; i < 2 * level; i++) {
            cp.src_off[i] = cp.dst_off[i] = uint16_t(i);
            cp.prime[i] = uint8_t(i % level);
        }
        TRY(launch_copy_limbs(c, k.dq, k.add, cp, uint32_t(2 * level) * count, s));
    }
    return moddown(c, k.y, k.lift, out, k.add, count, level, false, s);
}

// Two streams (and fork / join events) per device for split operations;
// the mutex is held while a split operation is enqueued.
struct SplitPool {
    bool ready = false;
    cudaStream_t st[2];
    cudaEvent_t fork, join[2];
};
static std::mutex g_split_mu;
static SplitPool g_split[64];

static int split_pool(SplitPool **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return CATFHE_ECUDA;
    SplitPool &p = g_split[dev];
    if (!p.ready) {
        for (int i = 0; i < 2; i++) {
            if (cudaStreamCreateWithFlags(&p.st[i], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&p.join[i], cudaEventDisableTiming) != cudaSuccess)
                return CATFHE_ECUDA;
        }
        if (cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming) != cudaSuccess)
            return CATFHE_ECUDA;
        p.ready = true;
    }
    *out = &p;
    return CATFHE_OK;
}

// Runs f(first, cnt, ws_base, stream) for the two halves of `count` items on
// the split streams, ordered after everything enqueued on s so far and before
// everything enqueued on s afterwards.
template <class F>
static int run_halves(const Context &c, uint32_t count, int level, bool fused, char *base,
                      cudaStream_t s, F f) {
    std::lock_guard<std::mutex> lock(g_split_mu);
    SplitPool *sp;
    TRY(split_pool(&sp));
    const uint32_t c0 = (count + 1) / 2;
    const uint32_t first[2] = {0, c0}, cnt[2] = {c0, count - c0};
    char *wb[2] = {base, base + ks_bytes(c, c0, level, fused)};
    if (cudaEventRecord(sp->fork, s) != cudaSuccess) return CATFHE_ECUDA;
    for (int h = 0; h < 2; h++) {
        if (cudaStreamWaitEvent(sp->st[h], sp->fork, 0) != cudaSuccess) return CATFHE_ECUDA;
        TRY(f(first[h], cnt[h], wb[h], sp->st[h]));
        if (cudaEventRecord(sp->join[h], sp->st[h]) != cudaSuccess) return CATFHE_ECUDA;
        if (cudaStreamWaitEvent(s, sp->join[h], 0) != cudaSuccess) return CATFHE_ECUDA;
    }
    return CATFHE_OK;
}

int op_mul_relin(Context &c, const Keys &keys, const uint64_t *a, const uint64_t *b,
                 uint64_t *out, uint32_t level, uint32_t count, bool fused, void *ws,
                 size_t ws_bytes_in, cudaStream_t s, const Gather *gth, bool split) {
    if (gth && gth->n && (c.scheme == CATFHE_BFV || gth->n != count || count > kGatherMax))
        return CATFHE_EINVAL;
    if (level < 1 || int(level) > c.L) return CATFHE_ELEVEL;
    if (fused && (c.scheme != CATFHE_CKKS)) return CATFHE_ESCHEME;
    if (fused && level < 2) return CATFHE_ELEVEL;
    if (count == 0) return CATFHE_OK;
    const size_t need = ws_bytes(c, fused ? CATFHE_OP_MUL_RELIN_RESCALE : CATFHE_OP_MUL_RELIN,
                                 level, count);
    char *base;
    TRY(get_ws(c, ws, ws_bytes_in, need, &base));
    const int lvl = int(level);
    auto run = [&](uint32_t first, uint32_t cnt, char *wbase, cudaStream_t st) -> int {
        Bump bump{wbase};
        KsBufs k{};
        ks_layout(c, bump, k, cnt, lvl, fused);
        const size_t n = c.n, lo = size_t(fused ? lvl - 1 : lvl);
        const uint64_t *ah = a + size_t(first) * 2 * lvl * n, *bh = b + size_t(first) * 2 * lvl * n;
        uint64_t *oh = out + size_t(first) * 2 * lo * n;
        if (c.scheme == CATFHE_BFV) return mul_relin_bfv(c, keys, ah, bh, oh, cnt, lvl, k, st);
        return mul_relin_ntt(c, keys, ah, bh, oh, cnt, lvl, fused, k, st, gth);
    };
    if (split && !(gth && gth->n) && split_ok(c, count))
        return run_halves(c, count, lvl, fused, base, s, run);
    return run(0, count, base, s);
}

// HRotate of count ciphertexts at lvl with the Galois key gk, workspace k.
static int rotate_run(Context &c, const uint64_t *gk, const uint64_t *a, uint64_t g, uint64_t *out,
                      int lvl, uint32_t count, KsBufs &k, cudaStream_t s, const Gather *gth) {
    const size_t n = c.n;
    if (c.scheme != CATFHE_BFV) {
        // sigma_g on both components in NTT form: d0 <- sigma(c0), d2 <- sigma(c1)
        for (uint32_t ct = 0; ct < count; ct++) {
            const uint64_t *src = (gth && gth->n) ? gth->a[ct] : a + size_t(ct) * 2 * lvl * n;
            TRY(launch_automorph_ntt(c, src, k.d0 + size_t(ct) * lvl * n, uint32_t(lvl), g, s));
            TRY(launch_automorph_ntt(c, src + size_t(lvl) * n, k.d2 + size_t(ct) * lvl * n,
                                     uint32_t(lvl), g, s));
        }
        LimbMap m = map_identity(uint32_t(lvl));
        TRY(launch_ntt_inv(c, k.d2, k.d2c, m, uint32_t(lvl) * count, s));
        TRY(modup(c, k.d2c, k.ext, count, lvl, false, s));
        TRY(ntt_ext(c, k.ext, count, lvl, false, s));
        TRY(inner_product(c, k.ext, k.d2, gk, k.d0, nullptr, k.y, count, lvl, s));
        return moddown(c, k.y, k.lift, out, nullptr, count, lvl, false, s, gth);
    }
    // BFV (coefficient form): (sigma(c0), 0) becomes the added pair of the
    // ModDown combine, sigma(c1) is key switched.
    uint64_t *addbuf = k.add;  // [count][2][level]
    {
        LimbMap m{};
        m.period = uint32_t(lvl);
        m.src_stride = uint32_t(2 * lvl);
        m.dst_stride = uint32_t(2 * lvl);
        for (int i = 0; i < lvl; i++) {
            m.src_off[i] = m.dst_off[i] = uint16_t(i);
            m.prime[i] = uint8_t(i);
        }
        TRY(launch_automorph_coeff(c, a, addbuf, m, uint32_t(lvl) * count, g, s));
        for (uint32_t ct = 0; ct < count; ct++)
            if (cudaMemsetAsync(addbuf + (size_t(ct) * 2 + 1) * lvl * n, 0, size_t(lvl) * n * 8, s) !=
                cudaSuccess)
                return CATFHE_ECUDA;
        LimbMap m1 = m;
        m1.dst_stride = uint32_t(lvl);
        for (int i = 0; i < lvl; i++) m1.src_off[i] = uint16_t(lvl + i);
        TRY(launch_automorph_coeff(c, a, k.d2c, m1, uint32_t(lvl) * count, g, s));
    }
    TRY(modup(c, k.d2c, k.ext, count, lvl, true, s));
    TRY(ntt_ext(c, k.ext, count, lvl, true, s));
    TRY(inner_product(c, k.ext, nullptr, gk, nullptr, nullptr, k.y, count, lvl, s));
    {
        const int M = lvl + c.K;
        LimbMap my = map_identity(uint32_t(M));
        for (int i = 0; i < M; i++) my.prime[i] = uint8_t(ext_prime(c, lvl, i));
        TRY(launch_ntt_inv(c, k.y, k.y, my, uint32_t(2 * M) * count, s));
    }
    return moddown(c, k.y, k.lift, out, addbuf, count, lvl, false, s);
}

int op_rotate(Context &c, const Keys &keys, const uint64_t *a, uint64_t g, uint64_t *out,
              uint32_t level, uint32_t count, void *ws, size_t ws_bytes_in, cudaStream_t s,
              const Gather *gth, bool split) {
    if (level < 1 || int(level) > c.L) return CATFHE_ELEVEL;
    if (gth && gth->n && (c.scheme == CATFHE_BFV || gth->n != count || count > kGatherMax))
        return CATFHE_EINVAL;
    g %= 2 * c.n;
    if (!(g & 1)) return CATFHE_EINVAL;
    const uint64_t *gk;
    TRY(key_for(keys, g, &gk));
    if (count == 0) return CATFHE_OK;
    char *base;
    TRY(get_ws(c, ws, ws_bytes_in, ws_bytes(c, CATFHE_OP_ROTATE, level, count), &base));
    const size_t n = c.n;
    const int lvl = int(level);
    auto run = [&](uint32_t first, uint32_t cnt, char *wbase, cudaStream_t st) -> int {
        Bump bump{wbase};
        KsBufs k{};
        ks_layout(c, bump, k, cnt, lvl, false);
        const uint64_t *ah = a + size_t(first) * 2 * lvl * n;
        uint64_t *oh = out + size_t(first) * 2 * lvl * n;
        return rotate_run(c, gk, ah, g, oh, lvl, cnt, k, st, gth);
    };
    if (split && !(gth && gth->n) && split_ok(c, count))
        return run_halves(c, count, lvl, false, base, s, run);
    return run(0, count, base, s);
}


// Hoisted rotations: one INTT + ModUp + NTT of a1, then per Galois element a
// permutation of a0, a1 and the lifted digits, the inner product and ModDown.
int op_rotate_hoisted(Context &c, const Keys &keys, const uint64_t *a, const uint64_t *gs,
                      uint32_t n_rot, uint64_t *out, uint32_t level, uint32_t count, void *ws,
                      size_t ws_bytes_in, cudaStream_t s) {
    if (c.scheme == CATFHE_BFV) return CATFHE_ESCHEME;
    if (level < 1 || int(level) > c.L) return CATFHE_ELEVEL;
    if (n_rot > 0 && !gs) return CATFHE_EINVAL;
    std::vector<const uint64_t *> gk(n_rot);
    std::vector<uint64_t> gv(n_rot);
    for (uint32_t r = 0; r < n_rot; r++) {
        gv[r] = gs[r] % (2 * c.n);
        if (!(gv[r] & 1)) return CATFHE_EINVAL;
        TRY(key_for(keys, gv[r], &gk[r]));
    }
    if (count == 0 || n_rot == 0) return CATFHE_OK;
    char *base;
    TRY(get_ws(c, ws, ws_bytes_in, ws_bytes(c, CATFHE_OP_ROTATE_HOISTED, level, count), &base));
    Bump bump{base};
    KsBufs ks[2];
    ks_layout(c, bump, ks[0], count, int(level), false);
    bump.off = ks_bytes(c, count, int(level), false);
    ks_layout(c, bump, ks[1], count, int(level), false);
    bump.off = 2 * ks_bytes(c, count, int(level), false);
    KsBufs &k = ks[0];
    const size_t n = c.n;
    const int lvl = int(level), M = lvl + c.K, beta = (lvl + c.alpha - 1) / c.alpha;
    uint64_t *ext0 = bump.take<uint64_t>(size_t(count) * beta * M * n);
    // a1 (NTT form) -> coefficient form -> lifted digits in NTT form, once
    LimbMap m1{};
    m1.period = uint32_t(lvl);
    m1.src_stride = uint32_t(2 * lvl);
    m1.dst_stride = uint32_t(lvl);
    for (int i = 0; i < lvl; i++) {
        m1.src_off[i] = uint16_t(lvl + i);
        m1.dst_off[i] = uint16_t(i);
        m1.prime[i] = uint8_t(i);
    }
    TRY(launch_ntt_inv(c, a, k.d2c, m1, uint32_t(lvl) * count, s));
    TRY(modup(c, k.d2c, ext0, count, lvl, false, s));
    TRY(ntt_ext(c, ext0, count, lvl, false, s));
    // the lifted positions of ext (as ntt_ext selects them)
    LimbMap me{};
    uint32_t e = 0;
    for (int j = 0; j < beta; j++) {
        const int lo = j * c.alpha, hi = std::min((j + 1) * c.alpha, lvl);
        for (int i = 0; i < M; i++) {
            if (i >= lo && i < hi) continue;
            if (e >= uint32_t(kMapMax)) return CATFHE_EINVAL;
            me.src_off[e] = me.dst_off[e] = uint16_t(j * M + i);
            me.prime[e] = uint8_t(ext_prime(c, lvl, i));
            e++;
        }
    }
    me.period = e;
    me.src_stride = me.dst_stride = uint32_t(beta * M);
    LimbMap m0 = m1;  // a0 -> d0
    for (int i = 0; i < lvl; i++) m0.src_off[i] = uint16_t(i);
    auto one = [&](uint32_t r, KsBufs &kb, cudaStream_t st) -> int {
        TRY(launch_automorph_ntt_map(c, a, kb.d0, m0, uint32_t(lvl) * count, gv[r], st));
        TRY(launch_automorph_ntt_map(c, a, kb.d2, m1, uint32_t(lvl) * count, gv[r], st));
        TRY(launch_automorph_ntt_map(c, ext0, kb.ext, me, e * count, gv[r], st));
        TRY(inner_product(c, kb.ext, kb.d2, gk[r], kb.d0, nullptr, kb.y, count, lvl, st));
        return moddown(c, kb.y, kb.lift, out + size_t(r) * count * 2 * lvl * n, nullptr, count,
                       lvl, false, st);
    };
    if (n_rot < 2 || c.log_n < 14) {
        for (uint32_t r = 0; r < n_rot; r++) TRY(one(r, k, s));
        return CATFHE_OK;
    }
    // rotations alternate over the two split streams, each with its own
    // buffer set (in order on its stream), after the shared ModUp on s
    std::lock_guard<std::mutex> lock(g_split_mu);
    SplitPool *sp;
    TRY(split_pool(&sp));
    if (cudaEventRecord(sp->fork, s) != cudaSuccess) return CATFHE_ECUDA;
    for (int h = 0; h < 2; h++)
        if (cudaStreamWaitEvent(sp->st[h], sp->fork, 0) != cudaSuccess) return CATFHE_ECUDA;
    for (uint32_t r = 0; r < n_rot; r++) TRY(one(r, ks[r & 1], sp->st[r & 1]));
    for (int h = 0; h < 2; h++) {
        if (cudaEventRecord(sp->join[h], sp->st[h]) != cudaSuccess) return CATFHE_ECUDA;
        if (cudaStreamWaitEvent(s, sp->join[h], 0) != cudaSuccess) return CATFHE_ECUDA;
    }
    return CATFHE_OK;
}

// CKKS rescale / BGV modulus switch: divide by q_{l-1}.
int op_rescale(Context &c, const uint64_t *a, uint64_t *out, uint32_t level, uint32_t count,
               void *ws, size_t ws_bytes_in, cudaStream_t s) {
    if (c.scheme == CATFHE_BFV) return CATFHE_ESCHEME;
    if (level < 2 || int(level) > c.L) return CATFHE_ELEVEL;
    if (count == 0) return CATFHE_OK;
    char *base;
    TRY(get_ws(c, ws, ws_bytes_in, ws_bytes(c, CATFHE_OP_RESCALE, level, count), &base));
    Bump bump{base};
    const size_t n = c.n;
    const int lvl = int(level), lo = lvl - 1;
    uint64_t *last = bump.take<uint64_t>(size_t(count) * 2 * n);
    uint64_t *lift = bump.take<uint64_t>(size_t(count) * 2 * lo * n);
    // INTT of the last limb of both polys: [count][2][level] -> [count][2][1]
    LimbMap m{};
    m.period = 2;
    m.src_stride = uint32_t(2 * lvl);
    m.dst_stride = 2;
    for (int p = 0; p < 2; p++) {
        m.src_off[p] = uint16_t(p * lvl + lvl - 1);
        m.dst_off[p] = uint16_t(p);
        m.prime[p] = uint8_t(lvl - 1);
    }
    TRY(launch_ntt_inv(c, a, last, m, 2 * count, s));
    PlanSpec sp;
    sp.lazy = true;  // NTT'd before the combine
    sp.src_mod.push_back(c.mod(lvl - 1));
    sp.src_off.push_back(0);
    for (int i = 0; i < lo; i++) {
        sp.dst_mod.push_back(c.mod(i));
        sp.dst_off.push_back(uint32_t(i));
    }
    if (c.scheme == CATFHE_BGV) {
        sp.pre.push_back(h_invmod(c.t % c.mod(lvl - 1), c.mod(lvl - 1)));
        for (int i = 0; i < lo; i++) sp.post.push_back(c.t % c.mod(i));
    }
    PlanList pl;
    TRY(make_list(c, {{"rescale/" + std::to_string(lvl), sp}}, pl));
    TRY(launch_conv(c, pl, last, n, 0, lift, size_t(lo) * n, 0, 2 * count, s));
    // NTT of the lift, its last pass writing (a - lift) q_{l-1}^-1 to out
    LimbMap m2{};
    NttEpilogue e{};
    m2.period = uint32_t(2 * lo);
    m2.src_stride = m2.dst_stride = uint32_t(2 * lo);
    e.y = a;
    e.out = out;
    e.status = c.d_status;
    e.y_stride = uint32_t(2 * lvl);
    e.out_stride = uint32_t(2 * lo);
    for (int p = 0; p < 2; p++)
        for (int i = 0; i < lo; i++) {
            const int r = p * lo + i;
            m2.src_off[r] = m2.dst_off[r] = uint16_t(r);
            m2.prime[r] = uint8_t(i);
            e.y_off[r] = uint16_t(p * lvl + i);
            e.out_off[r] = uint16_t(r);
            e.dinv[r] = h_invmod(c.mod(lvl - 1) % c.mod(i), c.mod(i));
            e.dinv_s[r] = h_shoup(e.dinv[r], c.mod(i));
        }
    return launch_ntt_fwd_combine(c, lift, m2, uint32_t(2 * lo) * count, e, s);
}

int op_add(Context &c, const uint64_t *a, const uint64_t *b, uint64_t *out, uint32_t level,
           uint32_t count, cudaStream_t s) {
    if (level < 1 || int(level) > c.L) return CATFHE_ELEVEL;
    if (count == 0) return CATFHE_OK;
    LimbMap m{};
    m.period = 2 * level;
    m.src_stride = m.dst_stride = 2 * level;
    for (uint32_t i = 0; i < 2 * level; i++) {
        m.src_off[i] = m.dst_off[i] = uint16_t(i);
        m.prime[i] = uint8_t(i % level);
    }
    return launch_add(c, a, b, out, m, 2 * level * count, s);
}

static LimbMap map_ct(uint32_t level) {
    LimbMap m{};
    m.period = 2 * level;
    m.src_stride = m.dst_stride = 2 * level;
    for (uint32_t i = 0; i < 2 * level; i++) {
        m.src_off[i] = m.dst_off[i] = uint16_t(i);
        m.prime[i] = uint8_t(i % level);
    }
    return m;
}

int op_sub(Context &c, const uint64_t *a, const uint64_t *b, uint64_t *out, uint32_t level,
           uint32_t count, cudaStream_t s) {
    if (level < 1 || int(level) > c.L) return CATFHE_ELEVEL;
    if (count == 0) return CATFHE_OK;
    return launch_sub(c, a, b, out, map_ct(level), 2 * level * count, s);
}

static uint64_t reduce_signed(int64_t v, uint64_t q) {
    const uint64_t mag = v < 0 ? uint64_t(0) - uint64_t(v) : uint64_t(v);
    const uint64_t r = mag % q;
    return (v < 0 && r) ? q - r : r;
}

// Both polynomials times the integer k (any scheme; no rescale).
int op_mul_int(Context &c, const uint64_t *a, int64_t k, uint64_t *out, uint32_t level,
               uint32_t count, cudaStream_t s) {
    if (level < 1 || int(level) > c.L) return CATFHE_ELEVEL;
    if (count == 0) return CATFHE_OK;
    const LimbMap m = map_ct(level);
    std::vector<uint64_t> kv(2 * level), ks(2 * level);
    std::vector<uint8_t> add(2 * level, 0);
    for (uint32_t i = 0; i < 2 * level; i++) {
        const uint64_t q = c.mod(int(i % level));
        kv[i] = reduce_signed(k, q);
        ks[i] = h_shoup(kv[i], q);
    }
    return launch_const_op(c, a, out, m, 2 * level * count, kv.data(), ks.data(), add.data(), s);
}

// Adds the plaintext constant k to every slot: c0 += k (the constant
// polynomial k, which is k at every evaluation point in NTT form) for CKKS
// and BGV; for BFV (coefficient form) c0 += Delta k at coefficient 0 is not
// an element-wise map, so BFV is not supported here.
int op_add_const(Context &c, const uint64_t *a, int64_t k, uint64_t *out, uint32_t level,
                 uint32_t count, cudaStream_t s) {
    if (c.scheme == CATFHE_BFV) return CATFHE_ESCHEME;
    if (level < 1 || int(level) > c.L) return CATFHE_ELEVEL;
    if (count == 0) return CATFHE_OK;
    const LimbMap m = map_ct(level);
    std::vector<uint64_t> kv(2 * level, 1), ks(2 * level);
    std::vector<uint8_t> add(2 * level, 0);
    for (uint32_t i = 0; i < 2 * level; i++) {
        const uint64_t q = c.mod(int(i % level));
        if (i < level) {
            kv[i] = reduce_signed(k, q);
            add[i] = 1;
        }
        ks[i] = h_shoup(kv[i], q);
    }
    return launch_const_op(c, a, out, m, 2 * level * count, kv.data(), ks.data(), add.data(), s);
}

// Plaintext upload: the signed coefficients are staged in the last limb of
// pt, converted to residues for the other limbs, then in place for the last
// (each thread reads its own coefficient before writing it), then NTT.
int op_plain_import(Context &c, const int64_t *coeffs, uint32_t level, uint64_t *pt,
                    cudaStream_t s) {
    if (level < 1 || int(level) > c.L) return CATFHE_ELEVEL;
    const size_t n = c.n;
    int64_t *stage = reinterpret_cast<int64_t *>(pt + size_t(level - 1) * n);
    if (cudaMemcpyAsync(stage, coeffs, n * 8, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return CATFHE_ECUDA;
    if (level > 1) {
        LimbMap m = map_identity(level - 1);
        TRY(launch_small_to_rns(c, stage, pt, m, level - 1, nullptr, nullptr, 0, s));
    }
    LimbMap ml{};
    ml.period = 1;
    ml.src_stride = ml.dst_stride = 1;
    ml.src_off[0] = ml.dst_off[0] = uint16_t(level - 1);
    ml.prime[0] = uint8_t(level - 1);
    TRY(launch_small_to_rns(c, stage, pt, ml, 1, nullptr, nullptr, 0, s));
    LimbMap m = map_identity(level);
    TRY(launch_ntt_fwd(c, pt, pt, m, level, s));
    return cudaStreamSynchronize(s) == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA;
}

// CKKS / BGV rest in NTT form: one limb-wise product.  BFV rests in
// coefficient form: the negacyclic product is NTT, limb-wise product, INTT,
// all in out (each transform is safe in place).
int op_mul_plain(Context &c, const uint64_t *a, const uint64_t *pt, uint64_t *out, uint32_t level,
                 uint32_t count, cudaStream_t s) {
    if (level < 1 || int(level) > c.L) return CATFHE_ELEVEL;
    if (count == 0) return CATFHE_OK;
    if (c.scheme != CATFHE_BFV) return launch_mul_plain(c, a, pt, out, level, 2 * level * count, s);
    const LimbMap m = map_identity(level);
    TRY(launch_ntt_fwd(c, a, out, m, 2 * level * count, s));
    TRY(launch_mul_plain(c, out, pt, out, level, 2 * level * count, s));
    return launch_ntt_inv(c, out, out, m, 2 * level * count, s);
}

// Keeps the first new_level limbs of each polynomial (dropping primes keeps
// the message and, in CKKS, the scale).
int op_drop_level(Context &c, const uint64_t *a, uint32_t level, uint32_t new_level,
                  uint64_t *out, uint32_t count, cudaStream_t s) {
    if (level < 1 || int(level) > c.L || new_level < 1 || new_level > level) return CATFHE_ELEVEL;
    if (count == 0) return CATFHE_OK;
    LimbMap m{};
    m.period = 2 * new_level;
    m.src_stride = 2 * level;
    m.dst_stride = 2 * new_level;
    for (uint32_t p = 0; p < 2; p++)
        for (uint32_t i = 0; i < new_level; i++) {
            m.src_off[p * new_level + i] = uint16_t(p * level + i);
            m.dst_off[p * new_level + i] = uint16_t(p * new_level + i);
            m.prime[p * new_level + i] = uint8_t(i);
        }
    return launch_copy_limbs(c, a, out, m, 2 * new_level * count, s);
}

int op_ntt(Context &c, uint64_t *limbs, uint32_t level, uint32_t count, int inverse,
           cudaStream_t s) {
    if (level < 1 || int(level) > c.L) return CATFHE_ELEVEL;
    LimbMap m = map_identity(level);
    return inverse ? launch_ntt_inv(c, limbs, limbs, m, level * count, s)
                   : launch_ntt_fwd(c, limbs, limbs, m, level * count, s);
}

// ----------------------------------------------------------------- keys

static SampleArgs sample_args(const Context &c, const uint8_t seed[32], uint32_t tag, uint32_t i0,
                              uint32_t i1, uint32_t kind) {
    SampleArgs a{};
    for (int i = 0; i < 8; i++)
        a.key[i] = uint32_t(seed[4 * i]) | (uint32_t(seed[4 * i + 1]) << 8) |
                   (uint32_t(seed[4 * i + 2]) << 16) | (uint32_t(seed[4 * i + 3]) << 24);
    a.tag = tag;
    a.i0 = i0;
    a.i1 = i1;
    a.kind = kind;
    memcpy(a.cdt, c.cdt, sizeof(a.cdt));
    return a;
}

enum { TAG_SK = 1, TAG_PK_A = 2, TAG_PK_E = 3, TAG_KSK_A = 4, TAG_KSK_E = 5, TAG_ENC_V = 6,
       TAG_ENC_E0 = 7, TAG_ENC_E1 = 8, TAG_CT_UNIFORM = 9 };

// Device array of t mod prime (Shoup pairs) for BGV error scaling.
struct DevConst {
    uint64_t *v = nullptr, *s = nullptr;
    ~DevConst() {
        cudaFree(v);
        cudaFree(s);
    }
    int set(const std::vector<uint64_t> &vals, const std::vector<uint64_t> &mods) {
        std::vector<uint64_t> sh(vals.size());
        for (size_t i = 0; i < vals.size(); i++) sh[i] = h_shoup(vals[i], mods[i]);
        if (cudaMalloc(&v, vals.size() * 8) != cudaSuccess) return CATFHE_ENOMEM;
        if (cudaMalloc(&s, vals.size() * 8) != cudaSuccess) return CATFHE_ENOMEM;
        if (cudaMemcpy(v, vals.data(), vals.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess)
            return CATFHE_ECUDA;
        if (cudaMemcpy(s, sh.data(), vals.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess)
            return CATFHE_ECUDA;
        return CATFHE_OK;
    }
};

static int gen_ksk(Context &c, Keys &k, uint64_t id, const uint64_t *sp, cudaStream_t s) {
    const size_t n = c.n;
    const int E = c.L + c.K;
    uint64_t *key = nullptr, *e = nullptr;
    if (cudaMalloc(&key, size_t(c.beta) * 2 * E * n * 8) != cudaSuccess) return CATFHE_ENOMEM;
    if (cudaMalloc(&e, size_t(E) * n * 8) != cudaSuccess) {
        cudaFree(key);
        return CATFHE_ENOMEM;
    }
    LimbMap m = map_identity(uint32_t(E));
    DevConst te, pf;
    std::vector<uint64_t> mods(E), tv(E);
    for (int i = 0; i < E; i++) {
        mods[i] = c.mod(i);
        tv[i] = c.scheme == CATFHE_BGV ? c.t % mods[i] : 1;
    }
    int rc = te.set(tv, mods);
    for (int j = 0; j < c.beta && rc == CATFHE_OK; j++) {
        uint64_t *bj = key + (size_t(j) * 2 + 0) * E * n;
        uint64_t *aj = key + (size_t(j) * 2 + 1) * E * n;
        rc = launch_sample(c, sample_args(c, k.seed, TAG_KSK_A, uint32_t(j), uint32_t(id), kUniform), aj,
                           m, uint32_t(E), nullptr, nullptr, s);
        if (!rc) rc = launch_ntt_fwd(c, aj, aj, m, uint32_t(E), s);
        if (!rc)
            rc = launch_sample(c, sample_args(c, k.seed, TAG_KSK_E, uint32_t(j), uint32_t(id), kGaussian),
                               e, m, uint32_t(E), c.scheme == CATFHE_BGV ? te.v : nullptr,
                               c.scheme == CATFHE_BGV ? te.s : nullptr, s);
        if (!rc) rc = launch_ntt_fwd(c, e, e, m, uint32_t(E), s);
        std::vector<uint64_t> pv(E, 0);
        for (int i = j * c.alpha; i < std::min((j + 1) * c.alpha, c.L); i++) pv[i] = pmod(c, c.mod(i));
        DevConst pfc;
        if (!rc) rc = pfc.set(pv, mods);
        if (!rc) rc = launch_ksk_row(c, aj, k.s_ntt, e, sp, bj, uint32_t(E), pfc.v, pfc.s, s);
        if (!rc) rc = cudaStreamSynchronize(s) == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA;
    }
    // Montgomery form: every limb times 2^64 mod its prime
    if (!rc) {
        std::vector<uint64_t> rv(E);
        for (int i = 0; i < E; i++) rv[i] = (uint64_t)(((unsigned __int128)1 << 64) % mods[i]);
        DevConst rm;
        rc = rm.set(rv, mods);
        if (!rc) rc = launch_scale_limbs(c, key, uint32_t(E), uint32_t(c.beta * 2), rm.v, rm.s, s);
        if (!rc) rc = cudaStreamSynchronize(s) == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA;
    }
    cudaFree(e);
    if (rc) {
        cudaFree(key);
        return rc;
    }
    auto it = k.ksk.find(id);
    if (it != k.ksk.end()) cudaFree(it->second);
    k.ksk[id] = key;
    return CATFHE_OK;
}

int op_keygen(Context &c, const uint8_t seed[32], Keys **out) {
    Keys *k = new Keys();
    memcpy(k->seed, seed, 32);
    const size_t n = c.n;
    const int E = c.L + c.K;
    cudaStream_t s = 0;
    uint64_t *a = nullptr, *e = nullptr, *sp = nullptr;
    int rc = CATFHE_OK;
    if (cudaMalloc(&k->s_ntt, size_t(E) * n * 8) != cudaSuccess ||
        cudaMalloc(&k->pk, size_t(2) * c.L * n * 8) != cudaSuccess ||
        cudaMalloc(&e, size_t(E) * n * 8) != cudaSuccess ||
        cudaMalloc(&sp, size_t(E) * n * 8) != cudaSuccess)
        rc = CATFHE_ENOMEM;
    LimbMap mE = map_identity(uint32_t(E)), mL = map_identity(uint32_t(c.L));
    if (!rc) rc = launch_sample(c, sample_args(c, seed, TAG_SK, 0, 0, kTernary), k->s_ntt, mE,
                                uint32_t(E), nullptr, nullptr, s);
    if (!rc) rc = launch_ntt_fwd(c, k->s_ntt, k->s_ntt, mE, uint32_t(E), s);
    // public key over Q_L
    a = k->pk + size_t(c.L) * n;
    if (!rc) rc = launch_sample(c, sample_args(c, seed, TAG_PK_A, 0, 0, kUniform), a, mL,
                                uint32_t(c.L), nullptr, nullptr, s);
    if (!rc) rc = launch_ntt_fwd(c, a, a, mL, uint32_t(c.L), s);
    DevConst te, zero;
    std::vector<uint64_t> mods(c.L), tv(c.L), zv(c.L, 0);
    for (int i = 0; i < c.L; i++) {
        mods[i] = c.mod(i);
        tv[i] = c.scheme == CATFHE_BGV ? c.t % mods[i] : 1;
    }
    if (!rc) rc = te.set(tv, mods);
    if (!rc) rc = zero.set(zv, mods);
    if (!rc) rc = launch_sample(c, sample_args(c, seed, TAG_PK_E, 0, 0, kGaussian), e, mL,
                                uint32_t(c.L), c.scheme == CATFHE_BGV ? te.v : nullptr,
                                c.scheme == CATFHE_BGV ? te.s : nullptr, s);
    if (!rc) rc = launch_ntt_fwd(c, e, e, mL, uint32_t(c.L), s);
    if (!rc) rc = launch_ksk_row(c, a, k->s_ntt, e, nullptr, k->pk, uint32_t(c.L), zero.v, zero.s, s);
    // relinearisation key: s' = s^2
    if (!rc) rc = launch_pointwise(c, k->s_ntt, k->s_ntt, sp, mE, uint32_t(E), s);
    if (!rc) rc = cudaStreamSynchronize(s) == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA;
    if (!rc) rc = gen_ksk(c, *k, 0, sp, s);
    cudaFree(e);
    cudaFree(sp);
    if (rc) {
        cudaFree(k->s_ntt);
        cudaFree(k->pk);
        for (auto &kv : k->ksk) cudaFree(kv.second);
        delete k;
        return rc;
    }
    *out = k;
    return CATFHE_OK;
}

int op_gen_galois(Context &c, Keys &k, uint64_t g) {
    g %= 2 * c.n;
    if (!(g & 1)) return CATFHE_EINVAL;
    if (k.ksk.count(g)) return CATFHE_OK;
    const int E = c.L + c.K;
    uint64_t *sp = nullptr;
    if (cudaMalloc(&sp, size_t(E) * c.n * 8) != cudaSuccess) return CATFHE_ENOMEM;
    int rc = launch_automorph_ntt(c, k.s_ntt, sp, uint32_t(E), g, 0);
    if (!rc) rc = gen_ksk(c, k, g, sp, 0);
    cudaFree(sp);
    return rc;
}

void keys_free(Keys *k) {
    if (!k) return;
    cudaFree(k->s_ntt);
    cudaFree(k->pk);
    for (auto &kv : k->ksk) cudaFree(kv.second);
    delete k;
}

// Coefficient-form copies of the keys to host memory.
int op_keys_export(Context &c, const Keys &k, uint64_t id, int64_t *s_out, uint64_t *pk_out,
                   uint64_t *ksk_out) {
    const size_t n = c.n;
    const int E = c.L + c.K;
    size_t need = size_t(c.beta) * 2 * E * n;
    uint64_t *tmp = nullptr;
    if (cudaMalloc(&tmp, need * 8) != cudaSuccess) return CATFHE_ENOMEM;
    int rc = CATFHE_OK;
    LimbMap mE = map_identity(uint32_t(E));
    if (s_out) {
        rc = launch_ntt_inv(c, k.s_ntt, tmp, mE, 1, 0);  // limb q_0 only
        std::vector<uint64_t> h(n);
        if (!rc && cudaMemcpy(h.data(), tmp, n * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = CATFHE_ECUDA;
        const uint64_t q0 = c.mod(0);
        for (size_t j = 0; j < n && !rc; j++) s_out[j] = h[j] > q0 / 2 ? int64_t(h[j]) - int64_t(q0) : int64_t(h[j]);
    }
    if (!rc && pk_out) {
        LimbMap mL = map_identity(uint32_t(c.L));
        rc = launch_ntt_inv(c, k.pk, tmp, mL, uint32_t(2 * c.L), 0);
        if (!rc && cudaMemcpy(pk_out, tmp, size_t(2) * c.L * n * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = CATFHE_ECUDA;
    }
    if (!rc && ksk_out) {
        auto it = k.ksk.find(id);
        if (it == k.ksk.end()) rc = CATFHE_ENOKEY;
        if (!rc) rc = launch_ntt_inv(c, it->second, tmp, mE, uint32_t(c.beta * 2 * E), 0);
        // undo the Montgomery form: times 2^-64 mod each prime
        std::vector<uint64_t> rv(E), mods(E);
        for (int i = 0; i < E && !rc; i++) {
            mods[i] = c.mod(i);
            rv[i] = h_invmod((uint64_t)(((unsigned __int128)1 << 64) % mods[i]), mods[i]);
        }
        DevConst ri;
        if (!rc) rc = ri.set(rv, mods);
        if (!rc) rc = launch_scale_limbs(c, tmp, uint32_t(E), uint32_t(c.beta * 2), ri.v, ri.s, 0);
        if (!rc && cudaMemcpy(ksk_out, tmp, need * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = CATFHE_ECUDA;
    }
    cudaFree(tmp);
    return rc;
}

// ----------------------------------------------------------------- encryption

int op_encrypt(Context &c, const Keys &k, const int64_t *msg, const uint8_t seed[32],
               uint64_t *ct, cudaStream_t s) {
    const size_t n = c.n;
    const int L = c.L;
    int64_t *dmsg = nullptr;
    uint64_t *v = nullptr, *tmp = nullptr;
    int rc = CATFHE_OK;
    if (cudaMalloc(&dmsg, n * 8) != cudaSuccess || cudaMalloc(&v, size_t(L) * n * 8) != cudaSuccess ||
        cudaMalloc(&tmp, size_t(2) * L * n * 8) != cudaSuccess)
        rc = CATFHE_ENOMEM;
    if (!rc && cudaMemcpyAsync(dmsg, msg, n * 8, cudaMemcpyHostToDevice, s) != cudaSuccess) rc = CATFHE_ECUDA;
    LimbMap mL = map_identity(uint32_t(L));
    std::vector<uint64_t> mods(L), tv(L), dv(L);
    uint64_t qmodt = 1;
    if (c.t)
        for (int i = 0; i < L; i++) qmodt = h_mulmod(qmodt, c.mod(i) % c.t, c.t);
    for (int i = 0; i < L; i++) {
        mods[i] = c.mod(i);
        tv[i] = c.scheme == CATFHE_BGV ? c.t % mods[i] : 1;
        // BFV Delta = floor(Q/t) = (Q - (Q mod t)) / t, mod q_i
        dv[i] = c.scheme == CATFHE_BFV
                    ? h_mulmod((mods[i] - qmodt % mods[i]) % mods[i], h_invmod(c.t % mods[i], mods[i]), mods[i])
                    : 1;
    }
    DevConst te, dl;
    if (!rc) rc = te.set(tv, mods);
    if (!rc) rc = dl.set(dv, mods);
    const bool bgv = c.scheme == CATFHE_BGV;
    uint64_t *t0 = tmp, *t1 = tmp + size_t(L) * n;
    if (!rc) rc = launch_sample(c, sample_args(c, seed, TAG_ENC_V, 0, 0, kTernary), v, mL, uint32_t(L),
                                nullptr, nullptr, s);
    if (!rc) rc = launch_ntt_fwd(c, v, v, mL, uint32_t(L), s);
    if (!rc) rc = launch_sample(c, sample_args(c, seed, TAG_ENC_E0, 0, 0, kGaussian), t0, mL,
                                uint32_t(L), bgv ? te.v : nullptr, bgv ? te.s : nullptr, s);
    if (!rc) rc = launch_sample(c, sample_args(c, seed, TAG_ENC_E1, 0, 0, kGaussian), t1, mL,
                                uint32_t(L), bgv ? te.v : nullptr, bgv ? te.s : nullptr, s);
    if (!rc) rc = launch_small_to_rns(c, dmsg, t0, mL, uint32_t(L),
                                      c.scheme == CATFHE_BFV ? dl.v : nullptr,
                                      c.scheme == CATFHE_BFV ? dl.s : nullptr, 1, s);
    uint64_t *c0 = ct, *c1 = ct + size_t(L) * n;
    if (c.scheme != CATFHE_BFV) {
        if (!rc) rc = launch_ntt_fwd(c, tmp, tmp, mL, uint32_t(2 * L), s);
        if (!rc) rc = launch_mul_add(c, t0, v, k.pk, c0, uint32_t(L), 0, s);
        if (!rc) rc = launch_mul_add(c, t1, v, k.pk + size_t(L) * n, c1, uint32_t(L), 0, s);
    } else {
        // v pk in NTT form, back to coefficients, plus (e0 + Delta m, e1)
        if (!rc) rc = launch_mul_add(c, nullptr, v, k.pk, c0, uint32_t(L), 0, s);
        if (!rc) rc = launch_mul_add(c, nullptr, v, k.pk + size_t(L) * n, c1, uint32_t(L), 0, s);
        if (!rc) rc = launch_ntt_inv(c, ct, ct, mL, uint32_t(2 * L), s);
        LimbMap m2{};
        m2.period = uint32_t(2 * L);
        m2.src_stride = m2.dst_stride = uint32_t(2 * L);
        for (int i = 0; i < 2 * L; i++) {
            m2.src_off[i] = m2.dst_off[i] = uint16_t(i);
            m2.prime[i] = uint8_t(i % L);
        }
        if (!rc) rc = launch_add(c, ct, tmp, ct, m2, uint32_t(2 * L), s);
    }
    if (!rc) rc = cudaStreamSynchronize(s) == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA;
    cudaFree(dmsg);
    cudaFree(v);
    cudaFree(tmp);
    return rc;
}

int op_ct_uniform(Context &c, const uint8_t seed[32], uint32_t index, uint32_t level, uint64_t *ct,
                  cudaStream_t s) {
    if (level < 1 || int(level) > c.L) return CATFHE_ELEVEL;
    LimbMap m = map_identity(level);
    for (uint32_t poly = 0; poly < 2; poly++)
        TRY(launch_sample(c, sample_args(c, seed, TAG_CT_UNIFORM, poly, index, kUniform),
                          ct + size_t(poly) * level * c.n, m, level, nullptr, nullptr, s));
    if (c.scheme != CATFHE_BFV) TRY(launch_ntt_fwd(c, ct, ct, m, 2 * level, s));
    return CATFHE_OK;
}

int op_import(Context &c, const uint64_t *host, uint32_t level, uint32_t count, int form,
              bool sync, uint64_t *ct, cudaStream_t s) {
    if (level < 1 || int(level) > c.L) return CATFHE_ELEVEL;
    const size_t bytes = size_t(count) * 2 * level * c.n * 8;
    if (cudaMemcpyAsync(ct, host, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return CATFHE_ECUDA;
    if (form == CATFHE_FORM_COEFF && c.scheme != CATFHE_BFV) {
        LimbMap m = map_identity(level);
        TRY(launch_ntt_fwd(c, ct, ct, m, 2 * level * count, s));
    }
    if (!sync) return CATFHE_OK;
    return cudaStreamSynchronize(s) == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA;
}

int op_export(Context &c, const uint64_t *ct, uint32_t level, uint32_t count, int form,
              bool sync, uint64_t *host, void *ws, size_t ws_bytes_in, cudaStream_t s) {
    if (level < 1 || int(level) > c.L) return CATFHE_ELEVEL;
    const size_t bytes = size_t(count) * 2 * level * c.n * 8;
    const uint64_t *src = ct;
    if (form == CATFHE_FORM_COEFF && c.scheme != CATFHE_BFV) {
        char *base;
        TRY(get_ws(c, ws, ws_bytes_in, ws_bytes(c, CATFHE_OP_EXPORT, level, count), &base));
        Bump b{base};
        uint64_t *tmp = b.take<uint64_t>(size_t(count) * 2 * level * c.n);
        LimbMap m = map_identity(level);
        TRY(launch_ntt_inv(c, ct, tmp, m, 2 * level * count, s));
        src = tmp;
    }
    if (cudaMemcpyAsync(host, src, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return CATFHE_ECUDA;
    if (!sync) return CATFHE_OK;
    return cudaStreamSynchronize(s) == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA;
}

// Packed transfers: the packed words are staged in the workspace (at least
// 2 count packed_words(level) words), copied and unpacked in stream order.
int op_import_packed(Context &c, const uint64_t *host, uint32_t level, uint32_t count, bool sync,
                     uint64_t *ct, void *ws, size_t ws_bytes_in, cudaStream_t s) {
    if (level < 1 || int(level) > c.L) return CATFHE_ELEVEL;
    if (count == 0) return CATFHE_OK;
    const size_t bytes = size_t(2) * count * packed_words(c, level) * 8;
    char *base;
    TRY(get_ws(c, ws, ws_bytes_in, bytes, &base));
    if (cudaMemcpyAsync(base, host, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return CATFHE_ECUDA;
    TRY(launch_unpack(c, reinterpret_cast<const uint64_t *>(base), ct, level, 2 * count, s));
    if (!sync) return CATFHE_OK;
    return cudaStreamSynchronize(s) == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA;
}

int op_export_packed(Context &c, const uint64_t *ct, uint32_t level, uint32_t count, bool sync,
                     uint64_t *host, void *ws, size_t ws_bytes_in, cudaStream_t s) {
    if (level < 1 || int(level) > c.L) return CATFHE_ELEVEL;
    if (count == 0) return CATFHE_OK;
    const size_t bytes = size_t(2) * count * packed_words(c, level) * 8;
    char *base;
    TRY(get_ws(c, ws, ws_bytes_in, bytes, &base));
    uint64_t *stage = reinterpret_cast<uint64_t *>(base);
    TRY(launch_pack(c, ct, stage, level, 2 * count, s));
    if (cudaMemcpyAsync(host, stage, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return CATFHE_ECUDA;
    if (!sync) return CATFHE_OK;
    return cudaStreamSynchronize(s) == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA;
}

// [c0 + c1 s]_{Q_l} per coefficient (CKKS: centred, two's complement; BFV:
// round(t x / Q) mod t; BGV: x mod t) into res (device int64[N]), using
// 2 level N words of scratch at base.
static int decrypt_device(Context &c, const Keys &k, const uint64_t *ct, uint32_t level,
                          int64_t *res, char *base, cudaStream_t s) {
    Bump b{base};
    const size_t n = c.n;
    uint64_t *x = b.take<uint64_t>(size_t(level) * n);
    uint64_t *tmp = b.take<uint64_t>(size_t(level) * n);
    LimbMap m = map_identity(level);
    if (c.scheme != CATFHE_BFV) {
        TRY(launch_mul_add(c, ct, ct + size_t(level) * n, k.s_ntt, x, level, 0, s));
        TRY(launch_ntt_inv(c, x, x, m, level, s));
    } else {
        TRY(launch_ntt_fwd(c, ct + size_t(level) * n, tmp, m, level, s));
        TRY(launch_mul_add(c, nullptr, tmp, k.s_ntt, tmp, level, 0, s));
        TRY(launch_ntt_inv(c, tmp, tmp, m, level, s));
        TRY(launch_add(c, ct, tmp, x, m, level, s));
    }
    PlanSpec sp;
    for (uint32_t i = 0; i < level; i++) {
        sp.src_mod.push_back(c.mod(int(i)));
        sp.src_off.push_back(i);
    }
    sp.dst_off.push_back(0);
    std::string key = "decrypt/" + std::to_string(level);
    if (c.scheme == CATFHE_CKKS) {
        sp.dst_mod.push_back(0);
    } else {
        sp.dst_mod.push_back(c.t);
        if (c.scheme == CATFHE_BFV) {
            // round(t x / Q) mod t = -[t x]_Q Q^-1 mod t
            for (uint32_t i = 0; i < level; i++) sp.pre.push_back(c.t % c.mod(int(i)));
            const uint64_t qt = prod_mod(c, 0, int(level), c.t);
            sp.post.push_back((c.t - h_invmod(qt, c.t)) % c.t);
        }
    }
    PlanList pl;
    TRY(make_list(c, {{key, sp}}, pl));
    return launch_conv(c, pl, x, 0, 0, reinterpret_cast<uint64_t *>(res), 0, 0, 1, s);
}

int op_decrypt(Context &c, const Keys &k, const uint64_t *ct, uint32_t level, uint64_t factor,
               int64_t *msg, void *ws, size_t ws_bytes_in, cudaStream_t s) {
    if (level < 1 || int(level) > c.L) return CATFHE_ELEVEL;
    if (c.scheme == CATFHE_BGV && (factor % c.t == 0 || h_invmod(factor % c.t, c.t) == 0))
        return CATFHE_EINVAL;
    char *base;
    TRY(get_ws(c, ws, ws_bytes_in, ws_bytes(c, CATFHE_OP_DECRYPT, level, 1), &base));
    const size_t n = c.n;
    int64_t *res = reinterpret_cast<int64_t *>(base + size_t(2) * level * n * 8);
    TRY(decrypt_device(c, k, ct, level, res, base, s));
    if (cudaMemcpyAsync(msg, res, n * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess) return CATFHE_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CATFHE_ECUDA;
    if (c.scheme == CATFHE_BGV) {
        const uint64_t finv = h_invmod(factor % c.t, c.t);
        for (size_t j = 0; j < n; j++) msg[j] = int64_t(h_mulmod(uint64_t(msg[j]), finv, c.t));
    }
    return CATFHE_OK;
}

// CKKS encode on the device: host slots (N/2 complex) -> plaintext in NTT form.
int op_encode_ckks(Context &c, const double *slots, double scale, uint32_t level, uint64_t *pt,
                   void *ws, size_t ws_bytes_in, cudaStream_t s) {
    if (c.scheme != CATFHE_CKKS) return CATFHE_ESCHEME;
    if (level < 1 || int(level) > c.L) return CATFHE_ELEVEL;
    if (!(scale > 0)) return CATFHE_EINVAL;
    TRY(enc_tables(c));
    char *base;
    TRY(get_ws(c, ws, ws_bytes_in, ws_bytes(c, CATFHE_OP_ENCODE, level, 1), &base));
    Bump b{base};
    const size_t n = c.n;
    double2 *dz = b.take<double2>(n / 2);
    double2 *b0 = b.take<double2>(n), *b1 = b.take<double2>(n);
    int64_t *m = b.take<int64_t>(n);
    if (cudaMemcpyAsync(dz, slots, n / 2 * sizeof(double2), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return CATFHE_ECUDA;
    TRY(launch_encode_ckks(c, dz, scale, b0, b1, m, s));
    LimbMap mp = map_identity(level);
    TRY(launch_small_to_rns(c, m, pt, mp, level, nullptr, nullptr, 0, s));
    TRY(launch_ntt_fwd(c, pt, pt, mp, level, s));
    return cudaStreamSynchronize(s) == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA;
}

// CKKS decrypt + decode: ciphertext -> host slots (N/2 complex) / scale.
int op_decode_ckks(Context &c, const Keys &k, const uint64_t *ct, uint32_t level, double scale,
                   double *slots, void *ws, size_t ws_bytes_in, cudaStream_t s) {
    if (c.scheme != CATFHE_CKKS) return CATFHE_ESCHEME;
    if (level < 1 || int(level) > c.L) return CATFHE_ELEVEL;
    if (!(scale > 0)) return CATFHE_EINVAL;
    TRY(enc_tables(c));
    char *base;
    TRY(get_ws(c, ws, ws_bytes_in, ws_bytes(c, CATFHE_OP_DECODE, level, 1), &base));
    Bump b{base};
    const size_t n = c.n;
    char *dec = reinterpret_cast<char *>(b.take<uint64_t>(size_t(2) * level * n));
    int64_t *m = b.take<int64_t>(n);
    double2 *b0 = b.take<double2>(n), *b1 = b.take<double2>(n);
    double2 *dz = b.take<double2>(n / 2);
    TRY(decrypt_device(c, k, ct, level, m, dec, s));
    TRY(launch_decode_ckks(c, m, 1.0 / scale, b0, b1, dz, s));
    if (cudaMemcpyAsync(slots, dz, n / 2 * sizeof(double2), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return CATFHE_ECUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA;
}

}  // namespace catfhe
