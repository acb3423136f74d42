// Context set-up: prime chain, NTT tables, base-conversion plans.
//
// Prime chain (paper Sec. 2.2 writes q as a product of word-sized coprime
// moduli without listing them): prime i of each list is the largest prime
// below 2^bits that is 1 mod 2^(log_n_max+1) and not taken yet; ciphertext
// primes first, then special primes, then BFV auxiliary primes.  The NTT
// root of each prime is its smallest primitive 2N-th root of unity.
#include <string.h>

#include <algorithm>

#include "internal.h"

namespace catfhe {

typedef unsigned __int128 u128;

static uint64_t next_prime_below(int bits, uint64_t two_n, const std::vector<uint64_t> &used) {
    const uint64_t top = (uint64_t(1) << bits) - 1;
    for (uint64_t c = ((top - 1) / two_n) * two_n + 1; c > two_n; c -= two_n) {
        if (std::find(used.begin(), used.end(), c) != used.end()) continue;
        if (h_is_prime(c)) return c;
    }
    return 0;
}

// Little-endian 64-bit-word products, for the BFV auxiliary basis rule.
static void mw_mul(std::vector<uint64_t> &a, uint64_t b) {
    u128 carry = 0;
    for (auto &w : a) {
        u128 t = (u128)w * b + carry;
        w = (uint64_t)t;
        carry = t >> 64;
    }
    if (carry) a.push_back((uint64_t)carry);
}

static int mw_cmp(const std::vector<uint64_t> &a, const std::vector<uint64_t> &b) {
    size_t na = a.size(), nb = b.size();
    while (na && !a[na - 1]) na--;
    while (nb && !b[nb - 1]) nb--;
    if (na != nb) return na < nb ? -1 : 1;
    for (size_t i = na; i-- > 0;)
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    return 0;
}

static int check(cudaError_t e) { return e == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA; }

int ctx_init(Context &c, const catfhe_params &p) {
    if (p.scheme < 0 || p.scheme > 2) return CATFHE_EINVAL;
    if (p.log_n < 12 || p.log_n > 16) return CATFHE_EINVAL;
    const int log_n_max = p.log_n_max ? p.log_n_max : p.log_n;
    if (log_n_max < p.log_n || log_n_max > 20) return CATFHE_EINVAL;
    if (p.L < 1 || p.L > kConvMaxK || p.K < 1 || p.K > 15) return CATFHE_EINVAL;
    if (p.dnum < 1 || p.dnum > p.L) return CATFHE_EINVAL;
    for (int i = 0; i < p.L; i++)
        if (p.q_bits[i] < 20 || p.q_bits[i] > 61) return CATFHE_EINVAL;
    for (int i = 0; i < p.K; i++)
        if (p.p_bits[i] < 20 || p.p_bits[i] > 61) return CATFHE_EINVAL;
    if (p.scheme != CATFHE_CKKS && (p.t < 3 || !(p.t & 1) || p.t >= (uint64_t(1) << 61)))
        return CATFHE_EINVAL;
    c.prm = p;
    c.scheme = p.scheme;
    c.log_n = p.log_n;
    c.n = uint64_t(1) << p.log_n;
    c.L = p.L;
    c.K = p.K;
    c.t = p.scheme == CATFHE_CKKS ? 0 : p.t;
    c.alpha = (p.L + p.dnum - 1) / p.dnum;
    c.beta = (p.L + c.alpha - 1) / c.alpha;
    if (c.beta > 32) return CATFHE_EINVAL;
    const uint64_t two_n = uint64_t(2) << log_n_max;

    std::vector<uint64_t> used;
    for (int i = 0; i < p.L; i++) {
        uint64_t q = next_prime_below(p.q_bits[i], two_n, used);
        if (!q) return CATFHE_EINVAL;
        used.push_back(q);
    }
    for (int i = 0; i < p.K; i++) {
        uint64_t q = next_prime_below(p.p_bits[i], two_n, used);
        if (!q) return CATFHE_EINVAL;
        used.push_back(q);
    }
    if (p.scheme == CATFHE_BFV) {
        const int bb = p.aux_bits ? p.aux_bits : 60;
        if (bb < 20 || bb > 61) return CATFHE_EINVAL;
        // smallest |B| with prod(B) > 2 t N Q (unless given)
        std::vector<uint64_t> bound{2 * c.t};
        mw_mul(bound, c.n);
        for (int i = 0; i < p.L; i++) mw_mul(bound, used[i]);
        std::vector<uint64_t> prod{1};
        int nb = 0;
        while (p.aux_count > 0 ? nb < p.aux_count : mw_cmp(prod, bound) <= 0) {
            uint64_t b = next_prime_below(bb, two_n, used);
            if (!b) return CATFHE_EINVAL;
            used.push_back(b);
            mw_mul(prod, b);
            nb++;
        }
        c.nb = nb;
        if (c.L + c.nb > kConvMaxK || c.nb > kConvMaxK) return CATFHE_EINVAL;
    }
    if (c.t) {
        for (uint64_t q : used)
            if (q % c.t == 0 || h_invmod(q % c.t, c.t) == 0) return CATFHE_EINVAL;
    }
    // the key-switching inner product sums beta + 1 products below 2^64 q
    for (uint64_t q : used)
        if ((u128)(c.beta + 1) * q >= ((u128)1 << 64)) return CATFHE_EINVAL;
    for (uint64_t q : used) c.primes.push_back(HostPrime{q, h_min_psi(q, c.log_n)});
    const size_t np = c.primes.size(), n = c.n;
    for (auto &hp : c.primes) c.hmods.push_back(h_devmod(hp.q, n, hp.psi));

    // NTT tables: psi^bitrev(i) and psi^-bitrev(i) with their Shoup quotients.
    std::vector<ulonglong2> twf(np * n), twi(np * n);
    std::vector<uint64_t> pw(n), pwi(n);
    for (size_t pi = 0; pi < np; pi++) {
        const uint64_t q = c.primes[pi].q, psi = c.primes[pi].psi, psii = h_invmod(psi, q);
        pw[0] = pwi[0] = 1;
        for (size_t i = 1; i < n; i++) {
            pw[i] = h_mulmod(pw[i - 1], psi, q);
            pwi[i] = h_mulmod(pwi[i - 1], psii, q);
        }
        for (size_t i = 0; i < n; i++) {
            uint32_t r = 0;
            for (int b = 0; b < c.log_n; b++) r |= ((i >> b) & 1) << (c.log_n - 1 - b);
            twf[pi * n + i] = make_ulonglong2(pw[r], h_shoup(pw[r], q));
            twi[pi * n + i] = make_ulonglong2(pwi[r], h_shoup(pwi[r], q));
        }
    }
    h_cdt(c.cdt);
    if (cudaGetDevice(&c.device) != cudaSuccess) return CATFHE_ECUDA;
    if (cudaMalloc(&c.d_status, sizeof(int)) != cudaSuccess) return CATFHE_ENOMEM;
    if (cudaMemset(c.d_status, 0, sizeof(int)) != cudaSuccess) return CATFHE_ECUDA;
    if (cudaMalloc(&c.d_mods, sizeof(DevMod) * np) != cudaSuccess) return CATFHE_ENOMEM;
    if (cudaMalloc(&c.d_twf, sizeof(ulonglong2) * np * n) != cudaSuccess) return CATFHE_ENOMEM;
    if (cudaMalloc(&c.d_twi, sizeof(ulonglong2) * np * n) != cudaSuccess) return CATFHE_ENOMEM;
    int rc = check(cudaMemcpy(c.d_mods, c.hmods.data(), sizeof(DevMod) * np, cudaMemcpyHostToDevice));
    if (!rc) rc = check(cudaMemcpy(c.d_twf, twf.data(), sizeof(ulonglong2) * np * n, cudaMemcpyHostToDevice));
    if (!rc) rc = check(cudaMemcpy(c.d_twi, twi.data(), sizeof(ulonglong2) * np * n, cudaMemcpyHostToDevice));
    return rc;
}

void ctx_free(Context &c) {
    cudaFree(c.d_status);
    cudaFree(c.d_enc);
    cudaFree(c.d_slot);
    cudaFree(c.d_mods);
    cudaFree(c.d_twf);
    cudaFree(c.d_twi);
    for (auto &kv : c.plans) cudaFree(kv.second);
    cudaFree(c.scratch.ptr);
    c.plans.clear();
}

// ----------------------------------------------------------------- conversion plans

static void put_mod(uint64_t *w, uint64_t q) {
    if (!q) {
        w[0] = w[1] = w[2] = w[3] = 0;
        return;
    }
    DevMod m = h_devmod(q, 0, 0);
    w[0] = m.q;
    w[1] = m.r64;
    w[2] = m.r64_s;
    w[3] = m.one_s;
}

static uint64_t neg_inv64(uint64_t m) {
    uint64_t x = m;  // m x = 1 mod 8 for odd m; each Newton step doubles the bits
    for (int i = 0; i < 6; i++) x *= 2 - m * x;
    return 0 - x;
}

static uint64_t r64_mod(uint64_t m) { return (uint64_t)(((u128)1 << 64) % m); }

bool plan_fits_mont(const PlanSpec &s) {
    u128 sum = 1;
    for (uint64_t m : s.src_mod) sum += m;
    return sum < ((u128)1 << 64);
}

bool plan_fits_split(const PlanSpec &s) {
    const uint64_t lim = uint64_t(1) << 60;
    if (!plan_fits_mont(s) || s.src_mod.empty() || s.src_mod.size() > 8) return false;
    for (uint64_t m : s.src_mod)
        if (m >= lim) return false;
    for (uint64_t p : s.dst_mod)
        if (p == 0 || p >= lim) return false;
    return true;
}

// A weight below 2^60 as its 30-bit halves, lo | hi << 32.
static uint64_t split30(uint64_t c) { return (c & ((uint64_t(1) << 30) - 1)) | ((c >> 30) << 32); }

std::vector<uint64_t> build_plan(const PlanSpec &s) {
    const uint32_t k = uint32_t(s.src_mod.size()), T = uint32_t(s.dst_mod.size());
    const bool mont = !s.exact && plan_fits_mont(s);
    const bool split = mont && s.split && plan_fits_split(s);
    bool wrap = false;
    for (uint64_t q : s.dst_mod) wrap |= (q == 0);
    const auto &m = s.src_mod;
    // plain constants shared by both layouts
    std::vector<uint64_t> pre(k), post(T), W(size_t(k) * k), Minv(k), h(k), Wt(size_t(k) * T), Mt(T);
    for (uint32_t i = 0; i < k; i++) pre[i] = s.pre.empty() ? 1 : s.pre[i] % m[i];
    for (uint32_t t = 0; t < T; t++) {
        const uint64_t p = s.dst_mod[t];
        post[t] = s.post.empty() ? 1 : (p ? s.post[t] % p : s.post[t]);
    }
    // W[i][j] = prod_{l<i} m_l mod m_j;  Minv[j] = (prod_{l<j} m_l)^-1 mod m_j
    for (uint32_t j = 0; j < k; j++) {
        uint64_t acc = 1 % m[j];
        for (uint32_t i = 0; i < k; i++) {
            W[size_t(i) * k + j] = acc;
            acc = h_mulmod(acc, m[i] % m[j], m[j]);
        }
        uint64_t prod = 1 % m[j];
        for (uint32_t l = 0; l < j; l++) prod = h_mulmod(prod, m[l] % m[j], m[j]);
        Minv[j] = h_invmod(prod, m[j]);
    }
    // mixed-radix digits of (M-1)/2, whose residues are (m_i - 1)/2
    for (uint32_t j = 0; j < k; j++) {
        const uint64_t r = (m[j] - 1) / 2;
        uint64_t s_mod = 0;
        for (uint32_t i = 0; i < j; i++)
            s_mod = (uint64_t)(((u128)h_mulmod(h[i] % m[j], W[size_t(i) * k + j], m[j]) + s_mod) % m[j]);
        h[j] = j == 0 ? r : h_mulmod((r + m[j] - s_mod) % m[j], Minv[j], m[j]);
    }
    // target weights prod_{l<i} m_l and M, mod p_t (mod 2^64 when p_t = 0)
    for (uint32_t t = 0; t < T; t++) {
        const uint64_t p = s.dst_mod[t];
        uint64_t acc = p ? 1 % p : 1;
        for (uint32_t i = 0; i < k; i++) {
            Wt[size_t(i) * T + t] = acc;
            acc = p ? h_mulmod(acc, m[i] % p, p) : acc * m[i];
        }
        Mt[t] = acc;
    }

    std::vector<uint64_t> out(plan_words(k, T, mont), 0);
    out[0] = uint64_t(k) | (uint64_t(T) << 16) | (uint64_t(wrap ? 1 : 0) << 32) |
             (uint64_t(s.lazy && !wrap ? 1 : 0) << 33) | (uint64_t(mont ? 1 : 0) << 34) |
             (uint64_t(split ? 1 : 0) << 35);
    uint64_t *c = out.data() + 1;
    for (uint32_t i = 0; i < k; i++) c[i] = s.src_off[i];
    c += k;
    for (uint32_t t = 0; t < T; t++) c[t] = s.dst_off[t];
    c += T;
    if (mont) {
        uint64_t *smod = c; c += 2 * k;
        uint64_t *dmod = c; c += 2 * T;
        uint64_t *C = c; c += size_t(k) * k;
        uint64_t *hh = c; c += k;
        uint64_t *Ct = c; c += size_t(k) * T;
        uint64_t *Mneg = c;
        for (uint32_t i = 0; i < k; i++) {
            smod[2 * i] = m[i];
            smod[2 * i + 1] = neg_inv64(m[i]);
        }
        for (uint32_t j = 0; j < k; j++) {
            const uint64_t R = r64_mod(m[j]);
            C[size_t(j) * k + j] = h_mulmod(h_mulmod(pre[j], Minv[j], m[j]), R, m[j]);
            for (uint32_t i = 0; i < j; i++) {
                const uint64_t wm = h_mulmod(W[size_t(i) * k + j], Minv[j], m[j]);
                C[size_t(i) * k + j] = h_mulmod((m[j] - wm) % m[j], R, m[j]);
            }
            hh[j] = h[j];
        }
        for (uint32_t t = 0; t < T; t++) {
            const uint64_t p = s.dst_mod[t];
            if (!p) {
                for (uint32_t i = 0; i < k; i++) Ct[size_t(i) * T + t] = Wt[size_t(i) * T + t];
                Mneg[t] = Mt[t];
                continue;
            }
            dmod[2 * t] = p;
            dmod[2 * t + 1] = neg_inv64(p);
            const uint64_t R = r64_mod(p), pr = h_mulmod(post[t], R, p);
            for (uint32_t i = 0; i < k; i++) Ct[size_t(i) * T + t] = h_mulmod(Wt[size_t(i) * T + t], pr, p);
            Mneg[t] = h_mulmod((p - Mt[t]) % p, pr, p);
        }
        if (split) {
            for (size_t i = 0; i < size_t(k) * k; i++) C[i] = split30(C[i]);
            for (size_t i = 0; i < size_t(k) * T; i++) Ct[i] = split30(Ct[i]);
        }
        return out;
    }
    uint64_t *smod = c; c += 4 * k;
    uint64_t *dmod = c; c += 4 * T;
    uint64_t *pre_v = c; c += k;
    uint64_t *pre_s = c; c += k;
    uint64_t *Wv = c; c += size_t(k) * k;
    uint64_t *Minv_v = c; c += k;
    uint64_t *Minv_s = c; c += k;
    uint64_t *hv = c; c += k;
    uint64_t *Wt_v = c; c += size_t(k) * T;
    uint64_t *Mt_v = c; c += T;
    uint64_t *post_v = c; c += T;
    uint64_t *post_s = c;
    for (uint32_t i = 0; i < k; i++) {
        put_mod(smod + 4 * i, m[i]);
        pre_v[i] = pre[i];
        pre_s[i] = h_shoup(pre[i], m[i]);
        Minv_v[i] = Minv[i];
        Minv_s[i] = h_shoup(Minv[i], m[i]);
        hv[i] = h[i];
    }
    for (size_t i = 0; i < W.size(); i++) Wv[i] = W[i];
    for (uint32_t t = 0; t < T; t++) {
        const uint64_t p = s.dst_mod[t];
        put_mod(dmod + 4 * t, p);
        post_v[t] = post[t];
        post_s[t] = p ? h_shoup(post[t], p) : 0;
        Mt_v[t] = Mt[t];
    }
    for (size_t i = 0; i < Wt.size(); i++) Wt_v[i] = Wt[i];
    return out;
}

static PlanRef upload_plan(Context &c, const std::string &key, std::vector<uint64_t> host,
                           const std::vector<uint64_t> &extra) {
    PlanRef ref;
    const size_t w = host.size();
    ref.mont = ((host[0] >> 34) & 1) != 0;
    ref.split = ((host[0] >> 35) & 1) != 0;
    host.insert(host.end(), extra.begin(), extra.end());
    uint64_t *dev = nullptr;
    if (cudaMalloc(&dev, host.size() * 8) != cudaSuccess) return ref;
    if (cudaMemcpy(dev, host.data(), host.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(dev);
        return ref;
    }
    c.plans[key] = dev;
    c.plan_sizes[key] = uint32_t(w) | (ref.mont ? 0x80000000u : 0u) | (ref.split ? 0x40000000u : 0u);
    ref.p = dev;
    ref.words = uint32_t(w);
    return ref;
}

PlanRef get_plan_extra(Context &c, const std::string &key0, const PlanSpec &spec,
                       const std::vector<uint64_t> &extra) {
    const std::string key = key0 + (spec.exact ? "/x" : spec.split ? "/s" : "");
    auto it = c.plans.find(key);
    if (it != c.plans.end()) {
        PlanRef ref;
        ref.p = it->second;
        ref.words = c.plan_sizes[key] & 0x3fffffffu;
        ref.mont = (c.plan_sizes[key] & 0x80000000u) != 0;
        ref.split = (c.plan_sizes[key] & 0x40000000u) != 0;
        return ref;
    }
    return upload_plan(c, key, build_plan(spec), extra);
}

PlanRef get_plan(Context &c, const std::string &key, const PlanSpec &spec) {
    return get_plan_extra(c, key, spec, {});
}

}  // namespace catfhe
