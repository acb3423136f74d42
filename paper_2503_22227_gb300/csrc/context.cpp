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
    if (cudaMalloc(&c.d_mods, sizeof(DevMod) * np) != cudaSuccess) return CATFHE_ENOMEM;
    if (cudaMalloc(&c.d_twf, sizeof(ulonglong2) * np * n) != cudaSuccess) return CATFHE_ENOMEM;
    if (cudaMalloc(&c.d_twi, sizeof(ulonglong2) * np * n) != cudaSuccess) return CATFHE_ENOMEM;
    int rc = check(cudaMemcpy(c.d_mods, c.hmods.data(), sizeof(DevMod) * np, cudaMemcpyHostToDevice));
    if (!rc) rc = check(cudaMemcpy(c.d_twf, twf.data(), sizeof(ulonglong2) * np * n, cudaMemcpyHostToDevice));
    if (!rc) rc = check(cudaMemcpy(c.d_twi, twi.data(), sizeof(ulonglong2) * np * n, cudaMemcpyHostToDevice));
    return rc;
}

void ctx_free(Context &c) {
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

std::vector<uint64_t> build_plan(const PlanSpec &s) {
    const uint32_t k = uint32_t(s.src_mod.size()), T = uint32_t(s.dst_mod.size());
    std::vector<uint64_t> out(plan_words(k, T), 0);
    bool wrap = false;
    for (uint64_t q : s.dst_mod) wrap |= (q == 0);
    out[0] = uint64_t(k) | (uint64_t(T) << 16) | (uint64_t(wrap ? 1 : 0) << 32) |
             (uint64_t(s.lazy && !wrap ? 1 : 0) << 33);
    uint64_t *c = out.data() + 1;
    uint64_t *src_off = c; c += k;
    uint64_t *dst_off = c; c += T;
    uint64_t *smod = c; c += 4 * k;
    uint64_t *dmod = c; c += 4 * T;
    uint64_t *pre = c; c += k;
    uint64_t *pre_s = c; c += k;
    uint64_t *W = c; c += size_t(k) * k;
    uint64_t *Minv = c; c += k;
    uint64_t *Minv_s = c; c += k;
    uint64_t *h = c; c += k;
    uint64_t *Wt = c; c += size_t(k) * T;
    uint64_t *Mt = c; c += T;
    uint64_t *post = c; c += T;
    uint64_t *post_s = c;
    const auto &m = s.src_mod;
    for (uint32_t i = 0; i < k; i++) {
        src_off[i] = s.src_off[i];
        put_mod(smod + 4 * i, m[i]);
        pre[i] = s.pre.empty() ? 1 : s.pre[i] % m[i];
        pre_s[i] = h_shoup(pre[i], m[i]);
    }
    for (uint32_t t = 0; t < T; t++) {
        dst_off[t] = s.dst_off[t];
        put_mod(dmod + 4 * t, s.dst_mod[t]);
        const uint64_t p = s.dst_mod[t];
        post[t] = s.post.empty() ? 1 : (p ? s.post[t] % p : s.post[t]);
        post_s[t] = p ? h_shoup(post[t], p) : 0;
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
        Minv_s[j] = h_shoup(Minv[j], m[j]);
    }
    // mixed-radix digits of (M-1)/2, whose residues are (m_i - 1)/2
    for (uint32_t j = 0; j < k; j++) {
        uint64_t r = (m[j] - 1) / 2;
        u128 sum = 0;
        uint64_t s_mod = 0;
        for (uint32_t i = 0; i < j; i++) {
            sum = (u128)h_mulmod(h[i] % m[j], W[size_t(i) * k + j], m[j]) + s_mod;
            s_mod = (uint64_t)(sum % m[j]);
        }
        h[j] = j == 0 ? r : h_mulmod((r + m[j] - s_mod) % m[j], Minv[j], m[j]);
    }
    // target weights
    for (uint32_t t = 0; t < T; t++) {
        const uint64_t p = s.dst_mod[t];
        uint64_t acc = p ? 1 % p : 1;
        for (uint32_t i = 0; i < k; i++) {
            Wt[size_t(i) * T + t] = acc;
            acc = p ? h_mulmod(acc, m[i] % p, p) : acc * m[i];
        }
        Mt[t] = acc;
    }
    return out;
}

const uint64_t *get_plan(Context &c, const std::string &key, const PlanSpec &spec,
                         uint32_t *words) {
    auto it = c.plans.find(key);
    if (it != c.plans.end()) {
        *words = c.plan_sizes[key];
        return it->second;
    }
    std::vector<uint64_t> host = build_plan(spec);
    uint64_t *dev = nullptr;
    if (cudaMalloc(&dev, host.size() * 8) != cudaSuccess) return nullptr;
    if (cudaMemcpy(dev, host.data(), host.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(dev);
        return nullptr;
    }
    c.plans[key] = dev;
    c.plan_sizes[key] = uint32_t(host.size());
    *words = uint32_t(host.size());
    return dev;
}

// Plan whose device copy is followed by `extra` words (BFV scale-and-round).
const uint64_t *get_plan_extra(Context &c, const std::string &key, const PlanSpec &spec,
                               const std::vector<uint64_t> &extra, uint32_t *words) {
    auto it = c.plans.find(key);
    if (it != c.plans.end()) {
        *words = c.plan_sizes[key];
        return it->second;
    }
    std::vector<uint64_t> host = build_plan(spec);
    const size_t w = host.size();
    host.insert(host.end(), extra.begin(), extra.end());
    uint64_t *dev = nullptr;
    if (cudaMalloc(&dev, host.size() * 8) != cudaSuccess) return nullptr;
    if (cudaMemcpy(dev, host.data(), host.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(dev);
        return nullptr;
    }
    c.plans[key] = dev;
    c.plan_sizes[key] = uint32_t(w);
    *words = uint32_t(w);
    return dev;
}

}  // namespace catfhe
