// Exact, centred RNS base conversion (the ModUp lift of a key-switching
// digit, the ModDown / rescale correction, the BFV scale-and-round and the
// decryption lift).
//
// Given residues r_i of x mod m_0 .. m_{k-1} (M = prod m_i), the centred
// representative x_c in (-M/2, M/2] is lifted to any target modulus p.
// The paper names these conversions only through its operators
// (relinearize, rescale, rotate in Tables 1-3; BFV multiplication through
// an auxiliary basis, Sec. 3.1); here they are computed exactly:
//
//   mixed radix (Garner): x = a_0 + a_1 m_0 + a_2 m_0 m_1 + ..., with
//     a_j = (r_j - sum_{i<j} a_i [prod_{l<i} m_l]_{m_j}) [prod_{l<j} m_l]^-1_{m_j}
//   centring: x > (M-1)/2 iff the digit vector (a_{k-1} .. a_0) exceeds the
//     digits of (M-1)/2 lexicographically; then x_c = x - M;
//   target: x_c mod p = sum_i a_i [prod_{l<i} m_l]_p - [x > (M-1)/2] [M]_p.
//
// Every sum is accumulated exactly in 128 bits and reduced once, so there is
// no floating-point estimate and no approximation: the result is the
// definition, bit for bit.  Two constant layouts exist (see internal.h):
//
//  - Montgomery (used whenever sum(m_i) + 1 < 2^64): every constant is
//    stored times 2^64 mod its modulus, the mixed-radix step of a_j is ONE
//    dot product over (r_j, a_0 .. a_{j-1}), a target is ONE dot product
//    (plus the folded -M term when x is above (M-1)/2), and each is reduced
//    by a single Montgomery reduction: u = lo * (-p^-1) mod 2^64,
//    (acc + u p) / 2^64 = hi + mulhi(u, p) + [lo != 0], in [0, 2p) because
//    acc < 2^64 p;
//  - exact (fallback): each sum reduced by hi*(2^64 mod p) + lo (Shoup).
//
// One thread handles one coefficient of one item; the packed plan (a few
// KB) sits in shared memory and every thread reads the same words
// (broadcast).
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include "launch.cuh"
#include "modarith.cuh"

namespace catfhe {

__device__ __forceinline__ void copy_plan(uint64_t *dst, const uint64_t *src, uint32_t words) {
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
}

// ================================================================== exact layout

struct ExactView {
    uint32_t k, T, wrap, lazy;
    const uint64_t *src_off, *dst_off, *smod, *dmod, *pre, *pre_s, *W, *Minv, *Minv_s, *h, *Wt,
        *Mt, *post, *post_s;
};

__device__ __forceinline__ ExactView exact_view(const uint64_t *p) {
    ExactView v;
    v.k = uint32_t(p[0] & 0xffff);
    v.T = uint32_t((p[0] >> 16) & 0xffff);
    v.wrap = uint32_t((p[0] >> 32) & 1);
    v.lazy = uint32_t((p[0] >> 33) & 1);
    const uint64_t *c = p + 1;
    const uint32_t k = v.k, T = v.T;
    v.src_off = c; c += k;
    v.dst_off = c; c += T;
    v.smod = c; c += 4 * k;
    v.dmod = c; c += 4 * T;
    v.pre = c; c += k;
    v.pre_s = c; c += k;
    v.W = c; c += size_t(k) * k;
    v.Minv = c; c += k;
    v.Minv_s = c; c += k;
    v.h = c; c += k;
    v.Wt = c; c += size_t(k) * T;
    v.Mt = c; c += T;
    v.post = c; c += T;
    v.post_s = c;
    return v;
}

__device__ __forceinline__ DevMod mod4(const uint64_t *w) {
    DevMod m;
    m.q = w[0];
    m.r64 = w[1];
    m.r64_s = w[2];
    m.one_s = w[3];
    return m;
}

// sum_{i < cnt} a[i] * w[i * stride], partial sums of <= 8 products of
// words < 2^62 reduced mod m so that 128 bits never overflow.
template <int KMAX>
__device__ __forceinline__ U128 dot_exact(const uint64_t (&a)[KMAX], const uint64_t *w,
                                          uint32_t stride, uint32_t cnt, const DevMod &m) {
    U128 acc{0, 0};
#pragma unroll(KMAX <= 16 ? KMAX : 1)
    for (int i = 0; i < KMAX; i++) {
        if (uint32_t(i) < cnt) {
            mac(acc, a[i], w[size_t(i) * stride]);
            if ((i & 7) == 7 && uint32_t(i + 1) < cnt) {
                acc.lo = reduce128(acc, m);
                acc.hi = 0;
            }
        }
    }
    return acc;
}

template <int KMAX>
__device__ __forceinline__ bool mixed_radix_exact(uint64_t (&a)[KMAX], const ExactView &P) {
#pragma unroll(KMAX <= 16 ? KMAX : 1)
    for (int i = 0; i < KMAX; i++)
        if (uint32_t(i) < P.k && P.pre[i] != 1)
            a[i] = shoup(a[i], P.pre[i], P.pre_s[i], P.smod[4 * i]);
#pragma unroll(KMAX <= 16 ? KMAX : 1)
    for (int j = 1; j < KMAX; j++) {
        if (uint32_t(j) < P.k) {
            const DevMod mj = mod4(P.smod + 4 * j);
            const uint64_t s = reduce128(dot_exact<KMAX>(a, P.W + j, P.k, uint32_t(j), mj), mj);
            a[j] = shoup(sub_mod(a[j], s, mj.q), P.Minv[j], P.Minv_s[j], mj.q);
        }
    }
    bool gt = false, decided = false;
#pragma unroll(KMAX <= 16 ? KMAX : 1)
    for (int i = KMAX - 1; i >= 0; i--) {
        if (uint32_t(i) < P.k && !decided && a[i] != P.h[i]) {
            gt = a[i] > P.h[i];
            decided = true;
        }
    }
    return gt;
}

// x_c mod p_t (times the post-multiplier), in [0, p_t).
template <int KMAX>
__device__ __forceinline__ uint64_t eval_exact(const uint64_t (&a)[KMAX], bool gt,
                                               const ExactView &P, uint32_t t) {
    if (P.wrap) {
        uint64_t r = 0;
#pragma unroll(KMAX <= 16 ? KMAX : 1)
        for (int i = 0; i < KMAX; i++)
            if (uint32_t(i) < P.k) r += a[i] * P.Wt[size_t(i) * P.T + t];
        return gt ? r - P.Mt[t] : r;
    }
    const DevMod mt = mod4(P.dmod + 4 * t);
    uint64_t r = reduce128(dot_exact<KMAX>(a, P.Wt + t, P.T, P.k, mt), mt);
    if (gt) r = sub_mod(r, P.Mt[t], mt.q);
    if (P.post[t] != 1) r = shoup(r, P.post[t], P.post_s[t], mt.q);
    return r;
}

// ================================================================== Montgomery layout

struct MontView {
    uint32_t k, T, wrap, lazy;
    const uint64_t *src_off, *dst_off, *smod, *dmod, *C, *h, *Ct, *Mneg;
};

__device__ __forceinline__ MontView mont_view(const uint64_t *p) {
    MontView v;
    v.k = uint32_t(p[0] & 0xffff);
    v.T = uint32_t((p[0] >> 16) & 0xffff);
    v.wrap = uint32_t((p[0] >> 32) & 1);
    v.lazy = uint32_t((p[0] >> 33) & 1);
    const uint64_t *c = p + 1;
    const uint32_t k = v.k, T = v.T;
    v.src_off = c; c += k;
    v.dst_off = c; c += T;
    v.smod = c; c += 2 * k;
    v.dmod = c; c += 2 * T;
    v.C = c; c += size_t(k) * k;
    v.h = c; c += k;
    v.Ct = c; c += size_t(k) * T;
    v.Mneg = c;
    return v;
}

template <int KMAX>
__device__ __forceinline__ bool mixed_radix_mont(uint64_t (&a)[KMAX], const MontView &P) {
#pragma unroll(KMAX <= 16 ? KMAX : 1)
    for (int j = 0; j < KMAX; j++) {
        if (uint32_t(j) < P.k) {
            const uint64_t mj = P.smod[2 * j], minv = P.smod[2 * j + 1];
            U128 acc{0, 0};
            mac(acc, a[j], P.C[size_t(j) * P.k + j]);
#pragma unroll(KMAX <= 16 ? KMAX : 1)
            for (int i = 0; i < KMAX; i++)
                if (i < j) mac(acc, a[i], P.C[size_t(i) * P.k + j]);
            a[j] = csub(redc(acc, mj, minv), mj);
        }
    }
    bool gt = false, decided = false;
#pragma unroll(KMAX <= 16 ? KMAX : 1)
    for (int i = KMAX - 1; i >= 0; i--) {
        if (uint32_t(i) < P.k && !decided && a[i] != P.h[i]) {
            gt = a[i] > P.h[i];
            decided = true;
        }
    }
    return gt;
}

// Two targets at once (two independent accumulation chains).
template <int KMAX>
__device__ __forceinline__ void eval_mont2(const uint64_t (&a)[KMAX], bool gt, const MontView &P,
                                           uint32_t t, uint64_t &r0, uint64_t &r1) {
    const uint32_t T = P.T;
    U128 acc0{0, 0}, acc1{0, 0};
#pragma unroll(KMAX <= 16 ? KMAX : 1)
    for (int i = 0; i < KMAX; i++) {
        if (uint32_t(i) < P.k) {
            mac(acc0, a[i], P.Ct[size_t(i) * T + t]);
            mac(acc1, a[i], P.Ct[size_t(i) * T + t + 1]);
        }
    }
    if (gt) {
        mac(acc0, 1, P.Mneg[t]);
        mac(acc1, 1, P.Mneg[t + 1]);
    }
    const uint64_t p0 = P.dmod[2 * t], p1 = P.dmod[2 * t + 2];
    r0 = redc(acc0, p0, P.dmod[2 * t + 1]);
    r1 = redc(acc1, p1, P.dmod[2 * t + 3]);
    if (!P.lazy) {
        r0 = csub(r0, p0);
        r1 = csub(r1, p1);
    }
}

// x_c mod p_t (times the post-multiplier): [0, p_t), or [0, 2 p_t) if lazy.
template <int KMAX>
__device__ __forceinline__ uint64_t eval_mont(const uint64_t (&a)[KMAX], bool gt,
                                              const MontView &P, uint32_t t) {
    const uint32_t T = P.T;
    if (P.wrap) {
        uint64_t r = 0;
#pragma unroll(KMAX <= 16 ? KMAX : 1)
        for (int i = 0; i < KMAX; i++)
            if (uint32_t(i) < P.k) r += a[i] * P.Ct[size_t(i) * T + t];
        return gt ? r - P.Mneg[t] : r;
    }
    U128 acc{0, 0};
#pragma unroll(KMAX <= 16 ? KMAX : 1)
    for (int i = 0; i < KMAX; i++)
        if (uint32_t(i) < P.k) mac(acc, a[i], P.Ct[size_t(i) * T + t]);
    if (gt) mac(acc, 1, P.Mneg[t]);
    const uint64_t p = P.dmod[2 * t];
    const uint64_t r = redc(acc, p, P.dmod[2 * t + 1]);
    return P.lazy ? r : csub(r, p);
}

// ================================================================== split weights

// Montgomery layout with k <= 8 and every modulus below 2^60: digits and
// weights are split into 30-bit halves (Acc3, mac3 and join3 in
// modarith.cuh).  With at most 8 products per sum, ll and hh stay below
// 2^63 and mm below 16 (2^30 - 1)^2 < 2^64.  The joined value is the same
// exact sum as in the Montgomery layout (below 2^64 times the modulus),
// reduced by one Montgomery reduction.


// A plan constant read from shared memory at its point of use.  The load is
// volatile so that the compiler keeps it there: with the exact-source-count
// instantiations fully unrolled it otherwise hoisted every constant of the
// mixed-radix steps and spilled (332 bytes per thread at k = 8); read in
// place, the k = 8 kernel fits in 64 registers at 4 CTAs per SM without
// spills (batched step 1491 -> 1455 us).
__device__ __forceinline__ uint64_t ld_plan(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.volatile.shared.u64 %0, [%1];"
                 : "=l"(v)
                 : "r"(uint32_t(__cvta_generic_to_shared(p))));
    return v;
}

// Mixed-radix digits as 30-bit halves, and the centring decision (the
// lexicographic comparison with the digits of (M-1)/2 runs from the least
// significant digit up: the last differing digit decides).
// EXACT: every plan of the launch has k = KMAX sources, so the source count
// and the constants' row stride are compile-time constants.
template <int KMAX, bool EXACT>
__device__ __forceinline__ bool mixed_radix_split(const uint64_t (&r)[KMAX], uint32_t (&al)[KMAX],
                                                  uint32_t (&ah)[KMAX], const MontView &P) {
    const uint32_t k = EXACT ? uint32_t(KMAX) : P.k;
    bool gt = false;
#pragma unroll
    for (int j = 0; j < KMAX; j++) {
        al[j] = ah[j] = 0;
        if (uint32_t(j) < k) {
            Acc3 acc{0, 0, 0};
            mac3(acc, uint32_t(r[j]) & kMask30, uint32_t(r[j] >> 30),
                 ld_plan(&P.C[size_t(j) * k + j]));
#pragma unroll
            for (int i = 0; i < KMAX; i++)
                if (i < j) mac3(acc, al[i], ah[i], ld_plan(&P.C[size_t(i) * k + j]));
            const uint64_t mj = P.smod[2 * j];
            const uint64_t aj = csub(redc(join3(acc), mj, P.smod[2 * j + 1]), mj);
            al[j] = uint32_t(aj) & kMask30;
            ah[j] = uint32_t(aj >> 30);
            if (aj != P.h[j]) gt = aj > P.h[j];
        }
    }
    return gt;
}

// Targets t and t+1 (two independent chains).
template <int KMAX, bool EXACT>
__device__ __forceinline__ void eval_split2(const uint32_t (&al)[KMAX], const uint32_t (&ah)[KMAX],
                                            bool gt, const MontView &P, uint32_t t, uint64_t &r0,
                                            uint64_t &r1) {
    const uint32_t T = P.T, k = EXACT ? uint32_t(KMAX) : P.k;
    Acc3 a0{0, 0, 0}, a1{0, 0, 0};
#pragma unroll
    for (int i = 0; i < KMAX; i++) {
        if (uint32_t(i) < k) {
            mac3(a0, al[i], ah[i], P.Ct[size_t(i) * T + t]);
            mac3(a1, al[i], ah[i], P.Ct[size_t(i) * T + t + 1]);
        }
    }
    if (gt) {  // below 2^60 each: ll stays below 2^64
        a0.ll += P.Mneg[t];
        a1.ll += P.Mneg[t + 1];
        a0.mm += P.Mneg[t];
        a1.mm += P.Mneg[t + 1];
    }
    const uint64_t p0 = P.dmod[2 * t], p1 = P.dmod[2 * t + 2];
    r0 = redc(join3(a0), p0, P.dmod[2 * t + 1]);
    r1 = redc(join3(a1), p1, P.dmod[2 * t + 3]);
    if (!P.lazy) {
        r0 = csub(r0, p0);
        r1 = csub(r1, p1);
    }
}

template <int KMAX, bool EXACT>
__device__ __forceinline__ uint64_t eval_split(const uint32_t (&al)[KMAX],
                                               const uint32_t (&ah)[KMAX], bool gt,
                                               const MontView &P, uint32_t t) {
    const uint32_t k = EXACT ? uint32_t(KMAX) : P.k;
    Acc3 a{0, 0, 0};
#pragma unroll
    for (int i = 0; i < KMAX; i++)
        if (uint32_t(i) < k) mac3(a, al[i], ah[i], P.Ct[size_t(i) * P.T + t]);
    if (gt) {
        a.ll += P.Mneg[t];
        a.mm += P.Mneg[t];
    }
    const uint64_t p = P.dmod[2 * t];
    const uint64_t r = redc(join3(a), p, P.dmod[2 * t + 1]);
    return P.lazy ? r : csub(r, p);
}

// Two adjacent coefficients per thread: every plan constant read from shared
// memory serves both coefficients' products (one load and one sum of halves
// instead of two), and sources and results move as 16-byte words.  The
// digits' sums of halves are formed once per digit.
struct Digits2 {
    template <int K>
    struct Of {
        uint32_t l[2][K], h[2][K], s[2][K];
    };
};

template <int K>
__device__ __forceinline__ void mixed_radix_split_pair(const ulonglong2 (&r)[K],
                                                       typename Digits2::template Of<K> &D,
                                                       bool (&gt)[2], const MontView &P) {
    gt[0] = gt[1] = false;
#pragma unroll
    for (int j = 0; j < K; j++) {
        Acc3 a0{0, 0, 0}, a1{0, 0, 0};
        const uint64_t wd = ld_plan(&P.C[size_t(j) * K + j]);
        const uint32_t dl = uint32_t(wd), dh = uint32_t(wd >> 32), ds = dl + dh;
        const uint32_t r0l = uint32_t(r[j].x) & kMask30, r0h = uint32_t(r[j].x >> 30);
        const uint32_t r1l = uint32_t(r[j].y) & kMask30, r1h = uint32_t(r[j].y >> 30);
        mac3s(a0, r0l, r0h, r0l + r0h, dl, dh, ds);
        mac3s(a1, r1l, r1h, r1l + r1h, dl, dh, ds);
#pragma unroll
        for (int i = 0; i < j; i++) {
            const uint64_t w = ld_plan(&P.C[size_t(i) * K + j]);
            const uint32_t wl = uint32_t(w), wh = uint32_t(w >> 32), ws = wl + wh;
            mac3s(a0, D.l[0][i], D.h[0][i], D.s[0][i], wl, wh, ws);
            mac3s(a1, D.l[1][i], D.h[1][i], D.s[1][i], wl, wh, ws);
        }
        const uint64_t mj = P.smod[2 * j], mq = P.smod[2 * j + 1];
        const uint64_t a0j = csub(redc(join3(a0), mj, mq), mj);
        const uint64_t a1j = csub(redc(join3(a1), mj, mq), mj);
        D.l[0][j] = uint32_t(a0j) & kMask30;
        D.h[0][j] = uint32_t(a0j >> 30);
        D.s[0][j] = D.l[0][j] + D.h[0][j];
        D.l[1][j] = uint32_t(a1j) & kMask30;
        D.h[1][j] = uint32_t(a1j >> 30);
        D.s[1][j] = D.l[1][j] + D.h[1][j];
        const uint64_t hj = P.h[j];
        if (a0j != hj) gt[0] = a0j > hj;
        if (a1j != hj) gt[1] = a1j > hj;
    }
}

template <int K>
__device__ __forceinline__ ulonglong2 eval_split_pair(const typename Digits2::template Of<K> &D,
                                                      const bool (&gt)[2], const MontView &P,
                                                      uint32_t t) {
    Acc3 a0{0, 0, 0}, a1{0, 0, 0};
#pragma unroll
    for (int i = 0; i < K; i++) {
        const uint64_t w = P.Ct[size_t(i) * P.T + t];
        const uint32_t wl = uint32_t(w), wh = uint32_t(w >> 32), ws = wl + wh;
        mac3s(a0, D.l[0][i], D.h[0][i], D.s[0][i], wl, wh, ws);
        mac3s(a1, D.l[1][i], D.h[1][i], D.s[1][i], wl, wh, ws);
    }
    const uint64_t mn = P.Mneg[t];
    if (gt[0]) {  // below 2^60 each: ll stays below 2^64
        a0.ll += mn;
        a0.mm += mn;
    }
    if (gt[1]) {
        a1.ll += mn;
        a1.mm += mn;
    }
    const uint64_t p = P.dmod[2 * t], pi = P.dmod[2 * t + 1];
    uint64_t r0 = redc(join3(a0), p, pi), r1 = redc(join3(a1), p, pi);
    if (!P.lazy) {
        r0 = csub(r0, p);
        r1 = csub(r1, p);
    }
    return make_ulonglong2(r0, r1);
}

// Targets t and t+1 for both coefficients (four independent sums).
template <int K>
__device__ __forceinline__ void eval_split_pair2(const typename Digits2::template Of<K> &D,
                                                 const bool (&gt)[2], const MontView &P,
                                                 uint32_t t, ulonglong2 &o0, ulonglong2 &o1) {
    Acc3 a0{0, 0, 0}, a1{0, 0, 0}, b0{0, 0, 0}, b1{0, 0, 0};
#pragma unroll
    for (int i = 0; i < K; i++) {
        const uint64_t w = P.Ct[size_t(i) * P.T + t], v = P.Ct[size_t(i) * P.T + t + 1];
        const uint32_t wl = uint32_t(w), wh = uint32_t(w >> 32), ws = wl + wh;
        const uint32_t vl = uint32_t(v), vh = uint32_t(v >> 32), vs = vl + vh;
        mac3s(a0, D.l[0][i], D.h[0][i], D.s[0][i], wl, wh, ws);
        mac3s(a1, D.l[1][i], D.h[1][i], D.s[1][i], wl, wh, ws);
        mac3s(b0, D.l[0][i], D.h[0][i], D.s[0][i], vl, vh, vs);
        mac3s(b1, D.l[1][i], D.h[1][i], D.s[1][i], vl, vh, vs);
    }
    const uint64_t mw = P.Mneg[t], mv = P.Mneg[t + 1];
    if (gt[0]) {  // below 2^60 each: ll stays below 2^64
        a0.ll += mw;
        a0.mm += mw;
        b0.ll += mv;
        b0.mm += mv;
    }
    if (gt[1]) {
        a1.ll += mw;
        a1.mm += mw;
        b1.ll += mv;
        b1.mm += mv;
    }
    const uint64_t p = P.dmod[2 * t], pi = P.dmod[2 * t + 1];
    const uint64_t pv = P.dmod[2 * t + 2], piv = P.dmod[2 * t + 3];
    uint64_t r0 = redc(join3(a0), p, pi), r1 = redc(join3(a1), p, pi);
    uint64_t s0 = redc(join3(b0), pv, piv), s1 = redc(join3(b1), pv, piv);
    if (!P.lazy) {
        r0 = csub(r0, p);
        r1 = csub(r1, p);
        s0 = csub(s0, pv);
        s1 = csub(s1, pv);
    }
    o0 = make_ulonglong2(r0, r1);
    o1 = make_ulonglong2(s0, s1);
}

// ================================================================== kernels

// Split-weight layout, every plan of the launch with exactly K sources, two
// adjacent coefficients per thread (128 threads cover 256 coefficients).
template <int K>
__global__ void __launch_bounds__(128, 4)
k_conv_pair(const PlanList plans, const uint64_t *__restrict__ src, size_t src_item,
            size_t src_plan, uint64_t *__restrict__ dst, size_t dst_item, size_t dst_plan,
            uint32_t log_n) {
    grid_dep_wait();
    extern __shared__ uint64_t splan[];
    const uint64_t *gp = plans.p[blockIdx.z];
    copy_plan(splan, gp, uint32_t(plan_words(gp[0])));
    __syncthreads();
    const size_t n = size_t(1) << log_n;
    const uint64_t *s = src + blockIdx.y * src_item + blockIdx.z * src_plan;
    uint64_t *d = dst + blockIdx.y * dst_item + blockIdx.z * dst_plan;
    const MontView P = mont_view(splan);
    const size_t x = 2 * (size_t(blockIdx.x) * blockDim.x + threadIdx.x);
    if (x >= n) return;
    ulonglong2 r[K];
#pragma unroll
    for (int i = 0; i < K; i++) r[i] = *reinterpret_cast<const ulonglong2 *>(s + P.src_off[i] * n + x);
    typename Digits2::template Of<K> D;
    bool gt[2];
    mixed_radix_split_pair<K>(r, D, gt, P);
    uint32_t t = 0;
    for (; t + 1 < P.T; t += 2) {
        ulonglong2 o0, o1;
        eval_split_pair2<K>(D, gt, P, t, o0, o1);
        *reinterpret_cast<ulonglong2 *>(d + P.dst_off[t] * n + x) = o0;
        *reinterpret_cast<ulonglong2 *>(d + P.dst_off[t + 1] * n + x) = o1;
    }
    if (t < P.T)
        *reinterpret_cast<ulonglong2 *>(d + P.dst_off[t] * n + x) = eval_split_pair<K>(D, gt, P, t);
}

template <int KMAX>
__device__ __forceinline__ void load_sources(uint64_t (&a)[KMAX], uint32_t k,
                                             const uint64_t *src_off, const uint64_t *s, size_t x,
                                             size_t n) {
#pragma unroll(KMAX <= 16 ? KMAX : 1)
    for (int i = 0; i < KMAX; i++) a[i] = uint32_t(i) < k ? s[src_off[i] * n + x] : 0;
}

template <int KMAX, bool MONT, bool SPLIT = false, bool EXACT = false>
__global__ void __launch_bounds__(256, 4)
k_conv(const PlanList plans, const uint64_t *__restrict__ src, size_t src_item, size_t src_plan,
       uint64_t *__restrict__ dst, size_t dst_item, size_t dst_plan, uint32_t log_n) {
    grid_dep_wait();
    extern __shared__ uint64_t splan[];
    const uint64_t *gp = plans.p[blockIdx.z];
    copy_plan(splan, gp, uint32_t(plan_words(gp[0])));
    __syncthreads();
    const size_t n = size_t(1) << log_n;
    const uint64_t *s = src + blockIdx.y * src_item + blockIdx.z * src_plan;
    uint64_t *d = dst + blockIdx.y * dst_item + blockIdx.z * dst_plan;
    if (SPLIT) {
        const MontView P = mont_view(splan);
        for (size_t x = size_t(blockIdx.x) * blockDim.x + threadIdx.x; x < n;
             x += size_t(gridDim.x) * blockDim.x) {
            uint64_t r[KMAX];
            load_sources<KMAX>(r, EXACT ? uint32_t(KMAX) : P.k, P.src_off, s, x, n);
            uint32_t al[KMAX], ah[KMAX];
            const bool gt = mixed_radix_split<KMAX, EXACT>(r, al, ah, P);
            uint32_t t = 0;
            for (; t + 1 < P.T; t += 2) {
                uint64_t r0, r1;
                eval_split2<KMAX, EXACT>(al, ah, gt, P, t, r0, r1);
                d[P.dst_off[t] * n + x] = r0;
                d[P.dst_off[t + 1] * n + x] = r1;
            }
            if (t < P.T) d[P.dst_off[t] * n + x] = eval_split<KMAX, EXACT>(al, ah, gt, P, t);
        }
    } else if (MONT) {
        const MontView P = mont_view(splan);
        for (size_t x = size_t(blockIdx.x) * blockDim.x + threadIdx.x; x < n;
             x += size_t(gridDim.x) * blockDim.x) {
            uint64_t a[KMAX];
            load_sources<KMAX>(a, P.k, P.src_off, s, x, n);
            const bool gt = mixed_radix_mont<KMAX>(a, P);
            uint32_t t = 0;
            if (!P.wrap) {
                for (; t + 1 < P.T; t += 2) {
                    uint64_t r0, r1;
                    eval_mont2<KMAX>(a, gt, P, t, r0, r1);
                    d[P.dst_off[t] * n + x] = r0;
                    d[P.dst_off[t + 1] * n + x] = r1;
                }
            }
            for (; t < P.T; t++) d[P.dst_off[t] * n + x] = eval_mont<KMAX>(a, gt, P, t);
        }
    } else {
        const ExactView P = exact_view(splan);
        for (size_t x = size_t(blockIdx.x) * blockDim.x + threadIdx.x; x < n;
             x += size_t(gridDim.x) * blockDim.x) {
            uint64_t a[KMAX];
            load_sources<KMAX>(a, P.k, P.src_off, s, x, n);
            const bool gt = mixed_radix_exact<KMAX>(a, P);
            for (uint32_t t = 0; t < P.T; t++) d[P.dst_off[t] * n + x] = eval_exact<KMAX>(a, gt, P, t);
        }
    }
}

// BFV scale-and-round: see launch_bfv_scale_round in internal.h.  Plan
// p_qb lifts [t x]_Q to B with t folded in as the source pre-multiplier and
// Q^-1 mod b_j as the target post-multiplier; its dst_off[] locate x_b
// inside the source item (nothing is written through it).  tq[2j], tq[2j+1]
// = t Q^-1 mod b_j and its Shoup quotient.  Plan p_bq lifts
// z = round(t x / Q) (centred in B) back to Q.  Both plans use the
// Montgomery layout (the host checks the bound).
template <int KQ, int KB>
__global__ void __launch_bounds__(256, 2)
k_bfv_scale_round(const uint64_t *__restrict__ p_qb, const uint64_t *__restrict__ p_bq,
                  const uint64_t *__restrict__ tq, uint32_t w_qb, uint32_t w_bq,
                  const uint64_t *__restrict__ src, size_t src_item, uint64_t *__restrict__ dst,
                  size_t dst_item, uint32_t log_n) {
    extern __shared__ uint64_t smem[];
    uint64_t *s_qb = smem, *s_bq = smem + w_qb, *s_tq = smem + w_qb + w_bq;
    copy_plan(s_qb, p_qb, w_qb);
    copy_plan(s_bq, p_bq, w_bq);
    const uint32_t nbq = uint32_t((p_qb[0] >> 16) & 0xffff);
    copy_plan(s_tq, tq, 2 * nbq);
    __syncthreads();
    const MontView A = mont_view(s_qb), B = mont_view(s_bq);
    const size_t n = size_t(1) << log_n;
    const uint64_t *s = src + blockIdx.y * src_item;
    uint64_t *d = dst + blockIdx.y * dst_item;
    for (size_t x = size_t(blockIdx.x) * blockDim.x + threadIdx.x; x < n;
         x += size_t(gridDim.x) * blockDim.x) {
        uint64_t a[KQ];
        load_sources<KQ>(a, A.k, A.src_off, s, x, n);
        const bool gt = mixed_radix_mont<KQ>(a, A);
        uint64_t z[KB];
#pragma unroll(KB <= 16 ? KB : 1)
        for (int j = 0; j < KB; j++) {
            if (uint32_t(j) < A.T) {
                // [t x]_Q Q^-1 mod b_j, and t Q^-1 x_b
                const uint64_t l = eval_mont<KQ>(a, gt, A, j);
                const uint64_t bq = A.dmod[2 * j];
                const uint64_t xb = s[A.dst_off[j] * n + x];
                const uint64_t txb = shoup(xb, s_tq[2 * j], s_tq[2 * j + 1], bq);
                z[j] = sub_mod(txb, l, bq);
            } else {
                z[j] = 0;
            }
        }
        const bool gz = mixed_radix_mont<KB>(z, B);
        for (uint32_t t = 0; t < B.T; t++) d[B.dst_off[t] * n + x] = eval_mont<KB>(z, gz, B, t);
    }
}

static int pick_kmax(uint32_t k) { return k <= 4 ? 4 : k <= 8 ? 8 : k <= 16 ? 16 : 32; }

template <bool MONT>
static void run_conv(int kmax, dim3 grid, size_t sm, cudaStream_t s, const PlanList &plans,
                     const uint64_t *src, size_t src_item, size_t src_plan, uint64_t *dst,
                     size_t dst_item, size_t dst_plan, uint32_t log_n) {
    switch (kmax) {
        case 4: launch_pdl(k_conv<4, MONT>, grid, dim3(256), sm, s, plans, src, src_item, src_plan, dst, dst_item, dst_plan, log_n); break;
        case 8: launch_pdl(k_conv<8, MONT>, grid, dim3(256), sm, s, plans, src, src_item, src_plan, dst, dst_item, dst_plan, log_n); break;
        case 16: launch_pdl(k_conv<16, MONT>, grid, dim3(256), sm, s, plans, src, src_item, src_plan, dst, dst_item, dst_plan, log_n); break;
        default: launch_pdl(k_conv<32, MONT>, grid, dim3(256), sm, s, plans, src, src_item, src_plan, dst, dst_item, dst_plan, log_n); break;
    }
}

int launch_conv(const Context &c, const PlanList &plans, const uint64_t *src, size_t src_item,
                size_t src_plan, uint64_t *dst, size_t dst_item, size_t dst_plan, uint32_t items,
                cudaStream_t s) {
    if (plans.n == 0 || items == 0) return CATFHE_OK;
    const size_t n = c.n;
    dim3 grid(unsigned((n + 255) / 256), items, plans.n);  // one coefficient per thread (fewer tail waves)
    const size_t sm = size_t(plans.words) * 8;
    if (plans.split) {
        if (plans.kmax > 8) return CATFHE_EINVAL;
        if (plans.kmin == plans.kmax && (reinterpret_cast<uintptr_t>(src) & 15) == 0 &&
            (reinterpret_cast<uintptr_t>(dst) & 15) == 0 && (src_item | src_plan | dst_item |
                                                              dst_plan) % 2 == 0 && n % 256 == 0) {
            // one source count for every plan, 16-byte aligned sources and
            // results: exact instantiation, two coefficients per thread
            const dim3 g2(unsigned(n / 256), items, plans.n);
            switch (plans.kmax) {
#define PAIRK(K)                                                                               \
    case K:                                                                                    \
        launch_pdl(k_conv_pair<K>, g2, dim3(128), sm, s, plans, src, src_item, src_plan, dst,  \
                   dst_item, dst_plan, c.log_n);                                               \
        break;
                PAIRK(1) PAIRK(2) PAIRK(3) PAIRK(4) PAIRK(5) PAIRK(6) PAIRK(7) PAIRK(8)
#undef PAIRK
                default:
                    return CATFHE_EINVAL;
            }
        } else if (plans.kmin == plans.kmax) {
            // one source count for every plan: exact instantiation
            switch (plans.kmax) {
#define EXACTK(K)                                                                              \
    case K:                                                                                    \
        launch_pdl(k_conv<K, true, true, true>, grid, dim3(256), sm, s, plans, src, src_item, src_plan, dst, \
                                                          dst_item, dst_plan, c.log_n);        \
        break;
                EXACTK(1) EXACTK(2) EXACTK(3) EXACTK(4) EXACTK(5) EXACTK(6) EXACTK(7) EXACTK(8)
#undef EXACTK
                default:
                    return CATFHE_EINVAL;
            }
        } else if (plans.kmax <= 4) {
            launch_pdl(k_conv<4, true, true>, grid, dim3(256), sm, s, plans, src, src_item, src_plan, dst,
                                                        dst_item, dst_plan, c.log_n);
        } else {
            launch_pdl(k_conv<8, true, true>, grid, dim3(256), sm, s, plans, src, src_item, src_plan, dst,
                                                        dst_item, dst_plan, c.log_n);
        }
    } else if (plans.mont)
        run_conv<true>(pick_kmax(plans.kmax), grid, sm, s, plans, src, src_item, src_plan, dst,
                       dst_item, dst_plan, c.log_n);
    else
        run_conv<false>(pick_kmax(plans.kmax), grid, sm, s, plans, src, src_item, src_plan, dst,
                        dst_item, dst_plan, c.log_n);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA;
}

// Coefficients per thread of a grid-stride launch over `items` rows of n
// coefficients, 256 threads per CTA: the count (1 to 8) whose last wave of
// CTAs is the fullest, given the resident CTAs per SM of `kernel` (more per
// thread on a tie, which spreads each CTA's plan copy over more work).  At
// N = 2^14 with 24 rows and 4 resident CTAs per SM on 152 SMs, 4 per thread
// (the fixed choice before) fills 63% of one wave; 3 per thread fills 87%.
int resident_slots(const void *kernel, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void *, int, size_t>, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    const auto key = std::make_tuple(dev, kernel, threads, smem);
    {
        std::lock_guard<std::mutex> g(mu);
        const auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    int sms = 0, occ = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) != cudaSuccess ||
        sms <= 0 || occ <= 0)
        return 0;
    std::lock_guard<std::mutex> g(mu);
    return cache[key] = sms * occ;
}

template <typename K>
static unsigned stride_columns(K kernel, size_t smem, size_t n, uint32_t items) {
    const int slots_i = resident_slots(reinterpret_cast<const void *>(kernel), 256, smem);
    if (slots_i <= 0) return unsigned((n + 1023) / 1024);
    const double slots = double(slots_i);
    double best = -1.0;
    unsigned cols = unsigned((n + 1023) / 1024);
    for (unsigned per = 1; per <= 8; per++) {
        const unsigned x = unsigned((n + 256 * per - 1) / (256 * per));
        const double waves = double(x) * items / slots;
        const double fill = waves / std::ceil(waves);
        if (fill >= best - 1e-9) {
            best = fill;
            cols = x;
        }
    }
    return cols;
}

int launch_bfv_scale_round(const Context &c, const uint64_t *q_to_b, uint32_t q_to_b_words,
                           const uint64_t *b_to_q, uint32_t b_to_q_words, const uint64_t *src,
                           size_t src_item, uint64_t *dst, size_t dst_item, uint32_t items,
                           cudaStream_t s) {
    // the t Q^-1 mod b_j pairs follow the q_to_b plan in the same allocation
    const uint64_t *tq = q_to_b + q_to_b_words;
    const size_t n = c.n;
    const uint32_t kq = uint32_t(c.L), kb = uint32_t(c.nb);
    const size_t sm = size_t(q_to_b_words + b_to_q_words + 2 * kb) * 8;
    if (kq <= 8 && kb <= 8) {
        const dim3 grid(stride_columns(k_bfv_scale_round<8, 8>, sm, n, items), items, 1);
        k_bfv_scale_round<8, 8><<<grid, 256, sm, s>>>(q_to_b, b_to_q, tq, q_to_b_words, b_to_q_words,
                                                     src, src_item, dst, dst_item, c.log_n);
    } else if (kq <= 16 && kb <= 16) {
        const dim3 grid(stride_columns(k_bfv_scale_round<16, 16>, sm, n, items), items, 1);
        k_bfv_scale_round<16, 16><<<grid, 256, sm, s>>>(q_to_b, b_to_q, tq, q_to_b_words,
                                                        b_to_q_words, src, src_item, dst, dst_item,
                                                        c.log_n);
    } else {
        const dim3 grid(stride_columns(k_bfv_scale_round<32, 32>, sm, n, items), items, 1);
        k_bfv_scale_round<32, 32><<<grid, 256, sm, s>>>(q_to_b, b_to_q, tq, q_to_b_words,
                                                        b_to_q_words, src, src_item, dst, dst_item,
                                                        c.log_n);
    }
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA;
}

}  // namespace catfhe
