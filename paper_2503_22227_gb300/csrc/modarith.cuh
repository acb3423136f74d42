// Modular arithmetic on 64-bit words for moduli q < 2^62 (device side).
//
// Products by a constant use Shoup's method: with w' = floor(w 2^64 / q),
// a*w - floor(a*w' / 2^64)*q lies in [0, 2q) for every 64-bit a.  Sums of
// products are accumulated exactly in 128 bits and reduced once: a 128-bit
// x = hi 2^64 + lo is congruent to hi*(2^64 mod q) + lo*1, both terms by
// Shoup, so the reduction needs only precomputed per-modulus constants.
#pragma once

#include <stdint.h>

#include "internal.h"

namespace catfhe {

__device__ __forceinline__ uint64_t mulhi(uint64_t a, uint64_t b) { return __umul64hi(a, b); }

__device__ __forceinline__ uint64_t csub(uint64_t x, uint64_t q) { return x >= q ? x - q : x; }

// Waits for the previous kernel on the stream (launches with programmatic
// dependent launch, launch.cuh); a no-op for ordinary launches.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ uint64_t add_mod(uint64_t a, uint64_t b, uint64_t q) {
    return csub(a + b, q);
}

__device__ __forceinline__ uint64_t sub_mod(uint64_t a, uint64_t b, uint64_t q) {
    return csub(a + q - b, q);
}

// The low 64 bits of a*w + e*n, as 32-bit multiply-adds: the low words'
// product widened, the second one accumulated onto it, then the four cross
// products into the high word.  Writing it out this way (instead of two
// 64-bit products and an add in C++) took the forward butterfly's
// multiply-pipe instructions from 11.8 to 10.1 and its rate from 1.05e12 to
// 1.20e12 per second on GB300 (ncu counts of a register-resident loop; the
// words are the same bit for bit).
__device__ __forceinline__ uint64_t lo_mul2(uint64_t a, uint64_t w, uint64_t e, uint64_t n) {
    uint64_t t;
    asm("{\n\t"
        ".reg .u32 a0, a1, w0, w1, e0, e1, n0, n1, t0, t1;\n\t"
        ".reg .u64 x;\n\t"
        "mov.b64 {a0, a1}, %1;\n\t"
        "mov.b64 {w0, w1}, %2;\n\t"
        "mov.b64 {e0, e1}, %3;\n\t"
        "mov.b64 {n0, n1}, %4;\n\t"
        "mul.wide.u32 x, a0, w0;\n\t"
        "mad.wide.u32 x, e0, n0, x;\n\t"
        "mov.b64 {t0, t1}, x;\n\t"
        "mad.lo.u32 t1, a0, w1, t1;\n\t"
        "mad.lo.u32 t1, a1, w0, t1;\n\t"
        "mad.lo.u32 t1, e0, n1, t1;\n\t"
        "mad.lo.u32 t1, e1, n0, t1;\n\t"
        "mov.b64 %0, {t0, t1};\n\t"
        "}"
        : "=l"(t)
        : "l"(a), "l"(w), "l"(e), "l"(n));
    return t;
}

// a*w mod q in [0, 2q); any 64-bit a, w < q, ws = floor(w 2^64 / q).
// Computed as a*w + floor(a ws / 2^64) * (2^64 - q) modulo 2^64.
__device__ __forceinline__ uint64_t shoup_lazy(uint64_t a, uint64_t w, uint64_t ws, uint64_t q) {
    return lo_mul2(a, w, mulhi(a, ws), 0 - q);
}

// floor(a b / 2^64) - e with e in {0, 1, 2}.  With a = a1 2^32 + a0 and
// b = b1 2^32 + b0, a b / 2^64 = a1 b1 + hi(a1 b0) + hi(a0 b1) + R / 2^64
// where R = (lo(a1 b0) + lo(a0 b1)) 2^32 + a0 b0 < 3 * 2^64; R is dropped.
// Two 32-bit high products and one widening multiply-add, against the
// exact high product's four partial products and their carries.
__device__ __forceinline__ uint64_t mulhi_approx(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("{\n\t"
        ".reg .u32 a0, a1, b0, b1, h1, h2, s, c;\n\t"
        ".reg .u64 t;\n\t"
        "mov.b64 {a0, a1}, %1;\n\t"
        "mov.b64 {b0, b1}, %2;\n\t"
        "mul.hi.u32 h1, a1, b0;\n\t"
        "mul.hi.u32 h2, a0, b1;\n\t"
        "add.cc.u32 s, h1, h2;\n\t"
        "addc.u32 c, 0, 0;\n\t"
        "mov.b64 t, {s, c};\n\t"
        "mad.wide.u32 %0, a1, b1, t;\n\t"
        "}"
        : "=l"(r)
        : "l"(a), "l"(b));
    return r;
}

// a*w mod q in [0, 4q); any 64-bit a, w < q, ws = floor(w 2^64 / q).  The
// quotient estimate is at most 2 below Shoup's, whose remainder is in
// [0, 2q); the subtraction is exact modulo 2^64 since the result is < 2^64.
__device__ __forceinline__ uint64_t shoup_lazy4(uint64_t a, uint64_t w, uint64_t ws, uint64_t q) {
    return lo_mul2(a, w, mulhi_approx(a, ws), 0 - q);
}

__device__ __forceinline__ uint64_t shoup(uint64_t a, uint64_t w, uint64_t ws, uint64_t q) {
    return csub(shoup_lazy(a, w, ws, q), q);
}

struct U128 {
    uint64_t lo, hi;
};

// acc += a * b (full 128-bit product) as 32-bit multiply-adds on a four-word
// carry chain (measured faster than the 64-bit mad.lo.cc / madc.hi pair).
__device__ __forceinline__ void mac(U128 &acc, uint64_t a, uint64_t b) {
    asm("{\n\t"
        ".reg .u32 a0, a1, b0, b1, r0, r1, r2, r3;\n\t"
        "mov.b64 {a0, a1}, %2;\n\t"
        "mov.b64 {b0, b1}, %3;\n\t"
        "mov.b64 {r0, r1}, %0;\n\t"
        "mov.b64 {r2, r3}, %1;\n\t"
        "mad.lo.cc.u32 r0, a0, b0, r0;\n\t"
        "madc.hi.cc.u32 r1, a0, b0, r1;\n\t"
        "madc.lo.cc.u32 r2, a1, b1, r2;\n\t"
        "madc.hi.u32 r3, a1, b1, r3;\n\t"
        "mad.lo.cc.u32 r1, a0, b1, r1;\n\t"
        "madc.hi.cc.u32 r2, a0, b1, r2;\n\t"
        "addc.u32 r3, r3, 0;\n\t"
        "mad.lo.cc.u32 r1, a1, b0, r1;\n\t"
        "madc.hi.cc.u32 r2, a1, b0, r2;\n\t"
        "addc.u32 r3, r3, 0;\n\t"
        "mov.b64 %0, {r0, r1};\n\t"
        "mov.b64 %1, {r2, r3};\n\t"
        "}"
        : "+l"(acc.lo), "+l"(acc.hi)
        : "l"(a), "l"(b));
}

// a -= b on 128 bits (a >= b).
__device__ __forceinline__ void sub128(U128 &a, const U128 &b) {
    asm("sub.cc.u64 %0, %0, %2;\n\t"
        "subc.u64 %1, %1, %3;"
        : "+l"(a.lo), "+l"(a.hi)
        : "l"(b.lo), "l"(b.hi));
}

// Exact x mod q for any 128-bit x.
__device__ __forceinline__ uint64_t reduce128(U128 x, const DevMod &m) {
    uint64_t r = shoup_lazy(x.hi, m.r64, m.r64_s, m.q) + shoup_lazy(x.lo, 1, m.one_s, m.q);
    r = csub(r, 2 * m.q);
    return csub(r, m.q);
}

// Montgomery reduction of acc < 2^64 q: acc 2^-64 mod q, in [0, 2q)
// (u = lo (-q^-1) mod 2^64 makes acc + u q divisible by 2^64).
__device__ __forceinline__ uint64_t redc(U128 acc, uint64_t q, uint64_t qinv) {
    const uint64_t u = acc.lo * qinv;
    return acc.hi + mulhi(u, q) + (acc.lo != 0 ? 1 : 0);
}

// ------------------------------------------------------------ split products
// Sums of products of words below 2^60, each split into 30-bit halves
// x = xh 2^30 + xl: the sum is ll + mm 2^30 + hh 2^60 with
//   ll = sum xl wl,  mm = sum (xl wh + xh wl),  hh = sum xh wh.
// The middle sum is formed by Karatsuba's identity: the accumulators hold
// ll, kk = sum (xl + xh)(wl + wh) and hh, three 32 x 32 -> 64-bit
// multiply-adds per product; kk may wrap modulo 2^64, but when mm is below
// 2^64 (the caller's bound) the difference kk - ll - hh taken modulo 2^64 is
// mm exactly.  A widening multiply-add occupies the integer multiply pipe
// as long as a 32-bit high product, so three of them cost less than the
// four low and four high products of mac() (measured per instruction on
// GB300: 2 pipe cycles per 32-bit low product, 4 per high or widening one).
// The conversions use them; in the HBM-bound inner product and tensor the
// extra splitting and joining measured slower (inner product 162 -> 172 us,
// tensor 122 -> 123 us per batched step).
struct Acc3 {
    uint64_t ll, mm, hh;  // mm holds kk until join3
};

// Three 32 x 32 -> 64-bit multiply-adds, written as PTX mad.wide.u32 (the
// four-product form in C++ measured slower than in PTX, 1788 vs 1743 us per
// batched step; Karatsuba's three products: 1498 -> 1488 us).  The sums of
// halves are below 2^31.
__device__ __forceinline__ void mac3(Acc3 &a, uint32_t xl, uint32_t xh, uint64_t w) {
    const uint32_t wl = uint32_t(w), wh = uint32_t(w >> 32);
    asm("{\n\t.reg .u32 xs, ws;\n\t"
        "add.u32 xs, %3, %4;\n\t"
        "add.u32 ws, %5, %6;\n\t"
        "mad.wide.u32 %0, %3, %5, %0;\n\t"
        "mad.wide.u32 %1, xs, ws, %1;\n\t"
        "mad.wide.u32 %2, %4, %6, %2;\n\t}"
        : "+l"(a.ll), "+l"(a.mm), "+l"(a.hh)
        : "r"(xl), "r"(xh), "r"(wl), "r"(wh));
}

// mac3 with both sums of halves (xs = xl + xh, ws = wl + wh) computed by the
// caller, once per digit and once per constant, when each serves several
// products.
__device__ __forceinline__ void mac3s(Acc3 &a, uint32_t xl, uint32_t xh, uint32_t xs, uint32_t wl,
                                      uint32_t wh, uint32_t ws) {
    asm("{\n\t"
        "mad.wide.u32 %0, %3, %6, %0;\n\t"
        "mad.wide.u32 %1, %5, %8, %1;\n\t"
        "mad.wide.u32 %2, %4, %7, %2;\n\t}"
        : "+l"(a.ll), "+l"(a.mm), "+l"(a.hh)
        : "r"(xl), "r"(xh), "r"(xs), "r"(wl), "r"(wh), "r"(ws));
}

// ll + mm 2^30 + hh 2^60 as 128 bits, mm recovered from kk first.  A term
// added to ll after the products (the folded -M of the centring) is added to
// kk too, so that the difference is unchanged.
__device__ __forceinline__ U128 join3(const Acc3 &a0) {
    Acc3 a = a0;
    a.mm = a0.mm - a0.ll - a0.hh;
    U128 x;
    asm("add.cc.u64 %0, %2, %3;\n\t"
        "addc.u64 %1, %4, 0;"
        : "=l"(x.lo), "=l"(x.hi)
        : "l"(a.ll), "l"(a.mm << 30), "l"(a.mm >> 34));
    asm("add.cc.u64 %0, %0, %2;\n\t"
        "addc.u64 %1, %1, %3;"
        : "+l"(x.lo), "+l"(x.hi)
        : "l"(a.hh << 60), "l"(a.hh >> 4));
    return x;
}

constexpr uint32_t kMask30 = (1u << 30) - 1;

// a*b mod q for a, b < 2^64 (exact).
__device__ __forceinline__ uint64_t mul_mod(uint64_t a, uint64_t b, const DevMod &m) {
    U128 x{a * b, mulhi(a, b)};
    return reduce128(x, m);
}

// x mod q for any 64-bit x.
__device__ __forceinline__ uint64_t reduce64(uint64_t x, const DevMod &m) {
    return csub(shoup_lazy(x, 1, m.one_s, m.q), m.q);
}

}  // namespace catfhe
