// NTT butterflies (device side), shared by the transform kernels and the
// integer-pipe ceiling microbenchmark so that both run the same instructions.
//
// Lazy reduction after Harvey ("Faster arithmetic for number-theoretic
// transforms", 2014), on Shoup products whose quotient estimate skips the
// low partial products (shoup_lazy4, result in [0, 4q)).  Every prime of a
// context is below 2^61, so 8q < 2^64:
//  - forward (Cooley-Tukey): words in [0, 8q) between stages, one
//    conditional subtraction of 4q per butterfly;
//  - forward for q < 2^57 ("wide"): no conditional subtraction at all; the
//    bound grows by 4q per stage, from below 4q to below 68q after 16
//    stages, which a 64-bit word still holds;
//  - inverse (Gentleman-Sande): words in [0, 4q), one conditional
//    subtraction of 4q per butterfly.
// The last stage of each transform reduces fully to [0, q).
#pragma once

#include "modarith.cuh"

namespace catfhe {

constexpr uint64_t kWideBound = uint64_t(1) << 57;

// a, b in [0, 8q) -> a + b w, a - b w (+4q), both in [0, 8q)
__device__ __forceinline__ void ct_bfly(uint64_t &a, uint64_t &b, ulonglong2 w, uint64_t q) {
    const uint64_t q4 = 4 * q;
    const uint64_t x = csub(a, q4);                  // [0, 4q)
    const uint64_t t = shoup_lazy4(b, w.x, w.y, q);  // [0, 4q)
    a = x + t;                                       // [0, 8q)
    b = x + q4 - t;                                  // (0, 8q)
}

// q < 2^57: no conditional subtraction; each output is below max(a) + 4q
__device__ __forceinline__ void ct_bfly_wide(uint64_t &a, uint64_t &b, ulonglong2 w, uint64_t q) {
    const uint64_t t = shoup_lazy4(b, w.x, w.y, q);  // [0, 4q)
    const uint64_t a0 = a;
    a = a0 + t;
    b = a0 + 4 * q - t;
}

template <bool WIDE>
__device__ __forceinline__ void fwd_bfly(uint64_t &a, uint64_t &b, ulonglong2 w, uint64_t q) {
    if (WIDE)
        ct_bfly_wide(a, b, w, q);
    else
        ct_bfly(a, b, w, q);
}

// a, b in [0, 4q) -> a + b, (a - b) w, both in [0, 4q)
__device__ __forceinline__ void gs_bfly(uint64_t &a, uint64_t &b, ulonglong2 w, uint64_t q) {
    const uint64_t q4 = 4 * q;
    const uint64_t a0 = a, b0 = b;
    a = csub(a0 + b0, q4);
    b = shoup_lazy4(a0 + q4 - b0, w.x, w.y, q);
}

}  // namespace catfhe
