// Integer-pipe ceilings of this device for the arithmetic the hot path is
// made of, measured by register-resident microbenchmarks (no memory traffic
// inside the timed loop): the 64-bit Shoup product by a constant, fully
// reduced (one per twiddle multiply, base-conversion weight, key product),
// and the forward NTT butterflies exactly as the transform runs them
// (butterfly.cuh): the one for primes below 2^57 (approximate-quotient
// Shoup product, the add and the subtract, no conditional subtraction; its
// words wrap modulo 2^64 after some tens of iterations here, which changes
// no instruction) and the one for larger primes (one conditional
// subtraction more, words in [0, 8q)).  These are the denominators of the
// "alu" roofline the benchmark reports.
//
// Also holds the library's kernel-launch counter.
#include <atomic>

#include "butterfly.cuh"
#include "modarith.cuh"

namespace catfhe {

static std::atomic<uint64_t> g_launches{0};
void note_launches(uint32_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
uint64_t launches_total() { return g_launches.load(std::memory_order_relaxed); }

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_peak_modmul(uint64_t *out, uint64_t q, uint64_t w,
                                                      uint64_t ws, int iters) {
    const uint64_t tid = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    uint64_t x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; j++) x[j] = (tid * 0x9E3779B97F4A7C15ull + j) % q;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int j = 0; j < kChains; j++) x[j] = shoup(x[j], w, ws, q);
    }
    uint64_t acc = 0;
#pragma unroll
    for (int j = 0; j < kChains; j++) acc ^= x[j];
    out[tid] = acc;
}

template <bool WIDE>
__global__ void __launch_bounds__(256) k_peak_bfly(uint64_t *out, uint64_t q, uint64_t w,
                                                    uint64_t ws, int iters) {
    const uint64_t tid = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    uint64_t a[kChains], b[kChains];
#pragma unroll
    for (int j = 0; j < kChains; j++) {
        a[j] = (tid * 0x9E3779B97F4A7C15ull + j) % q;
        b[j] = (tid * 0xC2B2AE3D27D4EB4Full + 3 * j) % q;
    }
    const ulonglong2 tw = make_ulonglong2(w, ws);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int j = 0; j < kChains; j++) fwd_bfly<WIDE>(a[j], b[j], tw, q);
    }
    uint64_t acc = 0;
#pragma unroll
    for (int j = 0; j < kChains; j++) acc ^= a[j] ^ b[j];
    out[tid] = acc;
}

// Rates of the single 32-bit multiply instructions the 64-bit arithmetic is
// built from, each in 8 independent chains per thread: the low product
// (mad.lo), the high product (mad.hi) and the widening product (mad.wide,
// whose 32-bit operand is the chain's own low word, so the loop issues no
// shift).  Their ratios are the multiply pipe's occupancy per instruction;
// with the counts of each kind per butterfly they bound the transform.
template <int KIND>
__global__ void __launch_bounds__(256) k_peak_imad(uint64_t *out, uint32_t c, int iters) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; j++) x[j] = tid * 7u + j + 0x80000000u;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int j = 0; j < kChains; j++) {
            if (KIND == 0) {
                uint32_t r;
                asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(uint32_t(x[j])), "r"(c), "r"(uint32_t(j)));
                x[j] = r;
            } else if (KIND == 1) {
                uint32_t r;
                asm volatile("mad.hi.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(uint32_t(x[j])), "r"(c), "r"(uint32_t(x[j])));
                x[j] = r;
            } else {
                uint64_t r;
                asm volatile("mad.wide.u32 %0, %1, %2, %3;" : "=l"(r) : "r"(uint32_t(x[j])), "r"(c), "l"(x[j]));
                x[j] = r;
            }
        }
    }
    uint64_t acc = 0;
#pragma unroll
    for (int j = 0; j < kChains; j++) acc ^= x[j];
    out[tid] = acc;
}

// Best of `reps` launches, in operations per second.
static int time_kernel(int which, cudaStream_t s, double *rate) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CATFHE_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CATFHE_ECUDA;
    const void *fn = which == 5   ? (const void *)k_peak_imad<2>
                     : which == 4 ? (const void *)k_peak_imad<1>
                     : which == 3 ? (const void *)k_peak_imad<0>
                     : which == 2 ? (const void *)k_peak_bfly<true>
                     : which == 1 ? (const void *)k_peak_bfly<false>
                                  : (const void *)k_peak_modmul;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0) != cudaSuccess)
        return CATFHE_ECUDA;
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    const size_t threads = size_t(blocks) * 256;
    const int iters = 2048;
    uint64_t *out = nullptr;
    if (cudaMalloc(&out, threads * 8) != cudaSuccess) return CATFHE_ENOMEM;
    // an odd modulus of a size each form serves: 60 bits, or 54 for the wide one
    const uint64_t q = which == 2 ? 0x3fffffffffe001ull : 0xffffffffffc0001ull;
    const uint64_t w = 0x1234567890abcdefull % q;
    const uint64_t ws = uint64_t(((unsigned __int128)w << 64) / q);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 0;
    int rc = CATFHE_OK;
    for (int rep = 0; rep < 6 && rc == CATFHE_OK; rep++) {
        cudaEventRecord(e0, s);
        if (which == 5)
            k_peak_imad<2><<<blocks, 256, 0, s>>>(out, 0x9E3779B1u, iters);
        else if (which == 4)
            k_peak_imad<1><<<blocks, 256, 0, s>>>(out, 0x9E3779B1u, iters);
        else if (which == 3)
            k_peak_imad<0><<<blocks, 256, 0, s>>>(out, 0x9E3779B1u, iters);
        else if (which == 2)
            k_peak_bfly<true><<<blocks, 256, 0, s>>>(out, q, w, ws, iters);
        else if (which == 1)
            k_peak_bfly<false><<<blocks, 256, 0, s>>>(out, q, w, ws, iters);
        else
            k_peak_modmul<<<blocks, 256, 0, s>>>(out, q, w, ws, iters);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = CATFHE_ECUDA;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        const double ops = double(threads) * iters * kChains;
        if (rep > 0 && ms > 0) best = std::max(best, ops / (ms * 1e-3));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    *rate = best;
    return rc;
}

int measure_int_peak(double *modmul_per_s, double *bfly_per_s, double *bfly_wide_per_s,
                     cudaStream_t s) {
    int rc = CATFHE_OK;
    if (modmul_per_s) rc = time_kernel(0, s, modmul_per_s);
    if (rc == CATFHE_OK && bfly_per_s) rc = time_kernel(1, s, bfly_per_s);
    if (rc == CATFHE_OK && bfly_wide_per_s) rc = time_kernel(2, s, bfly_wide_per_s);
    return rc;
}

int measure_imad_rates(double *lo_per_s, double *hi_per_s, double *wide_per_s, cudaStream_t s) {
    int rc = CATFHE_OK;
    if (lo_per_s) rc = time_kernel(3, s, lo_per_s);
    if (rc == CATFHE_OK && hi_per_s) rc = time_kernel(4, s, hi_per_s);
    if (rc == CATFHE_OK && wide_per_s) rc = time_kernel(5, s, wide_per_s);
    return rc;
}

}  // namespace catfhe
