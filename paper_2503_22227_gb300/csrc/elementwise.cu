// Element-wise kernels of the hot path: the fused tensor product (paper
// Sec. 3.1.4: the four products and the middle sum of a CKKS multiply in one
// kernel), the key-switching inner product, the ModDown combine, the
// automorphism X -> X^g, and ChaCha20 sampling for keys and encryption.
//
// All are HBM-bound streams over limb-major data: one thread per coefficient,
// consecutive threads on consecutive words, grids sized by the data (a whole
// batch of ciphertexts per launch).
#include <cmath>
#include "bulk.cuh"
#include "launch.cuh"
#include "modarith.cuh"

namespace catfhe {

static inline int ok() {
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA;
}

static inline dim3 coeff_grid(size_t n, uint32_t y, uint32_t z = 1) {
    return dim3(unsigned((n + 255) / 256), y, z);
}

// ------------------------------------------------------------------ tensor

__device__ __forceinline__ ulonglong2 ld2(const uint64_t *p) {
    return *reinterpret_cast<const ulonglong2 *>(p);
}
__device__ __forceinline__ void st2(uint64_t *p, uint64_t a, uint64_t b) {
    *reinterpret_cast<ulonglong2 *>(p) = make_ulonglong2(a, b);
}

// Two adjacent coefficients per thread (16-byte loads and stores).
__global__ void __launch_bounds__(256)
k_tensor(const TensorArgs A, const DevMod *__restrict__ mods, uint32_t log_n) {
    grid_dep_wait();
    const size_t n = size_t(1) << log_n;
    const size_t x = 2 * (size_t(blockIdx.x) * blockDim.x + threadIdx.x);
    const uint32_t i = blockIdx.y, item = blockIdx.z;
    if (x >= n) return;
    const DevMod m = mods[A.prime[i]];
    const uint64_t *a = A.gathered ? A.ga[item] : A.a + item * A.in_item;
    const uint64_t *b = A.gathered ? A.gb[item] : A.b + item * A.in_item;
    const size_t l0 = size_t(i) * n + x, l1 = (size_t(A.limbs) + i) * n + x;
    const ulonglong2 a0 = ld2(a + l0), a1 = ld2(a + l1), b0 = ld2(b + l0), b1 = ld2(b + l1);
    const size_t o = item * A.out_item + size_t(i) * n + x;
    // b in Montgomery form (b 2^64 mod q, in [0, 4q), one Shoup product each
    // on the approximate quotient), then one Montgomery reduction per output:
    // a b' < 4q^2 and the d1 sum < 8q^2, both below 2^64 q, so REDC returns
    // a b in [0, 2q) (measured: batched step 1438.5 -> 1435.2 us against two
    // Shoup products per 128-bit reduction)
    const uint64_t q = m.q;
    const ulonglong2 c0 = make_ulonglong2(shoup_lazy4(b0.x, m.r64, m.r64_s, q),
                                          shoup_lazy4(b0.y, m.r64, m.r64_s, q));
    const ulonglong2 c1 = make_ulonglong2(shoup_lazy4(b1.x, m.r64, m.r64_s, q),
                                          shoup_lazy4(b1.y, m.r64, m.r64_s, q));
    U128 p0{0, 0}, p1{0, 0};
    mac(p0, a0.x, c0.x);
    mac(p1, a0.y, c0.y);
    st2(A.d0 + o, csub(redc(p0, q, m.qinv), q), csub(redc(p1, q, m.qinv), q));
    U128 r0{0, 0}, r1{0, 0};
    mac(r0, a1.x, c1.x);
    mac(r1, a1.y, c1.y);
    st2(A.d2 + o, csub(redc(r0, q, m.qinv), q), csub(redc(r1, q, m.qinv), q));
    // d1 by Karatsuba: (a0 + a1)(b0' + b1') - a0 b0' - a1 b1' = a0 b1' + a1 b0',
    // one 64 x 64 product instead of two.  a0 + a1 < 2q and b0' + b1' < 8q
    // each fit one word (q < 2^61), their product (< 16 q^2) fits 128 bits,
    // and the difference is the same d1 sum as above, below 8 q^2
    U128 s0{0, 0}, s1{0, 0};
    mac(s0, a0.x + a1.x, c0.x + c1.x);
    mac(s1, a0.y + a1.y, c0.y + c1.y);
    sub128(s0, p0);
    sub128(s0, r0);
    sub128(s1, p1);
    sub128(s1, r1);
    st2(A.d1 + o, csub(redc(s0, q, m.qinv), q), csub(redc(s1, q, m.qinv), q));
}

int launch_tensor(const Context &c, const TensorArgs &a, uint32_t count, cudaStream_t s) {
    launch_pdl(k_tensor, coeff_grid(c.n / 2, a.limbs, count), dim3(256), 0, s, a, c.d_mods, c.log_n);
    return ok();
}

// ------------------------------------------------------------------ key-switch inner product

// y_p[i] = sum_j c_j[i] * key_j[p][i] (+ P * add_p[i] on ciphertext primes).
// The batch item is the fastest-varying block index, so the CTAs of all
// ciphertexts that read one block of the evaluation key are dispatched back
// to back: the key crosses HBM once per batch and is served from L2 after.
//
// Every load of a thread is issued before its first multiply (BETA is the
// exact digit count for the common small cases), so a warp keeps 2 + 3 BETA
// 16-byte loads in flight instead of stalling on each digit in turn.
template <int BETA>
__device__ __forceinline__ void ip_body(const IpArgs &A, const DevMod &m, uint32_t item,
                                        uint32_t i, size_t n, size_t x, uint32_t beta) {
    const uint32_t KL = A.L + A.K;
    const bool own_here = A.own != nullptr && i < A.level;
    const uint32_t own_digit = own_here ? i / A.alpha : 0xffffffffu;
    const uint64_t *ext = A.ext + item * A.ext_item;
    const bool fold = i < A.level && A.pfac[i] != 0;
    ulonglong2 d0 = make_ulonglong2(0, 0), d1 = make_ulonglong2(0, 0);
    if (fold && A.add0) d0 = ld2(A.add0 + item * A.add_item + size_t(i) * n + x);
    if (fold && A.add1) d1 = ld2(A.add1 + item * A.add_item + size_t(i) * n + x);
    ulonglong2 c[BETA], kb[BETA], ka[BETA];
#pragma unroll
    for (int j = 0; j < BETA; j++) {
        if (uint32_t(j) < beta) {
            c[j] = (uint32_t(j) == own_digit) ? ld2(A.own + item * A.own_item + size_t(i) * n + x)
                                              : ld2(ext + (size_t(j) * A.M + i) * n + x);
            kb[j] = ld2(A.key + ((size_t(j) * 2 + 0) * KL + A.key_limb[i]) * n + x);
            ka[j] = ld2(A.key + ((size_t(j) * 2 + 1) * KL + A.key_limb[i]) * n + x);
        }
    }
    // keys (and P) are in Montgomery form: one reduction per sum
    U128 a0{0, 0}, a1{0, 0}, b0{0, 0}, b1{0, 0};
    if (fold) {
        const uint64_t pf = A.pfac[i];
        mac(a0, d0.x, pf);
        mac(a1, d0.y, pf);
        mac(b0, d1.x, pf);
        mac(b1, d1.y, pf);
    }
#pragma unroll
    for (int j = 0; j < BETA; j++) {
        if (uint32_t(j) < beta) {
            mac(a0, c[j].x, kb[j].x);
            mac(a1, c[j].y, kb[j].y);
            mac(b0, c[j].x, ka[j].x);
            mac(b1, c[j].y, ka[j].y);
        }
    }
    uint64_t *y = A.y + item * A.y_item;
    st2(y + size_t(i) * n + x, csub(redc(a0, m.q, m.qinv), m.q), csub(redc(a1, m.q, m.qinv), m.q));
    st2(y + (size_t(A.M) + i) * n + x, csub(redc(b0, m.q, m.qinv), m.q),
        csub(redc(b1, m.q, m.qinv), m.q));
}

template <int BETA>
__global__ void __launch_bounds__(256)
k_ip(const IpArgs A, const DevMod *__restrict__ mods, uint32_t log_n) {
    grid_dep_wait();
    const size_t n = size_t(1) << log_n;
    const uint32_t item = blockIdx.x, i = blockIdx.z;
    const size_t x = 2 * (size_t(blockIdx.y) * blockDim.x + threadIdx.x);
    if (x >= n) return;
    const DevMod m = mods[A.prime[i]];
    ip_body<BETA>(A, m, item, i, n, x, A.beta);
}

// Many digits (beta > 8): digit by digit, loads interleaved with products,
// so registers stay bounded.
__global__ void __launch_bounds__(256)
k_ip_stream(const IpArgs A, const DevMod *__restrict__ mods, uint32_t log_n) {
    grid_dep_wait();
    const size_t n = size_t(1) << log_n;
    const uint32_t item = blockIdx.x, i = blockIdx.z;
    const size_t x = 2 * (size_t(blockIdx.y) * blockDim.x + threadIdx.x);
    if (x >= n) return;
    const DevMod m = mods[A.prime[i]];
    const uint32_t KL = A.L + A.K;
    const bool own_here = A.own != nullptr && i < A.level;
    const uint32_t own_digit = own_here ? i / A.alpha : 0xffffffffu;
    const uint64_t *ext = A.ext + item * A.ext_item;
    U128 a0{0, 0}, a1{0, 0}, b0{0, 0}, b1{0, 0};
    if (i < A.level && A.pfac[i] != 0) {
        if (A.add0) {
            const ulonglong2 d = ld2(A.add0 + item * A.add_item + size_t(i) * n + x);
            mac(a0, d.x, A.pfac[i]);
            mac(a1, d.y, A.pfac[i]);
        }
        if (A.add1) {
            const ulonglong2 d = ld2(A.add1 + item * A.add_item + size_t(i) * n + x);
            mac(b0, d.x, A.pfac[i]);
            mac(b1, d.y, A.pfac[i]);
        }
    }
    for (uint32_t j = 0; j < A.beta; j++) {
        const ulonglong2 c = (j == own_digit) ? ld2(A.own + item * A.own_item + size_t(i) * n + x)
                                              : ld2(ext + (size_t(j) * A.M + i) * n + x);
        const ulonglong2 kb = ld2(A.key + ((size_t(j) * 2 + 0) * KL + A.key_limb[i]) * n + x);
        const ulonglong2 ka = ld2(A.key + ((size_t(j) * 2 + 1) * KL + A.key_limb[i]) * n + x);
        mac(a0, c.x, kb.x);
        mac(a1, c.y, kb.y);
        mac(b0, c.x, ka.x);
        mac(b1, c.y, ka.y);
    }
    uint64_t *y = A.y + item * A.y_item;
    st2(y + size_t(i) * n + x, csub(redc(a0, m.q, m.qinv), m.q), csub(redc(a1, m.q, m.qinv), m.q));
    st2(y + (size_t(A.M) + i) * n + x, csub(redc(b0, m.q, m.qinv), m.q),
        csub(redc(b1, m.q, m.qinv), m.q));
}

// Inner product with bulk-copy staging: a CTA owns one extended limb i and
// a tile of kIpTile coefficients for every ciphertext of the batch.  Thread
// 0 loads the tile of the 2 BETA key rows once (bulk copies into shared
// memory) and streams each ciphertext's digit (and fold) tiles through two
// shared buffers, the next ciphertext's copies in flight while the threads
// compute on the current one; all threads then read shared memory only.
// Used when every address is 16-byte aligned (bulk-copy rule) and
// BETA <= 8; same arithmetic as k_ip, bit for bit.  Tiles of 512
// coefficients (256 threads) up to 4 digits; 256 coefficients (128 threads)
// for 5 to 8 digits, so that the 2 BETA key tiles and the two buffers
// (72 KB at BETA = 8) leave room for 3 CTAs per SM.
template <int BETA>
struct IpTile {
    static constexpr uint32_t value = BETA <= 4 ? 512 : 256;
};

// blockIdx.z: a group of consecutive ciphertexts of the launch (the host
// splits them when one group per tile would leave the last wave of CTAs
// mostly empty); each group's CTA loads its key tiles once.
template <int BETA>
__global__ void __launch_bounds__(IpTile<BETA>::value / 2)
k_ip_bulk(const IpArgs A, const DevMod *__restrict__ mods, uint32_t log_n, uint32_t count) {
    grid_dep_wait();
    const uint32_t per = (count + gridDim.z - 1) / gridDim.z;
    const uint32_t first = blockIdx.z * per;
    if (first >= count) return;  // an empty group (the whole CTA, before any barrier)
    const uint32_t nloc = count - first < per ? count - first : per;
    constexpr uint32_t kIpTile = IpTile<BETA>::value;
    extern __shared__ __align__(128) uint64_t sm[];
    __shared__ __align__(8) uint64_t bars[3];  // buffer 0, buffer 1, keys
    const size_t n = size_t(1) << log_n;
    const uint32_t i = blockIdx.y, tid = threadIdx.x;
    const size_t x0 = size_t(blockIdx.x) * kIpTile;
    const uint32_t beta = A.beta, KL = A.L + A.K;
    const DevMod m = mods[A.prime[i]];
    const bool fold = i < A.level && A.pfac[i] != 0;
    const bool f0 = fold && A.add0, f1 = fold && A.add1;
    const uint32_t own_digit = (A.own != nullptr && i < A.level) ? i / A.alpha : 0xffffffffu;
    constexpr uint32_t TB = kIpTile * 8;  // bytes per tile
    uint64_t *skey = sm;                                   // [2 BETA][tile]
    uint64_t *sbuf[2] = {sm + 2 * BETA * kIpTile, sm + (3 * BETA + 2) * kIpTile};
    const uint32_t item_bytes = (beta + (f0 ? 1 : 0) + (f1 ? 1 : 0)) * TB;

    auto issue_item = [&](uint32_t k, uint32_t b) {  // the group's k-th ciphertext
        const uint32_t item = first + k;
        uint64_t *dst = sbuf[b];
        mbar_expect_tx(&bars[b], item_bytes);
        const uint64_t *ext = A.ext + item * A.ext_item;
        for (uint32_t j = 0; j < beta; j++) {
            const uint64_t *src = (j == own_digit) ? A.own + item * A.own_item + size_t(i) * n
                                                   : ext + (size_t(j) * A.M + i) * n;
            bulk_load(dst + j * kIpTile, src + x0, TB, &bars[b]);
        }
        if (f0) bulk_load(dst + BETA * kIpTile, A.add0 + item * A.add_item + size_t(i) * n + x0, TB, &bars[b]);
        if (f1) bulk_load(dst + (BETA + 1) * kIpTile, A.add1 + item * A.add_item + size_t(i) * n + x0, TB, &bars[b]);
    };

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(&bars[2], 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_expect_tx(&bars[2], 2 * beta * TB);
        for (uint32_t j = 0; j < beta; j++) {
            bulk_load(skey + (2 * j) * kIpTile, A.key + ((size_t(j) * 2 + 0) * KL + A.key_limb[i]) * n + x0, TB, &bars[2]);
            bulk_load(skey + (2 * j + 1) * kIpTile, A.key + ((size_t(j) * 2 + 1) * KL + A.key_limb[i]) * n + x0, TB, &bars[2]);
        }
        issue_item(0, 0);
        if (nloc > 1) issue_item(1, 1);
    }
    // every wait is bounded, and the CTA decides together whether to go on
    // (__syncthreads_and), so no thread is left waiting at a barrier
    bool ok = __syncthreads_and(mbar_wait(&bars[2], 0));
    const uint32_t u = 2 * tid;  // this thread's two coefficients in the tile
    for (uint32_t k = 0; k < nloc && ok; k++) {
        const uint32_t item = first + k, b = k & 1;
        ok = __syncthreads_and(mbar_wait(&bars[b], (k >> 1) & 1));
        if (!ok) break;
        const uint64_t *buf = sbuf[b];
        U128 a0{0, 0}, a1{0, 0}, b0{0, 0}, b1{0, 0};
        if (f0) {
            const ulonglong2 d = ld2(buf + BETA * kIpTile + u);
            mac(a0, d.x, A.pfac[i]);
            mac(a1, d.y, A.pfac[i]);
        }
        if (f1) {
            const ulonglong2 d = ld2(buf + (BETA + 1) * kIpTile + u);
            mac(b0, d.x, A.pfac[i]);
            mac(b1, d.y, A.pfac[i]);
        }
#pragma unroll
        for (int j = 0; j < BETA; j++) {
            if (uint32_t(j) < beta) {
                const ulonglong2 c = ld2(buf + j * kIpTile + u);
                const ulonglong2 kb = ld2(skey + (2 * j) * kIpTile + u);
                const ulonglong2 ka = ld2(skey + (2 * j + 1) * kIpTile + u);
                mac(a0, c.x, kb.x);
                mac(a1, c.y, kb.y);
                mac(b0, c.x, ka.x);
                mac(b1, c.y, ka.y);
            }
        }
        uint64_t *y = A.y + item * A.y_item + x0 + u;
        st2(y + size_t(i) * n, csub(redc(a0, m.q, m.qinv), m.q), csub(redc(a1, m.q, m.qinv), m.q));
        st2(y + (size_t(A.M) + i) * n, csub(redc(b0, m.q, m.qinv), m.q),
            csub(redc(b1, m.q, m.qinv), m.q));
        __syncthreads();  // everyone is done with buffer b
        if (tid == 0 && k + 2 < nloc) {
            fence_proxy_async();
            issue_item(k + 2, b);
        }
    }
    if (!ok && tid == 0) {
        atomicOr(A.status, kStatusIpWait);
        // give this CTA's copies still in flight a bounded time to land
        mbar_wait(&bars[0], 0);
        mbar_wait(&bars[1], 0);
    }
}

// Watchdog self-test: a barrier that expects 16 bytes of bulk-copy data that
// no copy ever brings; the bounded wait must give up after limit_ns and the
// kernel must report it in the status word and return.
__global__ void k_wait_selftest(int *status, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_expect_tx(&bar, 16);
    const bool ok = __syncthreads_and(mbar_wait(&bar, 0, limit_ns));
    if (!ok && threadIdx.x == 0) atomicOr(status, kStatusSelfTestWait);
}

int launch_wait_selftest(const Context &c, uint64_t limit_ns, cudaStream_t s) {
    k_wait_selftest<<<1, 64, 0, s>>>(c.d_status, limit_ns);
    return ok();
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

static int launch_ip_regs(const Context &c, const IpArgs &a, uint32_t count, cudaStream_t s);

// Ciphertext groups of a bulk inner-product launch: 1 to 4, whichever fills
// the waves of CTAs best (resident CTAs per SM from the occupancy API), with
// the groups' uneven sizes counted, and only if that beats one group by 10%
// (each more group reloads its key tiles).  At N = 2^14 with 8 digits, 64
// tiles x 9 limbs at 3 CTAs per SM is 1.26 waves in one group, 2.53 in two.
template <typename K>
static unsigned ip_groups(K kernel, unsigned threads, size_t smem, size_t ctas, uint32_t count) {
    if (count < 2) return 1;
    const int slots_i = resident_slots(reinterpret_cast<const void *>(kernel), int(threads), smem);
    if (slots_i <= 0) return 1;
    const double slots = double(slots_i);
    auto score = [&](uint32_t g) {
        const double waves = double(ctas) * g / slots;
        const uint32_t per = (count + g - 1) / g;
        return waves / std::ceil(waves) * (double(count) / g / per);
    };
    unsigned best = 1;
    const double one = score(1);
    double top = one;
    for (uint32_t g = 2; g <= 4 && g <= count; g++)
        if (score(g) > top + 1e-9) {
            top = score(g);
            best = g;
        }
    return top >= 1.1 * one ? best : 1;
}

int launch_ip(const Context &c, const IpArgs &a, uint32_t count, cudaStream_t s) {
    const size_t n = c.n;
    bool bulk = a.beta <= 8 && a.status != nullptr && n % 512 == 0 && aligned16(a.ext) &&
                aligned16(a.key) && aligned16(a.y) && (!a.own || aligned16(a.own)) &&
                (!a.add0 || aligned16(a.add0)) && (!a.add1 || aligned16(a.add1)) &&
                (a.ext_item * 8) % 16 == 0 && (a.own_item * 8) % 16 == 0 &&
                (a.add_item * 8) % 16 == 0 && (a.y_item * 8) % 16 == 0;
    if (bulk) {
        switch (a.beta) {
#define IPB(B)                                                                                   \
    case B: {                                                                                    \
        constexpr uint32_t tile = IpTile<B>::value;                                              \
        const size_t smb = size_t(4 * B + 4) * tile * 8;                                         \
        if (cudaFuncSetAttribute(k_ip_bulk<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                                 int(smb)) != cudaSuccess)                                       \
            return CATFHE_ECUDA;                                                                 \
        const unsigned groups = ip_groups(k_ip_bulk<B>, tile / 2, smb, n / tile * a.M, count);   \
        launch_pdl(k_ip_bulk<B>, dim3(unsigned(n / tile), a.M, groups), dim3(tile / 2), smb, s,  \
                   a, c.d_mods, c.log_n, count);                                                 \
        break;                                                                                   \
    }
            IPB(1) IPB(2) IPB(3) IPB(4) IPB(5) IPB(6) IPB(7) IPB(8)
#undef IPB
            default: bulk = false;
        }
        if (bulk) return ok();
    }
    return launch_ip_regs(c, a, count, s);
}

static int launch_ip_regs(const Context &c, const IpArgs &a, uint32_t count, cudaStream_t s) {
    const dim3 g(count, unsigned((c.n / 2 + 255) / 256), a.M);
    switch (a.beta) {
        case 1: launch_pdl(k_ip<1>, g, dim3(256), 0, s, a, c.d_mods, c.log_n); break;
        case 2: launch_pdl(k_ip<2>, g, dim3(256), 0, s, a, c.d_mods, c.log_n); break;
        case 3: launch_pdl(k_ip<3>, g, dim3(256), 0, s, a, c.d_mods, c.log_n); break;
        case 4: launch_pdl(k_ip<4>, g, dim3(256), 0, s, a, c.d_mods, c.log_n); break;
        default:
            if (a.beta <= 8)
                launch_pdl(k_ip<8>, g, dim3(256), 0, s, a, c.d_mods, c.log_n);
            else
                launch_pdl(k_ip_stream, g, dim3(256), 0, s, a, c.d_mods, c.log_n);
    }
    return ok();
}

// ------------------------------------------------------------------ ModDown combine

// out_p[i] = (y_p[i] - lift_p[i]) * D^-1 (+ add_p[i]).
__global__ void __launch_bounds__(256)
k_combine(const CombineArgs A, const DevMod *__restrict__ mods, uint32_t log_n) {
    const size_t n = size_t(1) << log_n;
    const size_t x = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint32_t i = blockIdx.y % A.lo, p = blockIdx.y / A.lo, item = blockIdx.z;
    if (x >= n) return;
    const uint64_t q = mods[A.prime[i]].q;
    const uint64_t y = A.y[item * A.y_item + p * A.y_poly + size_t(i) * n + x];
    const uint64_t l = A.lift[item * A.lift_item + p * A.lift_poly + size_t(i) * n + x];
    uint64_t r = shoup(y + q - l, A.dinv[i], A.dinv_s[i], q);
    if (A.add) r = add_mod(r, A.add[item * A.add_item + p * A.add_poly + size_t(i) * n + x], q);
    A.out[item * A.out_item + p * A.out_poly + size_t(i) * n + x] = r;
}

int launch_combine(const Context &c, const CombineArgs &a, uint32_t count, cudaStream_t s) {
    k_combine<<<coeff_grid(c.n, 2 * a.lo, count), 256, 0, s>>>(a, c.d_mods, c.log_n);
    return ok();
}

// ------------------------------------------------------------------ automorphism

// NTT form: slot k = bitrev(i) holds a(psi^(2i+1)); sigma_g(a) there is
// a(psi^((2i+1) g)), a pure permutation of the slots.
__global__ void __launch_bounds__(256)
k_automorph_ntt(const uint64_t *__restrict__ in, uint64_t *__restrict__ out, uint64_t g,
                uint32_t log_n) {
    grid_dep_wait();
    const size_t n = size_t(1) << log_n;
    const size_t k = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint64_t mask2n = 2 * n - 1;
    const uint32_t i = __brev(uint32_t(k)) >> (32 - log_n);
    const uint64_t e = ((2 * uint64_t(i) + 1) * g) & mask2n;
    const uint32_t src = __brev(uint32_t((e - 1) >> 1)) >> (32 - log_n);
    const size_t limb = blockIdx.y;
    out[limb * n + k] = in[limb * n + src];
}

int launch_automorph_ntt(const Context &c, const uint64_t *in, uint64_t *out, uint32_t limbs_total,
                         uint64_t g, cudaStream_t s) {
    launch_pdl(k_automorph_ntt, coeff_grid(c.n, limbs_total), dim3(256), 0, s, in, out,
               uint64_t(g % (2 * c.n)), uint32_t(c.log_n));
    return ok();
}

__global__ void __launch_bounds__(256)
k_automorph_ntt_map(const uint64_t *__restrict__ in, uint64_t *__restrict__ out, const LimbMap map,
                    uint64_t g, uint32_t log_n) {
    grid_dep_wait();
    const size_t n = size_t(1) << log_n;
    const size_t k = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint32_t limb = blockIdx.y, grp = limb / map.period, r = limb % map.period;
    const uint64_t *src = in + (size_t(grp) * map.src_stride + map.src_off[r]) * n;
    uint64_t *dst = out + (size_t(grp) * map.dst_stride + map.dst_off[r]) * n;
    const uint64_t mask2n = 2 * n - 1;
    const uint32_t i = __brev(uint32_t(k)) >> (32 - log_n);
    const uint64_t e = ((2 * uint64_t(i) + 1) * g) & mask2n;
    dst[k] = src[__brev(uint32_t((e - 1) >> 1)) >> (32 - log_n)];
}

int launch_automorph_ntt_map(const Context &c, const uint64_t *in, uint64_t *out,
                             const LimbMap &map, uint32_t limbs_total, uint64_t g, cudaStream_t s) {
    if (limbs_total == 0) return CATFHE_OK;
    launch_pdl(k_automorph_ntt_map, coeff_grid(c.n, limbs_total), dim3(256), 0, s, in, out, map,
               uint64_t(g % (2 * c.n)), uint32_t(c.log_n));
    return ok();
}

// ------------------------------------------------------------------ plaintext product

__global__ void __launch_bounds__(256)
k_mul_plain(const uint64_t *__restrict__ a, const uint64_t *__restrict__ pt, uint64_t *out,
            uint32_t level, const DevMod *__restrict__ mods, uint32_t log_n) {
    const size_t n = size_t(1) << log_n;
    const size_t x = 2 * (size_t(blockIdx.x) * blockDim.x + threadIdx.x);
    if (x >= n) return;
    const uint32_t limb = blockIdx.y, i = limb % level;
    const DevMod m = mods[i];
    const ulonglong2 v = ld2(a + size_t(limb) * n + x), w = ld2(pt + size_t(i) * n + x);
    st2(out + size_t(limb) * n + x, mul_mod(v.x, w.x, m), mul_mod(v.y, w.y, m));
}

int launch_mul_plain(const Context &c, const uint64_t *a, const uint64_t *pt, uint64_t *out,
                     uint32_t level, uint32_t n_limbs, cudaStream_t s) {
    if (n_limbs == 0) return CATFHE_OK;
    k_mul_plain<<<coeff_grid(c.n / 2, n_limbs), 256, 0, s>>>(a, pt, out, level, c.d_mods, c.log_n);
    return ok();
}

// Coefficient form: out[k] = +in[i] if i g = k (mod 2N), -in[i] if i g = k + N.
__global__ void __launch_bounds__(256)
k_automorph_coeff(const uint64_t *__restrict__ in, uint64_t *__restrict__ out, const LimbMap map,
                  const DevMod *__restrict__ mods, uint64_t ginv, uint32_t log_n) {
    const size_t n = size_t(1) << log_n;
    const size_t k = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint32_t limb = blockIdx.y, g = limb / map.period, r = limb % map.period;
    const uint64_t *src = in + (size_t(g) * map.src_stride + map.src_off[r]) * n;
    uint64_t *dst = out + (size_t(g) * map.dst_stride + map.dst_off[r]) * n;
    const uint64_t q = mods[map.prime[r]].q;
    const uint64_t i1 = (uint64_t(k) * ginv) & (2 * n - 1);
    if (i1 < n) {
        dst[k] = src[i1];
    } else {
        const uint64_t v = src[i1 - n];
        dst[k] = v ? q - v : 0;
    }
}

static uint64_t inv_mod_pow2(uint64_t g, uint64_t two_n) {
    // g odd: Newton iteration for the inverse modulo a power of two
    uint64_t x = g;
    for (int i = 0; i < 6; i++) x *= 2 - g * x;
    return x & (two_n - 1);
}

int launch_automorph_coeff(const Context &c, const uint64_t *in, uint64_t *out,
                           const LimbMap &map, uint32_t n_limbs, uint64_t g, cudaStream_t s) {
    const uint64_t ginv = inv_mod_pow2(g % (2 * c.n), 2 * c.n);
    k_automorph_coeff<<<coeff_grid(c.n, n_limbs), 256, 0, s>>>(in, out, map, c.d_mods, ginv,
                                                               c.log_n);
    return ok();
}

// ------------------------------------------------------------------ simple maps

__global__ void __launch_bounds__(256)
k_add(const uint64_t *__restrict__ a, const uint64_t *__restrict__ b, uint64_t *out,
      const LimbMap map, const DevMod *__restrict__ mods, uint32_t log_n) {
    const size_t n = size_t(1) << log_n;
    const size_t x = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const uint32_t limb = blockIdx.y, g = limb / map.period, r = limb % map.period;
    const size_t o = (size_t(g) * map.src_stride + map.src_off[r]) * n + x;
    out[o] = add_mod(a[o], b[o], mods[map.prime[r]].q);
}

int launch_add(const Context &c, const uint64_t *a, const uint64_t *b, uint64_t *out,
               const LimbMap &map, uint32_t n_limbs, cudaStream_t s) {
    k_add<<<coeff_grid(c.n, n_limbs), 256, 0, s>>>(a, b, out, map, c.d_mods, c.log_n);
    return ok();
}

// out = a - b over a map (same layout for a, b, out).
__global__ void __launch_bounds__(256)
k_sub(const uint64_t *__restrict__ a, const uint64_t *__restrict__ b, uint64_t *out,
      const LimbMap map, const DevMod *__restrict__ mods, uint32_t log_n) {
    const size_t n = size_t(1) << log_n;
    const size_t x = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const uint32_t limb = blockIdx.y, g = limb / map.period, r = limb % map.period;
    const size_t o = (size_t(g) * map.src_stride + map.src_off[r]) * n + x;
    out[o] = sub_mod(a[o], b[o], mods[map.prime[r]].q);
}

int launch_sub(const Context &c, const uint64_t *a, const uint64_t *b, uint64_t *out,
               const LimbMap &map, uint32_t n_limbs, cudaStream_t s) {
    k_sub<<<coeff_grid(c.n, n_limbs), 256, 0, s>>>(a, b, out, map, c.d_mods, c.log_n);
    return ok();
}

// out = a * k_r (a constant per map entry, Shoup pair), or a + k_r on the
// entries with add_mask set (adding a constant polynomial in NTT form).
struct ConstArgs {
    uint64_t k[kMapMax], k_s[kMapMax];
    uint8_t add[kMapMax];
};

__global__ void __launch_bounds__(256)
k_const_op(const uint64_t *__restrict__ a, uint64_t *out, const LimbMap map, const ConstArgs C,
           const DevMod *__restrict__ mods, uint32_t log_n) {
    const size_t n = size_t(1) << log_n;
    const size_t x = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const uint32_t limb = blockIdx.y, g = limb / map.period, r = limb % map.period;
    const size_t o = (size_t(g) * map.src_stride + map.src_off[r]) * n + x;
    const uint64_t q = mods[map.prime[r]].q;
    out[o] = C.add[r] ? add_mod(a[o], C.k[r], q) : shoup(a[o], C.k[r], C.k_s[r], q);
}

int launch_const_op(const Context &c, const uint64_t *a, uint64_t *out, const LimbMap &map,
                    uint32_t n_limbs, const uint64_t *k, const uint64_t *k_s, const uint8_t *add,
                    cudaStream_t s) {
    ConstArgs C{};
    for (uint32_t r = 0; r < map.period; r++) {
        C.k[r] = k[r];
        C.k_s[r] = k_s[r];
        C.add[r] = add[r];
    }
    k_const_op<<<coeff_grid(c.n, n_limbs), 256, 0, s>>>(a, out, map, C, c.d_mods, c.log_n);
    return ok();
}

__global__ void __launch_bounds__(256)
k_copy(const uint64_t *__restrict__ src, uint64_t *__restrict__ dst, const LimbMap map,
       uint32_t log_n) {
    const size_t n = size_t(1) << log_n;
    const size_t x = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const uint32_t limb = blockIdx.y, g = limb / map.period, r = limb % map.period;
    dst[(size_t(g) * map.dst_stride + map.dst_off[r]) * n + x] =
        src[(size_t(g) * map.src_stride + map.src_off[r]) * n + x];
}

int launch_copy_limbs(const Context &c, const uint64_t *src, uint64_t *dst, const LimbMap &map,
                      uint32_t n_limbs, cudaStream_t s) {
    k_copy<<<coeff_grid(c.n, n_limbs), 256, 0, s>>>(src, dst, map, c.log_n);
    return ok();
}

__global__ void __launch_bounds__(256)
k_pointwise(const uint64_t *__restrict__ a, const uint64_t *__restrict__ b, uint64_t *out,
            const LimbMap map, const DevMod *__restrict__ mods, uint32_t log_n) {
    const size_t n = size_t(1) << log_n;
    const size_t x = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const uint32_t limb = blockIdx.y, g = limb / map.period, r = limb % map.period;
    const size_t ia = (size_t(g) * map.src_stride + map.src_off[r]) * n + x;
    const size_t io = (size_t(g) * map.dst_stride + map.dst_off[r]) * n + x;
    out[io] = mul_mod(a[ia], b[io], mods[map.prime[r]]);
}

// out[dst] = a[src] * b[dst] over the map
int launch_pointwise(const Context &c, const uint64_t *a, const uint64_t *b, uint64_t *out,
                     const LimbMap &map, uint32_t n_limbs, cudaStream_t s) {
    k_pointwise<<<coeff_grid(c.n, n_limbs), 256, 0, s>>>(a, b, out, map, c.d_mods, c.log_n);
    return ok();
}

// out[i] = c0[i] + c1[i] * sk[i] (or c0 - c1 sk), limbs 0..limbs-1 mod q_i.
__global__ void __launch_bounds__(256)
k_mul_add(const uint64_t *__restrict__ c0, const uint64_t *__restrict__ c1,
          const uint64_t *__restrict__ sk, uint64_t *out, int negate,
          const DevMod *__restrict__ mods, uint32_t log_n) {
    const size_t n = size_t(1) << log_n;
    const size_t x = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const uint32_t i = blockIdx.y;
    const DevMod m = mods[i];
    const size_t o = size_t(i) * n + x;
    const uint64_t prod = mul_mod(c1[o], sk[o], m);
    const uint64_t base = c0 ? c0[o] : 0;
    out[o] = negate ? sub_mod(base, prod, m.q) : add_mod(base, prod, m.q);
}

int launch_mul_add(const Context &c, const uint64_t *c0, const uint64_t *c1, const uint64_t *sk,
                   uint64_t *out, uint32_t limbs, int negate_product, cudaStream_t s) {
    k_mul_add<<<coeff_grid(c.n, limbs), 256, 0, s>>>(c0, c1, sk, out, negate_product, c.d_mods,
                                                     c.log_n);
    return ok();
}

// b[i] = -a[i] sk[i] + e[i] + pfac_i sp[i] (NTT form, limbs of Q_L u P).
__global__ void __launch_bounds__(256)
k_ksk_row(const uint64_t *__restrict__ a, const uint64_t *__restrict__ sk,
          const uint64_t *__restrict__ e, const uint64_t *__restrict__ sp, uint64_t *b,
          const uint64_t *__restrict__ pfac, const uint64_t *__restrict__ pfac_s,
          const DevMod *__restrict__ mods, uint32_t log_n) {
    const size_t n = size_t(1) << log_n;
    const size_t x = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const uint32_t i = blockIdx.y;
    const DevMod m = mods[i];
    const size_t o = size_t(i) * n + x;
    uint64_t v = sub_mod(e[o], mul_mod(a[o], sk[o], m), m.q);
    if (pfac[i]) v = add_mod(v, shoup(sp[o], pfac[i], pfac_s[i], m.q), m.q);
    b[o] = v;
}

__global__ void __launch_bounds__(256)
k_scale_limbs(uint64_t *x, uint32_t limbs, const uint64_t *__restrict__ w,
              const uint64_t *__restrict__ w_s, const DevMod *__restrict__ mods, uint32_t log_n) {
    const size_t n = size_t(1) << log_n;
    const size_t j = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t i = blockIdx.y % limbs;
    uint64_t *p = x + size_t(blockIdx.y) * n + j;
    *p = shoup(*p, w[i], w_s[i], mods[i].q);
}

int launch_scale_limbs(const Context &c, uint64_t *x, uint32_t limbs, uint32_t groups,
                       const uint64_t *w, const uint64_t *w_s, cudaStream_t s) {
    k_scale_limbs<<<coeff_grid(c.n, limbs * groups), 256, 0, s>>>(x, limbs, w, w_s, c.d_mods,
                                                                c.log_n);
    return ok();
}

int launch_ksk_row(const Context &c, const uint64_t *a, const uint64_t *sk, const uint64_t *e,
                   const uint64_t *sp, uint64_t *b, uint32_t limbs, const uint64_t *pfac,
                   const uint64_t *pfac_s, cudaStream_t s) {
    k_ksk_row<<<coeff_grid(c.n, limbs), 256, 0, s>>>(a, sk, e, sp, b, pfac, pfac_s, c.d_mods,
                                                     c.log_n);
    return ok();
}

// ------------------------------------------------------------------ sampling

__device__ __forceinline__ uint32_t rotl(uint32_t x, int r) { return (x << r) | (x >> (32 - r)); }

#define QR(a, b, c, d)                     \
    a += b; d ^= a; d = rotl(d, 16);       \
    c += d; b ^= c; b = rotl(b, 12);       \
    a += b; d ^= a; d = rotl(d, 8);        \
    c += d; b ^= c; b = rotl(b, 7);

// One ChaCha20 block (RFC 8439 Sec. 2.3): 16 output words.
__device__ __forceinline__ void chacha_block(const SampleArgs &A, uint32_t counter, uint32_t out[16]) {
    uint32_t s[16];
    s[0] = 0x61707865u; s[1] = 0x3320646eu; s[2] = 0x79622d32u; s[3] = 0x6b206574u;
#pragma unroll
    for (int i = 0; i < 8; i++) s[4 + i] = A.key[i];
    s[12] = counter; s[13] = A.tag; s[14] = A.i0; s[15] = A.i1;
    uint32_t x[16];
#pragma unroll
    for (int i = 0; i < 16; i++) x[i] = s[i];
#pragma unroll 1
    for (int r = 0; r < 10; r++) {
        QR(x[0], x[4], x[8], x[12]);
        QR(x[1], x[5], x[9], x[13]);
        QR(x[2], x[6], x[10], x[14]);
        QR(x[3], x[7], x[11], x[15]);
        QR(x[0], x[5], x[10], x[15]);
        QR(x[1], x[6], x[11], x[12]);
        QR(x[2], x[7], x[8], x[13]);
        QR(x[3], x[4], x[9], x[14]);
    }
#pragma unroll
    for (int i = 0; i < 16; i++) out[i] = x[i] + s[i];
}
#undef QR

// word w of the keystream = little-endian bytes 8w..8w+7: block w/8,
// 32-bit words 2(w%8) (low) and 2(w%8)+1 (high).
__global__ void __launch_bounds__(256)
k_sample(const SampleArgs A, uint64_t *out, const LimbMap map, const DevMod *__restrict__ mods,
         const uint64_t *__restrict__ mult, const uint64_t *__restrict__ mult_s, uint32_t n_limbs,
         uint32_t log_n) {
    const size_t n = size_t(1) << log_n;
    const size_t blk = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    uint32_t o[16];
    if (A.kind == kUniform) {
        // block b covers coefficients k = 4b .. 4b+3 (k = limb * N + j)
        if (blk * 4 >= size_t(n_limbs) * n) return;
        chacha_block(A, uint32_t(blk), o);
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const size_t k = blk * 4 + u;
            const uint32_t r = uint32_t(k / n);
            const size_t j = k % n;
            const uint64_t hi = uint64_t(o[4 * u]) | (uint64_t(o[4 * u + 1]) << 32);
            const uint64_t lo = uint64_t(o[4 * u + 2]) | (uint64_t(o[4 * u + 3]) << 32);
            const DevMod m = mods[map.prime[r % map.period]];
            const uint32_t g = r / map.period, rr = r % map.period;
            out[(size_t(g) * map.dst_stride + map.dst_off[rr]) * n + j] = reduce128(U128{lo, hi}, m);
        }
        return;
    }
    // block b covers coefficients j = 8b .. 8b+7 of the small polynomial
    if (blk * 8 >= n) return;
    chacha_block(A, uint32_t(blk), o);
    int64_t v[8];
#pragma unroll
    for (int u = 0; u < 8; u++) {
        const uint64_t w = uint64_t(o[2 * u]) | (uint64_t(o[2 * u + 1]) << 32);
        if (A.kind == kTernary) {
            v[u] = int64_t(w % 3) - 1;
        } else {
            const uint64_t low = w & ((uint64_t(1) << 40) - 1);
            int64_t mag = 0;
#pragma unroll
            for (int t = 0; t < 19; t++) mag += (low >= A.cdt[t]) ? 1 : 0;
            v[u] = (w >> 63) ? -mag : mag;
        }
    }
    for (uint32_t l = 0; l < n_limbs; l++) {
        const uint32_t g = l / map.period, rr = l % map.period;
        const DevMod m = mods[map.prime[rr]];
        uint64_t *dst = out + (size_t(g) * map.dst_stride + map.dst_off[rr]) * n + blk * 8;
#pragma unroll
        for (int u = 0; u < 8; u++) {
            uint64_t r = v[u] < 0 ? m.q - uint64_t(-v[u]) : uint64_t(v[u]);
            if (mult) r = shoup(r, mult[rr], mult_s[rr], m.q);
            dst[u] = r;
        }
    }
}

int launch_sample(const Context &c, const SampleArgs &a, uint64_t *out, const LimbMap &map,
                  uint32_t n_limbs, const uint64_t *mult, const uint64_t *mult_s,
                  cudaStream_t s) {
    size_t blocks = a.kind == kUniform ? (size_t(n_limbs) * c.n + 3) / 4 : (c.n + 7) / 8;
    k_sample<<<unsigned((blocks + 255) / 256), 256, 0, s>>>(a, out, map, c.d_mods, mult, mult_s,
                                                            n_limbs, c.log_n);
    return ok();
}

// int64 coefficients -> residues (times mult), optionally added to out.
__global__ void __launch_bounds__(256)
k_small_to_rns(const int64_t *__restrict__ in, uint64_t *out, const LimbMap map,
               const DevMod *__restrict__ mods, const uint64_t *__restrict__ mult,
               const uint64_t *__restrict__ mult_s, int accumulate, uint32_t log_n) {
    const size_t n = size_t(1) << log_n;
    const size_t x = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const uint32_t limb = blockIdx.y, g = limb / map.period, r = limb % map.period;
    const DevMod m = mods[map.prime[r]];
    const int64_t v = in[x];
    uint64_t res = v < 0 ? m.q - reduce64(uint64_t(-(v + 1)) + 1, m) : reduce64(uint64_t(v), m);
    res = csub(res, m.q);
    if (mult) res = shoup(res, mult[r], mult_s[r], m.q);
    uint64_t *o = out + (size_t(g) * map.dst_stride + map.dst_off[r]) * n + x;
    *o = accumulate ? add_mod(*o, res, m.q) : res;
}

int launch_small_to_rns(const Context &c, const int64_t *in, uint64_t *out, const LimbMap &map,
                        uint32_t n_limbs, const uint64_t *mult, const uint64_t *mult_s,
                        int accumulate, cudaStream_t s) {
    k_small_to_rns<<<coeff_grid(c.n, n_limbs), 256, 0, s>>>(in, out, map, c.d_mods, mult, mult_s,
                                                           accumulate, c.log_n);
    return ok();
}

}  // namespace catfhe
