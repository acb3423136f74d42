// Batched negacyclic NTT / inverse NTT over 64-bit primes (paper Sec.
// 3.1.3, the butterfly NTT "NTT_BM"), for N = 2^12 .. 2^16.
//
// Definition: out[bitrev(i)] = sum_j a_j psi^((2i+1) j) mod q.  Computed by
// Cooley-Tukey butterflies with twiddles psi^bitrev(m + i) at stage
// log2(m) (Gentleman-Sande with inverse twiddles for the inverse, N^-1
// folded into its last stage).
//
// GB300 layout.  A limb of N = 2^16 words is 512 KiB, more than one CTA's
// shared memory, so every transform is two passes over HBM:
//  - column pass: the first k1 stages only mix the 2^k1 elements that
//    share their low log N - k1 index bits (a strided "column"); a CTA
//    loads CW adjacent columns (coalesced rows of CW words) and runs the
//    k1 stages;
//  - row pass: the remaining k2 = log N - k1 stages act inside contiguous
//    chunks of 2^k2 words; a CTA loads several chunks.
// Inside a pass every thread holds E = 2^LOGE words in registers and runs
// LOGE stages on them without synchronisation; one shared-memory exchange
// regroups the words for the remaining (<= LOGE) stages.  The grid spans
// every limb of the batch (blockIdx.y), so one launch covers a whole batch
// of ciphertexts: no per-modulus kernels or streams (the paper's kernel
// segmentation, Sec. 3.1.4, is replaced by batching).
#include "bulk.cuh"
#include "butterfly.cuh"
#include "launch.cuh"
#include "modarith.cuh"

namespace catfhe {

// [0, 8q) -> [0, q)
__device__ __forceinline__ uint64_t reduce8(uint64_t x, uint64_t q) {
    return csub(csub(csub(x, 4 * q), 2 * q), q);
}

// Any word below 2^64 -> [0, q) (Shoup product by 1, then one subtraction).
__device__ __forceinline__ uint64_t reduce_any(uint64_t x, const DevMod &m) {
    return csub(shoup_lazy(x, 1, m.one_s, m.q), m.q);
}

// Limb of this CTA: group g (ciphertext or polynomial) and position r within
// the map's period.  PRIME_MAJOR (used by the forward transform, where it
// measured faster; the inverse is faster the other way): when the launch
// covers whole groups, consecutive blockIdx.y walk over the groups at one
// position (one prime), so the CTAs that read one prime's twiddle table run
// back to back and find it in L2.
template <bool PRIME_MAJOR>
__device__ __forceinline__ void limb_of(const LimbMap &map, uint32_t &g, uint32_t &r) {
    const uint32_t y = blockIdx.y, Y = gridDim.y;
    if (PRIME_MAJOR && Y % map.period == 0) {
        const uint32_t G = Y / map.period;
        g = y % G;
        r = y / G;
    } else {
        g = y / map.period;
        r = y % map.period;
    }
}

// (tau E + v) >> sh for 0 <= v < E = 2^LOGE: with v and sh known at compile
// time (unrolled loops) this folds to one shift of tau (and an OR).  Twiddle
// indexes stay in 32 bits (N <= 2^16).
template <int LOGE>
__device__ __forceinline__ uint32_t hi_bits(uint32_t tau, int v, int sh) {
    return sh >= LOGE ? (tau >> (sh - LOGE)) : ((tau << (LOGE - sh)) | uint32_t(v >> sh));
}

// ------------------------------------------------------------------ forward

template <int LOGR, int LOGE, bool WIDE>
__device__ __forceinline__ void fwd_cols_body(uint64_t (&x)[1 << LOGE], uint64_t *sm,
                                              const ulonglong2 *w, uint64_t q, int cl, int tau) {
    constexpr int R = 1 << LOGR, E = 1 << LOGE, T = R / E, CW = 256 / T;
    // stages 0 .. LOGE-1: partners at distance T*half are in this thread
#pragma unroll
    for (int st = 0; st < LOGE; st++) {
        const int half = E >> (st + 1);
#pragma unroll
        for (int v = 0; v < E; v++) {
            if (v & half) continue;
            fwd_bfly<WIDE>(x[v], x[v + half], w[(1 << st) + (v >> (LOGE - st))], q);
        }
    }
#pragma unroll
    for (int v = 0; v < E; v++) sm[(tau + T * v) * CW + cl] = x[v];
    __syncthreads();
#pragma unroll
    for (int v = 0; v < E; v++) x[v] = sm[(tau * E + v) * CW + cl];
    // stages LOGE .. LOGR-1: partners at distance < E
#pragma unroll
    for (int st = LOGE; st < LOGR; st++) {
        const int dist = 1 << (LOGR - 1 - st);
#pragma unroll
        for (int v = 0; v < E; v++) {
            if (v & dist) continue;
            const uint32_t idx = (1u << st) + hi_bits<LOGE>(uint32_t(tau), v, LOGR - st);
            fwd_bfly<WIDE>(x[v], x[v + dist], w[idx], q);
        }
    }
}

template <int LOGR, int LOGE>
__global__ void __launch_bounds__(256)
k_ntt_fwd_cols(const uint64_t *src, uint64_t *dst, const LimbMap map,
               const DevMod *__restrict__ mods, const ulonglong2 *__restrict__ tw, int log_n) {
    grid_dep_wait();
    constexpr int R = 1 << LOGR, E = 1 << LOGE, T = R / E, CW = 256 / T;
    __shared__ uint64_t sm[R * CW];
    uint32_t g, r;
    limb_of<true>(map, g, r);
    const size_t N = size_t(1) << log_n;
    const size_t S = N >> LOGR;
    const uint64_t *in = src + (size_t(g) * map.src_stride + map.src_off[r]) * N;
    uint64_t *out = dst + (size_t(g) * map.dst_stride + map.dst_off[r]) * N;
    const int p = map.prime[r];
    const uint64_t q = mods[p].q;
    const ulonglong2 *wg = tw + size_t(p) * N;
    const int cl = threadIdx.x % CW, tau = threadIdx.x / CW;
    const size_t c = size_t(blockIdx.x) * CW + cl;
    const uint32_t TS = uint32_t(T * S), SS = uint32_t(S);
    const uint64_t *ip = in + c + size_t(tau) * S;
    uint64_t *op = out + c + size_t(tau) * E * S;

    uint64_t x[E];
#pragma unroll
    for (int v = 0; v < E; v++) x[v] = ip[uint32_t(v) * TS];
    // the column stages use twiddles 1 .. R-1 only: staged in shared memory
    // once per CTA, after the data loads are issued (measured: forward 284 ->
    // 278 us, inverse 298 -> 294 us for 384 limbs)
    __shared__ ulonglong2 stw[R];
    for (int i = threadIdx.x; i < R; i += 256) stw[i] = wg[i];
    __syncthreads();
    const ulonglong2 *w = stw;
    // q < 2^57: no conditional subtractions; words leave below 4q + 4 LOGR q
    // (else below 8q) and the row pass reduces them after its stages
    if (q < kWideBound)
        fwd_cols_body<LOGR, LOGE, true>(x, sm, w, q, cl, tau);
    else
        fwd_cols_body<LOGR, LOGE, false>(x, sm, w, q, cl, tau);
#pragma unroll
    for (int v = 0; v < E; v++) op[uint32_t(v) * SS] = x[v];
}

template <int LOGR, int LOGE, bool WIDE>
__device__ __forceinline__ void fwd_rows_body(uint64_t (&x)[1 << LOGE], uint64_t *s,
                                              const ulonglong2 *w, uint64_t q, int k1, uint32_t h,
                                              int tau) {
    constexpr int R = 1 << LOGR, E = 1 << LOGE, T = R / E;
#define PAD(u) ((u) + ((u) >> LOGE))
#pragma unroll
    for (int st = 0; st < LOGE; st++) {
        const int half = E >> (st + 1);
        const uint32_t base = (1u << (k1 + st)) + (h << st);
#pragma unroll
        for (int v = 0; v < E; v++) {
            if (v & half) continue;
            fwd_bfly<WIDE>(x[v], x[v + half], w[base + uint32_t(v >> (LOGE - st))], q);
        }
    }
#pragma unroll
    for (int v = 0; v < E; v++) s[PAD(tau + T * v)] = x[v];
    __syncthreads();
#pragma unroll
    for (int v = 0; v < E; v++) x[v] = s[PAD(tau * E + v)];
#pragma unroll
    for (int st = LOGE; st < LOGR; st++) {
        const int dist = 1 << (LOGR - 1 - st);
        const uint32_t base = (1u << (k1 + st)) + (h << st);
#pragma unroll
        for (int v = 0; v < E; v++) {
            if (v & dist) continue;
            const uint32_t idx = base + hi_bits<LOGE>(uint32_t(tau), v, LOGR - st);
            fwd_bfly<WIDE>(x[v], x[v + dist], w[idx], q);
        }
    }
#undef PAD
}

// EPI: 0, the plain transform; 1, the ModDown combine epilogue with its y
// words loaded into registers before the butterflies; 2, the same epilogue
// with the CTA's y tile (its CC chunks of R words are contiguous) brought
// into shared memory by one bulk copy issued before the butterflies, so that
// no registers are held for it (y 16-byte aligned and a status word, checked
// on the host; the dynamic shared memory holds 256 E words).
template <int LOGR, int LOGE, int EPI>
__global__ void __launch_bounds__(256, 3)
k_ntt_fwd_rows(uint64_t *__restrict__ data, const LimbMap map, const DevMod *__restrict__ mods,
               const ulonglong2 *__restrict__ tw, int log_n, const NttEpilogue epi) {
    grid_dep_wait();
    constexpr int R = 1 << LOGR, E = 1 << LOGE, T = R / E, CC = 256 / T;
    constexpr int RP = R + R / E;
    __shared__ uint64_t sm[CC * RP];
    extern __shared__ __align__(16) uint64_t ytile[];
    __shared__ __align__(8) uint64_t ybar;
    uint32_t g, r;
    limb_of<true>(map, g, r);
    const size_t N = size_t(1) << log_n;
    uint64_t *out = data + (size_t(g) * map.dst_stride + map.dst_off[r]) * N;
    const int p = map.prime[r];
    const DevMod m = mods[p];
    const uint64_t q = m.q;
    const ulonglong2 *w = tw + size_t(p) * N;
    const int k1 = log_n - LOGR;
    const int chl = threadIdx.x / T, tau = threadIdx.x % T;
    const uint32_t h = blockIdx.x * CC + chl;
    uint64_t *base = out + size_t(h) * R;
    uint64_t *s = sm + chl * RP;
#define PAD(u) ((u) + ((u) >> LOGE))

    uint64_t x[E];
#pragma unroll
    for (int v = 0; v < E; v++) x[v] = base[tau + T * v];
    // combine epilogue: its y words are requested before the butterflies, so
    // the loads overlap them (measured, in registers: 1648 -> 1613 us per
    // batched step).  The barrier is initialised and the copy issued by the
    // same thread; the others reach the barrier after the exchange's
    // __syncthreads.
    uint64_t yv[EPI == 1 ? E : 1];
    if (EPI == 1) {
        const uint64_t *yp0 = epi.y + (size_t(g) * epi.y_stride + epi.y_off[r]) * N + size_t(h) * R;
#pragma unroll
        for (int v = 0; v < E; v++) yv[EPI == 1 ? v : 0] = yp0[tau + T * v];
    } else if (EPI == 2 && threadIdx.x == 0) {
        constexpr uint32_t bytes = uint32_t(CC) * R * 8;
        mbar_init(&ybar, 1);
        mbar_init_fence();
        mbar_expect_tx(&ybar, bytes);
        bulk_load(ytile,
                  epi.y + (size_t(g) * epi.y_stride + epi.y_off[r]) * N +
                      size_t(blockIdx.x) * CC * R,
                  bytes, &ybar);
    }
    // q < 2^57: no conditional subtractions in either pass, words stay below
    // 4q + 4 log2(N) q <= 68q < 2^64, then one Shoup reduction; else below
    // 8q, then three conditional subtractions.  (Each branch with its own
    // reduction, and 3 CTAs per SM: fewer register spills, measured
    // forward transform 297 -> 284 us.)
    if (q < kWideBound) {
        fwd_rows_body<LOGR, LOGE, true>(x, s, w, q, k1, h, tau);
#pragma unroll
        for (int v = 0; v < E; v++) s[PAD(tau * E + v)] = reduce_any(x[v], m);
    } else {
        fwd_rows_body<LOGR, LOGE, false>(x, s, w, q, k1, h, tau);
#pragma unroll
        for (int v = 0; v < E; v++) s[PAD(tau * E + v)] = reduce8(x[v], q);
    }
    __syncthreads();
    if (EPI == 0) {
#pragma unroll
        for (int v = 0; v < E; v++) base[tau + T * v] = s[PAD(tau + T * v)];
    } else {
        // a bounded wait that the CTA decides together (__syncthreads_and)
        if (EPI == 2 && !__syncthreads_and(mbar_wait(&ybar, 0))) {
            if (threadIdx.x == 0) {
                atomicOr(epi.status, kStatusNttWait);
                mbar_wait(&ybar, 0);  // a bounded time for the copy to land
            }
            return;
        }
        // ModDown combine: out = (y - lift) * D^-1 (+ add), lift now in NTT form
        const size_t off = size_t(h) * R;
        uint64_t *op = (epi.gathered ? epi.gout[g] : epi.out + size_t(g) * epi.out_stride * N) +
                       size_t(epi.out_off[r]) * N + off;
        const uint64_t *ap =
            epi.add ? epi.add + (size_t(g) * epi.add_stride + epi.add_off[r]) * N + off : nullptr;
        const uint64_t dv = epi.dinv[r], dvs = epi.dinv_s[r];
#pragma unroll
        for (int v = 0; v < E; v++) {
            const int u = tau + T * v;
            const uint64_t yw = EPI == 2 ? ytile[chl * R + u] : yv[EPI == 1 ? v : 0];
            uint64_t o = shoup(yw + q - s[PAD(u)], dv, dvs, q);
            if (ap) o = add_mod(o, ap[u], q);
            op[u] = o;
        }
    }
#undef PAD
}

// ------------------------------------------------------------------ inverse

template <int LOGR, int LOGE>
__global__ void __launch_bounds__(256)
k_ntt_inv_rows(const uint64_t *src, uint64_t *dst, const LimbMap map,
               const DevMod *__restrict__ mods, const ulonglong2 *__restrict__ tw, int log_n) {
    grid_dep_wait();
    constexpr int R = 1 << LOGR, E = 1 << LOGE, T = R / E, CC = 256 / T;
    constexpr int RP = R + R / E;
    __shared__ uint64_t sm[CC * RP];
    uint32_t g, r;
    limb_of<false>(map, g, r);
    const size_t N = size_t(1) << log_n;
    const uint64_t *in = src + (size_t(g) * map.src_stride + map.src_off[r]) * N;
    uint64_t *out = dst + (size_t(g) * map.dst_stride + map.dst_off[r]) * N;
    const int p = map.prime[r];
    const uint64_t q = mods[p].q;
    const ulonglong2 *w = tw + size_t(p) * N;
    const int k1 = log_n - LOGR;
    const int chl = threadIdx.x / T, tau = threadIdx.x % T;
    const uint32_t h = blockIdx.x * CC + chl;
    const uint64_t *ib = in + size_t(h) * R;
    uint64_t *ob = out + size_t(h) * R;
    uint64_t *s = sm + chl * RP;
#define PAD(u) ((u) + ((u) >> LOGE))

    uint64_t x[E];
#pragma unroll
    for (int v = 0; v < E; v++) s[PAD(tau + T * v)] = ib[tau + T * v];
    __syncthreads();
#pragma unroll
    for (int v = 0; v < E; v++) x[v] = s[PAD(tau * E + v)];
    // stages LOGR-1 .. LOGE (distances 1 .. E/2)
#pragma unroll
    for (int st = LOGR - 1; st >= LOGE; st--) {
        const int dist = 1 << (LOGR - 1 - st);
        const uint32_t base = (1u << (k1 + st)) + (h << st);
#pragma unroll
        for (int v = 0; v < E; v++) {
            if (v & dist) continue;
            const uint32_t idx = base + hi_bits<LOGE>(uint32_t(tau), v, LOGR - st);
            gs_bfly(x[v], x[v + dist], w[idx], q);
        }
    }
#pragma unroll
    for (int v = 0; v < E; v++) s[PAD(tau * E + v)] = x[v];
    __syncthreads();
#pragma unroll
    for (int v = 0; v < E; v++) x[v] = s[PAD(tau + T * v)];
#pragma unroll
    for (int st = LOGE - 1; st >= 0; st--) {
        const int half = E >> (st + 1);
        const uint32_t base = (1u << (k1 + st)) + (h << st);
#pragma unroll
        for (int v = 0; v < E; v++) {
            if (v & half) continue;
            gs_bfly(x[v], x[v + half], w[base + uint32_t(v >> (LOGE - st))], q);
        }
    }
#pragma unroll
    for (int v = 0; v < E; v++) ob[tau + T * v] = x[v];
#undef PAD
}

template <int LOGR, int LOGE>
__global__ void __launch_bounds__(256)
k_ntt_inv_cols(uint64_t *__restrict__ data, const LimbMap map, const DevMod *__restrict__ mods,
               const ulonglong2 *__restrict__ tw, int log_n) {
    grid_dep_wait();
    constexpr int R = 1 << LOGR, E = 1 << LOGE, T = R / E, CW = 256 / T;
    __shared__ uint64_t sm[R * CW];
    uint32_t g, r;
    limb_of<false>(map, g, r);
    const size_t N = size_t(1) << log_n;
    const size_t S = N >> LOGR;
    uint64_t *out = data + (size_t(g) * map.dst_stride + map.dst_off[r]) * N;
    const int p = map.prime[r];
    const DevMod m = mods[p];
    const uint64_t q = m.q;
    const ulonglong2 *wg = tw + size_t(p) * N;
    const int cl = threadIdx.x % CW, tau = threadIdx.x / CW;
    const size_t c = size_t(blockIdx.x) * CW + cl;
    const uint32_t TS = uint32_t(T * S), SS = uint32_t(S);
    uint64_t *ib = out + c + size_t(tau) * E * S;
    uint64_t *ob = out + c + size_t(tau) * S;

    uint64_t x[E];
#pragma unroll
    for (int v = 0; v < E; v++) x[v] = ib[uint32_t(v) * SS];
    // the column stages use twiddles 1 .. R-1 only: staged in shared memory
    // once per CTA, after the data loads are issued (measured: forward 284 ->
    // 278 us, inverse 298 -> 294 us for 384 limbs)
    __shared__ ulonglong2 stw[R];
    for (int i = threadIdx.x; i < R; i += 256) stw[i] = wg[i];
    __syncthreads();
    const ulonglong2 *w = stw;
#pragma unroll
    for (int st = LOGR - 1; st >= LOGE; st--) {
        const int dist = 1 << (LOGR - 1 - st);
#pragma unroll
        for (int v = 0; v < E; v++) {
            if (v & dist) continue;
            const uint32_t idx = (1u << st) + hi_bits<LOGE>(uint32_t(tau), v, LOGR - st);
            gs_bfly(x[v], x[v + dist], w[idx], q);
        }
    }
#pragma unroll
    for (int v = 0; v < E; v++) sm[(tau * E + v) * CW + cl] = x[v];
    __syncthreads();
#pragma unroll
    for (int v = 0; v < E; v++) x[v] = sm[(tau + T * v) * CW + cl];
#pragma unroll
    for (int st = LOGE - 1; st >= 1; st--) {
        const int half = E >> (st + 1);
#pragma unroll
        for (int v = 0; v < E; v++) {
            if (v & half) continue;
            gs_bfly(x[v], x[v + half], w[(1 << st) + (v >> (LOGE - st))], q);
        }
    }
    // stage 0 with N^-1 folded in: (a + b) N^-1, (a - b) psi^-bitrev(1) N^-1,
    // exact Shoup products of words below 8q, fully reduced
    {
        constexpr int half = E / 2;
#pragma unroll
        for (int v = 0; v < half; v++) {
            const uint64_t a0 = x[v], b0 = x[v + half];
            x[v] = shoup(a0 + b0, m.ninv, m.ninv_s, q);
            x[v + half] = shoup(a0 + 4 * q - b0, m.ninvw, m.ninvw_s, q);
        }
    }
#pragma unroll
    for (int v = 0; v < E; v++) ob[uint32_t(v) * TS] = x[v];
}

// ------------------------------------------------------------------ launchers

template <int R1, int E1, int R2, int E2>
static int run_fwd(const Context &c, const uint64_t *src, uint64_t *dst, const LimbMap &map,
                   uint32_t n_limbs, cudaStream_t s, const NttEpilogue *epi = nullptr) {
    const size_t N = c.n;
    dim3 g1(unsigned((N >> R1) / (256 / ((1 << R1) >> E1))), n_limbs);
    launch_pdl(k_ntt_fwd_cols<R1, E1>, g1, dim3(256), 0, s, src, dst, map, c.d_mods, c.d_twf, c.log_n);
    dim3 g2(unsigned((N >> R2) / (256 / ((1 << R2) >> E2))), n_limbs);
    if (epi && epi->status && (reinterpret_cast<uintptr_t>(epi->y) & 15) == 0) {
        constexpr int ybytes = 256 * (1 << E2) * 8;  // the CTA's y tile
        if (cudaFuncSetAttribute(k_ntt_fwd_rows<R2, E2, 2>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, ybytes) != cudaSuccess)
            return CATFHE_ECUDA;
        launch_pdl(k_ntt_fwd_rows<R2, E2, 2>, g2, dim3(256), ybytes, s, dst, map, c.d_mods,
                   c.d_twf, c.log_n, *epi);
    } else if (epi) {
        launch_pdl(k_ntt_fwd_rows<R2, E2, 1>, g2, dim3(256), 0, s, dst, map, c.d_mods, c.d_twf,
                   c.log_n, *epi);
    } else {
        launch_pdl(k_ntt_fwd_rows<R2, E2, 0>, g2, dim3(256), 0, s, dst, map, c.d_mods, c.d_twf,
                   c.log_n, NttEpilogue{});
    }
    note_launches(2);
    return cudaGetLastError() == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA;
}

template <int R1, int E1, int R2, int E2>
static int run_inv(const Context &c, const uint64_t *src, uint64_t *dst, const LimbMap &map,
                   uint32_t n_limbs, cudaStream_t s) {
    const size_t N = c.n;
    dim3 g2(unsigned((N >> R2) / (256 / ((1 << R2) >> E2))), n_limbs);
    launch_pdl(k_ntt_inv_rows<R2, E2>, g2, dim3(256), 0, s, src, dst, map, c.d_mods, c.d_twi, c.log_n);
    dim3 g1(unsigned((N >> R1) / (256 / ((1 << R1) >> E1))), n_limbs);
    launch_pdl(k_ntt_inv_cols<R1, E1>, g1, dim3(256), 0, s, dst, map, c.d_mods, c.d_twi, c.log_n);
    note_launches(2);
    return cudaGetLastError() == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA;
}

// (column pass log size, its LOGE, row pass log size, its LOGE) per log N
// Schedules per log N: (column-pass log size, its LOGE, row-pass log size,
// its LOGE).  Index 0 is the default; catfhe_tune_ntt times them all.
#define NTT_SCHEDULES(X)                                                        \
    X(12, 0, 6, 3, 6, 3) X(12, 1, 5, 3, 7, 4) X(12, 2, 7, 4, 5, 3)              \
    X(13, 0, 7, 4, 6, 3) X(13, 1, 6, 3, 7, 4) X(13, 2, 5, 3, 8, 4)              \
    X(14, 0, 7, 4, 7, 4) X(14, 1, 6, 3, 8, 4) X(14, 2, 8, 4, 6, 3)              \
    X(15, 0, 8, 4, 7, 4) X(15, 1, 7, 4, 8, 4)                                   \
    X(16, 0, 8, 4, 8, 4)

int ntt_schedule_count(int log_n) {
    switch (log_n) {
        case 12: case 13: case 14: return 3;
        case 15: return 2;
        case 16: return 1;
        default: return 0;
    }
}

void ntt_schedule_shape(int log_n, int sched, int shape[4]) {
#define SHAPE(LN, S, A, B, C, D) \
    if (log_n == LN && sched == S) { shape[0] = A; shape[1] = B; shape[2] = C; shape[3] = D; return; }
    NTT_SCHEDULES(SHAPE)
#undef SHAPE
    shape[0] = shape[1] = shape[2] = shape[3] = 0;
}

static int fwd_dispatch(const Context &c, const uint64_t *src, uint64_t *dst, const LimbMap &map,
                        uint32_t n_limbs, cudaStream_t s, const NttEpilogue *epi) {
    if (n_limbs == 0) return CATFHE_OK;
    const int sched = c.ntt_sched[ntt_class(n_limbs)];
#define FWD(LN, S, A, B, C, D) \
    if (c.log_n == LN && sched == S) return run_fwd<A, B, C, D>(c, src, dst, map, n_limbs, s, epi);
    NTT_SCHEDULES(FWD)
#undef FWD
    return CATFHE_EINVAL;
}

int launch_ntt_fwd(const Context &c, const uint64_t *src, uint64_t *dst, const LimbMap &map,
                   uint32_t n_limbs, cudaStream_t s) {
    return fwd_dispatch(c, src, dst, map, n_limbs, s, nullptr);
}

int launch_ntt_fwd_combine(const Context &c, uint64_t *lift, const LimbMap &map, uint32_t n_limbs,
                           const NttEpilogue &epi, cudaStream_t s) {
    return fwd_dispatch(c, lift, lift, map, n_limbs, s, &epi);
}

int launch_ntt_inv(const Context &c, const uint64_t *src, uint64_t *dst, const LimbMap &map,
                   uint32_t n_limbs, cudaStream_t s) {
    if (n_limbs == 0) return CATFHE_OK;
    const int sched = c.ntt_sched[ntt_class(n_limbs)];
#define INV(LN, S, A, B, C, D) \
    if (c.log_n == LN && sched == S) return run_inv<A, B, C, D>(c, src, dst, map, n_limbs, s);
    NTT_SCHEDULES(INV)
#undef INV
    return CATFHE_EINVAL;
}

// Times every schedule of this ring degree on `limbs` limbs (rounded up to
// whole groups of L; a forward and an inverse transform each, best of five)
// and keeps the fastest in the context for launches of that size class.
int tune_ntt(Context &c, uint32_t limbs, cudaStream_t s, int *chosen, float *us_out) {
    const int count = ntt_schedule_count(c.log_n);
    if (count == 0 || limbs == 0) return CATFHE_EINVAL;
    const uint32_t L = uint32_t(c.L);
    const uint32_t groups = (limbs + L - 1) / L;
    uint64_t *buf = nullptr;
    if (cudaMalloc(&buf, size_t(groups) * L * c.n * 8) != cudaSuccess) return CATFHE_ENOMEM;
    int rc = cudaMemsetAsync(buf, 0, size_t(groups) * L * c.n * 8, s) == cudaSuccess ? CATFHE_OK
                                                                                     : CATFHE_ECUDA;
    LimbMap m{};
    m.period = L;
    m.src_stride = m.dst_stride = L;
    for (uint32_t i = 0; i < L; i++) {
        m.src_off[i] = m.dst_off[i] = uint16_t(i);
        m.prime[i] = uint8_t(i);
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int cls = ntt_class(groups * L);
    const int keep = c.ntt_sched[cls];
    int best = keep;
    float best_ms = 1e30f;
    for (int k = 0; k < count && rc == CATFHE_OK; k++) {
        c.ntt_sched[cls] = k;
        float t_min = 1e30f;
        for (int rep = 0; rep < 6 && rc == CATFHE_OK; rep++) {
            cudaEventRecord(e0, s);
            rc = launch_ntt_fwd(c, buf, buf, m, groups * L, s);
            if (!rc) rc = launch_ntt_inv(c, buf, buf, m, groups * L, s);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = CATFHE_ECUDA;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) t_min = ms < t_min ? ms : t_min;
        }
        if (us_out) us_out[k] = t_min * 1e3f;
        if (t_min < best_ms) {
            best_ms = t_min;
            best = k;
        }
    }
    c.ntt_sched[cls] = rc == CATFHE_OK ? best : keep;
    if (chosen) *chosen = c.ntt_sched[cls];
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    return rc;
}

}  // namespace catfhe
