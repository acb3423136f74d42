// Batched negacyclic NTT / inverse NTT kernels and their launch templates
// (included by ntt.cu and by the ntt_n*.cu translation units, one per ring
// degree, which instantiate that degree's schedules; split so that the
// build compiles them in parallel).
#pragma once

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

// Any word below 2^64 -> [0, q) for q > 2^33, m64 = floor(2^64 / q) < 2^31:
// est = floor(hi32(x) m64 / 2^32) is at most floor(x/q) and at most 2 below
// it (x - hi32(x) 2^32 < 2^32 < q, m64 is short of 2^64/q by less than 1,
// which hi32(x) / 2^32 < 1 turns into less than 1, and the floor drops less
// than 1), so x - est q lies in [0, 3q).  Three 32-bit multiplies (one
// high, one wide, one low) instead of the 64-bit high product of the Shoup
// form: measured on the 384-limb forward row pass, 174 -> 166 us.
__device__ __forceinline__ uint64_t reduce_fast(uint64_t x, uint64_t q, uint32_t m64) {
    const uint32_t est = __umulhi(uint32_t(x >> 32), m64);
    const uint64_t r = x - uint64_t(est) * q;
    return csub(csub(r, 2 * q), q);
}

// The row pass's final reduction of a word of the forward transform: below
// 68q for primes under 2^57 (no subtractions in the butterflies), below 8q
// otherwise.
template <bool WIDE>
__device__ __forceinline__ uint64_t reduce_fwd(uint64_t x, const DevMod &m) {
    if (!WIDE) return reduce8(x, m.q);
    return m.m64 ? reduce_fast(x, m.q, uint32_t(m.m64)) : reduce_any(x, m);
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

// The last LOGE stages of an inverse row pass (like the first LOGE of a
// forward one) use twiddles that depend only on the chunk, not on the thread:
// E - 1 of them per chunk.  The inverse pass stages its chunks' ones in shared
// memory with its data, under the barrier it has anyway, one load per thread
// instead of E - 1; entry (1 << st) - 1 + i of chunk c is stage st's i-th
// twiddle.  (The forward pass would need one more barrier for it: the step
// measured 0.4% faster with it, the 384-limb forward transform 1% slower.)
template <int LOGN, int LOGR, int LOGE, int NT>
__device__ __forceinline__ void stage_chunk_twiddles(ulonglong2 *dst, const ulonglong2 *w) {
    constexpr int E = 1 << LOGE, T = (1 << LOGR) / E, CC = NT / T, NP = E - 1;
    constexpr int k1 = LOGN - LOGR;
    for (int i = threadIdx.x; i < CC * NP; i += NT) {
        const int c = i / NP, j = i % NP;
        const int st = 31 - __clz(j + 1);
        const uint32_t h = blockIdx.x * CC + c;
        dst[i] = w[(1u << (k1 + st)) + (h << st) + uint32_t(j + 1 - (1 << st))];
    }
}

// Twiddles a thread needs in the stages after a row pass's exchange, when
// there are at most 16 of them (else 0: they are read at their use).
template <int LOGR, int LOGE>
struct PrefetchCount {
    static constexpr int count() {
        int c = 0;
        for (int st = LOGE; st < LOGR; st++) c += (LOGR - st) >= LOGE ? 1 : ((1 << LOGE) >> (LOGR - st));
        return c;
    }
    static constexpr int value = count() <= 16 ? count() : 0;
};

template <int LOGR, int LOGE, int NT, bool WIDE>
__device__ __forceinline__ void fwd_cols_body(uint64_t (&x)[1 << LOGE], uint64_t *sm,
                                              const ulonglong2 *w, uint64_t q, int cl, int tau) {
    constexpr int R = 1 << LOGR, E = 1 << LOGE, T = R / E, CW = NT / T;
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

// The ring degree is a template parameter of every pass (one instantiation
// per schedule), so strides, shifts and twiddle offsets are compile-time
// constants and need no integer multiplies at run time: the multiply pipe
// is the one these kernels saturate.  NT threads per CTA: 256, or 128 for
// E = 32 words per thread (whose exchange buffer would not fit 48 KB of
// static shared memory at 256 threads).
template <int LOGN, int LOGR, int LOGE, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
k_ntt_fwd_cols(const uint64_t *src, uint64_t *dst, const LimbMap map,
               const DevMod *__restrict__ mods, const ulonglong2 *__restrict__ tw) {
    grid_dep_wait();
    constexpr int R = 1 << LOGR, E = 1 << LOGE, T = R / E, CW = NT / T;
    __shared__ uint64_t sm[R * CW];
    uint32_t g, r;
    limb_of<true>(map, g, r);
    constexpr size_t N = size_t(1) << LOGN;
    constexpr size_t S = N >> LOGR;
    const uint64_t *in = src + (size_t(g) * map.src_stride + map.src_off[r]) * N;
    uint64_t *out = dst + (size_t(g) * map.dst_stride + map.dst_off[r]) * N;
    const int p = map.prime[r];
    const uint64_t q = mods[p].q;
    const ulonglong2 *wg = tw + size_t(p) * N;
    const int cl = threadIdx.x % CW, tau = threadIdx.x / CW;
    const uint32_t c = blockIdx.x * CW + cl;
    constexpr uint32_t TS = uint32_t(T * S), SS = uint32_t(S);
    const uint64_t *ip = in + c + tau * SS;
    uint64_t *op = out + c + tau * (E * SS);

    uint64_t x[E];
#pragma unroll
    for (int v = 0; v < E; v++) x[v] = ip[v * TS];
    // the column stages use twiddles 1 .. R-1 only: staged in shared memory
    // once per CTA, after the data loads are issued (measured: forward 284 ->
    // 278 us, inverse 298 -> 294 us for 384 limbs)
    __shared__ ulonglong2 stw[R];
    for (int i = threadIdx.x; i < R; i += NT) stw[i] = wg[i];
    __syncthreads();
    const ulonglong2 *w = stw;
    // q < 2^57: no conditional subtractions; words leave below 4q + 4 LOGR q
    // (else below 8q) and the row pass reduces them after its stages
    if (q < kWideBound)
        fwd_cols_body<LOGR, LOGE, NT, true>(x, sm, w, q, cl, tau);
    else
        fwd_cols_body<LOGR, LOGE, NT, false>(x, sm, w, q, cl, tau);
#pragma unroll
    for (int v = 0; v < E; v++) op[v * SS] = x[v];
}

template <int LOGR, int LOGE, bool WIDE>
__device__ __forceinline__ void fwd_rows_body(uint64_t (&x)[1 << LOGE], uint64_t *s,
                                              const ulonglong2 *w, uint64_t q, int k1, uint32_t h,
                                              int tau) {
    constexpr int R = 1 << LOGR, E = 1 << LOGE, T = R / E;
#define PAD(u) ((u) + ((u) >> LOGE))
    // The stages after the exchange need E >> (LOGR - st) twiddles per thread
    // (at least one), read from L2.  When they are few (15 for 256-word rows
    // of 16 words per thread), all of them are requested here, before the
    // first stage, so their latency hides behind the stages before the
    // exchange instead of stalling the ones after it.
    constexpr int NPRE = PrefetchCount<LOGR, LOGE>::value;
    ulonglong2 pw[NPRE > 0 ? NPRE : 1];
    if (NPRE > 0) {
        int o = 0;
#pragma unroll
        for (int st = LOGE; st < LOGR; st++) {
            const int sh = LOGR - st;
            const int cnt = sh >= LOGE ? 1 : (E >> sh);
            const uint32_t base = (1u << (k1 + st)) + (h << st);
#pragma unroll
            for (int j = 0; j < cnt; j++)
                pw[NPRE > 0 ? o + j : 0] = w[base + hi_bits<LOGE>(uint32_t(tau), j << sh, sh)];
            o += cnt;
        }
    }
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
    int o = 0;
#pragma unroll
    for (int st = LOGE; st < LOGR; st++) {
        const int dist = 1 << (LOGR - 1 - st);
        const int sh = LOGR - st;
        const uint32_t base = (1u << (k1 + st)) + (h << st);
#pragma unroll
        for (int v = 0; v < E; v++) {
            if (v & dist) continue;
            if (NPRE > 0) {
                const int j = sh >= LOGE ? 0 : (v >> sh);
                fwd_bfly<WIDE>(x[v], x[v + dist], pw[NPRE > 0 ? o + j : 0], q);
            } else {
                const uint32_t idx = base + hi_bits<LOGE>(uint32_t(tau), v, sh);
                fwd_bfly<WIDE>(x[v], x[v + dist], w[idx], q);
            }
        }
        o += sh >= LOGE ? 1 : (E >> sh);
    }
#undef PAD
}

// EPI: 0, the plain transform; 1, the ModDown combine epilogue with its y
// words loaded into registers before the butterflies; 2, the same epilogue
// with the CTA's y tile (its CC chunks of R words are contiguous) brought
// into shared memory by one bulk copy issued before the butterflies, so that
// no registers are held for it (y 16-byte aligned and a status word, checked
// on the host; the dynamic shared memory holds 256 E words); 3, the plain
// transform with unreduced outputs for primes under 2^57 (words below 68q,
// for a consumer that reduces anyway: the key-switching inner product,
// whose host side checks that its sums stay below 2^64 q; larger primes are
// still reduced to [0, q)).
// The combine epilogues take the lift unreduced too: (y + 68q - lift) with
// y < q stays below 69q < 2^64 for primes under 2^57, and the Shoup product
// by D^-1 reduces any 64-bit word.
template <int LOGN, int LOGR, int LOGE, int NT, int MINB, int EPI>
__global__ void __launch_bounds__(NT, MINB)
k_ntt_fwd_rows(uint64_t *__restrict__ data, const LimbMap map, const DevMod *__restrict__ mods,
               const ulonglong2 *__restrict__ tw, const NttEpilogue epi) {
    grid_dep_wait();
    constexpr int R = 1 << LOGR, E = 1 << LOGE, T = R / E, CC = NT / T;
    constexpr int RP = R + R / E;
    __shared__ uint64_t sm[CC * RP];
    extern __shared__ __align__(16) uint64_t ytile[];
    __shared__ __align__(8) uint64_t ybar;
    uint32_t g, r;
    limb_of<true>(map, g, r);
    constexpr size_t N = size_t(1) << LOGN;
    uint64_t *out = data + (size_t(g) * map.dst_stride + map.dst_off[r]) * N;
    const int p = map.prime[r];
    const DevMod m = mods[p];
    const uint64_t q = m.q;
    const ulonglong2 *w = tw + size_t(p) * N;
    constexpr int k1 = LOGN - LOGR;
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
    // 4q + 4 log2(N) q <= 68q < 2^64, then one reduction (none for EPI 1-3);
    // else below 8q, then three conditional subtractions.  (Each branch with
    // its own reduction, and 3 CTAs per SM: fewer register spills, measured
    // forward transform 297 -> 284 us.)
    const bool wide = q < kWideBound;
    if (wide) {
        fwd_rows_body<LOGR, LOGE, true>(x, s, w, q, k1, h, tau);
#pragma unroll
        for (int v = 0; v < E; v++) s[PAD(tau * E + v)] = EPI == 0 ? reduce_fwd<true>(x[v], m) : x[v];
    } else {
        fwd_rows_body<LOGR, LOGE, false>(x, s, w, q, k1, h, tau);
#pragma unroll
        for (int v = 0; v < E; v++) s[PAD(tau * E + v)] = reduce8(x[v], q);
    }
    __syncthreads();
    if (EPI == 0 || EPI == 3) {
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
        const uint64_t cq = wide ? kWideWordsQ * q : q;  // above every lift word
#pragma unroll
        for (int v = 0; v < E; v++) {
            const int u = tau + T * v;
            const uint64_t yw = EPI == 2 ? ytile[chl * R + u] : yv[EPI == 1 ? v : 0];
            uint64_t o = csub(csub(shoup_lazy4(yw + cq - s[PAD(u)], dv, dvs, q), 2 * q), q);
            if (ap) o = add_mod(o, ap[u], q);
            op[u] = o;
        }
    }
#undef PAD
}

// ------------------------------------------------------------------ inverse

template <int LOGN, int LOGR, int LOGE, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
k_ntt_inv_rows(const uint64_t *src, uint64_t *dst, const LimbMap map,
               const DevMod *__restrict__ mods, const ulonglong2 *__restrict__ tw) {
    grid_dep_wait();
    constexpr int R = 1 << LOGR, E = 1 << LOGE, T = R / E, CC = NT / T;
    constexpr int RP = R + R / E;
    __shared__ uint64_t sm[CC * RP];
    uint32_t g, r;
    limb_of<false>(map, g, r);
    constexpr size_t N = size_t(1) << LOGN;
    const uint64_t *in = src + (size_t(g) * map.src_stride + map.src_off[r]) * N;
    uint64_t *out = dst + (size_t(g) * map.dst_stride + map.dst_off[r]) * N;
    const int p = map.prime[r];
    const uint64_t q = mods[p].q;
    const ulonglong2 *w = tw + size_t(p) * N;
    constexpr int k1 = LOGN - LOGR;
    const int chl = threadIdx.x / T, tau = threadIdx.x % T;
    const uint32_t h = blockIdx.x * CC + chl;
    const uint64_t *ib = in + size_t(h) * R;
    uint64_t *ob = out + size_t(h) * R;
    uint64_t *s = sm + chl * RP;
#define PAD(u) ((u) + ((u) >> LOGE))

    // the twiddles of the stages before the exchange (per thread, as in the
    // forward pass's stages after it) are requested with the data, so that
    // their latency overlaps the loads and the barrier
    constexpr int NPRE = PrefetchCount<LOGR, LOGE>::value;
    ulonglong2 pw[NPRE > 0 ? NPRE : 1];
    if (NPRE > 0) {
        int o = 0;
#pragma unroll
        for (int st = LOGR - 1; st >= LOGE; st--) {
            const int sh = LOGR - st;
            const int cnt = sh >= LOGE ? 1 : (E >> sh);
            const uint32_t base = (1u << (k1 + st)) + (h << st);
#pragma unroll
            for (int j = 0; j < cnt; j++)
                pw[NPRE > 0 ? o + j : 0] = w[base + hi_bits<LOGE>(uint32_t(tau), j << sh, sh)];
            o += cnt;
        }
    }
    uint64_t x[E];
#pragma unroll
    for (int v = 0; v < E; v++) s[PAD(tau + T * v)] = ib[tau + T * v];
    // the last LOGE stages' chunk twiddles, staged with the data (same barrier)
    __shared__ ulonglong2 tw1[CC * (E - 1)];
    stage_chunk_twiddles<LOGN, LOGR, LOGE, NT>(tw1, w);
    const ulonglong2 *w1 = tw1 + chl * (E - 1);
    __syncthreads();
#pragma unroll
    for (int v = 0; v < E; v++) x[v] = s[PAD(tau * E + v)];
    // stages LOGR-1 .. LOGE (distances 1 .. E/2)
    int o = 0;
#pragma unroll
    for (int st = LOGR - 1; st >= LOGE; st--) {
        const int dist = 1 << (LOGR - 1 - st);
        const int sh = LOGR - st;
        const uint32_t base = (1u << (k1 + st)) + (h << st);
#pragma unroll
        for (int v = 0; v < E; v++) {
            if (v & dist) continue;
            if (NPRE > 0) {
                const int j = sh >= LOGE ? 0 : (v >> sh);
                gs_bfly(x[v], x[v + dist], pw[NPRE > 0 ? o + j : 0], q);
            } else {
                const uint32_t idx = base + hi_bits<LOGE>(uint32_t(tau), v, sh);
                gs_bfly(x[v], x[v + dist], w[idx], q);
            }
        }
        o += sh >= LOGE ? 1 : (E >> sh);
    }
#pragma unroll
    for (int v = 0; v < E; v++) s[PAD(tau * E + v)] = x[v];
    __syncthreads();
#pragma unroll
    for (int v = 0; v < E; v++) x[v] = s[PAD(tau + T * v)];
#pragma unroll
    for (int st = LOGE - 1; st >= 0; st--) {
        const int half = E >> (st + 1);
#pragma unroll
        for (int v = 0; v < E; v++) {
            if (v & half) continue;
            gs_bfly(x[v], x[v + half], w1[(1 << st) - 1 + (v >> (LOGE - st))], q);
        }
    }
#pragma unroll
    for (int v = 0; v < E; v++) ob[tau + T * v] = x[v];
#undef PAD
}

template <int LOGN, int LOGR, int LOGE, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
k_ntt_inv_cols(uint64_t *__restrict__ data, const LimbMap map, const DevMod *__restrict__ mods,
               const ulonglong2 *__restrict__ tw) {
    grid_dep_wait();
    constexpr int R = 1 << LOGR, E = 1 << LOGE, T = R / E, CW = NT / T;
    __shared__ uint64_t sm[R * CW];
    uint32_t g, r;
    limb_of<false>(map, g, r);
    constexpr size_t N = size_t(1) << LOGN;
    constexpr size_t S = N >> LOGR;
    uint64_t *out = data + (size_t(g) * map.dst_stride + map.dst_off[r]) * N;
    const int p = map.prime[r];
    const DevMod m = mods[p];
    const uint64_t q = m.q;
    const ulonglong2 *wg = tw + size_t(p) * N;
    const int cl = threadIdx.x % CW, tau = threadIdx.x / CW;
    const uint32_t c = blockIdx.x * CW + cl;
    constexpr uint32_t TS = uint32_t(T * S), SS = uint32_t(S);
    uint64_t *ib = out + c + tau * (E * SS);
    uint64_t *ob = out + c + tau * SS;

    uint64_t x[E];
#pragma unroll
    for (int v = 0; v < E; v++) x[v] = ib[v * SS];
    // the column stages use twiddles 1 .. R-1 only: staged in shared memory
    // once per CTA, after the data loads are issued (measured: forward 284 ->
    // 278 us, inverse 298 -> 294 us for 384 limbs)
    __shared__ ulonglong2 stw[R];
    for (int i = threadIdx.x; i < R; i += NT) stw[i] = wg[i];
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
    // stage 0 with N^-1 folded in: (a + b) N^-1, (a - b) psi^-bitrev(1) N^-1
    // of words below 8q, by the approximate-quotient Shoup product (in
    // [0, 4q)) and two conditional subtractions: fully reduced
    {
        constexpr int half = E / 2;
        const uint64_t q2 = 2 * q;
#pragma unroll
        for (int v = 0; v < half; v++) {
            const uint64_t a0 = x[v], b0 = x[v + half];
            x[v] = csub(csub(shoup_lazy4(a0 + b0, m.ninv, m.ninv_s, q), q2), q);
            x[v + half] = csub(csub(shoup_lazy4(a0 + 4 * q - b0, m.ninvw, m.ninvw_s, q), q2), q);
        }
    }
#pragma unroll
    for (int v = 0; v < E; v++) ob[v * TS] = x[v];
}

// ------------------------------------------------------------------ launchers

// Forward transform modes: 0 plain, 3 unreduced outputs (see k_ntt_fwd_rows),
// or the ModDown combine epilogue when epi is given.
template <int LN, int R1, int E1, int T1, int B1, int R2, int E2, int T2, int B2>
static int run_fwd(const Context &c, const uint64_t *src, uint64_t *dst, const LimbMap &map,
                   uint32_t n_limbs, cudaStream_t s, const NttEpilogue *epi, bool lazy) {
    constexpr size_t N = size_t(1) << LN;
    const dim3 g1(unsigned((N >> R1) / (T1 / ((1 << R1) >> E1))), n_limbs);
    launch_pdl(k_ntt_fwd_cols<LN, R1, E1, T1, B1>, g1, dim3(T1), 0, s, src, dst, map, c.d_mods,
               c.d_twf);
    const dim3 g2(unsigned((N >> R2) / (T2 / ((1 << R2) >> E2))), n_limbs);
    if (epi && epi->status && (reinterpret_cast<uintptr_t>(epi->y) & 15) == 0) {
        constexpr int ybytes = T2 * (1 << E2) * 8;  // the CTA's y tile
        if (cudaFuncSetAttribute(k_ntt_fwd_rows<LN, R2, E2, T2, B2, 2>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, ybytes) != cudaSuccess)
            return CATFHE_ECUDA;
        launch_pdl(k_ntt_fwd_rows<LN, R2, E2, T2, B2, 2>, g2, dim3(T2), ybytes, s, dst, map,
                   c.d_mods, c.d_twf, *epi);
    } else if (epi) {
        launch_pdl(k_ntt_fwd_rows<LN, R2, E2, T2, B2, 1>, g2, dim3(T2), 0, s, dst, map, c.d_mods,
                   c.d_twf, *epi);
    } else if (lazy) {
        launch_pdl(k_ntt_fwd_rows<LN, R2, E2, T2, B2, 3>, g2, dim3(T2), 0, s, dst, map, c.d_mods,
                   c.d_twf, NttEpilogue{});
    } else {
        launch_pdl(k_ntt_fwd_rows<LN, R2, E2, T2, B2, 0>, g2, dim3(T2), 0, s, dst, map, c.d_mods,
                   c.d_twf, NttEpilogue{});
    }
    note_launches(2);
    return cudaGetLastError() == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA;
}

template <int LN, int R1, int E1, int T1, int B1, int R2, int E2, int T2, int B2>
static int run_inv(const Context &c, const uint64_t *src, uint64_t *dst, const LimbMap &map,
                   uint32_t n_limbs, cudaStream_t s) {
    constexpr size_t N = size_t(1) << LN;
    const dim3 g2(unsigned((N >> R2) / (T2 / ((1 << R2) >> E2))), n_limbs);
    launch_pdl(k_ntt_inv_rows<LN, R2, E2, T2, B2>, g2, dim3(T2), 0, s, src, dst, map, c.d_mods,
               c.d_twi);
    const dim3 g1(unsigned((N >> R1) / (T1 / ((1 << R1) >> E1))), n_limbs);
    launch_pdl(k_ntt_inv_cols<LN, R1, E1, T1, B1>, g1, dim3(T1), 0, s, dst, map, c.d_mods,
               c.d_twi);
    note_launches(2);
    return cudaGetLastError() == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA;
}

// Schedules per log N: (column-pass log size, its LOGE, its threads per CTA,
// its minimum CTAs per SM, then the same four for the row pass).  The
// minimum CTAs per SM sets a pass's register budget (65536 / (threads x
// CTAs)).  A pass of 2^LOGR words runs LOGE stages in registers, one
// exchange, then the rest, so LOGR <= 2 LOGE.  Index 0 is the default of
// every launch size class until catfhe_tune_ntt times them all; it is the
// schedule measured fastest for the largest class (32 ciphertexts) on
// GB300.  Row passes in small CTAs with up to 128 registers per thread
// measured faster than 80 registers in CTAs of 256 threads, although fewer
// warps are resident (forward plus inverse of 768 limbs at N = 2^16:
// 1102 us at 256 threads x 3 CTAs, 1039 at 128 x 4, 1022 at 64 x 8, 1018 at
// 32 x 16; with the later butterflies and twiddle prefetch 946 at 32 x 16).
// Column passes of 128 threads at 6 CTAs per SM (as many warps as 256 x 3,
// in CTAs of half the size, so that each exchange barrier holds 4 warps
// instead of 8) were faster than 256 x 3 in
// every size class at N = 2^16: forward plus inverse 481.8 against 484.5 us
// (largest class), 135.3 against 138.1 (up to 256 limbs), 77.3 against 79.3
// (up to 64).  At 2^13 - 2^15 the same column pass with row passes of 32
// threads x 16 CTAs per SM (up to 128 registers) was the fastest for the
// largest class: forward plus inverse 111.2 against 116.1 us (2^13, 16
// ciphertexts of 24 primes), 228.2 against 237.1 (2^14), 452.5 against
// 464.4 (2^15).
#define NTT_SCHEDULES(X)                                                                         \
    X(12, 0, 6, 3, 256, 3, 6, 3, 128, 4) X(12, 1, 6, 3, 256, 3, 6, 3, 256, 3)                    \
    X(12, 2, 5, 3, 256, 3, 7, 4, 128, 4) X(12, 3, 7, 4, 256, 3, 5, 3, 128, 4)                    \
    X(12, 4, 6, 3, 128, 6, 6, 3, 128, 4)                                                         \
    X(13, 0, 7, 4, 128, 6, 6, 3, 32, 16) X(13, 1, 7, 4, 256, 3, 6, 3, 64, 8)                     \
    X(13, 2, 7, 4, 256, 3, 6, 3, 256, 3) X(13, 3, 6, 3, 256, 3, 7, 4, 128, 4)                    \
    X(13, 4, 7, 4, 128, 6, 6, 3, 128, 4) X(13, 5, 7, 4, 256, 3, 6, 3, 128, 4)                    \
    X(13, 6, 7, 4, 128, 6, 6, 3, 64, 8)                                                          \
    X(14, 0, 8, 4, 128, 6, 6, 3, 32, 16) X(14, 1, 8, 4, 256, 3, 6, 3, 64, 8)                     \
    X(14, 2, 7, 4, 256, 3, 7, 4, 128, 4) X(14, 3, 8, 4, 256, 3, 6, 3, 256, 3)                    \
    X(14, 4, 6, 3, 256, 3, 8, 4, 128, 4) X(14, 5, 8, 4, 128, 6, 6, 3, 128, 4)                    \
    X(14, 6, 8, 4, 256, 3, 6, 3, 128, 4) X(14, 7, 8, 4, 128, 6, 6, 3, 64, 8)                     \
    X(15, 0, 7, 4, 128, 6, 8, 4, 32, 16) X(15, 1, 7, 4, 256, 3, 8, 4, 128, 4)                    \
    X(15, 2, 8, 4, 256, 3, 7, 4, 128, 4) X(15, 3, 7, 4, 256, 3, 8, 4, 256, 3)                    \
    X(15, 4, 6, 3, 256, 3, 9, 5, 128, 4) X(15, 5, 7, 4, 128, 6, 8, 4, 64, 8)                     \
    X(15, 6, 7, 4, 256, 3, 8, 4, 64, 8) X(15, 7, 7, 4, 128, 6, 8, 4, 128, 4)                     \
    X(16, 0, 8, 4, 128, 6, 8, 4, 32, 16) X(16, 1, 8, 4, 256, 3, 8, 4, 64, 8)                     \
    X(16, 2, 8, 4, 256, 3, 8, 4, 128, 4) X(16, 3, 8, 4, 256, 3, 8, 4, 256, 3)                    \
    X(16, 4, 8, 4, 256, 2, 8, 4, 64, 8) X(16, 5, 7, 4, 256, 3, 9, 5, 128, 4)                     \
    X(16, 6, 8, 4, 256, 3, 8, 4, 32, 16) X(16, 7, 8, 4, 128, 5, 8, 4, 32, 16)

}  // namespace catfhe
