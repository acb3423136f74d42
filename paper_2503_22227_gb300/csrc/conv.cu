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
// Every dot product is accumulated exactly in 128 bits (at most 8 products
// of < 2^62 words per partial sum) and reduced once, so there is no
// floating-point estimate and no approximation: the result is the
// definition, bit for bit, whatever the order of the work.
//
// One thread handles one coefficient of one item; the packed plan (a few
// KB) sits in shared memory and every thread reads the same words
// (broadcast).
#include "modarith.cuh"

namespace catfhe {

struct PlanView {
    uint32_t k, T, wrap, lazy;
    const uint64_t *src_off, *dst_off, *smod, *dmod, *pre, *pre_s, *W, *Minv, *Minv_s, *h, *Wt,
        *Mt, *post, *post_s;
};

__device__ __forceinline__ PlanView plan_view(const uint64_t *p) {
    PlanView v;
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

// sum_{i < cnt} a[i] * w[i * stride] mod m, exact.  KMAX <= 16 keeps the
// digits in registers (fully unrolled); the wide variant (KMAX = 32) keeps
// them in local memory with rolled loops.
template <int KMAX>
__device__ __forceinline__ uint64_t dot_mod(const uint64_t (&a)[KMAX], const uint64_t *w,
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
    return reduce128(acc, m);
}

// The same sum in [0, 4q) (no final conditional subtractions).
template <int KMAX>
__device__ __forceinline__ uint64_t dot_mod_lazy(const uint64_t (&a)[KMAX], const uint64_t *w,
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
    return shoup_lazy(acc.hi, m.r64, m.r64_s, m.q) + shoup_lazy(acc.lo, 1, m.one_s, m.q);
}

// Turns a[] (residues, already pre-multiplied) into mixed-radix digits and
// returns whether x > (M-1)/2.
template <int KMAX>
__device__ __forceinline__ bool mixed_radix(uint64_t (&a)[KMAX], const PlanView &P) {
#pragma unroll(KMAX <= 16 ? KMAX : 1)
    for (int j = 1; j < KMAX; j++) {
        if (uint32_t(j) < P.k) {
            const DevMod mj = mod4(P.smod + 4 * j);
            const uint64_t s = dot_mod<KMAX>(a, P.W + j, P.k, uint32_t(j), mj);
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

// x_c mod p_t (times the post-multiplier).
template <int KMAX>
__device__ __forceinline__ uint64_t eval_target(const uint64_t (&a)[KMAX], bool gt,
                                                const PlanView &P, uint32_t t) {
    if (P.wrap) {
        uint64_t r = 0;
#pragma unroll(KMAX <= 16 ? KMAX : 1)
        for (int i = 0; i < KMAX; i++)
            if (uint32_t(i) < P.k) r += a[i] * P.Wt[size_t(i) * P.T + t];
        return gt ? r - P.Mt[t] : r;
    }
    const DevMod mt = mod4(P.dmod + 4 * t);
    if (P.lazy) {
        // [0, 4q): one conditional subtraction fewer, for an NTT to consume
        uint64_t r = csub(dot_mod_lazy<KMAX>(a, P.Wt + t, P.T, P.k, mt), 2 * mt.q);
        if (gt) r += 2 * mt.q - P.Mt[t];
        if (P.post[t] != 1) r = shoup_lazy(r, P.post[t], P.post_s[t], mt.q);
        return r;
    }
    uint64_t r = dot_mod<KMAX>(a, P.Wt + t, P.T, P.k, mt);
    if (gt) r = sub_mod(r, P.Mt[t], mt.q);
    if (P.post[t] != 1) r = shoup(r, P.post[t], P.post_s[t], mt.q);
    return r;
}

template <int KMAX>
__device__ __forceinline__ void load_sources(uint64_t (&a)[KMAX], const PlanView &P,
                                             const uint64_t *s, size_t x, size_t n) {
#pragma unroll(KMAX <= 16 ? KMAX : 1)
    for (int i = 0; i < KMAX; i++) {
        if (uint32_t(i) < P.k) {
            uint64_t r = s[P.src_off[i] * n + x];
            if (P.pre[i] != 1) r = shoup(r, P.pre[i], P.pre_s[i], P.smod[4 * i]);
            a[i] = r;
        } else {
            a[i] = 0;
        }
    }
}

__device__ __forceinline__ void copy_plan(uint64_t *dst, const uint64_t *src, uint32_t words) {
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
}

template <int KMAX>
__global__ void __launch_bounds__(256)
k_conv(const PlanList plans, const uint64_t *__restrict__ src, size_t src_item, size_t src_plan,
       uint64_t *__restrict__ dst, size_t dst_item, size_t dst_plan, uint32_t log_n) {
    extern __shared__ uint64_t splan[];
    const uint64_t *gp = plans.p[blockIdx.z];
    const uint32_t k = uint32_t(gp[0] & 0xffff), T = uint32_t((gp[0] >> 16) & 0xffff);
    copy_plan(splan, gp, uint32_t(plan_words(k, T)));
    __syncthreads();
    const PlanView P = plan_view(splan);
    const size_t n = size_t(1) << log_n;
    const uint64_t *s = src + blockIdx.y * src_item + blockIdx.z * src_plan;
    uint64_t *d = dst + blockIdx.y * dst_item + blockIdx.z * dst_plan;
    for (size_t x = size_t(blockIdx.x) * blockDim.x + threadIdx.x; x < n;
         x += size_t(gridDim.x) * blockDim.x) {
        uint64_t a[KMAX];
        load_sources<KMAX>(a, P, s, x, n);
        const bool gt = mixed_radix<KMAX>(a, P);
        for (uint32_t t = 0; t < P.T; t++) d[P.dst_off[t] * n + x] = eval_target<KMAX>(a, gt, P, t);
    }
}

// BFV scale-and-round: see launch_bfv_scale_round in internal.h.  Plan
// p_qb lifts [t x]_Q to B: its pre[] is t mod q_i, its post[] Q^-1 mod b_j,
// and its dst_off[] locate x_b inside the source item (nothing is written
// through it).  tq[2j], tq[2j+1] = t Q^-1 mod b_j and its Shoup quotient.
// Plan p_bq lifts z = round(t x / Q) (centred in B) back to Q.
template <int KQ, int KB>
__global__ void __launch_bounds__(256)
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
    const PlanView A = plan_view(s_qb), B = plan_view(s_bq);
    const size_t n = size_t(1) << log_n;
    const uint64_t *s = src + blockIdx.y * src_item;
    uint64_t *d = dst + blockIdx.y * dst_item;
    for (size_t x = size_t(blockIdx.x) * blockDim.x + threadIdx.x; x < n;
         x += size_t(gridDim.x) * blockDim.x) {
        uint64_t a[KQ];
        load_sources<KQ>(a, A, s, x, n);  // t x_i mod q_i (pre = t)
        const bool gt = mixed_radix<KQ>(a, A);
        uint64_t z[KB];
#pragma unroll(KB <= 16 ? KB : 1)
        for (int j = 0; j < KB; j++) {
            if (uint32_t(j) < A.T) {
                // [t x]_Q Q^-1 mod b_j (post = Q^-1), and t Q^-1 x_b
                const uint64_t l = eval_target<KQ>(a, gt, A, j);
                const uint64_t bq = A.dmod[4 * j];
                const uint64_t xb = s[A.dst_off[j] * n + x];
                const uint64_t txb = shoup(xb, s_tq[2 * j], s_tq[2 * j + 1], bq);
                z[j] = sub_mod(txb, l, bq);
            } else {
                z[j] = 0;
            }
        }
        const bool gz = mixed_radix<KB>(z, B);
        for (uint32_t t = 0; t < B.T; t++) d[B.dst_off[t] * n + x] = eval_target<KB>(z, gz, B, t);
    }
}

static int pick_kmax(uint32_t k) { return k <= 4 ? 4 : k <= 8 ? 8 : k <= 16 ? 16 : 32; }

int launch_conv(const Context &c, const PlanList &plans, const uint64_t *src, size_t src_item,
                size_t src_plan, uint64_t *dst, size_t dst_item, size_t dst_plan, uint32_t items,
                cudaStream_t s) {
    if (plans.n == 0 || items == 0) return CATFHE_OK;
    const uint32_t kmax = plans.kmax, words = plans.words;
    const size_t n = c.n;
    dim3 grid(unsigned((n + 1023) / 1024), items, plans.n);
    const size_t sm = size_t(words) * 8;
    switch (pick_kmax(kmax)) {
        case 4: k_conv<4><<<grid, 256, sm, s>>>(plans, src, src_item, src_plan, dst, dst_item, dst_plan, c.log_n); break;
        case 8: k_conv<8><<<grid, 256, sm, s>>>(plans, src, src_item, src_plan, dst, dst_item, dst_plan, c.log_n); break;
        case 16: k_conv<16><<<grid, 256, sm, s>>>(plans, src, src_item, src_plan, dst, dst_item, dst_plan, c.log_n); break;
        default: k_conv<32><<<grid, 256, sm, s>>>(plans, src, src_item, src_plan, dst, dst_item, dst_plan, c.log_n); break;
    }
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA;
}

int launch_bfv_scale_round(const Context &c, const uint64_t *q_to_b, uint32_t q_to_b_words,
                           const uint64_t *b_to_q, uint32_t b_to_q_words, const uint64_t *src,
                           size_t src_item, uint64_t *dst, size_t dst_item, uint32_t items,
                           cudaStream_t s) {
    // the t Q^-1 mod b_j pairs follow the q_to_b plan in the same allocation
    const uint64_t *tq = q_to_b + q_to_b_words;
    const size_t n = c.n;
    const uint32_t kq = uint32_t(c.L), kb = uint32_t(c.nb);
    dim3 grid(unsigned((n + 1023) / 1024), items, 1);
    const size_t sm = size_t(q_to_b_words + b_to_q_words + 2 * kb) * 8;
    if (kq <= 8 && kb <= 8) {
        k_bfv_scale_round<8, 8><<<grid, 256, sm, s>>>(q_to_b, b_to_q, tq, q_to_b_words, b_to_q_words,
                                                     src, src_item, dst, dst_item, c.log_n);
    } else if (kq <= 16 && kb <= 16) {
        k_bfv_scale_round<16, 16><<<grid, 256, sm, s>>>(q_to_b, b_to_q, tq, q_to_b_words,
                                                        b_to_q_words, src, src_item, dst, dst_item,
                                                        c.log_n);
    } else {
        k_bfv_scale_round<32, 32><<<grid, 256, sm, s>>>(q_to_b, b_to_q, tq, q_to_b_words,
                                                        b_to_q_words, src, src_item, dst, dst_item,
                                                        c.log_n);
    }
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA;
}

}  // namespace catfhe
