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
#include "ntt_kernels.cuh"

namespace catfhe {

#define NTT_DECL(LN)                                                                          \
    int ntt_fwd_n##LN(const Context &c, const uint64_t *src, uint64_t *dst, const LimbMap &map, \
                      uint32_t n_limbs, cudaStream_t s, const NttEpilogue *epi, bool lazy,      \
                      int sched);                                                              \
    int ntt_inv_n##LN(const Context &c, const uint64_t *src, uint64_t *dst, const LimbMap &map, \
                      uint32_t n_limbs, cudaStream_t s, int sched);
NTT_DECL(12) NTT_DECL(13) NTT_DECL(14) NTT_DECL(15) NTT_DECL(16)
#undef NTT_DECL

int ntt_schedule_count(int log_n) {
    switch (log_n) {
        case 12: return 5;
        case 13: return 7;
        case 14: case 15: case 16: return 8;
        default: return 0;
    }
}

void ntt_schedule_shape(int log_n, int sched, int shape[4]) {
#define SHAPE(LN, S, A, B, TA, BA, C, D, TC, BC) \
    if (log_n == LN && sched == S) { shape[0] = A; shape[1] = B; shape[2] = C; shape[3] = D; return; }
    NTT_SCHEDULES(SHAPE)
#undef SHAPE
    shape[0] = shape[1] = shape[2] = shape[3] = 0;
}

static int fwd_dispatch(const Context &c, const uint64_t *src, uint64_t *dst, const LimbMap &map,
                        uint32_t n_limbs, cudaStream_t s, const NttEpilogue *epi, bool lazy) {
    if (n_limbs == 0) return CATFHE_OK;
    const int sched = c.ntt_sched[ntt_class(n_limbs)];
    switch (c.log_n) {
        case 12: return ntt_fwd_n12(c, src, dst, map, n_limbs, s, epi, lazy, sched);
        case 13: return ntt_fwd_n13(c, src, dst, map, n_limbs, s, epi, lazy, sched);
        case 14: return ntt_fwd_n14(c, src, dst, map, n_limbs, s, epi, lazy, sched);
        case 15: return ntt_fwd_n15(c, src, dst, map, n_limbs, s, epi, lazy, sched);
        case 16: return ntt_fwd_n16(c, src, dst, map, n_limbs, s, epi, lazy, sched);
        default: return CATFHE_EINVAL;
    }
}

int launch_ntt_fwd(const Context &c, const uint64_t *src, uint64_t *dst, const LimbMap &map,
                   uint32_t n_limbs, cudaStream_t s) {
    return fwd_dispatch(c, src, dst, map, n_limbs, s, nullptr, false);
}

int launch_ntt_fwd_lazy(const Context &c, const uint64_t *src, uint64_t *dst, const LimbMap &map,
                        uint32_t n_limbs, cudaStream_t s) {
    return fwd_dispatch(c, src, dst, map, n_limbs, s, nullptr, true);
}

int launch_ntt_fwd_combine(const Context &c, uint64_t *lift, const LimbMap &map, uint32_t n_limbs,
                           const NttEpilogue &epi, cudaStream_t s) {
    return fwd_dispatch(c, lift, lift, map, n_limbs, s, &epi, false);
}

int launch_ntt_inv(const Context &c, const uint64_t *src, uint64_t *dst, const LimbMap &map,
                   uint32_t n_limbs, cudaStream_t s) {
    if (n_limbs == 0) return CATFHE_OK;
    const int sched = c.ntt_sched[ntt_class(n_limbs)];
    switch (c.log_n) {
        case 12: return ntt_inv_n12(c, src, dst, map, n_limbs, s, sched);
        case 13: return ntt_inv_n13(c, src, dst, map, n_limbs, s, sched);
        case 14: return ntt_inv_n14(c, src, dst, map, n_limbs, s, sched);
        case 15: return ntt_inv_n15(c, src, dst, map, n_limbs, s, sched);
        case 16: return ntt_inv_n16(c, src, dst, map, n_limbs, s, sched);
        default: return CATFHE_EINVAL;
    }
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
