// Instantiates the NTT schedules of one ring degree (NTT_LOGN, defined by
// the including translation unit) and dispatches to them.
#include "ntt_kernels.cuh"

#define NTT_CAT2(a, b) a##b
#define NTT_CAT(a, b) NTT_CAT2(a, b)

namespace catfhe {

int NTT_CAT(ntt_fwd_n, NTT_LOGN)(const Context &c, const uint64_t *src, uint64_t *dst,
                                 const LimbMap &map, uint32_t n_limbs, cudaStream_t s,
                                 const NttEpilogue *epi, bool lazy, int sched) {
#define FWD(LN, S, A, B, TA, BA, C, D, TC, BC)                                              \
    if constexpr (LN == NTT_LOGN) {                                                        \
        if (sched == S)                                                                    \
            return run_fwd<LN, A, B, TA, BA, C, D, TC, BC>(c, src, dst, map, n_limbs, s, epi, \
                                                           lazy);                          \
    }
    NTT_SCHEDULES(FWD)
#undef FWD
    return CATFHE_EINVAL;
}

int NTT_CAT(ntt_inv_n, NTT_LOGN)(const Context &c, const uint64_t *src, uint64_t *dst,
                                 const LimbMap &map, uint32_t n_limbs, cudaStream_t s, int sched) {
#define INV(LN, S, A, B, TA, BA, C, D, TC, BC)                                               \
    if constexpr (LN == NTT_LOGN) {                                                         \
        if (sched == S)                                                                     \
            return run_inv<LN, A, B, TA, BA, C, D, TC, BC>(c, src, dst, map, n_limbs, s);   \
    }
    NTT_SCHEDULES(INV)
#undef INV
    return CATFHE_EINVAL;
}

}  // namespace catfhe
