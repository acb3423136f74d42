// NTT schedules of ring degree 2^14 (see ntt_part.cuh).
#define NTT_LOGN 14
#include "ntt_part.cuh"
