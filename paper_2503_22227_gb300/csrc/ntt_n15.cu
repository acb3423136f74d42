// NTT schedules of ring degree 2^15 (see ntt_part.cuh).
#define NTT_LOGN 15
#include "ntt_part.cuh"
