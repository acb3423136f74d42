// NTT schedules of ring degree 2^13 (see ntt_part.cuh).
#define NTT_LOGN 13
#include "ntt_part.cuh"
